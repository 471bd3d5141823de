"""Oracle for the matmul sumcheck of VeriLoRA (arXiv 2508.21393).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
CPU restatement of what the GPU prover computes: the sumcheck proof that
C = op(P) . op(Q) over the BLS12-381 scalar field (Sec. II-B, II-C, Eq.
eq:MLE and eq:zk-mle-matmul), with a SHA-256 Fiat-Shamir transcript (Sec. IV,
footnote on Fiat-Shamir), and the linear zkMat proofs of matrix additions
(sum_q c_q M_q = 0 by MLE linearity; the parameter update of Eq.
eq:grad_update_ab is one), and the lookup-argument sumcheck of Protocol 1
(Eq. eq:lookup-sumcheck) for range tables, and the batched-claim sumcheck
that proves many products with one transcript (Sec. IV, composition by
random aggregation), and the chained proof of one LoRA projection in which
the claims on intermediate tensors are reduced through the rescale
relations instead of being opened (Sec. IV, sequential composition).  It
uses Python integers and ``hashlib`` only,
with NumPy object arrays as the one library matmul step.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path (the CUDA library and its
Python binding) never imports, links or runs anything in here, and this
package imports nothing from the product.

Parity status per function is stated in each module header.  The transcript
byte format is this project's own convention (the paper fixes no hash,
serialisation or challenge sampling), so its *format* is "parity unpinned";
SHA-256 itself is pinned by the FIPS 180-4 test vectors.
"""

from .field import R_MOD, fr, fr_add, fr_sub, fr_mul, fr_inv, fr_to_bytes, fr_from_bytes
from .transcript import Transcript
from .mle import (eq_table, eq_value, eq_eval, mle_eval_bruteforce, mle_eval_bind, mle_eval_matrix,
                  fold_rows, fold_cols)
from .sumcheck import Proof, prove_matmul, verify_matmul, round_poly_eval
from .encode import encode_montgomery, limbs_le32
from .linear import LinearProof, prove_linear, verify_linear
from .lookup import LookupProof, prove_lookup, verify_lookup, cubic_eval
from .batch import BatchProof, prove_matmul_batch, verify_matmul_batch, merkle_root
from .chain import ChainProof, prove_chain, verify_chain

__all__ = [
    "R_MOD", "fr", "fr_add", "fr_sub", "fr_mul", "fr_inv", "fr_to_bytes", "fr_from_bytes",
    "Transcript", "eq_table", "eq_value", "eq_eval", "mle_eval_bruteforce", "mle_eval_bind", "mle_eval_matrix",
    "fold_rows", "fold_cols", "Proof", "prove_matmul", "verify_matmul", "round_poly_eval",
    "encode_montgomery", "limbs_le32", "LinearProof", "prove_linear", "verify_linear",
    "LookupProof", "prove_lookup", "verify_lookup", "cubic_eval",
    "BatchProof", "prove_matmul_batch", "verify_matmul_batch", "merkle_root",
    "ChainProof", "prove_chain", "verify_chain",
]
