"""Write tests/golden/proofs_small.json: small seeded statements of every
proof kind and the oracle's proof bytes for them.

The values come from the oracle only (this script imports nothing else of
the project but the seeded-input conventions below).  They freeze this
project's own transcript formats (the paper fixes none: matmul sumcheck,
linear zkMat, lookup argument, batched claims), so that a later change to
the oracle's byte layout shows up as a failing pin rather than passing
silently through the GPU parity tests.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def i16(rng, shape, lo=-(1 << 15), hi=1 << 15):
    return rng.integers(lo, hi, size=shape).astype(np.int16)


def main():
    rng = np.random.default_rng(20250821)
    out = {}
    # matmul sumcheck: op(P) . op(Q) with P transposed
    P, Q = i16(rng, (9, 5)), i16(rng, (9, 6))
    out["matmul"] = {"P": P.tolist(), "Q": Q.tolist(), "tp": 1, "tq": 0, "seed": 7,
                     "proof": oracle.prove_matmul(P, Q, 1, 0, seed=7).to_bytes().hex()}
    # linear zkMat: A' - A + G = 0
    A, G = i16(rng, (4, 6), -1000, 1000), i16(rng, (4, 6), -1000, 1000)
    A2 = (A - G).astype(np.int16)
    out["linear"] = {"mats": [A2.tolist(), A.tolist(), G.tolist()], "coeffs": [1, -1, 1], "seed": 8,
                     "proof": oracle.prove_linear([A2, A, G], [1, -1, 1], seed=8).to_bytes().hex()}
    # lookup argument: 13 values in [-4, 4)
    S = rng.integers(-4, 4, size=(13,)).astype(np.int16)
    out["lookup"] = {"S": S.tolist(), "t0": -4, "log2_n": 3, "seed": 9,
                     "proof": oracle.prove_lookup(S, -4, 3, seed=9).to_bytes().hex()}
    # batched claims: two products with inner dimension 5
    jobs = [{"P": i16(rng, (3, 5)), "Q": i16(rng, (5, 2)), "tp": 0, "tq": 0},
            {"P": i16(rng, (4, 5)), "Q": i16(rng, (5, 3)), "tp": 0, "tq": 0}]
    out["batch"] = {"jobs": [{"P": j["P"].tolist(), "Q": j["Q"].tolist()} for j in jobs], "seed": 10,
                    "proof": oracle.prove_matmul_batch(jobs, seed=10).to_bytes().hex()}
    with open(os.path.join(HERE, "proofs_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
