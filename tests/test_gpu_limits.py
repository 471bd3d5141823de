"""GPU parity at the limits the C header states, through the C ABI.

* VL_MAX_REDUCE = 2^16: a product with m = n = 2^16 (the fold reduces
  2^16 rows of op(P) and 2^16 columns of op(Q), the largest reductions the
  64-bit column sums of the int16 fold hold exactly), with random entries
  and with every entry at the int16 maximum (the largest column sums), in
  both storage orientations and on both fold engines; byte-equal to the
  oracle.  One more row or column is refused with VL_ESHAPE.
* VL_MAX_ROUNDS = 24: an inner dimension of k = 2^24 (24 sumcheck rounds);
  byte-equal to the oracle.  k = 2^24 + 1 is refused.
* VL_LOOKUP_MAX_LOG_D = 24: a range lookup of 2^24 int16 values in the
  table of all 2^16 int16 values.  The literal oracle sumcheck of seven
  2^24-entry vectors is out of reach here, so the proof is checked by
  properties that hold at any size, computed with the oracle's pieces: the
  transcript replayed from the statement (beta, alpha, u, every r_t, the
  final state), g_t(0) + g_t(1) equal to the running claim, the final claim
  equal to Eq. eq:lookup-sumcheck's polynomial at r from the four sent
  values and the verifier-side eq and table values, and the four values
  equal to the MLEs of A, S, B, m recomputed from S and T (variable-binding
  evaluation, pinned against brute-force eq:MLE).  2^24 + 1 values are
  refused.
"""
import numpy as np
import pytest

import oracle
from oracle import lookup as OL
from oracle.field import R_MOD, fr_inv
from paper_2508_21393_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

MAXR = 1 << 16


def _prove(P, Q, tp, tq, seed, engine=0):
    Pd, Qd = torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()
    j = B.job(Pd, Qd, tp, tq, seed)
    o = B.vl_batch_opts()
    o.fold_engine = engine
    n = B.vl_workspace_bytes([j], o)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    pf = B.vl_prove_batch([j], ws.data_ptr(), n, opts=o)[0]
    torch.cuda.synchronize()
    assert pf.status == 0
    return B.proof_bytes(pf)


def _oracle(P, Q, tp, tq, seed):
    return oracle.prove_matmul(P, Q, tp, tq, seed=seed).to_bytes()


@pytest.mark.parametrize("fill", ["random", "max"])
def test_max_reduce_both_sides(fill):
    rng = np.random.default_rng(21)
    k = 64
    if fill == "random":
        P = rng.integers(-(1 << 15), 1 << 15, size=(MAXR, k), dtype=np.int16)
        Q = rng.integers(-(1 << 15), 1 << 15, size=(k, MAXR), dtype=np.int16)
    else:  # p = x + 2^15 = 2^16 - 1 everywhere: the largest column sums
        P = np.full((MAXR, k), 32767, dtype=np.int16)
        Q = np.full((k, MAXR), 32767, dtype=np.int16)
    ref = _oracle(P, Q, 0, 0, 31)
    for engine in (0, 1):
        assert _prove(P, Q, 0, 0, 31, engine) == ref, f"engine {engine}"


def test_max_reduce_transposed_storage():
    rng = np.random.default_rng(22)
    k = 40  # ragged inner dimension
    P = rng.integers(-(1 << 15), 1 << 15, size=(k, MAXR), dtype=np.int16)  # op(P) = P^T: 2^16 x 40
    Q = rng.integers(-(1 << 15), 1 << 15, size=(MAXR, k), dtype=np.int16)  # op(Q) = Q^T: 40 x 2^16
    P[:, :3] = -32768
    Q[:5, :] = 32767
    ref = _oracle(P, Q, 1, 1, 32)
    for engine in (0, 1):
        assert _prove(P, Q, 1, 1, 32, engine) == ref, f"engine {engine}"


def test_one_past_max_reduce_is_refused():
    P = torch.zeros((MAXR + 1, 8), dtype=torch.int16, device="cuda")
    Q = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    j = B.job(P, Q, 0, 0, 1)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(j.P, j.Q, j.fs, ws.data_ptr(), 1 << 20)
    assert e.value.code == B.VL_ESHAPE


def test_max_rounds_k_2_24():
    rng = np.random.default_rng(23)
    k = 1 << 24
    P = rng.integers(-(1 << 15), 1 << 15, size=(1, k), dtype=np.int16)
    Q = rng.integers(-(1 << 15), 1 << 15, size=(1, k), dtype=np.int16)  # op(Q) = Q^T: k x 1
    got = _prove(P, Q, 0, 1, 33)
    assert int.from_bytes(got[16:20], "little") == 24  # d1
    assert got == _oracle(P, Q, 0, 1, 33)


def test_one_past_max_rounds_is_refused():
    k = (1 << 24) + 1
    P = torch.zeros((1, k), dtype=torch.int16, device="cuda")
    j = B.job(P, P, 0, 1, 1)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(j.P, j.Q, j.fs, ws.data_ptr(), 1 << 20)
    assert e.value.code == B.VL_ESHAPE


def _fr(x):
    return x.to_int()


def _lookup_properties(S, t0, log2_n, seed, pf):
    """The lookup verifier's checks written with the oracle's pieces."""
    N = 1 << log2_n
    n = S.size
    D, log2_d = OL.lookup_dims(n, log2_n)
    assert (pf.n, pf.log2_d, pf.log2_n, pf.t0) == (n, log2_d, log2_n, t0)
    T = OL._start(seed, n, log2_d, log2_n, t0, bytes(32))
    beta = T.squeeze(b"b", 1)[0]
    alpha = T.squeeze(b"a", 1)[0]
    u = T.squeeze(b"u", log2_d)
    claim = (alpha + alpha * alpha) % R_MOD
    rs = []
    for t in range(log2_d):
        g = [_fr(pf.g[t][q]) for q in range(4)]
        assert (g[0] + g[1]) % R_MOD == claim, f"round {t + 1}"
        T.absorb_fr(b"g", [g[0], g[2], g[3]])
        r = T.squeeze(b"r", 1)[0]
        rs.append(r)
        claim = OL.cubic_eval(g, r)
    a_r, s_r, b_r, m_r = (_fr(x) for x in (pf.a_r, pf.s_r, pf.b_r, pf.m_r))
    r_low, u_low = rs[log2_d - log2_n:], u[log2_d - log2_n:]
    t_r = oracle.mle_eval_bind([t0 + j for j in range(N)], r_low)
    c = N * fr_inv(D) % R_MOD
    final = OL.p_value({"A": a_r, "E": oracle.eq_eval(u, rs), "S": (s_r + beta) % R_MOD, "B": b_r,
                        "Ej": oracle.eq_eval(u_low, r_low), "T": (t_r + beta) % R_MOD, "m": m_r}, alpha, c)
    assert final == claim, "final claim"
    T.absorb_fr(b"f", [a_r, s_r, b_r, m_r])
    assert T.state == bytes(pf.state)
    # the four values against the vectors recomputed from S and T
    s = np.concatenate([S.reshape(-1).astype(np.int64), np.full(D - n, t0, dtype=np.int64)])  # padded with t0
    Binv = np.array([fr_inv((beta + t0 + j) % R_MOD) for j in range(N)], dtype=object)
    A = Binv[s - t0]
    assert a_r == oracle.mle_eval_bind(A, rs), "a_r"
    assert s_r == oracle.mle_eval_bind(s.astype(object) % R_MOD, rs), "s_r"
    assert b_r == oracle.mle_eval_bind(Binv, r_low), "b_r"
    m = np.bincount(s - t0, minlength=N)
    assert m_r == oracle.mle_eval_bind(m.tolist(), r_low), "m_r"


def test_lookup_max_log_d():
    rng = np.random.default_rng(24)
    S = rng.integers(-(1 << 15), 1 << 15, size=(4096, 4096), dtype=np.int16)  # 2^24 values, every int16 likely
    S[0, :4] = (-32768, 32767, 0, -1)
    Sd = torch.from_numpy(S).cuda()
    kj = B.lookup_job(B.mat(Sd), -32768, 16, seed=25)
    n = B.vl_lookup_workspace_bytes([kj])
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    pf = B.vl_prove_lookup([kj], ws.data_ptr(), n)[0]
    torch.cuda.synchronize()
    assert pf.log2_d == 24
    _lookup_properties(S, -32768, 16, 25, pf)


def test_lookup_one_past_max_log_d_is_refused():
    Sd = torch.zeros((1, (1 << 24) + 1), dtype=torch.int16, device="cuda")
    kj = B.lookup_job(B.mat(Sd), 0, 8, seed=1)
    with pytest.raises(B.VLError) as e:
        n = B.vl_lookup_workspace_bytes([kj])
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")
        B.vl_prove_lookup([kj], ws.data_ptr(), max(n, 256))
    assert e.value.code == B.VL_ESHAPE
