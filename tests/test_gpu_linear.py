"""GPU parity of the linear zkMat (sum_q c_q op(M_q) = 0, Sec. IV; the LoRA
parameter update of Eq. eq:grad_update_ab): every proof from the CUDA path
equals the oracle's proof byte for byte, through the C ABI.

Shapes cover both fold orientations (reduction over rows or over columns,
whichever is shorter), both fold engines (tensor cores; CUDA cores for
reductions of at most 128 entries), ragged tails of the 128-line tiles and
128-entry stages, several reduction segments per line (accumulator path), transposed,
host, unaligned and odd-pitch operands, extreme entries, batches of mixed
shapes, and the full-size parameter updates of a 7B LoRA step.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _rand(rng, shape, lo=-(1 << 15), hi=1 << 15):
    return rng.integers(lo, hi, size=shape).astype(np.int16)


def _ws(nbytes):
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")


class Stmt:
    """One relation: logical matrices, coefficients, seed, binds, and how each
    operand is handed to the library (transposed, on the host, unaligned)."""

    def __init__(self, mats, coeffs, seed=0, binds=None, trans=None, where=None):
        self.mats, self.coeffs, self.seed, self.binds = mats, coeffs, seed, binds
        self.trans = trans or [0] * len(mats)
        self.where = where or ["dev"] * len(mats)
        self.keep = []

    def operand(self, q):
        M = self.mats[q]
        S = np.ascontiguousarray(M.T) if self.trans[q] else M
        w = self.where[q]
        if w == "host":
            S = np.ascontiguousarray(S)
            self.keep.append(S)
            return B.mat(S, self.trans[q])
        if w == "dev":
            t = torch.from_numpy(np.ascontiguousarray(S)).cuda()
        elif w == "pitch":  # leading dimension cols + 3 (not a multiple of 8 entries)
            buf = torch.zeros((S.shape[0], S.shape[1] + 3), dtype=torch.int16, device="cuda")
            buf[:, :S.shape[1]] = torch.from_numpy(np.ascontiguousarray(S)).cuda()
            t = buf[:, :S.shape[1]]
        elif w == "offset":  # base 2 bytes past an aligned address
            flat = torch.zeros(S.size + 1, dtype=torch.int16, device="cuda")
            flat[1:] = torch.from_numpy(np.ascontiguousarray(S).ravel()).cuda()
            t = flat[1:].view(S.shape)
        else:
            raise ValueError(w)
        self.keep.append(t)
        return B.mat(t, self.trans[q])

    def job(self):
        return B.lin_job([self.operand(q) for q in range(len(self.mats))], self.coeffs, self.seed, self.binds)

    def oracle_bytes(self):
        return oracle.prove_linear(self.mats, self.coeffs, seed=self.seed, binds=self.binds).to_bytes()


def gpu_prove(stmts):
    jobs = [s.job() for s in stmts]
    n = B.vl_linear_workspace_bytes(jobs)
    assert n > 0
    ws = _ws(n)
    out = B.vl_prove_linear(jobs, ws.data_ptr(), n)
    torch.cuda.synchronize()
    assert all(p.status == 0 for p in out)
    return jobs, out


SHAPES = [
    # (rows, cols, nmats, transposes): reduction over the shorter side
    (1, 1, 1, [0]),
    (1, 300, 2, [0, 1]),
    (300, 1, 2, [0, 1]),
    (5, 7, 3, [0, 0, 0]),
    (129, 257, 3, [0, 1, 0]),       # ragged tiles and stages, reduction over rows
    (257, 129, 3, [1, 0, 0]),       # reduction over columns
    (16, 4096, 3, [0, 0, 0]),       # LoRA factor B' = B - G_B (r x k)
    (4096, 16, 3, [0, 1, 0]),       # LoRA factor A' = A - G_A (d x r)
    (1500, 1600, 2, [0, 1]),        # two reduction segments per line: accumulator path
    (2100, 2048, 2, [1, 0]),        # accumulator path, reduction over columns
    (200, 40000, 1, [0]),           # 313 line tiles
    (128, 3000, 3, [0, 1, 0]),      # the longest reduction folded on CUDA cores (rows)
    (3000, 127, 2, [1, 0]),         # CUDA-core fold over an odd number of columns
    (600, 72, 2, [0, 1]),           # CUDA-core fold: 16-byte loads of aligned rows, and columns
]


@pytest.mark.parametrize("rows,cols,q,trans", SHAPES)
def test_linear_parity(rows, cols, q, trans):
    rng = np.random.default_rng(rows * 7 + cols * 13 + q)
    mats = [_rand(rng, (rows, cols)) for _ in range(q)]
    coeffs = [int(c) for c in rng.integers(-(1 << 62), 1 << 62, size=q)]
    binds = [bytes([i + 1]) * 32 for i in range(q)]
    s = Stmt(mats, coeffs, seed=rows * cols, binds=binds, trans=trans)
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()


@pytest.mark.parametrize("where", ["host", "pitch", "offset"])
def test_linear_staged_operands(where):
    rng = np.random.default_rng(11)
    mats = [_rand(rng, (70, 333)) for _ in range(3)]
    s = Stmt(mats, [3, -1, 7], seed=5, trans=[0, 1, 0], where=["dev", where, where])
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()


def test_linear_extreme_entries():
    rows, cols = 300, 700
    mats = [np.full((rows, cols), -(1 << 15), np.int16), np.full((rows, cols), (1 << 15) - 1, np.int16),
            np.zeros((rows, cols), np.int16)]
    s = Stmt(mats, [1, 1, 1], seed=3)
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()


@pytest.mark.parametrize("rows,cols", [(100, 700), (700, 128)])
def test_linear_extreme_entries_short_reduction(rows, cols):
    """Reductions of at most 128 entries (CUDA-core fold): all-minimum and
    all-maximum entries, where the limb column sums are largest."""
    mats = [np.full((rows, cols), -(1 << 15), np.int16), np.full((rows, cols), (1 << 15) - 1, np.int16),
            np.zeros((rows, cols), np.int16)]
    s = Stmt(mats, [1, 1, 1], seed=4, trans=[0, 1, 0])
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()


@pytest.mark.parametrize("rows,cols,trans", [(1 << 16, 128, [0, 1, 0]), (128, 1 << 16, [1, 0, 0])])
def test_linear_short_reduction_at_max_lines(rows, cols, trans):
    """The CUDA-core fold at the header's limits: 2^16 lines (VL_MAX_REDUCE)
    with the longest reduction it takes (128 entries), both orientations."""
    rng = np.random.default_rng(rows + 3 * cols)
    mats = [_rand(rng, (rows, cols)) for _ in range(3)]
    s = Stmt(mats, [5, -2, 9], seed=rows ^ cols, trans=trans)
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()


def test_linear_batch_mixed_shapes_equals_single_proofs():
    rng = np.random.default_rng(12)
    stmts = []
    for i, (r, c) in enumerate([(3, 5), (4096, 8), (64, 4096), (1, 1), (1200, 1100), (17, 17)]):
        q = 1 + i % 4
        stmts.append(Stmt([_rand(rng, (r, c)) for _ in range(q)], list(range(1, q + 1)), seed=100 + i,
                          trans=[(i + j) % 2 for j in range(q)]))
    _, out = gpu_prove(stmts)
    for s, p in zip(stmts, out):
        assert B.lin_proof_bytes(p) == s.oracle_bytes()


def test_linear_true_and_false_relations_verify():
    """Completeness and soundness end to end: a true update relation's GPU
    proof verifies (library verifier and oracle verifier); a false one is
    rejected by both."""
    rng = np.random.default_rng(13)
    A = _rand(rng, (512, 64), -(1 << 14), 1 << 14)
    G = _rand(rng, (512, 64), -(1 << 13), 1 << 13)
    A2 = (A.astype(np.int32) - G).astype(np.int16)
    bad = A2.copy()
    bad[100, 7] += 1
    good, wrong = Stmt([A2, A, G], [1, -1, 1], seed=8), Stmt([bad, A, G], [1, -1, 1], seed=8)
    jobs, out = gpu_prove([good, wrong])
    hjobs = [B.lin_job([B.mat(m) for m in s.mats], s.coeffs, s.seed) for s in (good, wrong)]
    assert B.vl_verify_linear(hjobs[0], out[0])
    assert not B.vl_verify_linear(hjobs[1], out[1])
    for s, p, ok in ((good, out[0], True), (wrong, out[1], False)):
        proof = oracle.LinearProof(p.rows, p.cols, p.d0, p.d1, [p.evals[q].to_int() for q in range(p.nmats)],
                                   bytes(p.state))
        assert oracle.verify_linear(s.mats, s.coeffs, proof, seed=s.seed)[0] is ok


def test_linear_7b_step_updates_full_size():
    """All parameter updates of one 7B LoRA step layer set (4 projections x
    {A, B}, rank drawn per layer) in the batch launch the bench times; every
    proof verifies in the library's host verifier and a sample is byte-equal
    to the oracle."""
    layers = [0, 1]
    proj = W.make_step("7b", layers=layers)
    stmts = []
    for t in proj:
        for st in W.update_statements(t):
            stmts.append(Stmt(list(st["mats"]), list(st["coeffs"]), seed=st["seed"]))
    jobs, out = gpu_prove(stmts)
    for s, p in zip(stmts, out):
        hj = B.lin_job([B.mat(m) for m in s.mats], s.coeffs, s.seed)
        assert B.vl_verify_linear(hj, p)
    for i in (0, 1, len(stmts) - 1):
        assert B.lin_proof_bytes(out[i]) == stmts[i].oracle_bytes()


def test_linear_repeat_is_deterministic():
    rng = np.random.default_rng(14)
    s = Stmt([_rand(rng, (999, 1001)) for _ in range(2)], [1, 2], seed=1)
    _, a = gpu_prove([s])
    _, b = gpu_prove([s])
    assert B.lin_proof_bytes(a[0]) == B.lin_proof_bytes(b[0])


def test_linear_plan_reruns_rebinds_and_device_output():
    """A plan proves its batch at every run: the same proofs on repeated runs,
    after moving to another workspace, and with proofs left on the device;
    host operands are re-read at every run."""
    rng = np.random.default_rng(15)
    stmts = [Stmt([_rand(rng, (300, 40)) for _ in range(3)], [1, -2, 3], seed=4, where=["dev", "host", "pitch"]),
             Stmt([_rand(rng, (64, 2000)) for _ in range(2)], [5, 6], seed=5, trans=[1, 0])]
    jobs = [s.job() for s in stmts]
    plan = B.LinPlan(jobs)
    n = plan.workspace_bytes()
    ws1, ws2 = _ws(n), _ws(n)
    want = [s.oracle_bytes() for s in stmts]
    for ws in (ws1, ws1, ws2, ws1):
        out = plan.run(ws.data_ptr(), n)
        assert [B.lin_proof_bytes(p) for p in out] == want
    dout = torch.empty(2 * ctypes_sizeof_lin(), dtype=torch.uint8, device="cuda")
    plan.run(ws2.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE)
    torch.cuda.synchronize()
    raw = dout.cpu().numpy().tobytes()
    got = [B.lin_proof_bytes(B.vl_lin_proof.from_buffer_copy(raw, i * ctypes_sizeof_lin())) for i in range(2)]
    assert got == want
    ms = plan.phase_ms()
    assert all(x >= 0 for x in ms)
    # the host operand changes in place: the next run proves the new matrix
    host = stmts[0].keep[1]  # operand 1 of the first statement is the host array
    host[0, 0] ^= 1
    stmts[0].mats[1] = np.array(host)
    out = plan.run(ws1.data_ptr(), n)
    assert B.lin_proof_bytes(out[0]) == stmts[0].oracle_bytes()
    plan.destroy()


def ctypes_sizeof_lin():
    return ctypes.sizeof(B.vl_lin_proof)


def test_linear_sixteen_matrices():
    """VL_LIN_MAX matrices in one relation (the coefficient and bind lists at
    their longest)."""
    rng = np.random.default_rng(16)
    mats = [_rand(rng, (33, 47)) for _ in range(B.VL_LIN_MAX)]
    coeffs = [int(c) for c in rng.integers(-1000, 1000, size=B.VL_LIN_MAX)]
    binds = [bytes([i]) * 32 for i in range(B.VL_LIN_MAX)]
    s = Stmt(mats, coeffs, seed=16, binds=binds, trans=[i % 2 for i in range(B.VL_LIN_MAX)])
    _, out = gpu_prove([s])
    assert B.lin_proof_bytes(out[0]) == s.oracle_bytes()
