"""GPU parity of the lookup-argument sumcheck (Protocol 1, Eq.
eq:lookup-sumcheck): every proof from the CUDA path equals the oracle's byte
for byte, through the C ABI.

Cases: no high rounds (D = N), high rounds only after padding (n < N), one
and two rounds, a single entry, ragged n, negative t0, strided and host
operands, mixed batches equal to single proofs, plan reruns and rebinds,
device output, a value outside the table (VL_ELOOKUP), and the rescale
remainders of a 7B projection at full size (library verifier on every
proof, the oracle on a sample).
"""
import ctypes

import numpy as np
import pytest

from oracle import lookup as OL
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _ws(n):
    return torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")


class Look:
    def __init__(self, S, t0, ln, seed=0, bind=None, where="dev"):
        self.S = np.asarray(S, dtype=np.int16)
        if self.S.ndim == 1:
            self.S = self.S.reshape(1, -1)
        self.t0, self.ln, self.seed, self.bind, self.where = t0, ln, seed, bind, where
        self.keep = []

    def job(self):
        S = np.ascontiguousarray(self.S)
        if self.where == "host":
            self.keep.append(S)
            m = B.mat(S)
        elif self.where == "pitch":
            buf = torch.zeros((S.shape[0], S.shape[1] + 5), dtype=torch.int16, device="cuda")
            buf[:, :S.shape[1]] = torch.from_numpy(S).cuda()
            self.keep.append(buf)
            m = B.mat(buf[:, :S.shape[1]])
        else:
            t = torch.from_numpy(S).cuda()
            self.keep.append(t)
            m = B.mat(t)
        return B.lookup_job(m, self.t0, self.ln, self.seed, self.bind)

    def oracle_bytes(self):
        return OL.prove_lookup(self.S, self.t0, self.ln, seed=self.seed,
                               bind=self.bind if self.bind is not None else bytes(32)).to_bytes()


def gpu_prove(looks):
    jobs = [x.job() for x in looks]
    n = B.vl_lookup_workspace_bytes(jobs)
    assert n > 0
    ws = _ws(n)
    out = B.vl_prove_lookup(jobs, ws.data_ptr(), n)
    assert all(p.status == 0 for p in out)
    return jobs, out


CASES = [
    # (shape, log2_n, t0)
    ((1,), 0, 3),          # D = N = 1: no rounds
    ((2,), 1, 0),          # one round, a table round
    ((3,), 1, -1),         # two rounds: one high, one table
    ((16, 16), 8, 0),      # D = N = 256: table rounds only
    ((5, 7), 8, -128),     # n < N: padding fills the cube
    ((37, 29), 4, 0),      # ragged n, 7 high rounds
    ((64, 64), 6, 10),     # 6 high rounds, 6 table rounds
    ((1, 3000), 12, 0),    # N = 4096 > n
    ((4, 2048), 5, -16),   # several round items per pass
]


@pytest.mark.parametrize("shape,ln,t0", CASES)
def test_lookup_parity(shape, ln, t0):
    rng = np.random.default_rng(sum(shape) * 13 + ln)
    S = rng.integers(t0, t0 + (1 << ln), size=shape)
    x = Look(S, t0, ln, seed=ln * 1000 + sum(shape), bind=bytes([ln + 1]) * 32)
    _, out = gpu_prove([x])
    assert B.lookup_proof_bytes(out[0]) == x.oracle_bytes()


@pytest.mark.parametrize("where", ["host", "pitch"])
def test_lookup_operands(where):
    rng = np.random.default_rng(7)
    x = Look(rng.integers(0, 256, size=(33, 70)), 0, 8, seed=2, where=where)
    _, out = gpu_prove([x])
    assert B.lookup_proof_bytes(out[0]) == x.oracle_bytes()


def test_lookup_extreme_tables():
    """The whole int16 range as a table (N = 2^16) and values at both ends."""
    S = np.array([[-32768, 32767, 0, -1, 1, -32768, 32767, 5]], np.int16)
    x = Look(S, -32768, 16, seed=9)
    _, out = gpu_prove([x])
    assert B.lookup_proof_bytes(out[0]) == x.oracle_bytes()


def test_lookup_batch_equals_single_proofs():
    rng = np.random.default_rng(8)
    looks = [Look(rng.integers(0, 1 << ln, size=shape), 0, ln, seed=i)
             for i, (shape, ln) in enumerate([((9, 9), 3), ((1, 1), 0), ((200,), 8), ((64, 32), 4), ((3,), 2)])]
    _, out = gpu_prove(looks)
    for x, p in zip(looks, out):
        assert B.lookup_proof_bytes(p) == x.oracle_bytes()


def test_lookup_value_outside_table_reports_elookup():
    S = np.array([[0, 1, 2, 9]], np.int16)
    x = Look(S, 0, 3, seed=1)
    jobs = [x.job()]
    n = B.vl_lookup_workspace_bytes(jobs)
    ws = _ws(n)
    with pytest.raises(B.VLError) as e:
        B.vl_prove_lookup(jobs, ws.data_ptr(), n)
    assert e.value.code == B.VL_ELOOKUP
    # the context survives: a good proof right after
    y = Look(np.array([[0, 1, 2, 7]], np.int16), 0, 3, seed=1)
    _, out = gpu_prove([y])
    assert B.lookup_proof_bytes(out[0]) == y.oracle_bytes()


def test_lookup_plan_reruns_rebinds_device_output():
    rng = np.random.default_rng(10)
    looks = [Look(rng.integers(0, 16, size=(20, 20)), 0, 4, seed=3, where="host"),
             Look(rng.integers(-4, 4, size=(1, 500)), -4, 3, seed=4)]
    plan = B.LookupPlan([x.job() for x in looks])
    n = plan.workspace_bytes()
    ws1, ws2 = _ws(n), _ws(n)
    want = [x.oracle_bytes() for x in looks]
    for ws in (ws1, ws1, ws2, ws1):
        out = plan.run(ws.data_ptr(), n)
        assert [B.lookup_proof_bytes(p) for p in out] == want
    sz = ctypes.sizeof(B.vl_lookup_proof)
    dout = torch.empty(2 * sz, dtype=torch.uint8, device="cuda")
    plan.run(ws2.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE)
    torch.cuda.synchronize()
    raw = dout.cpu().numpy().tobytes()
    assert [B.lookup_proof_bytes(B.vl_lookup_proof.from_buffer_copy(raw, i * sz)) for i in range(2)] == want
    assert all(v >= 0 for v in plan.phase_ms())
    # host operand changed in place: the next run proves the new values
    host = looks[0].keep[0]
    host[0, 0] = (int(host[0, 0]) + 1) % 16
    looks[0].S = np.array(host)
    out = plan.run(ws1.data_ptr(), n)
    assert B.lookup_proof_bytes(out[0]) == looks[0].oracle_bytes()
    plan.destroy()


def test_lookup_7b_projection_remainders_full_size():
    """The four rescale-remainder lookups of two 7B projections, in the batch
    launch the bench times: every proof verifies in the library's host
    verifier; the two n x r lookups of the first projection are byte-equal
    to the oracle."""
    looks = []
    for t in W.make_step("7b", layers=[0])[:2]:
        for st in W.rescale_lookups(t):
            looks.append(Look(st["S"], st["t0"], st["log2_n"], seed=st["seed"]))
    jobs, out = gpu_prove(looks)
    for x, p in zip(looks, out):
        hj = B.lookup_job(B.mat(np.ascontiguousarray(x.S)), x.t0, x.ln, x.seed)
        assert B.vl_verify_lookup(hj, p)
    for i in (0, 1):
        assert B.lookup_proof_bytes(out[i]) == looks[i].oracle_bytes()


def test_plans_taking_turns_on_one_workspace():
    """A lookup plan, a linear plan and a claims plan alternate on one
    workspace: each run re-binds when another plan used the workspace since,
    and every proof stays equal to the oracle's."""
    rng = np.random.default_rng(21)
    x = Look(rng.integers(0, 64, size=(10, 30)), 0, 6, seed=2)
    lplan = B.LookupPlan([x.job()])
    A = rng.integers(-100, 100, size=(12, 20)).astype(np.int16)
    G = rng.integers(-100, 100, size=(12, 20)).astype(np.int16)
    A2 = (A - G).astype(np.int16)
    lin_t = [torch.from_numpy(m).cuda() for m in (A2, A, G)]
    linplan = B.LinPlan([B.lin_job([B.mat(t) for t in lin_t], [1, -1, 1], 5)])
    from oracle import prove_linear, prove_matmul_batch
    P = rng.integers(-1000, 1000, size=(9, 16)).astype(np.int16)
    Q = rng.integers(-1000, 1000, size=(16, 7)).astype(np.int16)
    bt = [torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()]
    cplan = B.ClaimsPlan([B.job(bt[0], bt[1], 0, 0, 0)], 8)
    n = max(lplan.workspace_bytes(), linplan.workspace_bytes(), cplan.workspace_bytes())
    ws = _ws(n)
    want_l = x.oracle_bytes()
    want_lin = prove_linear([A2, A, G], [1, -1, 1], seed=5).to_bytes()
    want_b = prove_matmul_batch([{"P": P, "Q": Q, "tp": 0, "tq": 0}], seed=8).to_bytes()
    for _ in range(2):
        assert B.lookup_proof_bytes(lplan.run(ws.data_ptr(), n)[0]) == want_l
        assert B.lin_proof_bytes(linplan.run(ws.data_ptr(), n)[0]) == want_lin
        assert cplan.run(ws.data_ptr(), n).to_bytes() == want_b
    lplan.destroy()
    linplan.destroy()
    cplan.destroy()


class _MatmulPlan:
    """A vl_plan with the other plans' method names."""

    def __init__(self, jobs):
        self.h, self.n = B.vl_plan_create(jobs), len(jobs)

    def workspace_bytes(self):
        return B.vl_plan_workspace_bytes(self.h)

    def first_proof(self, w, n):
        out = (B.vl_proof * self.n)()
        B.vl_plan_run(self.h, w, n, out, B.VL_HOST)
        return B.proof_bytes(out[0])

    def destroy(self):
        B.vl_plan_destroy(self.h)


def test_forgotten_workspace_is_bound_again():
    """vl_workspace_forget drops a workspace's record; the next run of any
    plan kind re-uploads its tables there (the record comes back, which only
    the binding step writes) and proves the same bytes; a destroyed plan
    leaves no record.  The workspace is never overwritten here."""
    rng = np.random.default_rng(22)
    x = Look(rng.integers(0, 32, size=(6, 20)), 0, 5, seed=3)
    A = rng.integers(-50, 50, size=(8, 12)).astype(np.int16)
    lin_t = [torch.from_numpy(m).cuda() for m in (A, A)]
    P = rng.integers(-100, 100, size=(5, 8)).astype(np.int16)
    Q = rng.integers(-100, 100, size=(8, 3)).astype(np.int16)
    bt = [torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()]
    plans = [(B.LookupPlan([x.job()]), lambda p, w, n: B.lookup_proof_bytes(p.run(w, n)[0])),
             (B.LinPlan([B.lin_job([B.mat(t) for t in lin_t], [1, -1], 6)]),
              lambda p, w, n: B.lin_proof_bytes(p.run(w, n)[0])),
             (B.ClaimsPlan([B.job(bt[0], bt[1], 0, 0, 0)], 9), lambda p, w, n: p.run(w, n).to_bytes()),
             (_MatmulPlan([B.job(bt[0], bt[1], 0, 0, 4)]), _MatmulPlan.first_proof)]
    for plan, run in plans:
        n = plan.workspace_bytes()
        ws = _ws(n)
        first = run(plan, ws.data_ptr(), n)
        assert B.vl_workspace_forget(ws.data_ptr())
        assert not B.vl_workspace_forget(ws.data_ptr())
        assert run(plan, ws.data_ptr(), n) == first
        assert B.vl_workspace_forget(ws.data_ptr())  # bound again by the second run
        run(plan, ws.data_ptr(), n)
        plan.destroy()
        assert not B.vl_workspace_forget(ws.data_ptr())
