"""The no-allocation entry point against the workspace entry point.

vl_prove_matmul_noalloc serves callers that cannot allocate device memory
(for example code embedded in an application that owns all device memory
through its own pool, or a loop that cannot afford the synchronisation
cudaMalloc implies): its scratch is a fixed array inside the library instead
of a caller workspace.  Its proofs must be byte-identical to
vl_prove_matmul's, on consecutive calls (the array keeps the previous
call's contents, so what must start at zero has to be cleared each call).

This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2508_21393_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _with_workspace(jb):
    n = B.vl_workspace_bytes([jb])
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    return B.proof_bytes(B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws.data_ptr(), n))


@pytest.mark.parametrize("m,k,n,tp,tq", [(64, 128, 64, 0, 0), (300, 1100, 70, 1, 0), (37, 2100, 29, 0, 1),
                                         (512, 4096, 16, 0, 0)])
def test_noalloc_matches_workspace_entry_point_twice(m, k, n, tp, tq):
    rng = np.random.default_rng(m + k + n + tp + tq)
    P = rng.integers(-(1 << 15), 1 << 15, size=(k, m) if tp else (m, k)).astype(np.int16)
    Q = rng.integers(-(1 << 15), 1 << 15, size=(n, k) if tq else (k, n)).astype(np.int16)
    Pd, Qd = torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()
    jb = B.job(Pd, Qd, tp, tq, seed=4242 + m)
    ref = _with_workspace(jb)
    first = B.proof_bytes(B.vl_prove_matmul_noalloc(jb.P, jb.Q, jb.fs))
    second = B.proof_bytes(B.vl_prove_matmul_noalloc(jb.P, jb.Q, jb.fs))
    assert first == ref
    assert second == ref


def test_noalloc_alternating_shapes_do_not_leak_state():
    rng = np.random.default_rng(5)
    jobs = []
    for (m, k, n) in ((40, 300, 20), (9, 33, 70)):
        Pd = torch.from_numpy(rng.integers(-(1 << 15), 1 << 15, size=(m, k)).astype(np.int16)).cuda()
        Qd = torch.from_numpy(rng.integers(-(1 << 15), 1 << 15, size=(k, n)).astype(np.int16)).cuda()
        jobs.append((B.job(Pd, Qd, 0, 0, seed=m), Pd, Qd))
    refs = [_with_workspace(j) for j, _, _ in jobs]
    for _ in range(2):
        for (j, _, _), ref in zip(jobs, refs):
            assert B.proof_bytes(B.vl_prove_matmul_noalloc(j.P, j.Q, j.fs)) == ref


def test_noalloc_refuses_jobs_beyond_the_fixed_scratch():
    k = 1 << 16  # two k x 8 accumulators alone are 8 MiB
    Pd = torch.zeros((1, k), dtype=torch.int16, device="cuda")
    Qd = torch.zeros((k, 1), dtype=torch.int16, device="cuda")
    jb = B.job(Pd, Qd, 0, 0, seed=1)
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul_noalloc(jb.P, jb.Q, jb.fs)
    assert e.value.code == B.VL_ENOMEM
    assert "scratch" in B.vl_last_error()
