"""Full-size parity at the benchmark's configurations, proved with one plan and
CUDA-graph replay exactly as bench.py runs them.

* The batched 7B-shaped LoRA step (32 layers x {q,k,v,o}, hidden 4096, seq
  512, ranks {8,16,64}; 1024 proofs): EVERY proof is recomputed by the oracle
  (one projection per worker process, spread over the host's cores) and
  compared byte for byte, for the default rounds and the batched rounds.
* The 13B-shaped step (40 layers x {q,k,v,o}, hidden 5120 padded to 8192,
  seq 2048, rank 16; 1280 proofs): every proof is replayed (below), and the
  eight proofs of 16 projections spread over the layers are compared byte for
  byte with the oracle.
* One 7B-shaped projection at seq 1024 (the plain per-matmul path of the
  benchmark's single-projection configuration): all eight proofs, byte for
  byte.

Replay (properties of every proof): dims and status, the transcript
replayed from the public statement (u, v, every r_i and the final state),
g_i(0) + g_i(1) equal to the running claim, and the final claim equal to
a_r . b_r.
"""
import ctypes

import pytest

import oracle
import oracle_pool
from oracle.field import R_MOD
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _fr(x):
    return x.to_int()


def _replay(job, pf):
    m, k, n = W.op_shape(job)
    d0, d1, d2 = (m - 1).bit_length(), (k - 1).bit_length(), (n - 1).bit_length()
    assert (pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2, pf.status) == (m, k, n, d0, d1, d2, 0)
    T = oracle.Transcript(job["seed"], m, k, n, job["tp"], job["tq"])
    T.squeeze(b"u", d0)
    T.squeeze(b"v", d2)
    claim = _fr(pf.c)
    T.absorb_fr(b"c", [claim])
    for i in range(d1):
        g = [_fr(pf.g[i][q]) for q in range(3)]
        assert (g[0] + g[1]) % R_MOD == claim, f"round {i}"
        T.absorb_fr(b"g", [g[0], g[2]])  # g(1) is fixed by the running claim
        r = T.squeeze(b"r", 1)[0]
        claim = oracle.round_poly_eval(*g, r)
    assert claim == _fr(pf.a_r) * _fr(pf.b_r) % R_MOD
    T.absorb_fr(b"f", [_fr(pf.a_r), _fr(pf.b_r)])
    assert T.state == bytes(pf.state)


def _prove_step(projs, opts=None):
    """All eight products of every projection, one plan, run twice (capture,
    then graph replay); returns (jobs, proofs)."""
    jobs = [j for t in projs for j in W.projection_products(t)]
    dev = {}
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    djobs = [B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
    plan = B.vl_plan_create(djobs, opts) if opts is not None else B.vl_plan_create(djobs)
    try:
        nws = B.vl_plan_workspace_bytes(plan)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        out = torch.empty(len(djobs) * ctypes.sizeof(B.vl_proof), dtype=torch.uint8, device="cuda")
        for _ in range(2):  # capture, then replay
            B.vl_plan_run(plan, ws.data_ptr(), nws, out.data_ptr(), B.VL_DEVICE)
        torch.cuda.synchronize()
        proofs = (B.vl_proof * len(djobs)).from_buffer_copy(out.cpu().numpy().tobytes())
    finally:
        B.vl_plan_destroy(plan)
        del dev
        torch.cuda.empty_cache()
    return jobs, proofs


def _compare(jobs, proofs, ref):
    by_name = {j["name"]: i for i, j in enumerate(jobs)}
    assert ref, "no oracle proofs"
    bad = [name for name, want in ref.items() if B.proof_bytes(proofs[by_name[name]]) != want]
    assert not bad, f"{len(bad)} of {len(ref)} proofs differ from the oracle, first: {bad[:4]}"


def test_7b_step_every_proof_equals_the_oracle():
    specs = W.step_layers("7b")
    pool, pending = oracle_pool.start(specs, W.GLOBAL_SEED)  # spawn workers; runs while the GPU proves
    try:
        projs = W.make_step("7b")
        jobs, proofs = _prove_step(projs)
        for j, pf in zip(jobs, proofs):
            _replay(j, pf)
        batched = B.vl_batch_opts()
        batched.rounds_variant = 8  # one launch per round over all proofs
        _, proofs8 = _prove_step(projs, batched)
    except BaseException:
        pool.terminate()
        raise
    ref = oracle_pool.finish(pool, pending)
    assert len(ref) == len(jobs) == 1024
    _compare(jobs, proofs, ref)
    _compare(jobs, proofs8, ref)


def test_13b_step_batched_graph():
    specs = W.step_layers("13b")
    sample = [s for s in specs if s[0] % 5 == 0 and s[1] in ("q", "o")]  # 16 projections over the 40 layers
    pool, pending = oracle_pool.start(sample, W.GLOBAL_SEED)
    try:
        projs = W.make_step("13b")
        jobs, proofs = _prove_step(projs)
        del projs
        assert len(jobs) == 1280
        for j, pf in zip(jobs, proofs):
            _replay(j, pf)
            m, k, n = W.op_shape(j)
            assert pf.d1 == (k - 1).bit_length()  # 5120 pads to 8192: 13 rounds
    except BaseException:
        pool.terminate()
        raise
    ref = oracle_pool.finish(pool, pending)
    assert len(ref) == 8 * len(sample)
    _compare(jobs, proofs, ref)


def test_7b_projection_seq1024_all_products():
    specs = W.step_layers("7b-proj")
    pool, pending = oracle_pool.start(specs, W.GLOBAL_SEED, procs=1)
    try:
        projs = W.make_step("7b-proj")
        jobs, proofs = _prove_step(projs)
        for j, pf in zip(jobs, proofs):
            _replay(j, pf)
    except BaseException:
        pool.terminate()
        raise
    ref = oracle_pool.finish(pool, pending)
    assert len(ref) == 8
    _compare(jobs, proofs, ref)
