"""GPU parity: every proof from the CUDA path equals the oracle's proof byte
for byte (transcript state included), through the C ABI.

Shapes span several fold tiles and ragged tails in every orientation
(column-sum tiles of 1024 columns x 256 rows, row-dot tiles of 32 rows x 2048
columns), transposed operands, unaligned leading dimensions and base
pointers, Montgomery-form operands, batches, graph replay and host-space
operands.
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


def _rand(rng, shape):
    return rng.integers(-(1 << 15), 1 << 15, size=shape).astype(np.int16)


def _ws(nbytes):
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")


def gpu_prove(P, Q, tp=0, tq=0, seed=0):
    Pd = torch.from_numpy(np.ascontiguousarray(P)).cuda()
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    jb = B.job(Pd, Qd, tp, tq, seed)
    n = B.vl_workspace_bytes([jb])
    assert n > 0
    ws = _ws(n)
    pf = B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws.data_ptr(), n)
    assert pf.status == 0
    return pf


def _shapes(m, k, n, tp, tq, rng):
    A = _rand(rng, (m, k))
    Bm = _rand(rng, (k, n))
    P = np.ascontiguousarray(A.T) if tp else A
    Q = np.ascontiguousarray(Bm.T) if tq else Bm
    return A, Bm, P, Q


def test_single_matmul_64x128x64():
    job = W.single_matmul()
    pf = gpu_prove(job["P"], job["Q"], 0, 0, job["seed"])
    ref = oracle.prove_matmul(job["P"], job["Q"], 0, 0, seed=job["seed"])
    assert B.proof_bytes(pf) == ref.to_bytes()


@pytest.mark.parametrize("m,k,n,tp,tq", [
    (37, 53, 29, 0, 0), (1, 1, 1, 0, 0), (5, 1, 3, 0, 0), (1, 64, 1, 0, 0), (2, 3, 1, 1, 1),
    (300, 1100, 70, 0, 0),     # column-sum: 2 column tiles x 2 row tiles; row-dot: 35 row tiles
    (70, 40, 2100, 0, 0),      # row-dot over 2100 columns: two column chunks
    (2100, 40, 70, 1, 1),      # transposed: row-dot over 2100 columns, column-sum of Q^T
    (257, 33, 300, 1, 1), (64, 128, 64, 1, 0), (64, 128, 64, 0, 1),
    (3, 4097, 5, 0, 0),        # k just above a power of two: d1 = 13, mostly padding
])
def test_ragged_and_transposed(m, k, n, tp, tq):
    rng = np.random.default_rng(m * 7919 + k * 31 + n + 100 * tp + 1000 * tq)
    A, Bm, P, Q = _shapes(m, k, n, tp, tq, rng)
    seed = m * k + n
    pf = gpu_prove(P, Q, tp, tq, seed)
    ref = oracle.prove_matmul(P, Q, tp, tq, seed=seed)
    assert B.proof_bytes(pf) == ref.to_bytes()


@pytest.mark.parametrize("m,k,n,tp,tq", [
    (600, 2056, 1032, 0, 0),   # bulk path: 3 row tiles, column tiles 1024/1024/8, 32 stages per tile
    (600, 2056, 1032, 1, 1),   # bulk path, transposed: row dots over 600 columns, column sums of Q^T
    (4096, 16, 40, 0, 0),      # narrow contiguous rows: one copy per stage
    (40, 4096, 16, 0, 0),      # narrow row dots (16 columns, a 32-byte copy per row)
    (24, 8, 8, 1, 1),          # smallest bulk-eligible shapes
])
def test_bulk_pipeline_shapes(m, k, n, tp, tq):
    rng = np.random.default_rng(m + 3 * k + 7 * n + tp)
    A, Bm, P, Q = _shapes(m, k, n, tp, tq, rng)
    pf = gpu_prove(P, Q, tp, tq, 99)
    assert B.proof_bytes(pf) == oracle.prove_matmul(P, Q, tp, tq, seed=99).to_bytes()


def test_bulk_eligible_cols_with_unaligned_ld_falls_back():
    rng = np.random.default_rng(8)
    big = _rand(rng, (64, 1030))
    Pd = torch.from_numpy(big).cuda()[:, :1024]      # cols % 8 == 0 but ld = 1030
    Q = _rand(rng, (1024, 24))
    Qd = torch.from_numpy(Q).cuda()  # kept alive: the job holds only its address
    jb = B.job(Pd, Qd, 0, 0, 5)
    n = B.vl_workspace_bytes([jb])
    ws = _ws(n)
    pf = B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws.data_ptr(), n)
    assert B.proof_bytes(pf) == oracle.prove_matmul(big[:, :1024], Q, 0, 0, seed=5).to_bytes()


def test_wait_limit_option_keeps_results():
    jobs = _lora_jobs(n=32, d=256, k=256, r=8, layer=5, proj="o")
    dj, keep = _dev_jobs(jobs)
    opts = B.vl_batch_opts()
    opts.wait_limit_us = 500000
    nb = B.vl_workspace_bytes(dj, opts)
    ws = _ws(nb)
    proofs = B.vl_prove_batch(dj, ws.data_ptr(), nb, opts=opts)
    for j, pf in zip(jobs, proofs):
        assert B.proof_bytes(pf) == oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()


def test_extreme_values():
    """All entries at the int16 extremes (the +2^15 offset and its correction)."""
    m, k, n = 33, 70, 40
    for val in (-(1 << 15), (1 << 15) - 1, 0):
        P = np.full((m, k), val, np.int16)
        Q = np.full((k, n), -(1 << 15), np.int16)
        pf = gpu_prove(P, Q, 0, 0, 5)
        assert B.proof_bytes(pf) == oracle.prove_matmul(P, Q, 0, 0, seed=5).to_bytes()


def test_unaligned_views():
    rng = np.random.default_rng(3)
    big = _rand(rng, (90, 203))
    Qbig = _rand(rng, (1 + 150 * 77,))
    Pd_full = torch.from_numpy(big).cuda()
    Pd = Pd_full[5:85, 3:153]                      # ld = 203 (odd), base offset 3 elements
    Qd = torch.from_numpy(Qbig).cuda()[1:].view(150, 77)  # base misaligned by 2 bytes
    jb = B.job(Pd, Qd, 0, 0, 42)
    n = B.vl_workspace_bytes([jb])
    ws = _ws(n)
    pf = B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws.data_ptr(), n)
    ref = oracle.prove_matmul(big[5:85, 3:153], Qbig[1:].reshape(150, 77), 0, 0, seed=42)
    assert B.proof_bytes(pf) == ref.to_bytes()


def _encode(Md):
    out = torch.empty((Md.shape[0], Md.shape[1], 8), dtype=torch.int32, device="cuda")
    B.vl_encode(B.mat(Md), out.data_ptr())
    return out


def test_encode_matches_definition():
    rng = np.random.default_rng(11)
    M = _rand(rng, (67, 45))
    M[0, :4] = [0, 1, -1, -(1 << 15)]
    out = _encode(torch.from_numpy(M).cuda()).cpu().numpy().view(np.uint32)
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            assert list(out[i, j]) == oracle.limbs_le32(oracle.encode_montgomery(int(M[i, j])))


@pytest.mark.parametrize("m,k,n,tp,tq", [(37, 53, 29, 0, 0), (300, 260, 20, 1, 1), (5, 600, 7, 0, 1)])
def test_montgomery_operands_prove_the_same_statement(m, k, n, tp, tq):
    rng = np.random.default_rng(m + k + n)
    A, Bm, P, Q = _shapes(m, k, n, tp, tq, rng)
    Pe = _encode(torch.from_numpy(P).cuda())
    Qe = _encode(torch.from_numpy(Q).cuda())
    jb = B.job(Pe, Qe, tp, tq, 77)
    nb = B.vl_workspace_bytes([jb])
    ws = _ws(nb)
    pf = B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws.data_ptr(), nb)
    ref = oracle.prove_matmul(P, Q, tp, tq, seed=77)
    assert B.proof_bytes(pf) == ref.to_bytes()


def _lora_jobs(n=64, d=256, k=256, r=8, layer=0, proj="q"):
    t = W.lora_projection(W.GLOBAL_SEED, layer, proj, n, d, k, r)
    return W.projection_products(t)


def _dev_jobs(jobs):
    keep, out = [], []
    cache = {}
    for j in jobs:
        for key in ("P", "Q"):
            a = j[key]
            if id(a) not in cache:
                cache[id(a)] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        Pd, Qd = cache[id(j["P"])], cache[id(j["Q"])]
        out.append(B.job(Pd, Qd, j["tp"], j["tq"], j["seed"]))
    keep.append(cache)
    return out, keep


def test_lora_step_batch_equals_alone_and_oracle():
    jobs = _lora_jobs() + _lora_jobs(n=32, d=128, k=192, r=16, layer=1, proj="o")
    dj, keep = _dev_jobs(jobs)
    nb = B.vl_workspace_bytes(dj)
    ws = _ws(nb)
    proofs = B.vl_prove_batch(dj, ws.data_ptr(), nb)
    for j, jb, pf in zip(jobs, dj, proofs):
        ref = oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
        assert B.proof_bytes(pf) == ref, j["name"]
        n1 = B.vl_workspace_bytes([jb])
        ws1 = _ws(n1)
        alone = B.vl_prove_matmul(jb.P, jb.Q, jb.fs, ws1.data_ptr(), n1)
        assert B.proof_bytes(alone) == ref, j["name"]


def test_plan_graph_replay_device_output():
    jobs = _lora_jobs(n=48, d=128, k=128, r=8)
    dj, keep = _dev_jobs(jobs)
    plan = B.vl_plan_create(dj)
    try:
        nb = B.vl_plan_workspace_bytes(plan)
        ws = _ws(nb)
        out = torch.zeros(len(dj) * ctypes.sizeof(B.vl_proof), dtype=torch.uint8, device="cuda")
        refs = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jobs]
        for _ in range(3):
            out.zero_()
            B.vl_plan_run(plan, ws.data_ptr(), nb, out.data_ptr(), B.VL_DEVICE)
            torch.cuda.synchronize()
            host = (B.vl_proof * len(dj)).from_buffer_copy(out.cpu().numpy().tobytes())
            for pf, ref in zip(host, refs):
                assert B.proof_bytes(pf) == ref
    finally:
        B.vl_plan_destroy(plan)


def test_host_operands_and_host_output():
    jobs = _lora_jobs(n=40, d=96, k=160, r=8, layer=2, proj="v")
    hj = [B.job(np.ascontiguousarray(j["P"]), np.ascontiguousarray(j["Q"]), j["tp"], j["tq"], j["seed"])
          for j in jobs]
    plan = B.vl_plan_create(hj)
    try:
        nb = B.vl_plan_workspace_bytes(plan)
        ws = _ws(nb)
        out = (B.vl_proof * len(hj))()
        for _ in range(2):
            B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
            for j, pf in zip(jobs, out):
                ref = oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
                assert B.proof_bytes(pf) == ref
    finally:
        B.vl_plan_destroy(plan)


def test_gpu_proofs_verify_and_perturbations_reject():
    rng = np.random.default_rng(19)
    A, Bm, P, Q = _shapes(24, 50, 12, 1, 0, rng)
    C = W.exact_matmul(A, Bm)
    pf = gpu_prove(P, Q, 1, 0, 314)
    fs = B.fs_init(314)
    assert B.vl_verify_matmul(B.mat(P, 1), B.mat(Q, 0), B.mat(C), fs, pf)
    opf = oracle.prove_matmul(P, Q, 1, 0, seed=314)
    assert oracle.verify_matmul(P, Q, C, opf, 1, 0, seed=314)[0]
    pf.g[2][1].limb[3] ^= 1
    assert not B.vl_verify_matmul(B.mat(P, 1), B.mat(Q, 0), B.mat(C), fs, pf)


def test_plans_taking_turns_on_one_workspace():
    """Two plans alternate on one workspace: each re-uploads its tables."""
    ja = _lora_jobs(n=32, d=64, k=96, r=8, layer=3, proj="k")
    jb_ = [_lora_jobs(n=24, d=80, k=48, r=16, layer=4, proj="q")[i] for i in (0, 3, 6)]
    da, ka = _dev_jobs(ja)
    db, kb = _dev_jobs(jb_)
    pa, pb = B.vl_plan_create(da), B.vl_plan_create(db)
    try:
        nb = max(B.vl_plan_workspace_bytes(pa), B.vl_plan_workspace_bytes(pb))
        ws = _ws(nb)
        ra = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in ja]
        rb = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jb_]
        for _ in range(2):
            for plan, refs in ((pa, ra), (pb, rb)):
                out = (B.vl_proof * len(refs))()
                B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
                assert [B.proof_bytes(p) for p in out] == refs
    finally:
        B.vl_plan_destroy(pa)
        B.vl_plan_destroy(pb)


def test_launch_modes_and_fold_engines_agree():
    """Persistent launch, phase launches with the tensor-core fold, phase
    launches with the CUDA-core fold, every rounds variant and thread count
    (8: batched rounds, one launch per round): the same proofs."""
    jobs = _lora_jobs(n=40, d=128, k=96, r=8, layer=6, proj="q")
    dj, keep = _dev_jobs(jobs)
    refs = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jobs]
    for mode, engine, rv, rt in ((1, 0, 0, 0), (2, 0, 0, 0), (2, 1, 0, 0), (0, 0, 0, 0), (2, 0, 4, 192),
                                 (2, 0, 3, 256), (2, 0, 2, 0), (2, 0, 4, 0), (2, 0, 5, 0), (2, 0, 6, 0),
                                 (2, 0, 8, 0), (2, 1, 8, 0)):
        opts = B.vl_batch_opts()
        opts.persistent = mode
        opts.fold_engine = engine
        opts.rounds_variant = rv
        opts.rounds_threads = rt
        nb = B.vl_workspace_bytes(dj, opts)
        ws = _ws(nb)
        proofs = B.vl_prove_batch(dj, ws.data_ptr(), nb, opts=opts)
        assert [B.proof_bytes(p) for p in proofs] == refs


def test_wait_that_runs_out_reports_timeout_and_context_survives():
    """A prologue that never signals ready (host-injected): the proof's fold
    tiles give up after the bounded wait, the proof reports VL_ETIMEOUT, the
    other proofs are unaffected, and the next run on the context is clean."""
    jobs = _lora_jobs(n=24, d=64, k=64, r=8, layer=7, proj="v")
    dj, keep = _dev_jobs(jobs)
    refs = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jobs]
    bad = 3
    opts = B.vl_batch_opts()
    opts.persistent = 1  # the hook delays a prologue inside the persistent step
    opts.wait_limit_us = 20000
    opts.test_never_ready = bad + 1
    plan = B.vl_plan_create(dj, opts)
    try:
        nb = B.vl_plan_workspace_bytes(plan)
        ws = _ws(nb)
        out = (B.vl_proof * len(dj))()
        with pytest.raises(B.VLError) as e:
            B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
        assert e.value.code == B.VL_ETIMEOUT
        assert out[bad].status == B.VL_ETIMEOUT
        for i, (pf, ref) in enumerate(zip(out, refs)):
            if i != bad:
                assert pf.status == 0 and B.proof_bytes(pf) == ref
    finally:
        B.vl_plan_destroy(plan)
    nb2 = B.vl_workspace_bytes(dj)
    ws2 = _ws(nb2)
    proofs = B.vl_prove_batch(dj, ws2.data_ptr(), nb2)
    assert [B.proof_bytes(p) for p in proofs] == refs


TC_SHAPES = [
    # (m, k, n, transP, transQ): ragged lines and reductions, both fold modes,
    # one or two TMA boxes per column-sum stage, reductions over one segment
    (1, 8, 1, 0, 0),
    (70, 200, 33, 0, 0),
    (64, 128, 64, 1, 1),
    (130, 136, 72, 0, 1),
    (200, 64, 300, 1, 0),
    (3, 512, 5, 0, 0),
    (129, 8, 257, 1, 1),
    (16500, 16, 8, 0, 0),
    (8, 24, 17000, 0, 0),
]


@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tensor_core_fold_matches_oracle_and_cuda_core_fold(shape):
    m, k, n, tp, tq = shape
    rng = np.random.default_rng(1000 + m + 7 * k + 13 * n)
    P = _rand(rng, (k, m) if tp else (m, k))
    Q = _rand(rng, (n, k) if tq else (k, n))
    ref = oracle.prove_matmul(P, Q, tp, tq, seed=m * 31 + n).to_bytes()
    Pd, Qd = torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()
    jb = [B.job(Pd, Qd, tp, tq, m * 31 + n)]
    for engine in (0, 1):
        opts = B.vl_batch_opts()
        opts.fold_engine = engine
        plan = B.vl_plan_create(jb, opts)
        try:
            ltc = B.vl_plan_launches(plan)
            nb = B.vl_plan_workspace_bytes(plan)
            ws = _ws(nb)
            out = (B.vl_proof * 1)()
            B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
            assert B.proof_bytes(out[0]) == ref, f"engine {engine}"
        finally:
            B.vl_plan_destroy(plan)
        # both operands are TMA-addressable (ld a multiple of 8) only when so
        tc_ok = (P.shape[1] % 8 == 0) and (Q.shape[1] % 8 == 0)
        if engine == 0 and tc_ok:
            assert ltc == 4  # prologue (transcripts, eq tables), tensor-core fold, rounds


def test_tensor_core_fold_extreme_entries():
    """Entries at the int16 extremes: every byte of p = x + 2^15 at 0 or 255,
    the largest per-stage accumulator values."""
    m, k, n = 200, 136, 72
    for pv, qv in ((-(1 << 15), (1 << 15) - 1), ((1 << 15) - 1, (1 << 15) - 1), (-(1 << 15), -(1 << 15))):
        P = np.full((m, k), pv, np.int16)
        Q = np.full((k, n), qv, np.int16)
        Pd, Qd = torch.from_numpy(P).cuda(), torch.from_numpy(Q).cuda()
        opts = B.vl_batch_opts()
        jb = [B.job(Pd, Qd, 0, 0, 9), B.job(Qd, Pd, 1, 1, 10)]
        nb = B.vl_workspace_bytes(jb, opts)
        ws = _ws(nb)
        proofs = B.vl_prove_batch(jb, ws.data_ptr(), nb, opts=opts)
        assert B.proof_bytes(proofs[0]) == oracle.prove_matmul(P, Q, 0, 0, seed=9).to_bytes()
        assert B.proof_bytes(proofs[1]) == oracle.prove_matmul(Q, P, 1, 1, seed=10).to_bytes()


def test_autotuned_options_prove_the_same_and_are_cached():
    jobs = _lora_jobs(n=64, d=256, k=512, r=16, layer=8, proj="k")
    dj, keep = _dev_jobs(jobs)
    refs = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jobs]
    # room for the largest candidate plan plus the proofs
    need = max(B.vl_workspace_bytes(dj, o) for o in _opt_variants())
    nb = need + 64 * 1024
    ws = _ws(nb)
    B.vl_autotune_clear()
    best, ms = B.vl_autotune(dj, ws.data_ptr(), nb, runs=2)
    assert ms > 0
    again, ms2 = B.vl_autotune(dj, ws.data_ptr(), nb, runs=2)
    assert bytes(again) == bytes(best) and ms2 == ms  # cached
    nbb = B.vl_workspace_bytes(dj, best)
    ws2 = _ws(nbb)
    proofs = B.vl_prove_batch(dj, ws2.data_ptr(), nbb, opts=best)
    assert [B.proof_bytes(p) for p in proofs] == refs


def _opt_variants():
    out = []
    for eng, pers, seg in ((0, 2, 0), (1, 2, 0), (0, 1, 0), (0, 2, 2048)):
        o = B.vl_batch_opts()
        o.fold_engine, o.persistent, o.tc_seg = eng, pers, seg
        out.append(o)
    return out


def test_paper_backward_route_products():
    """The paper's backward route (full dW' = X^T.dY, then dA = dW'.B^T and
    dB = A^T.dW'), nine products of one projection, byte-equal to the oracle
    and verified by the library's host verifier against the claimed products."""
    t = W.lora_projection(W.GLOBAL_SEED, 3, "v", 48, 160, 96, 8)
    jobs, dWr = W.paper_route_products(t)
    assert [j["name"].rsplit(".", 1)[1] for j in jobs] == list(W.ROUTE_PRODUCTS)
    assert dWr.shape == (160, 96)
    dj, keep = _dev_jobs(jobs)
    nb = B.vl_workspace_bytes(dj)
    ws = _ws(nb)
    proofs = B.vl_prove_batch(dj, ws.data_ptr(), nb)
    for j, pf in zip(jobs, proofs):
        ref = oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
        assert B.proof_bytes(pf) == ref, j["name"]
        C = W.claimed_product(j)
        assert B.vl_verify_matmul(B.mat(j["P"], j["tp"]), B.mat(j["Q"], j["tq"]), B.mat(C), B.fs_init(j["seed"]), pf)


def test_host_operands_packed_in_one_buffer_are_staged_together():
    """Host operands laid out back to back in one pinned buffer are staged
    with one copy per run of neighbouring matrices; a matrix at a 2-byte
    offset (not 16-byte aligned) starts a run of its own.  The proofs equal
    those of the same jobs with device operands, through a plan run twice."""
    jobs = _lora_jobs(n=48, d=96, k=80, r=8, layer=9, proj="k")
    mats, seen = [], set()
    for j in jobs:
        for key in ("P", "Q"):
            if id(j[key]) not in seen:
                seen.add(id(j[key]))
                mats.append(j[key])
    offs, tot = [], 0
    for i, a in enumerate(mats):
        offs.append(tot + (2 if i == 3 else 0))  # one matrix off the 16-byte grid
        tot = offs[-1] + (a.nbytes + 255) // 256 * 256
    arena = torch.empty(tot + 256, dtype=torch.uint8, pin_memory=True)
    host = {}
    for a, o in zip(mats, offs):
        h = arena[o:o + a.nbytes].view(torch.int16).view(a.shape)
        h.copy_(torch.from_numpy(np.ascontiguousarray(a)))
        host[id(a)] = h
    hj = [B.job(host[id(j["P"])], host[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
    dj, keep = _dev_jobs(jobs)
    nd = B.vl_workspace_bytes(dj)
    want = [B.proof_bytes(p) for p in B.vl_prove_batch(dj, _ws(nd).data_ptr(), nd)]
    plan = B.vl_plan_create(hj)
    try:
        nb = B.vl_plan_workspace_bytes(plan)
        ws = _ws(nb)
        for _ in range(2):
            out = (B.vl_proof * len(hj))()
            B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
            assert [B.proof_bytes(p) for p in out] == want
    finally:
        B.vl_plan_destroy(plan)
    ref = oracle.prove_matmul(jobs[0]["P"], jobs[0]["Q"], jobs[0]["tp"], jobs[0]["tq"], seed=jobs[0]["seed"])
    assert want[0] == ref.to_bytes()


@pytest.mark.parametrize("d,k,n,fill", [(256, 384, 64, "random"), (128, 128, 8, "random"), (512, 1024, 96, "random"),
                                        (256, 256, 40, "max"), (384, 128, 16, "min")])
def test_dual_fold_of_a_matrix_folded_both_ways(d, k, n, fill):
    """A stored matrix W that one product folds as row dots (X.W) and another
    as column sums (dY.W^T), rows and columns multiples of 128: the dual
    tensor-core tiles stream it once for both.  Proofs equal the oracle's,
    and the same plan without dual tiles, byte for byte; the dual launch is
    counted."""
    rng = np.random.default_rng(d * 7 + k + n)
    if fill == "random":
        Wm = _rand(rng, (d, k))
    else:
        Wm = np.full((d, k), 32767 if fill == "max" else -32768, np.int16)
    X, dY = _rand(rng, (n, d)), _rand(rng, (n, k))
    jobs = [{"P": X, "Q": Wm, "tp": 0, "tq": 0, "seed": 71}, {"P": dY, "Q": Wm, "tp": 0, "tq": 1, "seed": 72},
            {"P": X, "Q": X, "tp": 1, "tq": 0, "seed": 73}]  # X^T.X: two row dots of X, no pair
    refs = [oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes() for j in jobs]
    dj, keep = _dev_jobs(jobs)
    launches = {}
    for fd in (1, 0):
        opts = B.vl_batch_opts()
        opts.fold_dual = fd
        plan = B.vl_plan_create(dj, opts)
        try:
            launches[fd] = B.vl_plan_launches(plan)
            nb = B.vl_plan_workspace_bytes(plan)
            ws = _ws(nb)
            for _ in range(2):
                out = (B.vl_proof * len(dj))()
                B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
                assert [B.proof_bytes(p) for p in out] == refs, f"fold_dual {fd}"
        finally:
            B.vl_plan_destroy(plan)
    assert launches[1] == launches[0] + 1  # the dual kernel


def test_host_operands_separated_by_an_unmapped_page():
    """Two pageable host operands one unmapped page apart (the end of one
    mapping and the start of another): each is staged with its own copy,
    never with one copy over the gap, and the proof equals the oracle's."""
    import mmap
    libc = ctypes.CDLL(None, use_errno=True)
    libc.mmap.restype = ctypes.c_void_p
    libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long]
    libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    pg = mmap.PAGESIZE
    m, k, n = 64, 128, 64
    pbytes, qbytes = m * k * 2, k * n * 2
    pp, qp = -(-pbytes // pg), -(-qbytes // pg)  # pages of each operand
    total = (pp + 1 + qp) * pg
    base = libc.mmap(None, total, mmap.PROT_READ | mmap.PROT_WRITE, mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS, -1, 0)
    assert base not in (None, ctypes.c_void_p(-1).value)
    try:
        assert libc.munmap(base + pp * pg, pg) == 0  # the hole
        p_addr = base + pp * pg - pbytes              # P ends where the hole begins
        q_addr = base + (pp + 1) * pg                 # Q starts where it ends
        P = np.ctypeslib.as_array((ctypes.c_int16 * (m * k)).from_address(p_addr)).reshape(m, k)
        Q = np.ctypeslib.as_array((ctypes.c_int16 * (k * n)).from_address(q_addr)).reshape(k, n)
        rng = np.random.default_rng(91)
        P[:] = _rand(rng, (m, k))
        Q[:] = _rand(rng, (k, n))
        ref = oracle.prove_matmul(P.copy(), Q.copy(), 0, 0, seed=92).to_bytes()
        hj = [B.job(P, Q, 0, 0, 92)]
        plan = B.vl_plan_create(hj)
        try:
            nb = B.vl_plan_workspace_bytes(plan)
            ws = _ws(nb)
            for _ in range(2):
                out = (B.vl_proof * 1)()
                B.vl_plan_run(plan, ws.data_ptr(), nb, out, B.VL_HOST)
                torch.cuda.synchronize()
                assert B.proof_bytes(out[0]) == ref
        finally:
            B.vl_plan_destroy(plan)
        del P, Q, hj
    finally:
        libc.munmap(base, pp * pg)
        libc.munmap(base + (pp + 1) * pg, qp * pg)
