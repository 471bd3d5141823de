"""Serving: continuous batching under a device-memory budget (vl_server_*).

Requests of mixed shapes are submitted together into an arena too small to
hold them all, so admission waits for memory to free up and several batches
share the device; every request's proofs must equal the proofs of the same
jobs proved alone (and the oracle's, for two of them), byte for byte.  A
request that arrives while another batch is on the device is admitted at
once into a batch of its own, and the two batches' device intervals (CUDA
events on their streams) overlap.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _request(n, d, k, r, layer, proj, host):
    """One projection's products; W (frozen) resident on the device, the rest
    on the device or in pinned host memory."""
    t = W.lora_projection(W.GLOBAL_SEED, layer, proj, n, d, k, r)
    jobs = W.projection_products(t)
    keep, cache = [], {}
    out = []
    for j in jobs:
        for key in ("P", "Q"):
            a = j[key]
            if id(a) in cache:
                continue
            x = torch.from_numpy(np.ascontiguousarray(a))
            if host and a is not t["W"]:
                h = torch.empty(x.shape, dtype=torch.int16, pin_memory=True)
                h.copy_(x)
                cache[id(a)] = h
            else:
                cache[id(a)] = x.cuda()
        out.append(B.job(cache[id(j["P"])], cache[id(j["Q"])], j["tp"], j["tq"], j["seed"]))
    keep.append(cache)
    return jobs, out, keep


def _wait_all(server, tickets, timeout_s=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for tk, st, batch, lat, dev in B.vl_server_poll(server):
            done[tk] = (st, batch, lat, dev)
        assert time.time() - t0 < timeout_s, "server did not finish"
        time.sleep(0.002)
    return done


def test_requests_in_the_mix_equal_alone():
    specs = [(64, 256, 256, 8, 0, "q", False), (32, 128, 192, 16, 1, "k", True),
             (96, 256, 128, 64, 2, "v", True), (16, 64, 64, 8, 3, "o", False),
             (64, 128, 256, 16, 4, "q", True), (48, 192, 192, 8, 5, "k", False)]
    reqs = [_request(*s) for s in specs]
    # reference: each request proved alone
    alone = []
    need = 0
    for jobs, dj, keep in reqs:
        nb = B.vl_workspace_bytes(dj)
        need = max(need, nb)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        alone.append([B.proof_bytes(p) for p in B.vl_prove_batch(dj, ws.data_ptr(), nb)])
    # arena: room for about two of the largest requests at once
    arena_bytes = 2 * need + (1 << 20)
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    server = B.vl_server_create(arena.data_ptr(), arena_bytes, max_inflight=3, max_batch_requests=2)
    try:
        outs, tickets = [], []
        for jobs, dj, keep in reqs:
            out = (B.vl_proof * len(dj))()
            outs.append(out)
            tickets.append(B.vl_server_submit(server, dj, out))
        done = _wait_all(server, tickets)
        stats = B.vl_server_stats_get(server)
    finally:
        B.vl_server_destroy(server)
    batches = set()
    for tk, out, ref in zip(tickets, outs, alone):
        st, batch, lat, dev = done[tk]
        assert st == 0 and lat > 0 and dev[1] > dev[0]
        batches.add(batch)
        assert [B.proof_bytes(p) for p in out] == ref
    assert len(batches) >= 2  # the arena forced more than one batch
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["proofs"] == sum(len(r[1]) for r in reqs)
    # two requests against the oracle as well
    for (jobs, dj, keep), out in list(zip(reqs, outs))[:2]:
        for j, pf in list(zip(jobs, out))[:3]:
            assert B.proof_bytes(pf) == oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()


def test_request_larger_than_the_arena_is_refused():
    jobs, dj, keep = _request(64, 256, 256, 8, 0, "q", False)
    small = [dj[2]]  # F3 = H.B, rank-sized
    big_need = B.vl_workspace_bytes(dj)
    small_need = B.vl_workspace_bytes(small)
    assert small_need * 2 < big_need
    # between the two: the small request fits with its proof outputs, the big one never does
    arena_bytes = (small_need + big_need) // 2
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    server = B.vl_server_create(arena.data_ptr(), arena_bytes)
    try:
        out = (B.vl_proof * len(dj))()
        tk = B.vl_server_submit(server, dj, out)
        done = _wait_all(server, [tk])
        assert done[tk][0] == B.VL_ENOMEM and done[tk][1] == -1
        # the server keeps serving requests that fit
        out2 = (B.vl_proof * 1)()
        tk2 = B.vl_server_submit(server, small, out2)
        assert _wait_all(server, [tk2])[tk2][0] == 0
        ref = B.vl_prove_batch(small, torch.empty(small_need, dtype=torch.uint8, device="cuda").data_ptr(),
                               small_need)[0]
        assert B.proof_bytes(out2[0]) == B.proof_bytes(ref)
    finally:
        B.vl_server_destroy(server)


def test_request_arriving_while_a_batch_runs_overlaps_it():
    """Continuous batching: request B arrives only after request A's batch
    is on the device; B is admitted into a batch of its own on another
    stream at once (not after A), the two batches' device intervals overlap,
    and B's proofs equal B's proofs alone (and the oracle's)."""
    projs = W.make_step("7b", layers=range(16))  # A: 512 products, about 2 ms on the device
    dev = {}
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    a_jobs = [B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"], j["seed"])
              for t in projs for j in W.projection_products(t)]
    b_src, b_jobs, keep = _request(64, 256, 256, 16, 40, "v", True)
    nb = B.vl_workspace_bytes(b_jobs)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b_alone = [B.proof_bytes(p) for p in B.vl_prove_batch(b_jobs, ws.data_ptr(), nb)]
    need = B.vl_workspace_bytes(a_jobs) + nb + (64 << 20)
    arena = torch.empty(need, dtype=torch.uint8, device="cuda")
    server = B.vl_server_create(arena.data_ptr(), need, max_inflight=2, max_batch_requests=4)
    try:
        out_a = (B.vl_proof * len(a_jobs))()
        ta = B.vl_server_submit(server, a_jobs, out_a)
        t0 = time.time()
        while B.vl_server_stats_get(server)["launched"] < 1:  # A's batch is on the device
            assert time.time() - t0 < 60
            time.sleep(0.0002)
        out_b = (B.vl_proof * len(b_jobs))()
        tb = B.vl_server_submit(server, b_jobs, out_b)
        done = _wait_all(server, [ta, tb])
    finally:
        B.vl_server_destroy(server)
    (sa, ba, _, da), (sb, bb, _, db) = done[ta], done[tb]
    assert sa == 0 and sb == 0 and ba != bb
    assert db[0] < da[1], f"B's batch started at {db[0]:.3f} ms, after A's ended at {da[1]:.3f} ms"
    assert da[0] < db[1]
    assert [B.proof_bytes(p) for p in out_b] == b_alone
    for j, pf in list(zip(b_src, out_b))[:2]:
        assert B.proof_bytes(pf) == oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
    # A, spot-checked against the oracle
    j0 = [j for t in projs[:1] for j in W.projection_products(t)]
    for j, pf in list(zip(j0, out_a))[:2]:
        assert B.proof_bytes(pf) == oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
