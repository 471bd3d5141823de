#!/usr/bin/env python3
"""Benchmark: matmul-sumcheck proofs of a LoRA fine-tuning step on GB300.

Metric: matmul MACs proved per second (sum over the step's products of
m.k.n, divided by wall time), and ms per LoRA-step proof, batched (one plan,
CUDA-graph replay of the whole step) against the unbatched per-matmul path.
Every proof is bit-exact with the oracle (tests/test_gpu_parity.py,
tests/test_gpu_parity_fullsize.py).

Default workload: the 7B-shaped step -- 32 layers x {q,k,v,o}, hidden 4096,
sequence 512, LoRA rank per layer from {8, 16, 64}; eight products per
projection (1024 proofs).  Synthetic int16 fixed-point tensors (the paper's
LLaMA weights and C4 data are not available).  Inputs (~5.4 GB) are far
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank proves its own full step (independent proofs, no
collective: weak scaling); rank 0 prints one JSON line.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2508_21393_gb300 import workload as W  # noqa: E402

METRIC = "matmul MACs proved/sec and ms per LoRA step proof (batched vs unbatched), bit-exact"
UNIT = "MAC/s"
SMS = 152
SM_MAX_MHZ = 2070.0
# IMAD.WIDE.U32 (32x32->64 multiply-add) issue rate per SM per clock used for
# the ALU roofline of the int16 fold: 64 32-bit integer multiply-adds per SM
# per clock, a wide (64-bit result) one taking two of them.
MADWIDE_PER_SM_CLK = 32
STEP_KIND = {"7b-step": "7b", "7b-proj": "7b-proj", "13b-step": "13b", "serve": "7b-proj", "7b-update": "7b",
             "7b-step-paper-route": "7b", "7b-lookups": "7b", "7b-step-batched": "7b", "7b-step-all": "7b",
             "7b-step-chain": "7b"}
WORKLOADS = {
    "7b-step": "batched 7B-shaped LoRA step: 32 layers x {q,k,v,o}, hidden 4096, seq 512, ranks {8,16,64}",
    "7b-proj": "one 7B-shaped LoRA projection, n=1024, d=k=4096, r=16, eight products",
    "13b-step": "batched 13B-shaped LoRA step: 40 layers x {q,k,v,o}, hidden 5120, seq 2048, rank 16",
    "7b-step-paper-route": "batched 7B-shaped LoRA step along the paper's backward route (Eq. eq:grad_wl, "
                           "eq:grad_abl: full dW' = X^T.dY, then dA = dW'.B^T, dB = A^T.dW'), nine products per "
                           "projection, 32 layers x {q,k,v,o}, hidden 4096, seq 512, ranks {8,16,64}",
    "7b-lookups": "range lookups of the 7B-shaped LoRA step's rescale remainders (Protocol 1, Eq. "
                  "eq:lookup-sumcheck): 32 layers x {q,k,v,o} x {H, dH (512 x r, table 2^8), G_A (4096 x r), "
                  "G_B (r x 4096) (table 2^12)}, ranks {8,16,64}, one batched plan run",
    "7b-step-batched": "the batched 7B-shaped LoRA step's 1024 products as 5 batched-claim proofs (one per inner "
                       "dimension: 4096, 512, and the ranks 8, 16, 64), one transcript and one sumcheck each",
    "7b-step-all": "the built hot path of one 7B-shaped LoRA step: the 1024 matmul proofs (one plan, graph), the "
                   "256 parameter-update proofs and the 512 rescale-remainder range lookups, each plan on its own "
                   "stream",
    "7b-update": "parameter updates of the 7B-shaped LoRA step (Eq. eq:grad_update_ab): 32 layers x {q,k,v,o} x "
                 "{A' = A - G_A (4096 x r), B' = B - G_B (r x 4096)}, ranks {8,16,64}, linear zkMat, one batched call",
    "7b-step-chain": "the 7B-shaped LoRA step as 128 chained projection proofs (Sec. IV sequential composition): per "
                     "projection ten matmul sumchecks under one transcript, the claims on H and dH reduced through "
                     "the rescale relations to X.A and dY.B^T (proved at two points each) instead of being opened; "
                     "32 layers x {q,k,v,o}, hidden 4096, seq 512, ranks {8,16,64}",
    "serve": "serving stream: Poisson arrivals (20 jobs/s) of single-layer jobs (one projection's 8 products), "
             "hidden {4096, 5120}, seq {256, 512, 1024, 2048}, rank {8, 16, 64}, 120 GB admission budget",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="7b-step", choices=sorted(WORKLOADS))
    ap.add_argument("--no-unbatched", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-projections", type=int, default=2)
    ap.add_argument("--persistent", action="store_true",
                    help="one persistent launch per step (CUDA-core fold) instead of phase launches")
    ap.add_argument("--fold-engine", type=int, default=0, choices=[0, 1],
                    help="phase launches: 0 tensor-core fold where TMA can address the operand, 1 CUDA cores only")
    ap.add_argument("--groups", type=int, default=0,
                    help="phase launches: proof groups pipelined over three streams (0: library default)")
    ap.add_argument("--rounds-variant", type=int, default=0, choices=[0, 2, 3, 4, 5, 6, 7, 8],
                    help="rounds kernel register budget (CTAs per SM), or 8: batched rounds; 0 = library default")
    ap.add_argument("--fold-dual", action="store_true",
                    help="fold a matrix used as row dots and as column sums in one pass (dual tiles)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (it also stays off when launch or tile options are given)")
    ap.add_argument("--serve-jobs", type=int, default=200, help="serve workload: requests in the timed stream")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="serve workload: mean arrivals per second")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="serve workload: arena (admission budget)")
    ap.add_argument("--layers", type=int, default=0,
                    help="prove only the first L layers of the step (profiling captures); 0 = all")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_seed(rank):
    """Seed of rank `rank`'s replica: each rank proves its own step (weak scaling)."""
    return W.GLOBAL_SEED + 1000003 * rank


def max_over_ranks(x, world, device):
    """Maximum of a per-rank float over the process group (the job takes as
    long as its slowest rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, seconds_max):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def products(kind, t, seed):
    if kind == "7b-step-paper-route":
        jobs, dWr = W.paper_route_products(t, seed)
        t["dWr"] = dWr
        return jobs
    return W.projection_products(t, seed)


def step_jobs(kind, seed, layers=0):
    projs = W.make_step(STEP_KIND[kind], seed, layers=range(layers) if layers > 0 else None)
    jobs = [j for t in projs for j in products(kind, t, seed)]
    return projs, jobs


def _oracle_prove(kind, seed, jobs):
    import oracle
    if kind == "7b-step-batched":  # one batched proof per inner dimension
        groups = {}
        for j in jobs:
            groups.setdefault(W.op_shape(j)[1], []).append(j)
        for k, g in groups.items():
            oracle.prove_matmul_batch(g, seed=seed + k)
    else:
        for j in jobs:
            oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"])


def _oracle_projection_task(task):
    """Worker: regenerate one projection (untimed), then prove its products
    with the oracle; returns (seconds proving, MACs, proofs)."""
    kind, seed, spec = task
    t = W.lora_projection(seed, *spec)
    if kind == "7b-step-chain":
        import oracle
        t = W.chain_tensors(t)
        jobs = chain_products(t, seed)
        t0 = time.perf_counter()
        oracle.prove_chain(t, seed=W.proof_seed(seed, t["layer"], t["proj"], "chain"))
        return time.perf_counter() - t0, sum(W.macs(j) for j in jobs), len(jobs)
    jobs = products(kind, t, seed)
    t0 = time.perf_counter()
    _oracle_prove(kind, seed, jobs)
    return time.perf_counter() - t0, sum(W.macs(j) for j in jobs), len(jobs)


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / (1 << 20)
    except OSError:
        pass
    return None


class OracleCores:
    """The oracle over the host's cores: one worker process per core
    ('spawn' start: no CUDA state is inherited), each proving whole
    projections.  A sample proves one projection per worker at once; its
    time is the slowest worker's proving time (each worker regenerates its
    projection from the seeded recipe first, outside the timed part)."""

    def __init__(self, kind, procs=None):
        import multiprocessing as mp
        self.kind = kind
        spec_n = len(W.step_layers(STEP_KIND[kind], W.GLOBAL_SEED))
        n = procs or (os.cpu_count() or 1)
        gb = _mem_available_gb()
        per = 3.0 if kind == "13b-step" else 1.5  # oracle working set of one projection, GB
        if gb is not None:
            n = min(n, max(1, int(gb / 2 / per)))
        self.procs = max(1, min(n, spec_n))
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def sample(self, seed, first=0):
        """(seconds, MACs, proofs) of one projection per worker, projections
        first .. first + procs - 1 of the workload (wrapping around)."""
        specs = W.step_layers(STEP_KIND[self.kind], seed)
        tasks = [(self.kind, seed, specs[(first + i) % len(specs)]) for i in range(self.procs)]
        res = self.pool.map(_oracle_projection_task, tasks, chunksize=1)
        return max(r[0] for r in res), sum(r[1] for r in res), sum(r[2] for r in res)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def oracle_cores_baseline(kind, seed):
    """cpu_baseline of a matmul workload: the oracle on every host core."""
    oc = OracleCores(kind)
    try:
        dt, macs, nj = oc.sample(seed)
    finally:
        oc.close()
    return {"value": macs / dt, "unit": UNIT, "cores": oc.procs, "kind": "oracle",
            "sample": f"first {oc.procs} projections of the same workload, one per worker process "
                      f"({nj} proofs, {macs} MACs), proved at once on {oc.procs} cores in {dt:.1f} s "
                      f"(the slowest worker's proving time)"}


# Rounds of one matmul proof with d1 variables: round 1 evaluates g(0), g(1),
# g(2) on 2^(d1-1) pairs (three field products each); every later round t
# folds four values and evaluates three products on 2^(d1-t) pairs; the last
# fold is two products.
def rounds_products(d1):
    if d1 == 0:
        return 1
    return 3 * (1 << (d1 - 1)) + 7 * ((1 << (d1 - 1)) - 1) + 2


# One round's transcript step on the GPU (absorb g(0) || g(2): two SHA-256
# compressions; squeeze r: one more; the 512-bit reduction): a serial chain
# of 12.3 K cycles for one warp alone (clock64 over 200 dependent steps on the
# box, at 2.07 GHz 5.9 us).  The derived field-product peak: 152 SMs x 32
# IMAD.WIDE per clock x 2.07 GHz / 128 IMAD.WIDE per Montgomery product.
ROUND_HASH_CYCLES = 12300
PRODUCTS_PEAK = SMS * MADWIDE_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 128


def rounds_bound(jobs, rounds_ms):
    """Bounds of the claims-and-rounds phase: the field products of every
    proof's rounds against the derived product peak (throughput), and the
    longest proof's serial chain of transcript steps (latency)."""
    d1s = [(W.op_shape(j)[1] - 1).bit_length() for j in jobs]
    prods = sum(rounds_products(d) for d in d1s)
    thr_us = prods / PRODUCTS_PEAK * 1e6
    lat_us = max(d1s) * ROUND_HASH_CYCLES / (SM_MAX_MHZ * 1e6) * 1e6
    bound_us = max(thr_us, lat_us)
    return {"field_products": prods, "throughput_bound_us": thr_us, "latency_bound_us": lat_us,
            "bound_us": bound_us, "measured_us": 1e3 * rounds_ms, "frac": bound_us / (1e3 * rounds_ms),
            "note": "products at the derived ALU peak (152 SMs x 32 IMAD.WIDE/clk x 2070 MHz / 128 per product); "
                    "latency = max d1 x 12.3 K-cycle transcript step (measured single-warp chain)"}


def pinned_h2d_gbs(stream, nbytes=1 << 30, reps=3):
    """Plain host-to-device copy rate of this machine: one cudaMemcpyAsync of a
    pinned 1 GiB buffer, best of `reps`, timed with CUDA events."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h.fill_(1)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.copy_(h, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del d, h
    return nbytes / (best / 1e3) / 1e9


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def run_reference(args, rank, world):
    """The oracle (pure-Python CPU prover), timed on this host, as the reference arm."""
    if rank != 0:
        return
    cores = 1
    if args.workload == "7b-lookups":
        per_step = []
        for _ in range(args.warmup):
            oracle_lookup_sample(W.GLOBAL_SEED, 1)
        for _ in range(args.steps):
            rate, dt, nj, ent = oracle_lookup_sample(W.GLOBAL_SEED, 1)
            per_step.append(dt)
        total = sum(per_step)
        value = ent * args.steps / total
        sample = f"the two n x r remainder lookups of the first projection ({nj} proofs, {ent} entries) per step"
        print(json.dumps({
            "impl": "reference", "metric": LK_METRIC, "value": value, "unit": LK_UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (Fr, 255-bit)",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
            "cpu_baseline": {"value": value, "unit": LK_UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": LK_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    if args.workload == "7b-update":
        nproj = 8
        per_step = []
        for _ in range(args.warmup):
            oracle_update_sample(W.GLOBAL_SEED, nproj)
        for _ in range(args.steps):
            rate, dt, nj, ent = oracle_update_sample(W.GLOBAL_SEED, nproj)
            per_step.append(dt)
        total = sum(per_step)
        value = ent * args.steps / total
        sample = f"update relations of the first {nproj} projections ({nj} proofs, {ent} entries) per step"
        print(json.dumps({
            "impl": "reference", "metric": LIN_METRIC, "value": value, "unit": LIN_UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (Fr, 255-bit)",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
            "cpu_baseline": {"value": value, "unit": LIN_UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": LIN_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    # every host core proves one projection per step (worker processes)
    oc = OracleCores(args.workload)
    cores = oc.procs
    try:
        specs_n = len(W.step_layers(STEP_KIND[args.workload], W.GLOBAL_SEED))
        for i in range(args.warmup):
            oc.sample(W.GLOBAL_SEED, first=(i * cores) % specs_n)
        per_step, macs_total, nj = [], 0, 0
        for i in range(args.steps):
            dt, macs, nj = oc.sample(W.GLOBAL_SEED, first=((args.warmup + i) * cores) % specs_n)
            per_step.append(dt)
            macs_total += macs
    finally:
        oc.close()
    total = sum(per_step)
    value = macs_total / total
    sample = (f"{cores} projections per step ({nj} proofs), one per worker process on {cores} cores, "
              f"cycling through the {args.workload} workload's projections; a step's time is the slowest "
              f"worker's proving time")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int (Fr, 255-bit)",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def serve_main(args, rank, world, local):
    """Serving stream through vl_server_*: Poisson arrivals, continuous batching
    under the admission budget; frozen W resident on the device, activations
    copied from pinned host memory per request.  Reports proofs/s and p50/p99
    submit-to-completion latency."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    B.lib()
    arrivals = W.serving_jobs(args.serve_jobs, W.GLOBAL_SEED + rank, rate=args.serve_rate)
    shapes = sorted({sh for _, sh in arrivals})
    pool = {}
    for i, (h, n, r) in enumerate(shapes):  # job pool: generated before timing
        t = W.lora_projection(W.GLOBAL_SEED, 100 + i, "q", n, h, h, r)
        jobs = W.projection_products(t, W.GLOBAL_SEED)
        hold = {}
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            x = torch.from_numpy(np.ascontiguousarray(t[key]))
            if key == "W":
                hold[key] = x.cuda()  # frozen weight: resident
            else:
                hp = torch.empty(x.shape, dtype=torch.int16, pin_memory=True)
                hp.copy_(x)
                hold[key] = hp
        by_id = {id(t[k]): hold[k] for k in hold}
        vj = [B.job(by_id[id(j["P"])], by_id[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
        h2d = sum(v.numel() * 2 for k, v in hold.items() if k != "W")
        pool[(h, n, r)] = (vj, sum(W.macs(j) for j in jobs), h2d, hold)
    budget = int(args.serve_budget_gb * (1 << 30))
    arena = torch.empty(budget, dtype=torch.uint8, device="cuda")
    server = B.vl_server_create(arena.data_ptr(), budget)

    def submit(vj, seed):
        jobs = []
        for j in vj:
            c = B.vl_job.from_buffer_copy(j)
            c.fs.seed = seed
            jobs.append(c)
        out = (B.vl_proof * len(jobs))()
        return B.vl_server_submit(server, jobs, out), out

    done = {}
    # warm-up: one request of each shape (plan building, attribute setup)
    warm_outs = [submit(pool[sh][0], 7 + i) for i, sh in enumerate(shapes)]  # outputs live until done
    warm = [tk for tk, _ in warm_outs]
    while len(done) < len(warm):
        for tk, st, b, lat, _ in B.vl_server_poll(server):
            done[tk] = (st, b, lat)
        time.sleep(0.001)
    torch.cuda.synchronize()
    done.clear()
    clocks = Clocks(local)
    time.sleep(0.6)
    sub = {}
    outs = []
    t0 = time.perf_counter()
    for i, (ta, sh) in enumerate(arrivals):
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
            for tk, st, b, lat, _ in B.vl_server_poll(server):
                done[tk] = (st, b, lat, time.perf_counter() - t0)
            time.sleep(min(0.0005, ta - now))
        tk, out = submit(pool[sh][0], 1000003 * (i + 1))
        sub[tk] = (time.perf_counter() - t0, sh)
        outs.append(out)
    while len(done) < len(sub):
        for tk, st, b, lat, _ in B.vl_server_poll(server):
            done[tk] = (st, b, lat, time.perf_counter() - t0)
        time.sleep(0.0005)
    clk = clocks.stop()
    stats = B.vl_server_stats_get(server)
    B.vl_server_destroy(server)
    lat = sorted(v[2] for v in done.values())
    assert all(v[0] == 0 for v in done.values()), "a request failed"
    end = max(sub[tk][0] + done[tk][2] / 1e3 for tk in sub)
    nproofs = sum(len(pool[sh][0]) for _, sh in sub.values())
    macs = sum(pool[sh][1] for _, sh in sub.values())
    h2d = sum(pool[sh][2] for _, sh in sub.values())
    pct = lambda q: float(np.percentile(lat, q))
    if rank != 0:
        return
    line = {
        "metric": "serving: proofs/s with p50/p99 proof latency (continuous batching, bit-exact)",
        "value": nproofs / end, "unit": "proofs/s", "n_gpus": world, "steps": len(sub), "warmup": len(warm),
        "ms_per_step": 1e3 * end / len(sub), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["serve"].replace("(20 jobs/s)", f"({args.serve_rate:g} jobs/s)"),
                   "requests": len(sub), "proofs": nproofs,
                   "distinct_shapes": len(shapes), "admission_budget_gb": args.serve_budget_gb,
                   "batches": stats["batches"], "l2": "inputs larger than L2 (no flush)"},
        "latency_ms": {"p50": pct(50), "p99": pct(99), "mean": float(np.mean(lat)), "max": lat[-1]},
        "macs_per_s": macs / end,
        "roofline": None,
        "cpu_baseline": None,
        "e2e": {"value": nproofs / end, "unit": "proofs/s", "h2d_bytes_per_step": h2d // len(sub),
                "d2h_bytes_per_step": int(ctypes.sizeof(B.vl_proof) * nproofs // len(sub))},
        "clocks": clk,
        "gpu_launches": None,
    }
    print(json.dumps(line))


LIN_METRIC = "linear-relation matrix entries proved/sec (parameter-update proofs of a LoRA step), bit-exact"
LIN_UNIT = "entries/s"


def update_statements(seed, layers=0, nproj=None):
    spec = W.step_layers("7b", seed)
    if layers > 0:
        spec = [s for s in spec if s[0] < layers]
    if nproj is not None:
        spec = spec[:nproj]
    stmts = []
    for s in spec:
        stmts += W.update_statements(W.lora_projection(seed, *s), seed)
    return stmts


def oracle_update_sample(seed, nproj):
    """Time the oracle on the update relations of the first `nproj` projections."""
    import oracle
    stmts = update_statements(seed, nproj=nproj)
    entries = sum(m.size for st in stmts for m in st["mats"])
    t0 = time.perf_counter()
    for st in stmts:
        oracle.prove_linear(list(st["mats"]), list(st["coeffs"]), seed=st["seed"])
    dt = time.perf_counter() - t0
    return entries / dt, dt, len(stmts), entries


def update_main(args, rank, world, local, cpu):
    """Parameter-update proofs of the 7B step: 256 linear relations (three
    int16 matrices each) proved by one plan run (five launches) per step."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    stmts = update_statements(rank_seed(rank), args.layers)
    entries = sum(m.size for st in stmts for m in st["mats"])
    dev = [[torch.from_numpy(m).cuda() for m in st["mats"]] for st in stmts]
    jobs = [B.lin_job([B.mat(t) for t in d], list(st["coeffs"]), st["seed"]) for d, st in zip(dev, stmts)]
    plan = B.LinPlan(jobs)
    n = plan.workspace_bytes()
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    dout = torch.empty(len(jobs) * ctypes.sizeof(B.vl_lin_proof), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):  # the first run binds the plan to the workspace
        plan.run(ws.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE, stream)
    torch.cuda.synchronize()
    raw = dout.cpu().numpy().tobytes()
    out = [B.vl_lin_proof.from_buffer_copy(raw, i * ctypes.sizeof(B.vl_lin_proof)) for i in range(len(jobs))]
    assert all(p.status == 0 for p in out)
    # every warm-up proof verifies in the library's host verifier (not timed)
    hj = [B.lin_job([B.mat(m) for m in st["mats"]], list(st["coeffs"]), st["seed"]) for st in stmts]
    assert all(B.vl_verify_linear(j, p) for j, p in zip(hj, out))
    # a buffer larger than L2 written between steps: the operands (~0.2 GB) would otherwise stay in L2
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)
    total_ms, phases = 0.0, []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(ws.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        phases.append(plan.phase_ms())
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = total_ms / args.steps
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(entries, world, ms_max / 1e3)
    fold_ms = statistics.mean(p[1] for p in phases)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak, hbm_note = (peaks["hbm_gbs"], "measured") if "hbm_gbs" in peaks else (6800.0, "fallback")
    hbm_gbs = 2 * entries / (fold_ms / 1e3) / 1e9
    # The LoRA factors reduce over the rank (at most 64 entries): the fold runs
    # on CUDA cores (lin_short_kernel), one thread per line: eight 32 x 32 ->
    # 64-bit multiply-adds per entry and one REDC (64 more) per line.  Bound:
    # those multiply-adds at the derived ALU peak; the 2 B per entry of HBM
    # traffic would take a fifth of that time.
    lines = sum(len(st["mats"]) * max(st["mats"][0].shape) for st in stmts)
    madw = 8 * entries + 64 * lines
    alu_peak = SMS * MADWIDE_PER_SM_CLK * SM_MAX_MHZ * 1e6
    roof = {"bound": "alu", "kernel": "lin_short_kernel", "achieved": madw / (fold_ms / 1e3) / 1e12,
            "peak": alu_peak / 1e12, "unit": "T mad.wide/s", "frac": madw / (fold_ms / 1e3) / alu_peak,
            "traffic": None,
            "peak_note": f"derived: {SMS} SMs x {MADWIDE_PER_SM_CLK} IMAD.WIDE/clk x {SM_MAX_MHZ} MHz",
            "algorithmic_madwide_per_launch": madw,
            "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                    "algorithmic_bytes_per_launch": 2 * entries,
                    "peak_note": f"{hbm_note} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}
    # End to end: pinned host operands in (staged by the library), host proofs out.
    host = [[torch.from_numpy(m).pin_memory() for m in st["mats"]] for st in stmts]
    hjobs = [B.lin_job([B.mat(t) for t in h], list(st["coeffs"]), st["seed"]) for h, st in zip(host, stmts)]
    hplan = B.LinPlan(hjobs)
    hn = hplan.workspace_bytes()
    plan.destroy()
    del ws
    hws = torch.empty(hn, dtype=torch.uint8, device="cuda")
    hplan.run(hws.data_ptr(), hn, stream=stream)
    ksteps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(ksteps):
        hplan.run(hws.data_ptr(), hn, stream=stream)  # operands copied in, proofs read back, every run
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ksteps, world, "cuda")
    hplan.destroy()
    e2e = {"value": job_value(entries, world, e2e_s), "unit": LIN_UNIT,
           "h2d_bytes_per_step": int(2 * entries), "d2h_bytes_per_step": int(ctypes.sizeof(B.vl_lin_proof) * len(jobs)),
           "ms_per_step": 1e3 * e2e_s, "steps": ksteps}
    if rank != 0:
        return
    print(json.dumps({
        "metric": LIN_METRIC, "value": value, "unit": LIN_UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["7b-update"] + (f", first {args.layers} layers" if args.layers else ""),
                   "proofs_per_step": len(jobs), "matrices_per_step": 3 * len(jobs), "entries_per_step": entries,
                   "l2": "256 MB buffer written between steps (operands smaller than L2)",
                   "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                   "phase_ms": {"start+eq": statistics.mean(p[0] for p in phases), "fold": fold_ms,
                                "dots+proofs": statistics.mean(p[2] for p in phases)}},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": 5 * args.steps,
    }))


LK_METRIC = "lookup-argument entries proved/sec (range checks of a LoRA step's rescale remainders), bit-exact"
LK_UNIT = "entries/s"
# Montgomery products per second the SMs can issue: 152 SMs x 32 IMAD.WIDE
# per clock x 2070 MHz, 128 IMAD.WIDE per 8-limb Montgomery product (64 for
# the product, 64 for the reduction).
MONT_PEAK = SMS * MADWIDE_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 128


def lookup_statements(seed, layers=0, nproj=None):
    spec = W.step_layers("7b", seed)
    if layers > 0:
        spec = [s for s in spec if s[0] < layers]
    if nproj is not None:
        spec = spec[:nproj]
    looks = []
    for s in spec:
        looks += W.rescale_lookups(W.lora_projection(seed, *s), seed)
    return looks


def lookup_cube(x):
    n = int(x["S"].size)
    return 1 << max(x["log2_n"], (n - 1).bit_length())


def oracle_lookup_sample(seed, nproj):
    """Time the oracle on the two n x r remainder lookups of the first `nproj` projections."""
    import oracle
    looks = [x for x in lookup_statements(seed, nproj=nproj) if x["log2_n"] == W.RESCALE_SHIFT]
    entries = sum(int(x["S"].size) for x in looks)
    t0 = time.perf_counter()
    for x in looks:
        oracle.prove_lookup(x["S"], x["t0"], x["log2_n"], seed=x["seed"])
    dt = time.perf_counter() - t0
    return entries / dt, dt, len(looks), entries


def lookups_main(args, rank, world, local, cpu):
    """Range lookups of the 7B step's rescale remainders: 512 proofs per
    step, one plan run (setup, three launches per round, finish)."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    looks = lookup_statements(rank_seed(rank), args.layers)
    entries = sum(int(x["S"].size) for x in looks)
    cube = sum(lookup_cube(x) for x in looks)
    dev = [torch.from_numpy(np.ascontiguousarray(x["S"])).cuda() for x in looks]
    jobs = [B.lookup_job(B.mat(d), x["t0"], x["log2_n"], x["seed"]) for d, x in zip(dev, looks)]
    plan = B.LookupPlan(jobs)
    n = plan.workspace_bytes()
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    sz = ctypes.sizeof(B.vl_lookup_proof)
    dout = torch.empty(len(jobs) * sz, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        plan.run(ws.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE, stream)
    torch.cuda.synchronize()
    raw = dout.cpu().numpy().tobytes()
    out = [B.vl_lookup_proof.from_buffer_copy(raw, i * sz) for i in range(len(jobs))]
    assert all(p.status == 0 for p in out)
    # a sample of the warm-up proofs verifies in the library's host verifier (not timed)
    for i in range(0, len(looks), max(1, len(looks) // 16)):
        hj = B.lookup_job(B.mat(np.ascontiguousarray(looks[i]["S"])), looks[i]["t0"], looks[i]["log2_n"],
                          looks[i]["seed"])
        assert B.vl_verify_lookup(hj, out[i])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)
    total_ms, phases = 0.0, []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(ws.data_ptr(), n, dout.data_ptr(), B.VL_DEVICE, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        phases.append(plan.phase_ms())
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = total_ms / args.steps
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(entries, world, ms_max / 1e3)
    # the sumcheck rounds: batched passes plus each proof's tail rounds
    rounds_ms = statistics.mean(p[1] + p[2] for p in phases)
    # algorithmic field products of the rounds: per round and pair, 3 folds +
    # 3 evaluation points x 2 products (9 per pair; sum over rounds 9 D), plus
    # the eq(u, .) entry (1 per cube entry): 10 per cube entry
    achieved = 10 * cube / (rounds_ms / 1e3)
    roof = {"bound": "alu", "kernel": "lk_pass_kernel + lk_round_kernel + lk_tail_kernel (all rounds)",
            "achieved": achieved / 1e9,
            "peak": MONT_PEAK / 1e9, "unit": "G Montgomery products/s", "frac": achieved / MONT_PEAK,
            "traffic": None, "peak_note": "derived: 152 SMs x 32 IMAD.WIDE/clk x 2070 MHz / 128 per product",
            "algorithmic_products_per_step": 10 * cube}
    host = [torch.from_numpy(np.ascontiguousarray(x["S"])).pin_memory() for x in looks]
    hjobs = [B.lookup_job(B.mat(h), x["t0"], x["log2_n"], x["seed"]) for h, x in zip(host, looks)]
    hplan = B.LookupPlan(hjobs)
    hn = hplan.workspace_bytes()
    plan.destroy()
    del ws
    hws = torch.empty(hn, dtype=torch.uint8, device="cuda")
    hplan.run(hws.data_ptr(), hn, stream=stream)
    ksteps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(ksteps):
        hplan.run(hws.data_ptr(), hn, stream=stream)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ksteps, world, "cuda")
    hplan.destroy()
    e2e = {"value": job_value(entries, world, e2e_s), "unit": LK_UNIT, "h2d_bytes_per_step": int(2 * entries),
           "d2h_bytes_per_step": int(sz * len(jobs)), "ms_per_step": 1e3 * e2e_s, "steps": ksteps}
    max_l = max((lookup_cube(x) - 1).bit_length() for x in looks)
    if rank != 0:
        return
    print(json.dumps({
        "metric": LK_METRIC, "value": value, "unit": LK_UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 values, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["7b-lookups"] + (f", first {args.layers} layers" if args.layers else ""),
                   "proofs_per_step": len(jobs), "entries_per_step": entries, "cube_entries_per_step": cube,
                   "l2": "256 MB buffer written between steps",
                   "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                   "phase_ms": {"setup": statistics.mean(p[0] for p in phases),
                                "batched rounds": statistics.mean(p[1] for p in phases),
                                "tail rounds + proofs": statistics.mean(p[2] for p in phases)}},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": (5 + 3 * max_l) * args.steps,
    }))


def batched_main(args, rank, world, local, cpu=None):
    """The 7B step's products grouped by inner dimension, each group one
    batched-claim proof (a vl_claims_plan per group, replayed every step)."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    seed = rank_seed(rank)
    projs, jobs = step_jobs("7b-step", seed, args.layers)
    macs_step = sum(W.macs(j) for j in jobs)
    dev = {}
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    groups = {}
    for j in jobs:
        groups.setdefault(W.op_shape(j)[1], []).append(B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"],
                                                             j["seed"]))
    keys = sorted(groups)
    plans = {k: B.ClaimsPlan(groups[k], seed + k) for k in keys}
    sizes = {k: plans[k].workspace_bytes() for k in keys}
    # one workspace per batch (plans stay bound), proofs and values on the device
    wss = {k: torch.empty(sizes[k], dtype=torch.uint8, device="cuda") for k in keys}
    outs = {k: (torch.empty(ctypes.sizeof(B.vl_batch_proof), dtype=torch.uint8, device="cuda"),
                torch.empty(3 * 32 * len(groups[k]), dtype=torch.uint8, device="cuda")) for k in keys}
    stream = torch.cuda.current_stream()

    def dev_out(k):
        pr, vals = outs[k]
        base, K = vals.data_ptr(), len(groups[k])
        return (pr.data_ptr(), base, base + 32 * K, base + 64 * K)

    # each batch on its own stream: one batch's latency-bound rounds overlap
    # another's fold; the step forks from and joins the timing stream
    streams = {k: torch.cuda.Stream() for k in keys}
    fork = torch.cuda.Event()
    joins = {k: torch.cuda.Event() for k in keys}

    def step():
        fork.record(stream)
        for k in keys:
            streams[k].wait_event(fork)
            plans[k].run(wss[k].data_ptr(), sizes[k], streams[k], device_out=dev_out(k))
            joins[k].record(streams[k])
        for k in keys:
            stream.wait_event(joins[k])

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    for k in keys:  # statuses of the warm-up proofs; the host-output run gives the proof bytes below
        assert int(np.frombuffer(outs[k][0].cpu().numpy().tobytes()[12:16], dtype=np.int32)[0]) == 0
    res = [plans[k].run(wss[k].data_ptr(), sizes[k], stream) for k in keys]
    assert all(r.proof.status == 0 for r in res)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(macs_step, world, ms_max / 1e3)
    # end to end: the same batches from pinned host operands, host proofs, synchronous
    e2e = None
    if not args.no_e2e:
        host = {}
        for t in projs:
            for key in ("X", "W", "A", "B", "dY", "H", "dH"):
                host[id(t[key])] = torch.from_numpy(t[key]).pin_memory()
        hgroups = {}
        for j in jobs:
            hgroups.setdefault(W.op_shape(j)[1], []).append(
                B.job(host[id(j["P"])], host[id(j["Q"])], j["tp"], j["tq"], j["seed"]))
        hplans = {k: B.ClaimsPlan(hgroups[k], seed + k) for k in keys}
        hsizes = {k: hplans[k].workspace_bytes() for k in keys}
        del wss
        hws = {k: torch.empty(hsizes[k], dtype=torch.uint8, device="cuda") for k in keys}
        for k in keys:  # bind (first run on each workspace)
            hplans[k].run(hws[k].data_ptr(), hsizes[k], stream)
        ksteps = max(1, min(args.steps, 3))
        t1 = time.perf_counter()
        for _ in range(ksteps):
            for k in keys:
                hplans[k].run(hws[k].data_ptr(), hsizes[k], stream)
        e2e_s = max_over_ranks((time.perf_counter() - t1) / ksteps, world, "cuda")
        e2e = {"value": job_value(macs_step, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(h.numel() * 2 for h in host.values())),
               "d2h_bytes_per_step": int(sum(ctypes.sizeof(B.vl_batch_proof) + 96 * len(hgroups[k]) for k in keys)),
               "ms_per_step": 1e3 * e2e_s, "steps": ksteps,
               "note": "one synchronous plan run per batch (host outputs), operands copied in every run"}
        for k in keys:
            hplans[k].destroy()
    launches = args.steps * sum(7 + 2 * (k - 1).bit_length() for k in keys)
    proof_bytes = sum(len(r.to_bytes()) for r in res)
    # the same products as separate proofs: dims, c, three values per round, a_r, b_r, state
    separate_bytes = sum(24 + 32 + 96 * (W.op_shape(j)[1] - 1).bit_length() + 64 + 32 for j in jobs)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["7b-step-batched"] + (f", first {args.layers} layers" if args.layers else ""),
                   "products_per_step": len(jobs), "batched_proofs_per_step": len(keys),
                   "products_per_batch": {str(k): len(groups[k]) for k in keys}, "macs_per_step": macs_step,
                   "proof_bytes_per_step": proof_bytes, "separate_proofs_bytes_per_step": separate_bytes,
                   "l2": "inputs larger than L2 (no flush)",
                   "host_ms_per_step": 1e3 * wall,
                   "note": "one plan run per batch, each batch on its own stream (plans bound to their "
                           "workspaces, proofs left on the device)"},
        "roofline": None, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": launches,
    }))
    for k in keys:
        plans[k].destroy()


def chain_products(t, seed):
    """The ten products of one projection's chained proof, as oracle jobs
    (the member operands; the chain draws their points itself)."""
    X, W_, A, B_, dY, H, dH = (t[x] for x in ("X", "W", "A", "B", "dY", "H", "dH"))
    spec = [(X, W_, 0, 0), (H, B_, 0, 0), (dY, W_, 0, 1), (dH, A, 0, 1), (X, dH, 1, 0), (H, dY, 1, 0),
            (X, A, 0, 0), (X, A, 0, 0), (dY, B_, 0, 1), (dY, B_, 0, 1)]
    return [{"P": P, "Q": Q, "tp": tp, "tq": tq} for P, Q, tp, tq in spec]


def chain_main(args, rank, world, local, cpu=None):
    """The 7B step as one batch of chained projection proofs (a vl_chain_plan,
    rerun every step; each run ends with the proofs copied to the host)."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    seed = rank_seed(rank)
    projs = [W.chain_tensors(t) for t in W.make_step("7b", seed, layers=range(args.layers) if args.layers else None)]
    macs_step = sum(W.macs(j) for t in projs for j in chain_products(t, seed))
    entries = sum(W.fold_entries(j) for t in projs for j in chain_products(t, seed))
    dev = [{k: torch.from_numpy(np.ascontiguousarray(t[k])).cuda() for k in B.CHAIN_MATS} for t in projs]
    jobs = [B.chain_job(d, seed=W.proof_seed(seed, t["layer"], t["proj"], "chain")) for d, t in zip(dev, projs)]
    plan = B.ChainPlan(jobs)
    nws = plan.workspace_bytes()
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        out = plan.run(ws.data_ptr(), nws, stream)
    assert all(p.status == 0 for p in out)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run(ws.data_ptr(), nws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(macs_step, world, ms_max / 1e3)
    plan.destroy()
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["7b-step-chain"] + (f", first {args.layers} layers" if args.layers else ""),
                   "chains_per_step": len(jobs), "sumchecks_per_step": 10 * len(jobs), "macs_per_step": macs_step,
                   "fold_entries_per_step": entries, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                   "timed": "vl_chain_plan_run per step, including its synchronising copy of the proofs to the host"},
        "roofline": None, "cpu_baseline": cpu, "e2e": None, "clocks": clk,
        "gpu_launches": None,
    }))


def all_main(args, rank, world, local):
    """Matmul proofs, parameter-update proofs and remainder lookups of one 7B
    step, each as its plan on its own stream; ms_per_step is the fork-join
    time on the timing stream."""
    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    seed = rank_seed(rank)
    projs, jobs = step_jobs("7b-step", seed, args.layers)
    macs_step = sum(W.macs(j) for j in jobs)
    dev = {}
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    djobs = [B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
    opts = B.vl_batch_opts()
    opts.persistent = 2
    opts.timing_runs = 1
    mplan = B.vl_plan_create(djobs, opts)
    mn = B.vl_plan_workspace_bytes(mplan)
    mws = torch.empty(mn, dtype=torch.uint8, device="cuda")
    mout = torch.empty(len(djobs) * ctypes.sizeof(B.vl_proof), dtype=torch.uint8, device="cuda")
    ustm = [st for t in projs for st in W.update_statements(t, seed)]
    udev = [[torch.from_numpy(m).cuda() for m in st["mats"]] for st in ustm]
    uplan = B.LinPlan([B.lin_job([B.mat(x) for x in d], list(st["coeffs"]), st["seed"]) for d, st in zip(udev, ustm)])
    un = uplan.workspace_bytes()
    uws = torch.empty(un, dtype=torch.uint8, device="cuda")
    uout = torch.empty(len(ustm) * ctypes.sizeof(B.vl_lin_proof), dtype=torch.uint8, device="cuda")
    looks = [x for t in projs for x in W.rescale_lookups(t, seed)]
    ldev = [torch.from_numpy(np.ascontiguousarray(x["S"])).cuda() for x in looks]
    lplan = B.LookupPlan([B.lookup_job(B.mat(d), x["t0"], x["log2_n"], x["seed"]) for d, x in zip(ldev, looks)])
    ln = lplan.workspace_bytes()
    lws = torch.empty(ln, dtype=torch.uint8, device="cuda")
    lout = torch.empty(len(looks) * ctypes.sizeof(B.vl_lookup_proof), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    sm, su, sl = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    fork, jm, ju, jl = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()

    def step():
        fork.record(stream)
        for s2 in (sm, su, sl):
            s2.wait_event(fork)
        B.vl_plan_run(mplan, mws.data_ptr(), mn, mout.data_ptr(), B.VL_DEVICE, sm)
        jm.record(sm)
        uplan.run(uws.data_ptr(), un, uout.data_ptr(), B.VL_DEVICE, su)
        ju.record(su)
        lplan.run(lws.data_ptr(), ln, lout.data_ptr(), B.VL_DEVICE, sl)
        jl.record(sl)
        for e in (jm, ju, jl):
            stream.wait_event(e)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    st_m = np.frombuffer(mout.cpu().numpy().tobytes(), dtype=np.int32).reshape(len(djobs), -1)[:, 6]
    st_u = [B.vl_lin_proof.from_buffer_copy(uout.cpu().numpy().tobytes(), i * ctypes.sizeof(B.vl_lin_proof)).status
            for i in range(len(ustm))]
    st_l = [B.vl_lookup_proof.from_buffer_copy(lout.cpu().numpy().tobytes(), i * ctypes.sizeof(B.vl_lookup_proof)).status
            for i in range(len(looks))]
    assert (st_m == 0).all() and not any(st_u) and not any(st_l)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(macs_step, world, ms_max / 1e3)
    uplan.destroy()
    lplan.destroy()
    B.vl_plan_destroy(mplan)
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS["7b-step-all"] + (f", first {args.layers} layers" if args.layers else ""),
                   "matmul_proofs": len(djobs), "update_proofs": len(ustm), "lookup_proofs": len(looks),
                   "macs_per_step": macs_step, "l2": "inputs larger than L2 (no flush)",
                   "note": "value counts the matmul MACs only; the update and lookup proofs ride along"},
        "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": None,
    }))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serve":
        return serve_main(args, rank, world, local)
    if args.workload == "7b-step-all":
        return all_main(args, rank, world, local)
    if args.workload == "7b-step-chain":
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = oracle_cores_baseline(args.workload, W.GLOBAL_SEED)
            cpu["sample"] += "; chained proofs"
        return chain_main(args, rank, world, local, cpu)
    if args.workload == "7b-step-batched":
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = oracle_cores_baseline(args.workload, W.GLOBAL_SEED)
            cpu["sample"] += "; batched proofs, one per inner dimension of each projection"
        return batched_main(args, rank, world, local, cpu)
    if args.workload == "7b-lookups":
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            rate, dt, nj, ent = oracle_lookup_sample(W.GLOBAL_SEED, 1)
            cpu = {"value": rate, "unit": LK_UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the two n x r remainder lookups of the first projection ({nj} proofs, {ent} "
                             f"entries), single process, {dt:.1f} s"}
        return lookups_main(args, rank, world, local, cpu)
    if args.workload == "7b-update":
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            rate, dt, nj, ent = oracle_update_sample(W.GLOBAL_SEED, args.cpu_sample_projections)
            cpu = {"value": rate, "unit": LIN_UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"update relations of the first {args.cpu_sample_projections} projections "
                             f"({nj} proofs, {ent} entries), single process, {dt:.1f} s"}
        return update_main(args, rank, world, local, cpu)

    # The oracle CPU baseline runs before any CUDA work (no forked pools after it).
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_cores_baseline(args.workload, W.GLOBAL_SEED)

    import torch
    from paper_2508_21393_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.lib()
    seed = rank_seed(rank)
    projs, jobs = step_jobs(args.workload, seed, args.layers)
    macs_step = sum(W.macs(j) for j in jobs)
    entries = sum(W.fold_entries(j) for j in jobs)

    dev, keep = {}, []
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH", "dWr"):
            if key in t:
                dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    djobs = [B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
    in_bytes = sum(x.numel() * 2 for x in dev.values())

    stream = torch.cuda.current_stream()
    opts = B.vl_batch_opts()
    opts.rounds_variant = args.rounds_variant
    opts.persistent = 1 if args.persistent else 2
    opts.fold_engine = args.fold_engine
    opts.groups = args.groups
    opts.fold_dual = 1 if args.fold_dual else 0
    forced = args.persistent or args.fold_engine or args.rounds_variant or args.groups or args.fold_dual
    tuned = None
    if not args.no_autotune and not forced:
        # Launch and tile options by timing candidates on this workload (not timed).
        need = 0
        for eng, pers, seg in ((0, 2, 0), (1, 2, 0), (0, 1, 0), (0, 2, 2048)):
            o = B.vl_batch_opts()
            o.fold_engine, o.persistent, o.tc_seg = eng, pers, seg
            need = max(need, B.vl_workspace_bytes(djobs, o))
        need += len(djobs) * ctypes.sizeof(B.vl_proof) + (1 << 20)
        tws = torch.empty(need, dtype=torch.uint8, device="cuda")
        t0 = time.perf_counter()
        opts, tune_ms = B.vl_autotune(djobs, tws.data_ptr(), need, base=opts, stream=stream, runs=3)
        tuned = {"seconds": time.perf_counter() - t0, "ms_per_step_at_tuning": tune_ms,
                 **{k: getattr(opts, k) for k in ("fold_engine", "tc_seg", "rounds_variant", "rounds_threads", "persistent",
                                                  "colsum_rows", "rowdot_cols", "groups")}}
        del tws
    cuda_core = opts.persistent == 1 or opts.fold_engine == 1
    persistent = opts.persistent == 1
    opts.timing_runs = max(args.steps, 1)
    plan = B.vl_plan_create(djobs, opts)
    nws = B.vl_plan_workspace_bytes(plan)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    out = torch.empty(len(djobs) * ctypes.sizeof(B.vl_proof), dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        B.vl_plan_run(plan, ws.data_ptr(), nws, out.data_ptr(), B.VL_DEVICE, stream)
    torch.cuda.synchronize()
    status = np.frombuffer(out.cpu().numpy().tobytes(), dtype=np.int32).reshape(len(djobs), -1)[:, 6]
    assert (status == 0).all(), "a proof reported a non-OK status"
    B.vl_plan_phase_ms(plan, 0, reset=1)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.6)  # let the sampler take its first reading before the timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        B.vl_plan_run(plan, ws.data_ptr(), nws, out.data_ptr(), B.VL_DEVICE, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    status = np.frombuffer(out.cpu().numpy().tobytes(), dtype=np.int32).reshape(len(djobs), -1)[:, 6]
    assert (status == 0).all(), "a proof of the timed steps reported a non-OK status"
    ms = e0.elapsed_time(e1) / args.steps
    phases = B.vl_plan_phase_ms(plan, args.steps, reset=1)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_value(macs_step, world, ms_max / 1e3)

    fold_ms = statistics.mean(p[1] for p in phases)
    pro_ms = statistics.mean(p[0] for p in phases)
    rnd_ms = statistics.mean(p[2] for p in phases)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak, hbm_note = (peaks["hbm_gbs"], "measured") if "hbm_gbs" in peaks else (6800.0, "fallback")
    hbm_gbs = 2 * entries / (fold_ms / 1e3) / 1e9  # each int16 operand entry read once
    if cuda_core:
        # CUDA-core fold: bound by 32x32->64 multiply-adds (eight per entry).
        if persistent:
            kernel, phase_ms = "step_kernel (persistent)", {"clear": pro_ms, "step_kernel": fold_ms}
        else:
            kernel, phase_ms = "fold_kernel", {"clear+prologue": pro_ms, "fold": fold_ms, "rounds": rnd_ms}
        peak = SMS * MADWIDE_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
        achieved = 8 * entries / (fold_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "Tmadwide/s",
                "frac": achieved / peak, "traffic": None, "hbm_gbs_algorithmic": hbm_gbs,
                "peak_note": "152 SMs x 32 IMAD.WIDE/clk x 2070 MHz (derived)"}
    else:
        # Tensor-core fold: streams every operand entry once from HBM.
        kernel, phase_ms = "fold_tc_kernel", {"clear+prologue": pro_ms, "fold": fold_ms, "rounds": rnd_ms}
        # 64 fp16 MACs per entry (two bytes x 32 weight bytes) plus the two
        # constant MMAs of each 128-entry stage (2 x 128 x 32 x 16 MACs per
        # 128 x 128 entries: 8 per entry)
        tflops = 2 * (64 + 8) * entries / (fold_ms / 1e3) / 1e12
        # DRAM traffic per launch: ncu capture of the same kernel on the first
        # two layers (profiles/fold_tc_kernel_7b_2layers.md), 444.4 MB for 750 MB
        # algorithmic, scaled by entries (the tile mix repeats per projection).
        traffic = 0.5926 * 2 * entries if args.workload == "7b-step" else None
        roof = {"bound": "hbm", "kernel": kernel, "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_gbs / hbm_peak, "traffic": traffic,
                "peak_note": f"{hbm_note} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": 2 * entries,
                "unique_input_bytes": in_bytes,
                "frac_of_unique_bytes": in_bytes / (fold_ms / 1e3) / 1e9 / hbm_peak,
                "tensor_tflops_fp16": tflops}
    rounds_roof = rounds_bound(jobs, rnd_ms)

    # Unbatched per-matmul path: each product proved by its own plan (graph),
    # one after another on the same stream.
    unbatched_ms = None
    if not args.no_unbatched:
        one = B.vl_batch_opts()
        one.timing_runs = 1
        plans = [B.vl_plan_create([j], one) for j in djobs]
        sizes = [(B.vl_plan_workspace_bytes(p) + 255) // 256 * 256 for p in plans]
        offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        ws1 = torch.empty(int(sum(sizes)), dtype=torch.uint8, device="cuda")  # one slice per plan
        base = ws1.data_ptr()
        for p, sz, o in zip(plans, sizes, offs):
            B.vl_plan_run(p, base + int(o), sz, out.data_ptr(), B.VL_DEVICE, stream)
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        for p, sz, o in zip(plans, sizes, offs):
            B.vl_plan_run(p, base + int(o), sz, out.data_ptr(), B.VL_DEVICE, stream)
        u1.record(stream)
        torch.cuda.synchronize()
        unbatched_ms = u0.elapsed_time(u1)
        for p in plans:
            B.vl_plan_destroy(p)
        del ws1

    # End to end through the C ABI: pinned host operands in, host proofs out.
    e2e = None
    if not args.no_e2e:
        # The step in chunks of whole projections (4 layers each), one plan
        # per chunk, on two streams: a chunk's host operands are copied in
        # while the previous chunk is proved.  Each chunk's operands sit in
        # one pinned host buffer (256-byte aligned, back to back), which the
        # library stages with one copy.  Proofs go to device memory and come
        # back in one copy at the end of the step.
        pper = min(16, len(projs))
        host, arenas = {}, []
        for c0 in range(0, len(projs), pper):
            mats = [t[key] for t in projs[c0:c0 + pper]
                    for key in ("X", "W", "A", "B", "dY", "H", "dH", "dWr") if key in t]
            offs, tot = [], 0
            for a in mats:
                offs.append(tot)
                tot += (a.nbytes + 255) // 256 * 256
            arena = torch.empty(tot, dtype=torch.uint8, pin_memory=True)
            arenas.append(arena)
            for a, o in zip(mats, offs):
                h = arena[o:o + a.nbytes].view(torch.int16).view(a.shape)
                h.copy_(torch.from_numpy(a))
                host[id(a)] = h
        hjobs = [B.job(host[id(j["P"])], host[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
        hopts = B.vl_batch_opts.from_buffer_copy(opts)  # the same (tuned) options
        hopts.timing_runs = 1
        per = len(jobs) // len(projs) * pper
        chunks = [hjobs[i:i + per] for i in range(0, len(hjobs), per)]
        hplans = [B.vl_plan_create(c, hopts) for c in chunks]
        hsizes = [B.vl_plan_workspace_bytes(p) for p in hplans]
        del ws
        hwss = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in hsizes]
        psz = ctypes.sizeof(B.vl_proof)
        dproofs = torch.empty(len(hjobs) * psz, dtype=torch.uint8, device="cuda")
        hproofs = torch.empty(len(hjobs) * psz, dtype=torch.uint8, pin_memory=True)
        pipes = [torch.cuda.Stream(), torch.cuda.Stream()]
        fork, joins = torch.cuda.Event(), [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_step(plans=None, sizes=None):
            plans, sizes = plans or hplans, sizes or hsizes
            fork.record(stream)
            off = 0
            for i, (hp, c) in enumerate(zip(plans, chunks)):
                s2 = pipes[i % 2]
                s2.wait_event(fork)
                B.vl_plan_run(hp, hwss[i].data_ptr(), sizes[i], dproofs.data_ptr() + off, B.VL_DEVICE, s2)
                off += len(c) * psz
            for ev, s2 in zip(joins, pipes):
                ev.record(s2)
                stream.wait_event(ev)
            hproofs.copy_(dproofs, non_blocking=True)
            stream.synchronize()

        for _ in range(2):
            e2e_step()
        st_h = np.frombuffer(hproofs.numpy().tobytes(), dtype=np.int32).reshape(len(hjobs), -1)[:, 6]
        assert (st_h == 0).all(), "a proof reported a non-OK status (end to end)"
        ksteps = max(1, min(args.steps, 5))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            e2e_step()
        e2e_s = (time.perf_counter() - t0) / ksteps
        e2e_max = max_over_ranks(e2e_s, world, "cuda")
        h2d = int(sum(h.numel() * 2 for h in host.values()))
        rate = pinned_h2d_gbs(stream)
        e2e = {"value": job_value(macs_step, world, e2e_max), "unit": UNIT,
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(psz * len(hjobs)),
               "ms_per_step": 1e3 * e2e_max, "steps": ksteps,
               "pinned_h2d_gbs": rate, "copy_bound_ms": 1e3 * h2d / (rate * 1e9),
               "pipeline": f"{len(chunks)} plans of {pper} projections on 2 streams (copy of chunk i+1 overlaps the "
                           f"proving of chunk i; each chunk's operands in one pinned buffer, staged by one copy), "
                           f"one proof copy-out per step"}
        # The same step with the frozen W kept on the device, as a
        # fine-tuning loop keeps it: every other operand (activations,
        # gradients, LoRA factors, rescaled products) copied in per step.
        if any("W" in t for t in projs):
            frozen = {id(t["W"]) for t in projs if "W" in t}
            host2, arenas2 = {}, []
            for c0 in range(0, len(projs), pper):
                mats = [t[key] for t in projs[c0:c0 + pper]
                        for key in ("X", "A", "B", "dY", "H", "dH", "dWr") if key in t]
                offs, tot = [], 0
                for a in mats:
                    offs.append(tot)
                    tot += (a.nbytes + 255) // 256 * 256
                arena = torch.empty(tot, dtype=torch.uint8, pin_memory=True)
                arenas2.append(arena)
                for a, o in zip(mats, offs):
                    h = arena[o:o + a.nbytes].view(torch.int16).view(a.shape)
                    h.copy_(torch.from_numpy(a))
                    host2[id(a)] = h

            def src(a):
                return dev[id(a)] if id(a) in frozen else host2[id(a)]
            rjobs = [B.job(src(j["P"]), src(j["Q"]), j["tp"], j["tq"], j["seed"]) for j in jobs]
            rplans = [B.vl_plan_create(rjobs[i:i + per], hopts) for i in range(0, len(rjobs), per)]
            rsizes = [B.vl_plan_workspace_bytes(p) for p in rplans]
            assert all(r <= h for r, h in zip(rsizes, hsizes))  # the end-to-end workspaces serve
            for _ in range(2):
                e2e_step(rplans, rsizes)
            st_r = np.frombuffer(hproofs.numpy().tobytes(), dtype=np.int32).reshape(len(rjobs), -1)[:, 6]
            assert (st_r == 0).all(), "a proof reported a non-OK status (end to end, W resident)"
            t0 = time.perf_counter()
            for _ in range(ksteps):
                e2e_step(rplans, rsizes)
            r_s = max_over_ranks((time.perf_counter() - t0) / ksteps, world, "cuda")
            h2d_r = int(sum(h.numel() * 2 for h in host2.values()))
            e2e["frozen_w_resident"] = {
                "value": job_value(macs_step, world, r_s), "unit": UNIT, "ms_per_step": 1e3 * r_s,
                "h2d_bytes_per_step": h2d_r, "d2h_bytes_per_step": int(psz * len(rjobs)),
                "copy_bound_ms": 1e3 * h2d_r / (rate * 1e9),
                "note": "the frozen W on the device across steps (copied once, outside the timed region); the "
                        "other operands from pinned host memory every step, same pipeline"}
            for rp in rplans:
                B.vl_plan_destroy(rp)
        for hp in hplans:
            B.vl_plan_destroy(hp)

    launches = args.steps * B.vl_plan_launches(plan)
    B.vl_plan_destroy(plan)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16 operands, Fr (255-bit) arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + (f", first {args.layers} layers" if args.layers else ""),
                   "proofs_per_step": len(jobs),
                   "macs_per_step": macs_step, "fold_entries_per_step": entries,
                   "input_bytes_per_step": in_bytes, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                   "batched_ms_per_step": ms_max, "unbatched_ms_per_step": unbatched_ms,
                   "launch_mode": "one persistent launch" if persistent else "phase launches (CUDA graph)",
                   "fold_engine": "CUDA cores" if cuda_core else "tensor cores",
                   "autotuned": tuned,
                   "phase_ms": phase_ms, "rounds_bound": rounds_roof},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
