"""Oracle proofs of whole LoRA projections in worker processes (test helper).

The oracle proves one 7B-shaped projection (eight products) in a few seconds
on one core, so comparing every proof of a full step with it is a matter of
spreading projections over the host's cores.  Workers are started with the
'spawn' method: they share nothing with the parent (in particular no CUDA
context), import only the oracle and the seeded input generators, and
regenerate each projection's tensors from its recipe (workload.lora_projection)
instead of receiving them through a pipe.
"""
import multiprocessing as mp
import os


def _projection_proofs(task):
    seed, spec = task
    import oracle
    from paper_2508_21393_gb300 import workload as W

    t = W.lora_projection(seed, *spec)
    return [(j["name"], oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes())
            for j in W.projection_products(t, seed)]


def cores():
    return os.cpu_count() or 1


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / (1 << 20)
    except OSError:
        pass
    return None


def workers(n_tasks, gb_per_task=2.0):
    """Worker count: one per core, at most one per task, and no more than
    half the host's available memory allows (a 13B-shaped projection's
    oracle holds about 1.2 GB of Python integers)."""
    n = min(cores(), n_tasks)
    gb = _mem_available_gb()
    if gb is not None:
        n = min(n, max(1, int(gb / 2 / gb_per_task)))
    return max(1, n)


def start(specs, seed, procs=None):
    """Start proving the projections `specs` ((layer, proj, n, d, k, r) tuples)
    in a spawn pool; returns (pool, async result).  Call finish() on them."""
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(procs or workers(len(specs)))
    res = pool.map_async(_projection_proofs, [(seed, s) for s in specs], chunksize=1)
    return pool, res


def finish(pool, res, timeout=1800):
    """{proof name: oracle proof bytes} of every started projection."""
    try:
        out = {}
        for part in res.get(timeout):
            out.update(part)
        return out
    finally:
        pool.terminate()
        pool.join()
