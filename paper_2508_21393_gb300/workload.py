"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the proving method: it only draws
fixed-point integer tensors, forms the exact integer products a LoRA step
would claim, and names the matrix products of one LoRA step.  Both the CUDA
path and the oracle receive the arrays made here; neither is imported here.

Stand-ins: the paper trains LLaMA-2/3.2 and OPT models on C4 (Sec. VI-A).
Neither the weights nor the data are available, so tensors are synthetic with
LLaMA shapes: hidden size 4096 (7B) or 5120 (13B), LoRA rank r in {8,16,64},
activations and upstream gradients ~ round(N(0, 2^8)), weights and LoRA
factors ~ round(N(0, 0.02 * 2^8)), all clamped to int16 (fixed point with
scale 2^8).  The single-matmul case draws int16 uniformly in [-2^15, 2^15).

The LoRA step (Sec. III-B, III-C; LoRA factors in the X.A.B convention):
    Y = X.W + (X.A).B,   H = rescale(X.A),   dH = rescale(dY.B^T)
and the eight products proved per projection (F = forward, B = backward):
    F1 X.W    F2 X.A    F3 H.B    B1 dY.B^T
    B2 H^T.dY B3 X^T.dH B4 dY.W^T B5 dH.A^T
B2, B3 and B4 give dB, dA and the frozen-weight part of dX; B1 (dH) and B5
(the LoRA part of dX) are the two rank-r products the chain needs.  A
transpose is never materialised: a product names the stored matrix and a
transpose flag.

Rescale (workload only; it is a lookup-proved step in the paper, Sec. IV-A,
zkSwiGLU quantisation): z' = floor((z + 2^7) / 2^8), clamped to int16.

Parameter update (Eq. eq:grad_update_ab, in fixed point): the learning rate
is eta = 2^-UPDATE_SHIFT at the tensor scale, so the step of a LoRA factor is
G = rescale(dFactor, UPDATE_SHIFT) (the exact gradient product, rounded half
up, clamped to +-2^14) and the updated factor is Factor' = Factor - G.  The
update is then the linear relation Factor' - Factor + G = 0, proved by the
linear zkMat with coefficients (1, -1, 1); the rescale itself is a
lookup-proved step.
"""

import hashlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GLOBAL_SEED = 250821393
ACT_SIGMA = 256.0
WEIGHT_SIGMA = 0.02 * 256.0
PRODUCTS = ("F1", "F2", "F3", "B1", "B2", "B3", "B4", "B5")
PROJECTIONS = ("q", "k", "v", "o")
I16_MIN, I16_MAX = -(1 << 15), (1 << 15) - 1


def _rng(*key):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


def uniform_int16(rng, shape):
    return rng.integers(I16_MIN, I16_MAX + 1, size=shape, dtype=np.int16)


def gauss_int16(rng, shape, sigma):
    x = rng.standard_normal(size=shape, dtype=np.float32)
    x *= np.float32(sigma)
    np.rint(x, out=x)
    np.clip(x, I16_MIN, I16_MAX, out=x)
    return x.astype(np.int16)


def exact_matmul(A, B):
    """Exact integer product of two integer matrices, as int64.

    Uses float64 BLAS when every partial sum is below 2^53 (then exact), else
    falls back to Python integers.
    """
    A = np.asarray(A)
    B = np.asarray(B)
    amax = int(np.abs(A.astype(np.int64)).max()) if A.size else 0
    bmax = int(np.abs(B.astype(np.int64)).max()) if B.size else 0
    if A.shape[1] * amax * bmax < (1 << 53):
        return (A.astype(np.float64) @ B.astype(np.float64)).astype(np.int64)
    return (A.astype(object) @ B.astype(object)).astype(np.int64)


def rescale(Z, shift=8):
    Z = np.asarray(Z, dtype=np.int64)
    return np.clip((Z + (1 << (shift - 1))) >> shift, I16_MIN, I16_MAX).astype(np.int16)


def proof_seed(global_seed, layer, proj, product):
    """Per-proof transcript seed: first 8 bytes (LE) of SHA256 of the job key.

    A public, deterministic seed per proof is what makes a proof made in a
    batch byte-identical to the same proof made alone.
    """
    key = f"{int(global_seed)}/{int(layer)}/{proj}/{product}".encode()
    return int.from_bytes(hashlib.sha256(key).digest()[:8], "little")


def single_matmul(seed=GLOBAL_SEED, m=64, k=128, n=64):
    """One matmul C = A.B with int16 entries uniform in [-2^15, 2^15)."""
    rng = _rng(seed, 1)
    A = uniform_int16(rng, (m, k))
    B = uniform_int16(rng, (k, n))
    return {"P": A, "Q": B, "tp": 0, "tq": 0, "seed": proof_seed(seed, 0, "x", "M"),
            "name": f"matmul{m}x{k}x{n}"}


def lora_projection(seed, layer, proj, n, d, k, r):
    """Tensors of one LoRA projection: X n x d, W d x k, A d x r, B r x k, dY n x k, H, dH."""
    pid = PROJECTIONS.index(proj) if proj in PROJECTIONS else 9
    rng = _rng(seed, 2, layer, pid)
    X = gauss_int16(rng, (n, d), ACT_SIGMA)
    W = gauss_int16(rng, (d, k), WEIGHT_SIGMA)
    A = gauss_int16(rng, (d, r), WEIGHT_SIGMA)
    B = gauss_int16(rng, (r, k), WEIGHT_SIGMA)
    dY = gauss_int16(rng, (n, k), ACT_SIGMA)
    H = rescale(exact_matmul(X, A))
    dH = rescale(exact_matmul(dY, B.T))
    return {"X": X, "W": W, "A": A, "B": B, "dY": dY, "H": H, "dH": dH,
            "layer": layer, "proj": proj, "n": n, "d": d, "k": k, "r": r}


def projection_products(t, seed=GLOBAL_SEED):
    """The eight (P, Q, transP, transQ) products of one projection, with seeds."""
    X, W, A, B, dY, H, dH = (t[x] for x in ("X", "W", "A", "B", "dY", "H", "dH"))
    spec = {
        "F1": (X, W, 0, 0), "F2": (X, A, 0, 0), "F3": (H, B, 0, 0),
        "B1": (dY, B, 0, 1), "B2": (H, dY, 1, 0), "B3": (X, dH, 1, 0),
        "B4": (dY, W, 0, 1), "B5": (dH, A, 0, 1),
    }
    out = []
    for name in PRODUCTS:
        P, Q, tp, tq = spec[name]
        out.append({"P": P, "Q": Q, "tp": tp, "tq": tq, "name": f"L{t['layer']}.{t['proj']}.{name}",
                    "seed": proof_seed(seed, t["layer"], t["proj"], name)})
    return out


UPDATE_SHIFT = 12
UPDATE_CLAMP = 1 << 14


def update_statements(t, seed=GLOBAL_SEED):
    """The two parameter-update relations of one projection: A' = A - G_A
    (d x r) and B' = B - G_B (r x k), with G = rescale(gradient) as above.
    Each is {"mats": (A', A, G), "coeffs": (1, -1, 1), "seed", "name"}."""
    X, A, B, dY, H, dH = (t[x] for x in ("X", "A", "B", "dY", "H", "dH"))
    out = []
    for name, F, grad in (("A", A, lambda: exact_matmul(X.T, dH)), ("B", B, lambda: exact_matmul(H.T, dY))):
        G = np.clip(rescale(grad(), UPDATE_SHIFT), -UPDATE_CLAMP, UPDATE_CLAMP).astype(np.int16)
        F2 = (F.astype(np.int32) - G.astype(np.int32))
        assert F2.min() >= I16_MIN and F2.max() <= I16_MAX
        out.append({"mats": (F2.astype(np.int16), F, G), "coeffs": (1, -1, 1),
                    "seed": proof_seed(seed, t["layer"], t["proj"], "U" + name),
                    "name": f"L{t['layer']}.{t['proj']}.U{name}"})
    return out


ROUTE_PRODUCTS = ("F1", "F2", "F3", "B1", "B4", "B5", "R1", "R2", "R3")


def paper_route_products(t, seed=GLOBAL_SEED):
    """The products of one projection along the paper's backward route
    (Eq. eq:grad_wl, eq:grad_abl), which forms the full d x k gradient of the
    adapted weight W' = W + A.B and derives the LoRA gradients from it:
        R1 dW' = X^T.dY (d x n x k),  dWr = rescale(dW')
        R2 dA  = dWr.B^T (d x k x r)
        R3 dB  = A^T.dWr (r x d x k)
    replacing B2 and B3 of the eight-product set; F1-F3, B1, B4, B5 stay (the
    input gradient needs dH).  Returns (products, dWr)."""
    X, A, B, dY = (t[x] for x in ("X", "A", "B", "dY"))
    dWr = rescale(exact_matmul(X.T, dY))
    base = {j["name"].rsplit(".", 1)[1]: j for j in projection_products(t, seed)}
    spec = {"R1": (X, dY, 1, 0), "R2": (dWr, B, 0, 1), "R3": (A, dWr, 1, 0)}
    out = []
    for name in ROUTE_PRODUCTS:
        if name in base:
            out.append(base[name])
            continue
        P, Q, tp, tq = spec[name]
        out.append({"P": P, "Q": Q, "tp": tp, "tq": tq, "name": f"L{t['layer']}.{t['proj']}.{name}",
                    "seed": proof_seed(seed, t["layer"], t["proj"], name)})
    return out, dWr


RESCALE_SHIFT = 8


def remainder(Z, shift):
    """rho = (z + 2^(shift-1)) mod 2^shift, the remainder the rescale
    z' = floor((z + 2^(shift-1)) / 2^shift) drops: z + 2^(shift-1) = 2^shift z' + rho."""
    Z = np.asarray(Z, dtype=np.int64)
    return ((Z + (1 << (shift - 1))) & ((1 << shift) - 1)).astype(np.int16)


def rescale_lookups(t, seed=GLOBAL_SEED):
    """Range checks of one projection's rescale remainders (the lookup
    arguments that prove the fixed-point rescales, Sec. IV-A): H = rescale(X.A)
    and dH = rescale(dY.B^T) (n x r, remainders in [0, 2^8)), and the
    parameter-update steps G_A, G_B (d x r and r x k, remainders in
    [0, 2^12)).  Each is {"S", "t0", "log2_n", "seed", "name"}."""
    X, A, B, dY, H, dH = (t[x] for x in ("X", "A", "B", "dY", "H", "dH"))
    out = []
    for name, Z, shift in (("H", lambda: exact_matmul(X, A), RESCALE_SHIFT),
                           ("dH", lambda: exact_matmul(dY, B.T), RESCALE_SHIFT),
                           ("GA", lambda: exact_matmul(X.T, dH), UPDATE_SHIFT),
                           ("GB", lambda: exact_matmul(H.T, dY), UPDATE_SHIFT)):
        out.append({"S": remainder(Z(), shift), "t0": 0, "log2_n": shift,
                    "seed": proof_seed(seed, t["layer"], t["proj"], "R" + name),
                    "name": f"L{t['layer']}.{t['proj']}.R{name}"})
    return out


def chain_tensors(t):
    """The projection's tensors plus the rescale remainders the chained proof
    needs: rhoH = (X.A + 2^7) mod 2^8, rhodH = (dY.B^T + 2^7) mod 2^8, so that
    X.A + 2^7 = 2^8 H + rhoH and dY.B^T + 2^7 = 2^8 dH + rhodH hold exactly
    (checked: a clamped rescale would break them)."""
    X, A, B, dY, H, dH = (t[x] for x in ("X", "A", "B", "dY", "H", "dH"))
    out = dict(t)
    for name, Z, Hs in (("rhoH", exact_matmul(X, A), H), ("rhodH", exact_matmul(dY, B.T), dH)):
        rho = remainder(Z, RESCALE_SHIFT)
        assert np.array_equal(Z + (1 << (RESCALE_SHIFT - 1)),
                              (Hs.astype(np.int64) << RESCALE_SHIFT) + rho), "rescale clamped"
        out[name] = rho
    return out


def chain_outputs(t):
    """The claimed outputs of one projection: Y = X.W + H.B, dX = dY.W^T +
    dH.A^T, dA = X^T.dH, dB = H^T.dY (exact int64)."""
    X, W, A, B, dY, H, dH = (t[x] for x in ("X", "W", "A", "B", "dY", "H", "dH"))
    return {"Y": exact_matmul(X, W) + exact_matmul(H, B), "dX": exact_matmul(dY, W.T) + exact_matmul(dH, A.T),
            "dA": exact_matmul(X.T, dH), "dB": exact_matmul(H.T, dY)}


def op_shape(job):
    P, Q = job["P"], job["Q"]
    m, k = (P.shape[1], P.shape[0]) if job["tp"] else P.shape
    k2, n = (Q.shape[1], Q.shape[0]) if job["tq"] else Q.shape
    assert k == k2
    return m, k, n


def claimed_product(job):
    """C = op(P).op(Q) exactly (the claimed output the verifier checks)."""
    P = job["P"].T if job["tp"] else job["P"]
    Q = job["Q"].T if job["tq"] else job["Q"]
    return exact_matmul(P, Q)


def macs(job):
    m, k, n = op_shape(job)
    return m * k * n


def fold_entries(job):
    return job["P"].size + job["Q"].size


def step_layers(kind, seed=GLOBAL_SEED):
    """Layer list of a LoRA step: (layer, proj, n, d, k, r) tuples.

    '7b'  : 32 layers x {q,k,v,o}, hidden 4096, seq 512, rank per layer drawn
            from {8, 16, 64} with the seed.
    '13b' : 40 layers x {q,k,v,o}, hidden 5120, seq 2048, rank 16.
    """
    if kind == "7b":
        rng = _rng(seed, 3)
        ranks = rng.choice(np.array([8, 16, 64]), size=32)
        return [(l, p, 512, 4096, 4096, int(ranks[l])) for l in range(32) for p in PROJECTIONS]
    if kind == "13b":
        return [(l, p, 2048, 5120, 5120, 16) for l in range(40) for p in PROJECTIONS]
    if kind == "7b-proj":
        return [(0, "v", 1024, 4096, 4096, 16)]
    raise ValueError(kind)


def make_step(kind, seed=GLOBAL_SEED, layers=None, threads=16):
    """All projections (tensors) of a step; generated in parallel threads."""
    spec = step_layers(kind, seed)
    if layers is not None:
        spec = [s for s in spec if s[0] in layers]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda s: lora_projection(seed, *s), spec))


def serving_jobs(count, seed=GLOBAL_SEED, rate=20.0):
    """Poisson arrivals of single-projection proving jobs (mixed 7B / 13B shapes).

    Returns (arrival_time_s, (hidden, seq, rank)) per job; shapes are uniform
    over hidden in {4096, 5120}, seq in {256, 512, 1024, 2048}, rank in {8, 16, 64}.
    """
    rng = _rng(seed, 5)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    hid = rng.choice(np.array([4096, 5120]), size=count)
    seq = rng.choice(np.array([256, 512, 1024, 2048]), size=count)
    rank = rng.choice(np.array([8, 16, 64]), size=count)
    return [(float(t[i]), (int(hid[i]), int(seq[i]), int(rank[i]))) for i in range(count)]
