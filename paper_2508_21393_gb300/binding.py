"""ctypes binding of libverilora.so (include/verilora.h), same names as the C ABI.

Argument marshalling only: every step of the proving path runs in the CUDA
library.  PyTorch is used for device memory and streams.  If the library is
missing the calls raise; there is no fallback.

Helpers: ``mat`` wraps a torch tensor (device or host) or a NumPy array
(host) as a ``vl_mat``; ``fs_init`` builds transcript inputs;
``proof_bytes`` serialises a proof canonically (six u32le dims, c, the d1
round triples, a_r, b_r, the final transcript state).
"""

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libverilora.so")

VL_OK, VL_EINVAL, VL_ESHAPE, VL_ENOMEM, VL_ECUDA, VL_ETIMEOUT, VL_REJECT, VL_ELOOKUP = range(8)
VL_I16, VL_I64, VL_FR_MONT = 1, 2, 3
VL_DEVICE, VL_HOST = 0, 1
VL_MAX_ROUNDS = 24
VL_MAX_REDUCE = 1 << 16

# Every symbol include/verilora.h declares.
EXPORTS = ("vl_version", "vl_strerror", "vl_last_error", "vl_workspace_bytes", "vl_prove_matmul", "vl_prove_batch",
           "vl_plan_create", "vl_plan_workspace_bytes", "vl_plan_run", "vl_plan_launches", "vl_plan_phase_ms",
           "vl_plan_destroy", "vl_verify_matmul", "vl_encode", "vl_prove_matmul_noalloc",
           "vl_server_create", "vl_server_submit", "vl_server_poll", "vl_server_stats_get", "vl_server_destroy",
           "vl_autotune", "vl_autotune_clear", "vl_linear_workspace_bytes", "vl_prove_linear", "vl_verify_linear",
           "vl_lin_plan_create", "vl_lin_plan_workspace_bytes", "vl_lin_plan_run", "vl_lin_plan_phase_ms",
           "vl_lin_plan_destroy", "vl_lookup_workspace_bytes", "vl_lookup_plan_create",
           "vl_lookup_plan_workspace_bytes", "vl_lookup_plan_run", "vl_lookup_plan_phase_ms",
           "vl_lookup_plan_destroy", "vl_prove_lookup", "vl_verify_lookup", "vl_batch_workspace_bytes",
           "vl_prove_matmul_batched", "vl_verify_matmul_batched", "vl_claims_plan_create",
           "vl_claims_plan_workspace_bytes", "vl_claims_plan_run", "vl_claims_plan_destroy",
           "vl_workspace_forget", "vl_chain_workspace_bytes", "vl_prove_chain", "vl_verify_chain",
           "vl_chain_plan_create", "vl_chain_plan_workspace_bytes", "vl_chain_plan_run", "vl_chain_plan_destroy")
VL_NOALLOC_SCRATCH_BYTES = 8 << 20
VL_LIN_MAX = 16
VL_LOOKUP_MAX_LOG_D = 24
VL_LOOKUP_MAX_LOG_N = 16
R_MOD = 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001


class vl_fr(ctypes.Structure):
    _fields_ = [("limb", ctypes.c_uint32 * 8)]

    def to_int(self):
        return sum(int(self.limb[i]) << (32 * i) for i in range(8))


class vl_mat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32), ("trans", ctypes.c_int32),
                ("space", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class vl_fs_init(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("bind", (ctypes.c_uint8 * 32) * 3)]


class vl_proof(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("k", ctypes.c_int32), ("n", ctypes.c_int32),
                ("d0", ctypes.c_int32), ("d1", ctypes.c_int32), ("d2", ctypes.c_int32),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("c", vl_fr), ("g", (vl_fr * 3) * VL_MAX_ROUNDS), ("a_r", vl_fr), ("b_r", vl_fr),
                ("state", ctypes.c_uint8 * 32)]


class vl_lin_job(ctypes.Structure):
    _fields_ = [("mats", ctypes.POINTER(vl_mat)), ("coeffs", ctypes.POINTER(vl_fr)),
                ("binds", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("nmats", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class vl_lin_proof(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("d0", ctypes.c_int32), ("d1", ctypes.c_int32),
                ("nmats", ctypes.c_int32), ("status", ctypes.c_int32), ("evals", vl_fr * VL_LIN_MAX),
                ("state", ctypes.c_uint8 * 32)]


class vl_lookup_job(ctypes.Structure):
    _fields_ = [("S", vl_mat), ("t0", ctypes.c_int64), ("log2_n", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("bind", ctypes.c_uint8 * 32)]


class vl_lookup_proof(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("log2_d", ctypes.c_int32), ("log2_n", ctypes.c_int32),
                ("status", ctypes.c_int32), ("t0", ctypes.c_int64),
                ("g", (vl_fr * 4) * VL_LOOKUP_MAX_LOG_D), ("a_r", vl_fr), ("s_r", vl_fr), ("b_r", vl_fr),
                ("m_r", vl_fr), ("state", ctypes.c_uint8 * 32)]


class vl_batch_proof(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("k", ctypes.c_int32), ("d1", ctypes.c_int32), ("status", ctypes.c_int32),
                ("g", (vl_fr * 3) * VL_MAX_ROUNDS), ("state", ctypes.c_uint8 * 32)]


class vl_job(ctypes.Structure):
    _fields_ = [("P", vl_mat), ("Q", vl_mat), ("fs", vl_fs_init)]


VL_CHAIN_MEMBERS = 10
VL_CHAIN_MAX_RANK = 256
CHAIN_MATS = ("X", "W", "A", "B", "dY", "H", "dH", "rhoH", "rhodH")


class vl_chain_job(ctypes.Structure):
    _fields_ = [(name, vl_mat) for name in CHAIN_MATS] + [("seed", ctypes.c_uint64),
                                                          ("bind", (ctypes.c_uint8 * 32) * 7)]


class vl_chain_proof(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("d", ctypes.c_int32), ("k", ctypes.c_int32), ("r", ctypes.c_int32),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sub", vl_proof * VL_CHAIN_MEMBERS), ("e", vl_fr * 4), ("state", ctypes.c_uint8 * 32)]


class vl_server_opts(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_batch_requests", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class vl_server_done(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("latency_ms", ctypes.c_double), ("dev_start_ms", ctypes.c_double), ("dev_end_ms", ctypes.c_double)]


class vl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("proofs", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("launched", ctypes.c_int64)]


class vl_batch_opts(ctypes.Structure):
    _fields_ = [("colsum_rows", ctypes.c_int32), ("rowdot_cols", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("groups", ctypes.c_int32), ("fold_engine", ctypes.c_int32),
                ("use_graph", ctypes.c_int32),
                ("timing_runs", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("rounds_variant", ctypes.c_int32), ("rounds_threads", ctypes.c_int32), ("tc_seg", ctypes.c_int32),
                ("test_never_ready", ctypes.c_int32), ("fold_dual", ctypes.c_int32)]


class VLError(RuntimeError):
    def __init__(self, code, what):
        detail = f" [{vl_last_error()}]" if code == VL_ECUDA else ""
        super().__init__(f"{what}: {vl_strerror(code)} ({code}){detail}")
        self.code = code


_lib = None


def lib():
    """Load libverilora.so once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libverilora.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.vl_version.restype = ctypes.c_int32
    L.vl_strerror.argtypes = [ctypes.c_int32]
    L.vl_strerror.restype = ctypes.c_char_p
    L.vl_last_error.restype = ctypes.c_char_p
    L.vl_workspace_bytes.argtypes = [P(vl_job), ctypes.c_int32, P(vl_batch_opts)]
    L.vl_workspace_bytes.restype = ctypes.c_size_t
    L.vl_prove_matmul.argtypes = [P(vl_mat), P(vl_mat), P(vl_fs_init), ctypes.c_void_p, ctypes.c_size_t,
                                  P(vl_proof), ctypes.c_void_p]
    L.vl_prove_matmul.restype = ctypes.c_int32
    L.vl_prove_batch.argtypes = [P(vl_job), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                 ctypes.c_int32, ctypes.c_void_p, P(vl_batch_opts)]
    L.vl_prove_batch.restype = ctypes.c_int32
    L.vl_plan_create.argtypes = [P(vl_job), ctypes.c_int32, P(vl_batch_opts), P(ctypes.c_void_p)]
    L.vl_plan_create.restype = ctypes.c_int32
    L.vl_plan_workspace_bytes.argtypes = [ctypes.c_void_p]
    L.vl_plan_workspace_bytes.restype = ctypes.c_size_t
    L.vl_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int32,
                              ctypes.c_void_p]
    L.vl_plan_run.restype = ctypes.c_int32
    L.vl_plan_launches.argtypes = [ctypes.c_void_p]
    L.vl_plan_launches.restype = ctypes.c_int32
    L.vl_plan_phase_ms.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.c_int32]
    L.vl_plan_phase_ms.restype = ctypes.c_int32
    L.vl_plan_destroy.argtypes = [ctypes.c_void_p]
    L.vl_plan_destroy.restype = None
    L.vl_autotune.argtypes = [P(vl_job), ctypes.c_int32, P(vl_batch_opts), ctypes.c_void_p, ctypes.c_size_t,
                              ctypes.c_void_p, ctypes.c_int32, P(vl_batch_opts), P(ctypes.c_float)]
    L.vl_autotune.restype = ctypes.c_int32
    L.vl_autotune_clear.argtypes = []
    L.vl_autotune_clear.restype = None
    L.vl_server_create.argtypes = [P(vl_server_opts), P(ctypes.c_void_p)]
    L.vl_server_create.restype = ctypes.c_int32
    L.vl_server_submit.argtypes = [ctypes.c_void_p, P(vl_job), ctypes.c_int32, P(vl_proof), P(ctypes.c_uint64)]
    L.vl_server_submit.restype = ctypes.c_int32
    L.vl_server_poll.argtypes = [ctypes.c_void_p, P(vl_server_done), ctypes.c_int32, P(ctypes.c_int32)]
    L.vl_server_poll.restype = ctypes.c_int32
    L.vl_server_stats_get.argtypes = [ctypes.c_void_p, P(vl_server_stats)]
    L.vl_server_stats_get.restype = ctypes.c_int32
    L.vl_server_destroy.argtypes = [ctypes.c_void_p]
    L.vl_server_destroy.restype = ctypes.c_int32
    L.vl_verify_matmul.argtypes = [P(vl_mat), P(vl_mat), P(vl_mat), P(vl_fs_init), P(vl_proof)]
    L.vl_verify_matmul.restype = ctypes.c_int32
    L.vl_prove_matmul_noalloc.argtypes = [P(vl_mat), P(vl_mat), P(vl_fs_init), P(vl_proof), ctypes.c_void_p]
    L.vl_prove_matmul_noalloc.restype = ctypes.c_int32
    L.vl_encode.argtypes = [P(vl_mat), ctypes.c_void_p, ctypes.c_void_p]
    L.vl_linear_workspace_bytes.argtypes = [P(vl_lin_job), ctypes.c_int32]
    L.vl_linear_workspace_bytes.restype = ctypes.c_size_t
    L.vl_prove_linear.argtypes = [P(vl_lin_job), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                  P(vl_lin_proof), ctypes.c_void_p]
    L.vl_prove_linear.restype = ctypes.c_int32
    L.vl_verify_linear.argtypes = [P(vl_lin_job), P(vl_lin_proof)]
    L.vl_lin_plan_create.argtypes = [P(vl_lin_job), ctypes.c_int32, P(ctypes.c_void_p)]
    L.vl_lin_plan_create.restype = ctypes.c_int32
    L.vl_lin_plan_workspace_bytes.argtypes = [ctypes.c_void_p]
    L.vl_lin_plan_workspace_bytes.restype = ctypes.c_size_t
    L.vl_lin_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                  ctypes.c_int32, ctypes.c_void_p]
    L.vl_lin_plan_run.restype = ctypes.c_int32
    L.vl_lin_plan_phase_ms.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    L.vl_lin_plan_phase_ms.restype = ctypes.c_int32
    L.vl_lin_plan_destroy.argtypes = [ctypes.c_void_p]
    L.vl_lin_plan_destroy.restype = None
    L.vl_lookup_workspace_bytes.argtypes = [P(vl_lookup_job), ctypes.c_int32]
    L.vl_lookup_workspace_bytes.restype = ctypes.c_size_t
    L.vl_lookup_plan_create.argtypes = [P(vl_lookup_job), ctypes.c_int32, P(ctypes.c_void_p)]
    L.vl_lookup_plan_create.restype = ctypes.c_int32
    L.vl_lookup_plan_workspace_bytes.argtypes = [ctypes.c_void_p]
    L.vl_lookup_plan_workspace_bytes.restype = ctypes.c_size_t
    L.vl_lookup_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_void_p]
    L.vl_lookup_plan_run.restype = ctypes.c_int32
    L.vl_lookup_plan_phase_ms.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    L.vl_lookup_plan_phase_ms.restype = ctypes.c_int32
    L.vl_lookup_plan_destroy.argtypes = [ctypes.c_void_p]
    L.vl_lookup_plan_destroy.restype = None
    L.vl_prove_lookup.argtypes = [P(vl_lookup_job), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                  P(vl_lookup_proof), ctypes.c_void_p]
    L.vl_prove_lookup.restype = ctypes.c_int32
    L.vl_verify_lookup.argtypes = [P(vl_lookup_job), P(vl_lookup_proof)]
    L.vl_verify_lookup.restype = ctypes.c_int32
    L.vl_batch_workspace_bytes.argtypes = [P(vl_job), ctypes.c_int32]
    L.vl_batch_workspace_bytes.restype = ctypes.c_size_t
    L.vl_prove_matmul_batched.argtypes = [P(vl_job), ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_size_t, P(vl_batch_proof), P(vl_fr), P(vl_fr), P(vl_fr),
                                          ctypes.c_void_p]
    L.vl_prove_matmul_batched.restype = ctypes.c_int32
    L.vl_verify_matmul_batched.argtypes = [P(vl_job), P(vl_mat), ctypes.c_int32, ctypes.c_uint64,
                                           P(vl_batch_proof), P(vl_fr), P(vl_fr), P(vl_fr)]
    L.vl_verify_matmul_batched.restype = ctypes.c_int32
    L.vl_claims_plan_create.argtypes = [P(vl_job), ctypes.c_int32, ctypes.c_uint64, P(ctypes.c_void_p)]
    L.vl_claims_plan_create.restype = ctypes.c_int32
    L.vl_claims_plan_workspace_bytes.argtypes = [ctypes.c_void_p]
    L.vl_claims_plan_workspace_bytes.restype = ctypes.c_size_t
    L.vl_claims_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p]
    L.vl_claims_plan_run.restype = ctypes.c_int32
    L.vl_claims_plan_destroy.argtypes = [ctypes.c_void_p]
    L.vl_claims_plan_destroy.restype = None
    L.vl_verify_linear.restype = ctypes.c_int32
    L.vl_encode.restype = ctypes.c_int32
    L.vl_workspace_forget.argtypes = [ctypes.c_void_p]
    L.vl_workspace_forget.restype = ctypes.c_int32
    L.vl_chain_workspace_bytes.argtypes = [P(vl_chain_job), ctypes.c_int32]
    L.vl_chain_workspace_bytes.restype = ctypes.c_size_t
    L.vl_prove_chain.argtypes = [P(vl_chain_job), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                 P(vl_chain_proof), ctypes.c_void_p]
    L.vl_prove_chain.restype = ctypes.c_int32
    L.vl_verify_chain.argtypes = [P(vl_chain_job), P(vl_mat), P(vl_mat), P(vl_mat), P(vl_mat), P(vl_chain_proof)]
    L.vl_verify_chain.restype = ctypes.c_int32
    L.vl_chain_plan_create.argtypes = [P(vl_chain_job), ctypes.c_int32, P(ctypes.c_void_p)]
    L.vl_chain_plan_create.restype = ctypes.c_int32
    L.vl_chain_plan_workspace_bytes.argtypes = [ctypes.c_void_p]
    L.vl_chain_plan_workspace_bytes.restype = ctypes.c_size_t
    L.vl_chain_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, P(vl_chain_proof),
                                    ctypes.c_void_p]
    L.vl_chain_plan_run.restype = ctypes.c_int32
    L.vl_chain_plan_destroy.argtypes = [ctypes.c_void_p]
    L.vl_chain_plan_destroy.restype = None
    _lib = L
    return L


def _check(code, what):
    if code != VL_OK:
        raise VLError(code, what)


# ------------------------------------------------------------------ helpers --

def _torch():
    import torch
    return torch


def mat(a, trans=0, dtype=None):
    """vl_mat view of a 2-D torch tensor (device or host) or NumPy array (host).

    int16 -> VL_I16, int64 -> VL_I64; a tensor/array of shape (rows, cols, 8)
    with 4-byte elements holds Montgomery field elements (VL_FR_MONT).
    Rows must be contiguous (unit column stride).
    """
    m = vl_mat()
    if isinstance(a, np.ndarray):
        if a.ndim == 3:
            assert a.shape[2] == 8 and a.dtype.itemsize == 4 and a.flags["C_CONTIGUOUS"]
            m.dtype, m.ld = VL_FR_MONT, a.shape[1]
        else:
            # a single column may report any column stride
            assert a.ndim == 2 and (a.strides[1] == a.itemsize or a.shape[1] == 1), "unit column stride required"
            m.dtype = {np.dtype(np.int16): VL_I16, np.dtype(np.int64): VL_I64}[a.dtype]
            m.ld = a.strides[0] // a.itemsize
        m.data = a.ctypes.data
        m.space = VL_HOST
    else:
        torch = _torch()
        if a.dim() == 3:
            assert a.shape[2] == 8 and a.element_size() == 4 and a.is_contiguous()
            m.dtype, m.ld = VL_FR_MONT, a.shape[1]
        else:
            assert a.dim() == 2 and (a.stride(1) == 1 or a.shape[1] == 1), "unit column stride required"
            m.dtype = {torch.int16: VL_I16, torch.int64: VL_I64}[a.dtype]
            m.ld = a.stride(0)
        m.data = a.data_ptr()
        m.space = VL_DEVICE if a.is_cuda else VL_HOST
    m.rows, m.cols = int(a.shape[0]), int(a.shape[1])
    if m.rows == 1 and m.ld < m.cols:
        m.ld = m.cols  # a size-1 dimension may report any stride
    m.trans = int(trans)
    m.reserved = 0
    if dtype is not None:
        m.dtype = dtype
    m._keep = a  # the array or tensor stays alive as long as this descriptor
    return m


def fs_init(seed, binds=None):
    f = vl_fs_init()
    f.seed = int(seed) & ((1 << 64) - 1)
    for i in range(3):
        b = bytes(32) if binds is None else bytes(binds[i])
        for j in range(32):
            f.bind[i][j] = b[j]
    return f


def job(P, Q, tp=0, tq=0, seed=0, binds=None):
    j = vl_job()
    j.P = mat(P, tp)
    j.Q = mat(Q, tq)
    j.fs = fs_init(seed, binds)
    j._keep = (P, Q)  # the operands stay alive as long as the job
    return j


def jobs_array(jobs):
    arr = (vl_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j
    return arr


def proof_bytes(p):
    """Canonical proof serialisation (same layout as the oracle's Proof.to_bytes)."""
    out = b"".join(int(x).to_bytes(4, "little") for x in (p.m, p.k, p.n, p.d0, p.d1, p.d2))
    out += bytes(p.c)
    for i in range(p.d1):
        for q in range(3):
            out += bytes(p.g[i][q])
    out += bytes(p.a_r) + bytes(p.b_r) + bytes(p.state)
    return out


def fr(x):
    """vl_fr holding the canonical residue of the integer x (negative allowed)."""
    v = vl_fr()
    x = int(x) % R_MOD
    for i in range(8):
        v.limb[i] = (x >> (32 * i)) & 0xFFFFFFFF
    return v


def lin_proof_bytes(p):
    """Linear proof serialisation (same layout as the oracle's LinearProof.to_bytes)."""
    out = b"".join(int(x).to_bytes(4, "little") for x in (p.rows, p.cols, p.d0, p.d1, p.nmats))
    return out + b"".join(bytes(p.evals[q]) for q in range(p.nmats)) + bytes(p.state)


def lin_job(mats, coeffs, seed=0, binds=None):
    """vl_lin_job for sum_q coeffs[q] * op(mats[q]) = 0.  mats: vl_mat list;
    coeffs: Python ints (reduced mod r); binds: None or one 32-byte string per
    matrix.  The returned structure keeps its arrays alive."""
    if len(mats) != len(coeffs):
        raise ValueError("one coefficient per matrix")
    j = vl_lin_job()
    j._keep = [getattr(m, "_keep", None) for m in mats]  # the operands stay alive as long as the job
    j._mats = (vl_mat * len(mats))(*mats)
    j._coeffs = (vl_fr * len(coeffs))(*[fr(c) for c in coeffs])
    j.mats = ctypes.cast(j._mats, ctypes.POINTER(vl_mat))
    j.coeffs = ctypes.cast(j._coeffs, ctypes.POINTER(vl_fr))
    j._binds = None
    if binds is not None:
        raw = b"".join(bytes(b) for b in binds)
        if len(raw) != 32 * len(mats):
            raise ValueError("one 32-byte bind per matrix")
        j._binds = ctypes.create_string_buffer(raw, len(raw))
        j.binds = ctypes.addressof(j._binds)
    j.seed = int(seed) & ((1 << 64) - 1)
    j.nmats = len(mats)
    j.reserved = 0
    return j


def lin_jobs_array(jobs):
    arr = (vl_lin_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j
    arr._keep = list(jobs)  # the copies point at the jobs' arrays
    return arr


def lookup_job(S, t0, log2_n, seed=0, bind=None):
    """vl_lookup_job: every entry of S (a vl_mat of int16, row-major) in
    [t0, t0 + 2^log2_n)."""
    j = vl_lookup_job()
    j.S = S
    j._keep = getattr(S, "_keep", None)  # the values stay alive as long as the job
    j.t0 = int(t0)
    j.log2_n = int(log2_n)
    j.reserved = 0
    j.seed = int(seed) & ((1 << 64) - 1)
    b = bytes(32) if bind is None else bytes(bind)
    for i in range(32):
        j.bind[i] = b[i]
    return j


def lookup_jobs_array(jobs):
    arr = (vl_lookup_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j
    return arr


def lookup_proof_bytes(p):
    """Lookup proof serialisation (same layout as the oracle's LookupProof.to_bytes)."""
    out = b"".join(int(x).to_bytes(4, "little") for x in (p.n, p.log2_d, p.log2_n))
    out += int(p.t0).to_bytes(8, "little", signed=True)
    for t in range(p.log2_d):
        out += b"".join(bytes(p.g[t][q]) for q in range(4))
    return out + bytes(p.a_r) + bytes(p.s_r) + bytes(p.b_r) + bytes(p.m_r) + bytes(p.state)


def _stream_ptr(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------- C ABI, by name --

def vl_version():
    return lib().vl_version()


def vl_strerror(code):
    return lib().vl_strerror(int(code)).decode()


def vl_last_error():
    return lib().vl_last_error().decode()


def vl_workspace_forget(workspace):
    """Forget which plan's tables a workspace (a device pointer) holds: True
    if a record was dropped.  Call it after writing to a workspace outside a
    plan run, or before reusing a freed buffer's address for a plan."""
    code = lib().vl_workspace_forget(workspace)
    if code < 0:
        raise VLError(-code, "vl_workspace_forget")
    return code == 1


def vl_workspace_bytes(jobs, opts=None):
    arr = jobs_array(jobs)
    return lib().vl_workspace_bytes(arr, len(jobs), ctypes.byref(opts) if opts is not None else None)


def vl_prove_matmul(P, Q, fs, workspace, workspace_bytes, stream=None):
    """Prove one product; returns a host vl_proof.  P, Q: vl_mat."""
    out = vl_proof()
    _check(lib().vl_prove_matmul(ctypes.byref(P), ctypes.byref(Q), ctypes.byref(fs), workspace,
                                 workspace_bytes, ctypes.byref(out), _stream_ptr(stream)), "vl_prove_matmul")
    return out


def vl_prove_matmul_noalloc(P, Q, fs, stream=None):
    """Prove one product of device matrices with no workspace and no device
    allocation (scratch is a fixed array inside the library); host vl_proof."""
    out = vl_proof()
    _check(lib().vl_prove_matmul_noalloc(ctypes.byref(P), ctypes.byref(Q), ctypes.byref(fs), ctypes.byref(out),
                                         _stream_ptr(stream)), "vl_prove_matmul_noalloc")
    return out


def vl_prove_batch(jobs, workspace, workspace_bytes, out=None, out_space=VL_HOST, stream=None, opts=None):
    """Prove a batch.  For VL_HOST returns the ctypes array of proofs; for
    VL_DEVICE `out` is a device pointer (int) to len(jobs) proofs."""
    arr = jobs_array(jobs)
    if out_space == VL_HOST:
        res = (vl_proof * len(jobs))()
        ptr = ctypes.addressof(res)
    else:
        res, ptr = None, int(out)
    _check(lib().vl_prove_batch(arr, len(jobs), workspace, workspace_bytes, ptr, out_space, _stream_ptr(stream),
                                ctypes.byref(opts) if opts is not None else None), "vl_prove_batch")
    return res


def vl_plan_create(jobs, opts=None):
    arr = jobs_array(jobs)
    h = ctypes.c_void_p()
    _check(lib().vl_plan_create(arr, len(jobs), ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(h)), "vl_plan_create")
    return h.value


def vl_plan_workspace_bytes(plan):
    return lib().vl_plan_workspace_bytes(plan)


def vl_plan_run(plan, workspace, workspace_bytes, out, out_space=VL_DEVICE, stream=None):
    ptr = ctypes.addressof(out) if out_space == VL_HOST else int(out)
    _check(lib().vl_plan_run(plan, workspace, workspace_bytes, ptr, out_space, _stream_ptr(stream)), "vl_plan_run")


def vl_plan_launches(plan):
    return lib().vl_plan_launches(plan)


def vl_plan_phase_ms(plan, max_runs, reset=1):
    """Per-run phase times [(clear+prologue, fold, rounds) ms, ...] of the last runs."""
    buf = (ctypes.c_float * (3 * max(max_runs, 1)))()
    n = lib().vl_plan_phase_ms(plan, buf, max_runs, reset)
    if n < 0:
        raise VLError(-n, "vl_plan_phase_ms")
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


def vl_plan_destroy(plan):
    lib().vl_plan_destroy(plan)


def vl_autotune(jobs, ws_ptr, ws_bytes, base=None, stream=None, runs=0):
    """Options for `jobs` chosen by timing candidate plans (cached per shape signature).
    Returns (vl_batch_opts, ms per run)."""
    arr = jobs_array(jobs)
    best = vl_batch_opts()
    ms = ctypes.c_float()
    _check(lib().vl_autotune(arr, len(jobs), ctypes.byref(base) if base is not None else None, ws_ptr, ws_bytes,
                             _stream_ptr(stream), runs, ctypes.byref(best), ctypes.byref(ms)), "vl_autotune")
    return best, ms.value


def vl_autotune_clear():
    lib().vl_autotune_clear()


def vl_server_create(arena_ptr, arena_bytes, max_inflight=0, max_batch_requests=0, wait_limit_us=0):
    """Start a proving server over the caller's device arena (its admission budget)."""
    o = vl_server_opts()
    o.arena = arena_ptr
    o.arena_bytes = arena_bytes
    o.max_inflight = max_inflight
    o.max_batch_requests = max_batch_requests
    o.wait_limit_us = wait_limit_us
    s = ctypes.c_void_p()
    _check(lib().vl_server_create(ctypes.byref(o), ctypes.byref(s)), "vl_server_create")
    return s


def vl_server_submit(server, jobs, out):
    """Queue one request (a list of vl_job); `out` receives len(jobs) proofs. Returns its ticket."""
    arr = jobs_array(jobs)
    t = ctypes.c_uint64()
    _check(lib().vl_server_submit(server, arr, len(jobs), out, ctypes.byref(t)), "vl_server_submit")
    return t.value


def vl_server_poll(server, max_done=1024):
    """Completed requests since the last poll: list of (ticket, status, batch,
    latency_ms, (dev_start_ms, dev_end_ms)) -- the last item is the batch's
    device interval on the GPU's clock since the server started."""
    buf = (vl_server_done * max_done)()
    n = ctypes.c_int32()
    _check(lib().vl_server_poll(server, buf, max_done, ctypes.byref(n)), "vl_server_poll")
    return [(buf[i].ticket, buf[i].status, buf[i].batch, buf[i].latency_ms, (buf[i].dev_start_ms, buf[i].dev_end_ms))
            for i in range(n.value)]


def vl_server_stats_get(server):
    st = vl_server_stats()
    _check(lib().vl_server_stats_get(server, ctypes.byref(st)), "vl_server_stats_get")
    return {k: getattr(st, k) for k, _ in vl_server_stats._fields_}


def vl_server_destroy(server):
    _check(lib().vl_server_destroy(server), "vl_server_destroy")


def vl_verify_matmul(P, Q, C, fs, proof):
    """Host verifier: True (accept) / False (reject); raises on input errors."""
    code = lib().vl_verify_matmul(ctypes.byref(P), ctypes.byref(Q), ctypes.byref(C), ctypes.byref(fs),
                                  ctypes.byref(proof))
    if code == VL_REJECT:
        return False
    _check(code, "vl_verify_matmul")
    return True


def vl_linear_workspace_bytes(jobs):
    """Workspace bytes vl_prove_linear needs for these vl_lin_job (0 if invalid)."""
    return lib().vl_linear_workspace_bytes(lin_jobs_array(jobs), len(jobs))


def vl_prove_linear(jobs, workspace, workspace_bytes, stream=None):
    """Prove a batch of linear relations; returns the ctypes array of host proofs."""
    arr = lin_jobs_array(jobs)
    out = (vl_lin_proof * len(jobs))()
    _check(lib().vl_prove_linear(arr, len(jobs), workspace, workspace_bytes, out, _stream_ptr(stream)),
           "vl_prove_linear")
    return out


class LinPlan:
    """A vl_lin_plan (keeps the jobs' arrays alive as long as the plan)."""

    def __init__(self, jobs):
        self.arr = lin_jobs_array(jobs)
        self.ptr = ctypes.c_void_p()
        _check(lib().vl_lin_plan_create(self.arr, len(jobs), ctypes.byref(self.ptr)), "vl_lin_plan_create")
        self.n = len(jobs)

    def workspace_bytes(self):
        return lib().vl_lin_plan_workspace_bytes(self.ptr)

    def run(self, workspace, workspace_bytes, out=None, out_space=VL_HOST, stream=None):
        """VL_HOST: returns the ctypes array of proofs; VL_DEVICE: `out` is a
        device pointer (int) to n proofs and the run is asynchronous."""
        if out_space == VL_HOST:
            res = (vl_lin_proof * self.n)()
            ptr = ctypes.addressof(res)
        else:
            res, ptr = None, int(out)
        _check(lib().vl_lin_plan_run(self.ptr, workspace, workspace_bytes, ptr, out_space, _stream_ptr(stream)),
               "vl_lin_plan_run")
        return res

    def phase_ms(self):
        ms = (ctypes.c_float * 3)()
        _check(lib().vl_lin_plan_phase_ms(self.ptr, ms), "vl_lin_plan_phase_ms")
        return tuple(ms)

    def destroy(self):
        if self.ptr:
            lib().vl_lin_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()


def vl_lookup_workspace_bytes(jobs):
    return lib().vl_lookup_workspace_bytes(lookup_jobs_array(jobs), len(jobs))


def vl_prove_lookup(jobs, workspace, workspace_bytes, stream=None):
    """Prove a batch of range lookups; returns the ctypes array of host proofs."""
    out = (vl_lookup_proof * len(jobs))()
    _check(lib().vl_prove_lookup(lookup_jobs_array(jobs), len(jobs), workspace, workspace_bytes, out,
                                 _stream_ptr(stream)), "vl_prove_lookup")
    return out


def vl_verify_lookup(job, proof):
    """Host verifier of a lookup proof: True / False; raises on input errors."""
    code = lib().vl_verify_lookup(ctypes.byref(job), ctypes.byref(proof))
    if code == VL_REJECT:
        return False
    _check(code, "vl_verify_lookup")
    return True


class LookupPlan:
    """A vl_lookup_plan."""

    def __init__(self, jobs):
        self.arr = lookup_jobs_array(jobs)
        self.ptr = ctypes.c_void_p()
        _check(lib().vl_lookup_plan_create(self.arr, len(jobs), ctypes.byref(self.ptr)), "vl_lookup_plan_create")
        self.n = len(jobs)

    def workspace_bytes(self):
        return lib().vl_lookup_plan_workspace_bytes(self.ptr)

    def run(self, workspace, workspace_bytes, out=None, out_space=VL_HOST, stream=None):
        if out_space == VL_HOST:
            res = (vl_lookup_proof * self.n)()
            ptr = ctypes.addressof(res)
        else:
            res, ptr = None, int(out)
        _check(lib().vl_lookup_plan_run(self.ptr, workspace, workspace_bytes, ptr, out_space, _stream_ptr(stream)),
               "vl_lookup_plan_run")
        return res

    def phase_ms(self):
        ms = (ctypes.c_float * 3)()
        _check(lib().vl_lookup_plan_phase_ms(self.ptr, ms), "vl_lookup_plan_phase_ms")
        return tuple(ms)

    def destroy(self):
        if self.ptr:
            lib().vl_lookup_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()


class BatchedProof:
    """A batched-claim proof: the vl_batch_proof and the per-product claims,
    a_i, b_i (ctypes arrays, job order)."""

    def __init__(self, K):
        self.proof = vl_batch_proof()
        self.claims = (vl_fr * K)()
        self.a = (vl_fr * K)()
        self.b = (vl_fr * K)()

    def to_bytes(self):
        """Same layout as the oracle's BatchProof.to_bytes."""
        p = self.proof
        out = b"".join(int(x).to_bytes(4, "little") for x in (p.K, p.k, p.d1))
        out += b"".join(bytes(c) for c in self.claims)
        for t in range(p.d1):
            out += b"".join(bytes(p.g[t][q]) for q in range(3))
        for x, y in zip(self.a, self.b):
            out += bytes(x) + bytes(y)
        return out + bytes(p.state)


class ClaimsPlan:
    """A vl_claims_plan (keeps its job array alive)."""

    def __init__(self, jobs, seed):
        self.arr = jobs_array(jobs)
        self.K = len(jobs)
        self.ptr = ctypes.c_void_p()
        _check(lib().vl_claims_plan_create(self.arr, self.K, int(seed) & ((1 << 64) - 1), ctypes.byref(self.ptr)),
               "vl_claims_plan_create")

    def workspace_bytes(self):
        return lib().vl_claims_plan_workspace_bytes(self.ptr)

    def run(self, workspace, workspace_bytes, stream=None, device_out=None):
        """Host outputs (a BatchedProof) by default; device_out = (proof, claims,
        a, b) device pointers for an asynchronous run."""
        if device_out is None:
            res = BatchedProof(self.K)
            ptrs = [ctypes.addressof(res.proof), ctypes.addressof(res.claims), ctypes.addressof(res.a),
                    ctypes.addressof(res.b)]
            space = VL_HOST
        else:
            res, ptrs, space = None, [int(x) for x in device_out], VL_DEVICE
        _check(lib().vl_claims_plan_run(self.ptr, workspace, workspace_bytes, *ptrs, space, _stream_ptr(stream)),
               "vl_claims_plan_run")
        return res

    def destroy(self):
        if self.ptr:
            lib().vl_claims_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()


def vl_batch_workspace_bytes(jobs):
    return lib().vl_batch_workspace_bytes(jobs_array(jobs), len(jobs))


def vl_prove_matmul_batched(jobs, seed, workspace, workspace_bytes, stream=None):
    res = BatchedProof(len(jobs))
    _check(lib().vl_prove_matmul_batched(jobs_array(jobs), len(jobs), int(seed) & ((1 << 64) - 1), workspace,
                                         workspace_bytes, ctypes.byref(res.proof), res.claims, res.a, res.b,
                                         _stream_ptr(stream)), "vl_prove_matmul_batched")
    return res


def vl_verify_matmul_batched(jobs, Cs, seed, res):
    """Host verifier: True / False; Cs are vl_mat of the claimed products."""
    cs = (vl_mat * len(Cs))(*Cs)
    code = lib().vl_verify_matmul_batched(jobs_array(jobs), cs, len(jobs), int(seed) & ((1 << 64) - 1),
                                          ctypes.byref(res.proof), res.claims, res.a, res.b)
    if code == VL_REJECT:
        return False
    _check(code, "vl_verify_matmul_batched")
    return True


def vl_verify_linear(job, proof):
    """Host verifier of a linear proof: True / False; raises on input errors."""
    code = lib().vl_verify_linear(ctypes.byref(job), ctypes.byref(proof))
    if code == VL_REJECT:
        return False
    _check(code, "vl_verify_linear")
    return True


def vl_encode(src, dst, stream=None):
    """Encode a device int16 vl_mat into dst (device pointer, rows*cols*32 bytes)."""
    _check(lib().vl_encode(ctypes.byref(src), int(dst), _stream_ptr(stream)), "vl_encode")


# ------------------------------------------------------------ chained proofs --

def chain_job(t, seed=0, binds=None):
    """vl_chain_job of one projection: t maps X, W, A, B, dY, H, dH, rhoH,
    rhodH to 2-D int16 torch tensors (device, for the prover) or NumPy arrays
    (host, for the verifier); binds: None or seven 32-byte strings."""
    j = vl_chain_job()
    j._keep = []
    for name in CHAIN_MATS:
        m = mat(t[name])
        j._keep.append(m._keep)  # the operands stay alive as long as the job
        setattr(j, name, m)
    j.seed = int(seed) & ((1 << 64) - 1)
    for i in range(7):
        b = bytes(32) if binds is None else bytes(binds[i])
        for q in range(32):
            j.bind[i][q] = b[q]
    return j


def chain_jobs_array(jobs):
    arr = (vl_chain_job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j
    arr._keep = list(jobs)
    return arr


def chain_proof_bytes(p):
    """Chained proof serialisation (same layout as the oracle's ChainProof.to_bytes)."""
    out = b"".join(int(x).to_bytes(4, "little") for x in (p.n, p.d, p.k, p.r))
    out += b"".join(proof_bytes(p.sub[i]) for i in range(VL_CHAIN_MEMBERS))
    return out + b"".join(bytes(p.e[q]) for q in range(4)) + bytes(p.state)


def vl_chain_workspace_bytes(jobs):
    return lib().vl_chain_workspace_bytes(chain_jobs_array(jobs), len(jobs))


def vl_prove_chain(jobs, workspace, workspace_bytes, stream=None):
    """Prove a batch of chained projection proofs; returns the ctypes array of host proofs."""
    out = (vl_chain_proof * len(jobs))()
    _check(lib().vl_prove_chain(chain_jobs_array(jobs), len(jobs), workspace, workspace_bytes, out,
                                _stream_ptr(stream)), "vl_prove_chain")
    return out


class ChainPlan:
    """A vl_chain_plan: the same batch of chained proofs, proved repeatedly."""

    def __init__(self, jobs):
        self._jobs = chain_jobs_array(jobs)  # keeps the operands alive
        h = ctypes.c_void_p()
        _check(lib().vl_chain_plan_create(self._jobs, len(jobs), ctypes.byref(h)), "vl_chain_plan_create")
        self.h, self.n = h.value, len(jobs)

    def workspace_bytes(self):
        return lib().vl_chain_plan_workspace_bytes(self.h)

    def run(self, workspace, workspace_bytes, stream=None):
        out = (vl_chain_proof * self.n)()
        _check(lib().vl_chain_plan_run(self.h, workspace, workspace_bytes, out, _stream_ptr(stream)),
               "vl_chain_plan_run")
        return out

    def destroy(self):
        if self.h:
            lib().vl_chain_plan_destroy(self.h)
            self.h = None


def vl_verify_chain(job, outputs, proof):
    """Host verifier of a chained proof: job with host matrices, outputs maps
    Y, dX, dA, dB to int64 NumPy arrays.  True / False; raises on input errors."""
    ms = [mat(np.ascontiguousarray(outputs[k])) for k in ("Y", "dX", "dA", "dB")]
    code = lib().vl_verify_chain(ctypes.byref(job), *[ctypes.byref(m) for m in ms], ctypes.byref(proof))
    if code == VL_REJECT:
        return False
    _check(code, "vl_verify_chain")
    return True
