"""The no-allocation entry point's fixed scratch array holds any single
product of the benchmark's LoRA projections (7B-shaped at seq 512 and 1024,
ranks 8, 16, 64; 13B-shaped at seq 2048, rank 16), in every orientation the
step uses: the scratch it needs (the workspace of a one-job plan with the
launch options that entry point uses, device operands, so no staging) is at
most VL_NOALLOC_SCRATCH_BYTES.  Host-side plan sizing only: no GPU."""
import ctypes

import pytest

from paper_2508_21393_gb300 import binding as B

SPEC = {"F1": ("X", "W", 0, 0), "F2": ("X", "A", 0, 0), "F3": ("H", "B", 0, 0), "B1": ("dY", "B", 0, 1),
        "B2": ("H", "dY", 1, 0), "B3": ("X", "dH", 1, 0), "B4": ("dY", "W", 0, 1), "B5": ("dH", "A", 0, 1)}


def _dmat(rows, cols, trans):
    m = B.vl_mat()
    m.data = 1 << 20  # a device address is never dereferenced by the sizing
    m.rows, m.cols, m.ld = rows, cols, cols
    m.dtype, m.trans, m.space, m.reserved = B.VL_I16, trans, B.VL_DEVICE, 0
    return m


@pytest.mark.parametrize("n,d,k,r", [(512, 4096, 4096, 8), (512, 4096, 4096, 16), (512, 4096, 4096, 64),
                                     (1024, 4096, 4096, 16), (2048, 5120, 5120, 16)])
def test_every_projection_product_fits_the_scratch_array(n, d, k, r):
    shapes = {"X": (n, d), "W": (d, k), "A": (d, r), "B": (r, k), "dY": (n, k), "H": (n, r), "dH": (n, r)}
    o = B.vl_batch_opts()
    o.persistent, o.fold_engine = 2, 1  # phase launches, CUDA-core fold: what the entry point runs
    for name, (p, q, tp, tq) in SPEC.items():
        j = B.vl_job()
        j.P, j.Q, j.fs = _dmat(*shapes[p], tp), _dmat(*shapes[q], tq), B.fs_init(1)
        need = B.lib().vl_workspace_bytes(ctypes.byref(j), 1, ctypes.byref(o))
        assert 0 < need <= B.VL_NOALLOC_SCRATCH_BYTES, (name, need)
