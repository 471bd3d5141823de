"""No C++ exception crosses the C ABI: a host allocation that fails inside
the library comes back as VL_ENOMEM with a message, and the process goes on.

A child process caps its address space just above what it uses, then asks
the host lookup verifier to check a 2^24-entry statement (its index table
alone needs 64 MB).  Without the guard, std::bad_alloc would unwind into the
C caller and abort the process."""
import os
import subprocess
import sys

import pytest

from paper_2508_21393_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, resource, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_2508_21393_gb300 import binding as B
L = B.lib()
S = np.zeros((4096, 4096), np.int16)
job = B.lookup_job(B.mat(S), 0, 8, 0)
p = B.vl_lookup_proof()
p.n, p.log2_d, p.log2_n, p.t0, p.status = S.size, 24, 8, 0, 0
vm = next(int(l.split()[1]) for l in open("/proc/self/status") if l.startswith("VmSize")) * 1024
hard = resource.getrlimit(resource.RLIMIT_AS)[1]
resource.setrlimit(resource.RLIMIT_AS, (vm + (16 << 20), hard))
code = L.vl_verify_lookup(ctypes.byref(job), ctypes.byref(p))
msg = L.vl_last_error().decode()
resource.setrlimit(resource.RLIMIT_AS, (hard, hard))
print(code, msg)
"""


@pytest.mark.skipif(not sys.platform.startswith("linux"), reason="needs RLIMIT_AS and /proc")
def test_failed_host_allocation_returns_enomem():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    res = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr[-2000:]
    code, msg = res.stdout.strip().split(" ", 1)
    assert int(code) == B.VL_ENOMEM
    assert msg == "host memory allocation failed"
