"""A plain C program uses the library through the C ABI alone: it includes
include/verilora.h, links libverilora.so with gcc (no Python, no torch), and
calls the host-only entry points.  It verifies a matmul proof that the oracle
made (written to a file as a vl_proof struct), rejects the same proof with
one bit of c flipped, sizes a workspace, and gets VL_EINVAL from the prover
for a missing operand before any CUDA call."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "verilora.h"

static void* slurp(const char* dir, const char* name, size_t bytes) {
  char path[4096];
  snprintf(path, sizeof(path), "%s/%s", dir, name);
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  void* p = malloc(bytes);
  if (p && fread(p, 1, bytes, f) != bytes) {
    free(p);
    p = NULL;
  }
  fclose(f);
  return p;
}

int main(int argc, char** argv) {
  if (argc != 6) return 2;
  const char* dir = argv[1];
  const int64_t m = atoll(argv[2]), k = atoll(argv[3]), n = atoll(argv[4]);
  int16_t* P = slurp(dir, "P.bin", (size_t)(m * k) * 2);
  int16_t* Q = slurp(dir, "Q.bin", (size_t)(k * n) * 2);
  int64_t* C = slurp(dir, "C.bin", (size_t)(m * n) * 8);
  vl_proof* proof = slurp(dir, "proof.bin", sizeof(vl_proof));
  if (!P || !Q || !C || !proof) return 3;
  vl_mat mp = {P, m, k, k, VL_I16, 0, VL_HOST, 0};
  vl_mat mq = {Q, k, n, n, VL_I16, 0, VL_HOST, 0};
  vl_mat mc = {C, m, n, n, VL_I64, 0, VL_HOST, 0};
  vl_fs_init fs;
  memset(&fs, 0, sizeof(fs));
  fs.seed = strtoull(argv[5], NULL, 10);
  const int32_t accept = vl_verify_matmul(&mp, &mq, &mc, &fs, proof);
  proof->c.limb[0] ^= 1u;
  const int32_t flipped = vl_verify_matmul(&mp, &mq, &mc, &fs, proof);
  vl_job job;
  job.P = mp;
  job.Q = mq;
  job.fs = fs;
  const size_t ws = vl_workspace_bytes(&job, 1, NULL);
  const int32_t missing = vl_prove_matmul(NULL, &mq, &fs, NULL, 0, proof, NULL);
  printf("%d %d %d %d %d %s\n", vl_version(), accept, flipped, ws > 0 ? 1 : 0, missing, vl_strerror(flipped));
  free(P);
  free(Q);
  free(C);
  free(proof);
  return 0;
}
"""


def _vl_proof(pf):
    out = B.vl_proof()
    out.m, out.k, out.n, out.d0, out.d1, out.d2 = pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2
    out.status = 0
    out.c = B.fr(pf.c)
    for i, tri in enumerate(pf.g):
        for q in range(3):
            out.g[i][q] = B.fr(tri[q])
    out.a_r, out.b_r = B.fr(pf.a_r), B.fr(pf.b_r)
    for i in range(32):
        out.state[i] = pf.state[i]
    return out


def test_c_program_verifies_through_the_abi(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    libdir = os.path.dirname(B.LIB_PATH)
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lverilora", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    rng = np.random.default_rng(31)
    m, k, n, seed = 6, 19, 5, 77
    P = rng.integers(-(1 << 15), 1 << 15, size=(m, k)).astype(np.int16)
    Q = rng.integers(-(1 << 15), 1 << 15, size=(k, n)).astype(np.int16)
    C = W.exact_matmul(P, Q).astype(np.int64)
    pf = oracle.prove_matmul(P, Q, 0, 0, seed=seed)
    vp = _vl_proof(pf)
    assert B.proof_bytes(vp) == pf.to_bytes()
    (tmp_path / "P.bin").write_bytes(P.tobytes())
    (tmp_path / "Q.bin").write_bytes(Q.tobytes())
    (tmp_path / "C.bin").write_bytes(C.tobytes())
    (tmp_path / "proof.bin").write_bytes(bytes(vp))
    res = subprocess.run([str(exe), str(tmp_path), str(m), str(k), str(n), str(seed)], capture_output=True,
                         text=True, check=True)
    version, accept, flipped, sized, missing, msg = res.stdout.split(maxsplit=5)
    assert int(version) == B.vl_version()
    assert int(accept) == B.VL_OK
    assert int(flipped) == B.VL_REJECT and msg.strip() == "proof rejected"
    assert int(sized) == 1
    assert int(missing) == B.VL_EINVAL
