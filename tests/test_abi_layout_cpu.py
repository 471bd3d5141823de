"""The ctypes structures of the binding match the C header: the header is
compiled as C by gcc into a tiny program that prints every structure's size
and every field's offset, and the binding's ctypes layout must agree.  (The
binding is argument marshalling only, so a layout mismatch would silently
corrupt every call.)"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2508_21393_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["vl_fr", "vl_mat", "vl_fs_init", "vl_proof", "vl_job", "vl_batch_opts", "vl_lin_job", "vl_lin_proof",
           "vl_lookup_job", "vl_lookup_proof", "vl_batch_proof", "vl_server_opts", "vl_server_done",
           "vl_server_stats", "vl_chain_job", "vl_chain_proof"]


def _ctypes_layout():
    out = {}
    for name in STRUCTS:
        cls = getattr(B, name)
        out[name] = (ctypes.sizeof(cls), {f[0]: getattr(cls, f[0]).offset for f in cls._fields_})
    return out


def test_binding_structs_match_the_header(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    layout = _ctypes_layout()
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "verilora.h"', "int main(void) {"]
    for name, (_, fields) in layout.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in res:
        if not line:
            continue
        name, field, value = line.split()
        want = int(value)
        got = layout[name][0] if field == "size" else layout[name][1][field]
        assert got == want, f"{name}.{field}: ctypes {got}, C {want}"
        seen += 1
    assert seen == sum(1 + len(f) for _, f in layout.values())
