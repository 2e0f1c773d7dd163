"""The ctypes structures of the binding have the layout of the C header's.

A small C program compiled with gcc against include/gridspt.h prints the size
and field offsets of gridspt_desc, gridspt_cosmo and gridspt_kernel_stat; the
binding's ctypes definitions must agree field by field (a mismatch would pass
wrong plan parameters silently). Host only, no GPU.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "gridspt_desc": ("GridsptDesc", ["n", "n_max", "batch", "form", "box", "kcut_lin", "kcut_nl", "truncate",
                                     "accum"]),
    "gridspt_cosmo": ("GridsptCosmo", ["omega_m", "h", "n_s", "sigma8", "gamma"]),
    "gridspt_kernel_stat": ("GridsptKernelStat", ["name", "launches", "reserved", "ms", "bytes"]),
}


def _c_layout(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gridspt.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        layout[(cname, key)] = int(val)
    return layout


def test_binding_structures_match_the_header(tmp_path):
    from paper_1807_04215_gb300 import _lib
    layout = _c_layout(tmp_path)
    for cname, (pyname, fields) in STRUCTS.items():
        cls = getattr(_lib, pyname)
        assert [f[0] for f in cls._fields_] == fields, cname
        assert ctypes.sizeof(cls) == layout[(cname, "size")], cname
        for f in fields:
            assert getattr(cls, f).offset == layout[(cname, f)], (cname, f)
