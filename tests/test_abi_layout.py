"""The ctypes structures of the binding have the layout of the C header:
every field at the offset a C compiler gives it, and the same sizes (a plain C
program compiled against include/tsvd.h prints them)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2208_08410_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [B.tsvd_matrix, B.tsvd_options, B.tsvd_report, B.tsvd_server_options, B.tsvd_request_info,
           B.tsvd_server_stats]


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tsvd.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for st in STRUCTS:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
