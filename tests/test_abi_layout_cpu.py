"""The ctypes mirrors of the C ABI structs match include/micropolar.h.

A small C program, generated from the binding's field lists, is compiled
against the header with the host compiler and prints sizeof / offsetof of
every struct and field; a field the header lacks fails to compile, a field
at another offset or a struct of another size fails the comparison.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["mp_phase", "mp_problem", "mp_result", "mp_alloc", "mp_batch_stats", "mp_server_opts",
           "mp_server_stats"]
C_NAME = {"lambda_": "lambda"}  # Python keyword renamed in the binding


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__._build_module().build()  # the binding loads the library on import
    from paper_2409_10774_gb300 import binding
    return binding


def _fields(B, name):
    return [f[0] for f in getattr(B, name)._fields_]


@pytest.fixture(scope="module")
def c_layout(B, tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "micropolar.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f in _fields(B, s):
            cf = C_NAME.get(f, f)
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {cf}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, k, v = line.split()
        table[(s, k)] = int(v)
    return table


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_layout_matches_header(B, c_layout, name):
    st = getattr(B, name)
    assert C.sizeof(st) == c_layout[(name, "size")], name
    for f in _fields(B, name):
        assert getattr(st, f).offset == c_layout[(name, f)], (name, f)
