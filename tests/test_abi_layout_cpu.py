"""The ctypes binding's structures have the C ABI's layout: every field of bilu_params,
sqmr_info, gmres_info, bilu_stats_t and bilu_mlp_train_cfg at the offset the C compiler gives it
(include/bilu.h compiled as plain C with gcc), and the same total size."""
import ctypes as ct
import os
import shutil
import subprocess

import pytest

import paper_1908_10169_gb300 as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["bilu_params", "sqmr_info", "gmres_info", "bilu_stats_t", "bilu_mlp_train_cfg"]


def test_struct_layouts_match_the_header(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "bilu.h"', "int main(void) {"]
    for name in STRUCTS:
        py = getattr(B, name)
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for name in STRUCTS:
        py = getattr(B, name)
        assert got[(name, "size")] == ct.sizeof(py), name
        for field, _ in py._fields_:
            assert got[(name, field)] == getattr(py, field).offset, (name, field)
