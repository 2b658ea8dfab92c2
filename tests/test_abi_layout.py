"""The C ABI's structs as the ctypes binding lays them out.

A small C program, compiled against include/ei.h with the host C compiler,
prints sizeof of each struct the binding mirrors (ei_options, ei_stats,
ei_mlp_decision, ei_batch_problem, ei_batch_stats) and offsetof of every one
of its fields.  The binding's ctypes structures must agree field by field:
a field added, removed or retyped on one side only fails here instead of
shifting every later field silently.  Host code only: no GPU.
"""
import ctypes as C
import shutil
import subprocess
from pathlib import Path

import pytest

from paper_1309_4616_gb300 import ei

STRUCTS = [
    ("ei_options", ei.Options),
    ("ei_stats", ei.Stats),
    ("ei_mlp_decision", ei.MlpDecision),
    ("ei_batch_problem", ei.BatchProblem),
    ("ei_batch_stats", ei.BatchStats),
]


def _c_layout(tmp_path, repo_root):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ei.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", str(repo_root / "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        layout[(cname, field)] = int(value)
    return layout


def test_struct_layouts_match_header(tmp_path):
    layout = _c_layout(tmp_path, Path(__file__).resolve().parents[1])
    for cname, cls in STRUCTS:
        assert layout[(cname, "sizeof")] == C.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert layout[(cname, field)] == getattr(cls, field).offset, (cname, field)
