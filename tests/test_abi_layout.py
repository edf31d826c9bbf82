"""The ctypes structures of the Python binding have the layout of the C
structures in include/hfp.h: every field at the same offset, every structure
of the same size (CPU only: a small C program compiled with gcc prints the
header's sizeof/offsetof)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# binding structure -> header typedef
PAIRS = {
    "_Hypergraph": "hfp_hypergraph",
    "_NetInfo": "hfp_net_info",
    "_Stats": "hfp_stats",
    "Tuning": "hfp_tuning",
    "RefineParams": "hfp_refine_params",
    "PairResult": "hfp_pair_result",
    "RoundStats": "hfp_round_stats",
    "AdamParams": "hfp_adam_params",
    "_NetworkView": "hfp_flow_network_view",
    "FcParams": "hfp_fc_params",
    "_FcResult": "hfp_fc_result",
    "_FcTask": "hfp_fc_task",
}


def _c_layout(hfp):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hfp.h"', "int main(void) {"]
    for py, c in PAIRS.items():
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(hfp, py)._fields_:
            lines.append(f'  printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        r = subprocess.run([cc, "-std=c11", "-I" + os.path.join(ROOT, "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, "the header lacks a field the binding names:\n" + r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        py, name, val = line.split()
        layout[(py, name)] = int(val)
    return layout


def test_binding_structs_match_the_header():
    from paper_2201_01556_gb300 import hfp
    layout = _c_layout(hfp)
    for py in PAIRS:
        cls = getattr(hfp, py)
        assert ctypes.sizeof(cls) == layout[(py, "size")], f"{py}: size"
        for name, _ in cls._fields_:
            assert getattr(cls, name).offset == layout[(py, name)], f"{py}.{name}: offset"
