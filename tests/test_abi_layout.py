"""The Python binding's ctypes structures match the C structures of
include/cs_omp.h field by field (offsets and sizes as a C compiler lays them
out), so parameters cross the boundary unchanged."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "cs_omp_params": ("OmpParams", ["k", "tol", "max_iter", "prec", "topc"]),
    "cs_clomp_params": ("ClompParams", ["base", "steps", "lr", "beta1", "beta2", "eps",
                                        "reset_adam_each_iter", "form", "select_threshold", "tv_weight",
                                        "tv_D", "tv_N", "tv_ldd", "image_width", "lv_weight", "lv_eps"]),
    "cs_iht_params": ("IhtParams", ["k", "tol", "max_iter", "step"]),
    "cs_instance": ("Instance", ["A", "m", "n", "lda", "y", "k", "support", "coef", "n_iter", "res_norm",
                                 "sig_status"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cs_omp.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields or []:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0;\n}")
    src = d / "layout.c"
    src.write_text("\n".join(lines))
    exe = d / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    return {line.rsplit(" ", 1)[0]: int(line.rsplit(" ", 1)[1]) for line in out.splitlines()}


def test_struct_layouts_match(c_layout):
    import paper_2501_11592_gb300 as cs
    for cname, (pyname, fields) in STRUCTS.items():
        py = getattr(cs, pyname)
        assert [f[0] for f in py._fields_] == fields, f"{pyname} fields differ from the checked list"
        assert ctypes.sizeof(py) == c_layout[f"{cname} size"], cname
        for f in fields or []:
            assert getattr(py, f).offset == c_layout[f"{cname}.{f}"], f"{cname}.{f}"
