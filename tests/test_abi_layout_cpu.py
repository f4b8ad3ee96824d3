"""The Python binding's ctypes structures have the layout of the C header's
structs: a small C program compiled against include/pmf.h prints sizeof and
offsetof of every field, which must equal the ctypes figures (a field added
on one side only, or in another order, shifts every later offset)."""
import os
import shutil
import subprocess

import pytest

from paper_1105_4840_gb300 import pmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "pmf_system_desc": pmf.SystemDesc,
    "pmf_run_params": pmf.RunParams,
    "pmf_batch_item": pmf.BatchItem,
    "pmf_hist_params": pmf.HistParams,
    "pmf_run_info": pmf.RunInfo,
    "pmf_free_energy_result": pmf.FreeEnergyResult,
    "pmf_adaptive_trace": pmf.AdaptiveTrace,
    "pmf_adaptive_params": pmf.AdaptiveParams,
    "pmf_adaptive_info": pmf.AdaptiveInfo,
}


def _c_name(field):
    return "lambda" if field == "lambda_" else field


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pmf.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {_c_name(f)}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        s, f, v = line.split()
        layout[(s, f)] = int(v)
    return layout


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_layout_matches_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert c_layout[(cname, "sizeof")] == pmf.C.sizeof(cls)
    for f, _ in cls._fields_:
        assert c_layout[(cname, f)] == getattr(cls, f).offset, (cname, f)
