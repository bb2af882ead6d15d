"""The Python binding's ctypes structures have the C header's layout: every field at the
offset, and every structure of the size, that a C compiler gives include/dlx.h (compiled
here with gcc), so a binding that drifts from the header fails here, not inside a call."""

import ctypes as C
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]

# C typedef name -> ctypes class name in paper_2406_08703_gb300._native
STRUCTS = {
    "dlx_mft_desc": "MftDesc",
    "dlx_params": "Params",
    "dlx_grads": "Grads",
    "dlx_plan_info": "PlanInfo",
    "dlx_kernel_times": "KernelTimes",
    "dlx_request": "Request",
    "dlx_result": "Result",
    "dlx_server_stats": "ServerStats",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_2406_08703_gb300 import _native as N

    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dlx.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in getattr(N, pyname)._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0; }"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lay = {}
    for ln in out.splitlines():
        s, f, v = ln.split()
        lay[(s, f)] = int(v)
    return lay


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    from paper_2406_08703_gb300 import _native as N

    cls = getattr(N, STRUCTS[cname])
    assert C.sizeof(cls) == c_layout[(cname, "sizeof")], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c_layout[(cname, f)], (cname, f)
