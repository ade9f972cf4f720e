"""The ctypes structures of the Python binding have the same layout as the C
structures of include/sfhk.h: a small C program compiled against the header
prints sizeof and the offset of every field, and both must agree with ctypes.
A field appended on one side only would otherwise shift every later field
silently."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2608_13686_b300 import sfhk as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# ctypes names that differ from the C ones (Python keywords)
C_NAME = {"yield_": "yield"}
STRUCTS = ["sfhk_target_desc", "sfhk_pulse_desc", "sfhk_align_desc", "sfhk_run_opts",
           "sfhk_stats", "sfhk_server_opts", "sfhk_request", "sfhk_result",
           "sfhk_server_stats"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sfhk.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'printf("{name} . %zu\\n", sizeof({name}));')
        for field, _ in getattr(S, name)._fields_:
            cf = C_NAME.get(field, field)
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {cf}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines))
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for ln in out.splitlines():
        name, field, value = ln.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_layout_matches_the_header(c_layout, name):
    cls = getattr(S, name)
    assert C.sizeof(cls) == c_layout[(name, ".")], name
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], (name, field)
