"""The ctypes mirrors of the C-ABI structs (paper_2507_04115_gb300/tdse.py) against include/tdse.h
(no GPU): a C program compiled with the host compiler prints every struct's size and every field's
offset, which must equal ctypes' layout of the same fields."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_struct_layouts_match_the_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_2507_04115_gb300 import tdse
    structs = [tdse.tdse_instance, tdse.tdse_absorber, tdse.tdse_plan_info, tdse.tdse_pipe_rates,
               tdse.tdse_tune_trial]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tdse.h"', "int main(void) {"]
    want = []
    for S in structs:
        name = S.__name__
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (name, name))
        want.append("%s %d" % (name, ctypes.sizeof(S)))
        for fname, _ in S._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (name, fname, name, fname))
            want.append("%s.%s %d" % (name, fname, getattr(S, fname).offset))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    assert [g for g in got if g] == want
