"""The ctypes mirrors of the C ABI structs (paper_1907_01252_gb300/fsi.py) against the
header itself: include/fsi.h compiled with the system C compiler reports the size of
every struct and the offset of every field, which must equal the ctypes layout (a
field added on one side only would shift everything after it)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1907_01252_gb300 import fsi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["fsi_mesh", "fsi_params", "fsi_stats", "fsi_parareal_stats", "fsi_mesh3d", "fsi_instance"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fsi.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in getattr(fsi, name)._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_mirror_matches_the_header(c_layout, name):
    cls = getattr(fsi, name)
    assert c_layout[(name, "size")] == C.sizeof(cls)
    for field, _ in cls._fields_:
        assert c_layout[(name, field)] == getattr(cls, field).offset, field
