"""The C-ABI library builds, loads and exports every symbol include/fsi.h declares (CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    pat = r"^\s*(?:const\s+)?(?:unsigned\s+|long\s+)*[a-z_]+\s*\*?\s*((?:fsi|fsi3|fsi3d)_\w+|parareal_\w+)\s*\("
    return sorted(set(re.findall(pat, src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("fsi_setup", "fsi_fine", "fsi_coarse", "parareal_iterate", "fsi_destroy", "fsi_last_error",
              "fsi_launch_count", "fsi3_setup", "fsi3_theta_step", "fsi3_parareal", "fsi3_launch_count",
              "fsi3d_mesh_size"):
        assert n in names, n


def test_library_loads_and_exports_all_symbols():
    from paper_1907_01252_gb300 import build, fsi
    path = build.build_library()
    lib = fsi.load_library(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in fsi.SIGNATURES, name
    # no compute call here: the error path needs no GPU
    assert lib.fsi_setup(None, None, None) == fsi.FSI_EINVAL
    assert b"null" in lib.fsi_last_error()
