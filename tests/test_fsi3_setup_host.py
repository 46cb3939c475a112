"""Host-side checks of the 3D entry points that need no GPU: fsi3_setup rejects bad
meshes and parameters with FSI_EINVAL (and a message) before it touches the device."""
import ctypes as C

import numpy as np
import pytest

from paper_1907_01252_gb300 import workloads as wl


@pytest.fixture(scope="module")
def fsi():
    from paper_1907_01252_gb300 import build, fsi as f
    build.build_library()
    f.load_library()
    return f


def try_setup(fsi, w, **overrides):
    mesh, keep = fsi._mesh3d_struct(w)
    base = wl.Workload("3d", nx=1, ny=1, T=w.T, n_slices=w.n_slices, m_fine=w.m_fine)
    p = fsi._params(base, 2, dict(dict(mg_coarsest_max_dofs=2000, precision=2), **overrides))
    prm = fsi.fsi_params(**p)
    h = C.c_void_p()
    rc = fsi.load_library().fsi3_setup(C.byref(mesh), C.byref(prm), C.byref(h))
    return rc, fsi.load_library().fsi_last_error().decode(), h


@pytest.mark.parametrize("overrides,msg", [
    (dict(precision=1), "precision"),
    (dict(gmres_restart=64), "gmres_restart"),
    (dict(mg_smoother=2), "mg_smoother"),
    (dict(max_batch=0), "invalid"),
    (dict(newton_tol=0.0), "invalid"),
    (dict(mg_coarse_sweeps=-1), "mg_coarse_sweeps"),
])
def test_fsi3_setup_rejects_bad_parameters(fsi, overrides, msg):
    rc, err, h = try_setup(fsi, wl.SMALL3D_8x4x4, **overrides)
    assert rc == fsi.FSI_EINVAL and msg in err and not h.value


def test_fsi3_setup_needs_a_coarser_level(fsi):
    """3 x 2 x 3 cells is the coarsest interface-fitted mesh of the channel (one cell
    per segment): 1715 dofs, nothing to coarsen, so no multigrid hierarchy."""
    w = wl.Workload3D("min", nx=3, ny=2, nz=3, T=1.0, n_slices=2, m_fine=2)
    assert w.segments == ((1, 1, 1), (1, 1), (1, 1, 1))
    rc, err, h = try_setup(fsi, w, mg_coarsest_max_dofs=1000)
    assert rc == fsi.FSI_EINVAL and "coarser level" in err


def test_fsi3_setup_rejects_a_bad_mesh(fsi):
    mesh, keep = fsi._mesh3d_struct(wl.SMALL3D_8x4x4)
    bad = (C.c_int * 3)(2, 0, 5)   # a segment without cells
    mesh.nx_seg = bad
    prm = fsi.fsi_params(**fsi._params(wl.SMALL_16x4, 1, {}))
    h = C.c_void_p()
    rc = fsi.load_library().fsi3_setup(C.byref(mesh), C.byref(prm), C.byref(h))
    assert rc == fsi.FSI_EINVAL and "segment" in fsi.load_library().fsi_last_error().decode()


def test_fsi3_launch_accounting_on_the_host(fsi):
    """The 3D kernel table and its accounting work without a device: every 3D kernel has a
    name, nothing ran in this process, and enabling and reading records is harmless."""
    names = fsi.kernel_names3()
    assert len(names) == len(set(names)) and all(n.startswith("k3_") for n in names)
    assert {"k3_cell_jacobian", "k3_vanka_apply", "k3_vanka_setup", "k3_spmv"} <= set(names)
    assert fsi.launch_count3() == 0
    fsi.profile3(True)
    assert all(v == (0.0, 0) for v in fsi.profile3_read().values())
    fsi.profile3(False)
    lib = fsi.load_library()
    assert lib.fsi3_kernel_name(len(names)) is None and lib.fsi3_launch_count(len(names)) == -1
    ms, n = C.c_double(), C.c_longlong()
    assert lib.fsi3_profile_read(-1, C.byref(ms), C.byref(n)) == fsi.FSI_EINVAL
