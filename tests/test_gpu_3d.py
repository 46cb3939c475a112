"""Parity of the 3D CUDA path (the fsi3_* entry points of the C ABI) with the FP64 3D
oracle (oracle/fsi_nd.py at d = 3).

Tolerances as in 2D: the residual and the Jacobian are the same finite sums in another
order (1e-12 relative to the largest entry of a field; 1e-10 per field block of the
Jacobian, whose entries span ~16 decades); Newton-solved states to 1e-9 per field.

The cooperative cell routines the kernels run are also checked on the CPU: against
the oracle (tests/test_element3d_host.py) and for races with one host thread per
CUDA thread (tests/test_cta_races.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi_nd as on  # noqa: E402
from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"
FIELDS = {"v": slice(0, 3), "u": slice(3, 6), "p": slice(6, 7)}
# 5 x 2 x 3 cells (2695 dofs): levels 2695 -> 2205 -> 1715 dofs with a 2000-dof coarsest bound
TINY = wl.Workload3D("tiny3d", nx=5, ny=2, nz=3, T=0.04, n_slices=2, m_fine=2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def ctx_for(w, S, **kw):
    from paper_1907_01252_gb300 import fsi
    return fsi.Context3D(w, max_batch=S, **kw)


def oracle_mesh(w):
    return on.make_mesh_nd(w.breaks, w.segments, wl.SOLID_BOX_3D)


def state(n_nodes, seed):
    rng = np.random.default_rng(seed)
    U = np.empty((n_nodes, 7))
    U[:, 0:3] = rng.uniform(-1, 1, (n_nodes, 3))
    U[:, 3:6] = 2e-3 * rng.uniform(-1, 1, (n_nodes, 3))
    U[:, 6] = 100 * rng.uniform(-1, 1, n_nodes)
    return U


def dev(a):
    return torch.tensor(np.ascontiguousarray(a).reshape(a.shape[0], -1), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("w", [TINY, wl.SMALL3D_8x4x4], ids=lambda w: w.name)
def test_3d_residual_matches_oracle(w):
    mesh = oracle_mesh(w)
    S, k, theta = 2, 0.02, 0.52
    mat = w.material
    U = np.stack([state(mesh.n_nodes, 1 + s) for s in range(S)])
    Uo = np.stack([state(mesh.n_nodes, 11 + s) for s in range(S)])
    t_new = np.array([0.13, 0.3])
    ctx = ctx_for(w, S)
    assert ctx.n_dofs == mesh.n_dofs
    R = ctx.fsi3_residual(dev(U), dev(Uo), t_new, k, theta).cpu().numpy().reshape(S, -1, 7)
    for s in range(S):
        ref = on.StepProblemND(mesh, mat, Uo[s], t_new[s], k, theta).residual(U[s])
        scale = np.abs(ref).max(axis=0)
        assert np.all(np.abs(R[s] - ref).max(axis=0) <= 1e-12 * scale), s


def test_3d_jacobian_matches_oracle():
    import scipy.sparse as sp
    w = TINY
    mesh = oracle_mesh(w)
    U, Uo = state(mesh.n_nodes, 3), state(mesh.n_nodes, 4)
    k, theta = 0.02, 0.52
    ctx = ctx_for(w, 1)
    vals = ctx.fsi3_jacobian(dev(U[None]), dev(Uo[None]), k, theta).cpu().numpy()[0]
    rowptr, colidx = ctx.fsi3_bsr_pattern()
    A = sp.bsr_matrix((vals, colidx, rowptr), shape=(mesh.n_dofs, mesh.n_dofs)).toarray()
    ref = on.StepProblemND(mesh, w.material, Uo, 0.2, k, theta).jacobian(U).toarray()
    for ci in range(7):
        for cj in range(7):
            blk_ref, blk = ref[ci::7, cj::7], A[ci::7, cj::7]
            sc = max(np.abs(blk_ref).max(), 1e-12 * np.abs(ref).max())
            assert np.abs(blk - blk_ref).max() <= 1e-10 * sc, (ci, cj)


@pytest.fixture(scope="module")
def oracle_step():
    """The oracle's exact-Newton step from rest to t = 0.52 at full inflow."""
    w = TINY
    mesh = oracle_mesh(w)
    Uo = np.zeros((mesh.n_nodes, 7))
    model = on.FSIModelND(mesh, w.material, newton_tol=1e-12)
    return mesh, Uo, model.step(Uo, 0.5, 0.02, 0.52)


@pytest.mark.parametrize("precision,smoother,coarse_sweeps", [(0, 0, 0), (2, 0, 0), (2, 1, 0), (2, 1, 8)])
def test_3d_theta_step_matches_oracle(oracle_step, precision, smoother, coarse_sweeps):
    mesh, Uo, ref = oracle_step
    ctx = ctx_for(TINY, 2, precision=precision, mg_smoother=smoother, mg_coarse_sweeps=coarse_sweeps,
                  mg_omega=1.0 if smoother else 0.6, mg_smooth=1 if smoother else 2)
    U0 = dev(np.stack([Uo, Uo]))
    U1, st = ctx.fsi3_theta_step(U0, [0.5, 0.5], 0.02, 0.52)
    assert st["slice_status"] == [0, 0]
    got = U1.cpu().numpy().reshape(2, -1, 7)
    for s in range(2):
        for name, sl in FIELDS.items():
            err = np.abs(got[s][:, sl] - ref[:, sl]).max() / np.abs(ref[:, sl]).max()
            assert err <= 1e-9, (s, name, err)


def test_3d_parareal_with_n_iterations_is_the_fine_solution():
    """Parareal run for n_slices iterations reproduces the serial fine propagation."""
    w = TINY
    ctx = ctx_for(w, w.n_slices)
    n = ctx.n_dofs
    U = torch.zeros((w.n_slices + 1, n), dtype=torch.float64, device=DEV)
    U, st = ctx.fsi3_parareal(U, w.n_slices, 0.0)
    assert st["iterations"] == w.n_slices
    serial = torch.zeros((1, n), dtype=torch.float64, device=DEV)
    dt = w.T / w.n_slices
    for i in range(w.n_slices):
        serial, _ = ctx.fsi3_fine(serial, [i * dt])
        ref = serial[0].cpu().numpy().reshape(-1, 7)
        got = U[i + 1].cpu().numpy().reshape(-1, 7)
        for name, sl in FIELDS.items():
            den = max(np.abs(ref[:, sl]).max(), 1e-300)
            assert np.abs(got[:, sl] - ref[:, sl]).max() <= 1e-12 * den, (i, name)


def test_3d_parareal_iterate_matches_oracle():
    """One Parareal iteration (predictor sweep with C, batched fine solves, corrected
    sweep F + (C_new - C_old)) equals the oracle's iterate at every slice boundary."""
    from oracle import parareal as opr
    w = wl.Workload3D("tiny3d_pr", nx=5, ny=2, nz=3, T=0.06, n_slices=3, m_fine=1)
    mesh = oracle_mesh(w)
    model = on.FSIModelND(mesh, w.material, newton_tol=1e-12)
    dt = w.T / w.n_slices
    coarse = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, w.m_coarse, theta=1.0)  # noqa: E731
    fine = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, w.m_fine)  # noqa: E731
    U0 = np.zeros((mesh.n_nodes, 7))
    ref = opr.parareal(U0, w.n_slices, coarse, fine, 1)[1]
    # the velocities are small at these early times (max 0.07), so the GPU solves its Newton
    # systems to the oracle's 1e-12 too (the tolerance is absolute below a unit residual)
    ctx = ctx_for(w, w.n_slices, newton_tol=1e-12)
    U = torch.zeros((w.n_slices + 1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    U, st = ctx.fsi3_parareal(U, 1, 0.0)
    assert st["iterations"] == 1
    for i in range(1, w.n_slices + 1):
        got = U[i].cpu().numpy().reshape(-1, 7)
        for name, sl in FIELDS.items():
            den = max(np.abs(ref[i][:, sl]).max(), 1e-300)
            assert np.abs(got[:, sl] - ref[i][:, sl]).max() <= 1e-9 * den, (i, name)


def test_3d_failures_are_reported_per_slice():
    """A non-finite state in one slice ends that slice with FSI_ENAN (per-slice status) while
    the other slice completes; a batch larger than max_batch is rejected with FSI_EINVAL."""
    from paper_1907_01252_gb300 import fsi
    ctx = ctx_for(TINY, 2)
    U = torch.zeros((2, ctx.n_dofs), dtype=torch.float64, device=DEV)
    U[1, 7 * (5 + 11 * (2 + 5 * 3)) + 6] = float("nan")   # the pressure of an interior node (i, j, k) = (5, 2, 3)
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi3_theta_step(U, [0.0, 0.0], 0.01, 0.51)
    assert e.value.code == fsi.FSI_ENAN
    assert e.value.slice_status == [0, fsi.FSI_ENAN]
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi3_theta_step(torch.zeros((3, ctx.n_dofs), dtype=torch.float64, device=DEV), [0.0] * 3, 0.01, 0.51)
    assert e.value.code == fsi.FSI_EINVAL
