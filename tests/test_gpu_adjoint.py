"""Discrete adjoint on the GPU (through the C ABI) against the FP64 oracle's
adjoint and against central differences of the GPU functional."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as oa  # noqa: E402
from oracle import fsi as of  # noqa: E402
from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def small_case():
    # 8 x 2 mesh, fine step 1/200 (T = 0.04, 2 slices x 4 steps)
    w = wl.Workload("adj", nx=8, ny=2, T=0.04, n_slices=2, m_fine=4, newton_tol=1e-13)
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    model = of.FSIModel(mesh, w.material, newton_tol=1e-13)
    k = w.k_fine
    Us = oa.trajectory(model, np.zeros((mesh.n_nodes, 5)), 0.0, k, 3)
    return w, mesh, model, k, Us


def test_old_state_jacobian_matches_oracle():
    from paper_1907_01252_gb300 import fsi
    w, mesh, model, k, Us = small_case()
    ctx = fsi.Context(w, max_batch=1)
    U = torch.tensor(Us[3].reshape(1, -1), device=DEV)
    Uo = torch.tensor(Us[2].reshape(1, -1), device=DEV)
    vals = ctx.fsi_jacobian_old(U, Uo, k, 0.5 + k).cpu().numpy()
    rowptr, colidx = ctx.fsi_bsr_pattern()
    import scipy.sparse as sp
    B = sp.bsr_matrix((vals[0], colidx, rowptr), shape=(mesh.n_dofs, mesh.n_dofs)).toarray()
    ref = oa.old_state_jacobian(mesh, model.tab, w.material, Us[3], Us[2], 3 * k, k, 0.5 + k).toarray()
    assert np.abs(B - ref).max() <= 1e-12 * np.abs(ref).max()


def test_adjoint_gradient_matches_oracle_and_finite_differences():
    from paper_1907_01252_gb300 import fsi
    w, mesh, model, k, Us = small_case()
    tip = oa.tip_node(mesh, wl.SOLID_BOX)
    M = 6                                  # two checkpointed slices (4 + 2 steps)
    J_ref, g_ref = oa.adjoint_gradient(model, Us[3], 3 * k, k, M, tip)
    # central differences of J need forward solves converged to round-off: every
    # Newton correction is solved exactly (no inexact-Newton forcing)
    ctx = fsi.Context(w, max_batch=1, newton_eta=0.0)
    U0 = torch.tensor(Us[3].ravel(), device=DEV)
    J, g, _ = ctx.fsi_adjoint(U0, 3 * k, M)
    assert J == pytest.approx(J_ref, rel=1e-9)
    for i in range(3):
        assert g[i] == pytest.approx(g_ref[i], rel=1e-8), i
    # central differences of the GPU functional (h = 1e-4 relative)
    m = w.material
    base = [m.mu_s, m.lambda_s, m.vbar]
    for i in range(3):
        vals = []
        for sgn in (1, -1):
            p = list(base)
            p[i] += sgn * 1e-4 * base[i]
            ctx.fsi_set_material(*p)
            vals.append(ctx.fsi_adjoint(U0, 3 * k, M)[0])
        ctx.fsi_set_material(*base)
        fd = (vals[0] - vals[1]) / (2e-4 * base[i])
        assert abs(g[i] - fd) <= 1e-6 * abs(fd), (i, g[i], fd)
    # the autograd wrapper returns the same gradient
    fn = fsi.tip_functional(ctx, U0, 3 * k, M)
    params = torch.tensor(base, dtype=torch.float64, requires_grad=True)
    Jt = fn(params)
    Jt.backward()
    assert Jt.item() == pytest.approx(J, rel=1e-14)
    assert np.allclose(params.grad.numpy(), g, rtol=1e-14, atol=0)


def test_adjoint_gradient_on_the_16x4_workload_matches_finite_differences():
    """Beyond the toy mesh: the 16 x 4 workload's mesh and fine step (k = 1/128),
    from a developed state (an oracle implicit-Euler step from rest to t = 0.25,
    the inflow at full strength), 32 fine steps in two checkpointed slices; the
    gradient against central differences of the GPU functional at h = 1e-4
    relative, with every Newton system solved to 1e-12 and exact linear solves
    (a difference quotient needs forward solves converged to round-off)."""
    from paper_1907_01252_gb300 import fsi
    import dataclasses
    w = dataclasses.replace(wl.SMALL_16x4, newton_tol=1e-12)
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    model = of.FSIModel(mesh, w.material, newton_tol=1e-12)
    U_dev = model.step(np.zeros((mesh.n_nodes, 5)), 0.15, 0.1, 1.0)
    k = w.k_fine
    M = 2 * w.m_fine
    ctx = fsi.Context(w, max_batch=1, newton_eta=0.0)
    U0 = torch.tensor(U_dev.ravel(), device=DEV)
    J, g, _ = ctx.fsi_adjoint(U0, 0.25, M)
    assert J > 0.0
    m = w.material
    base = [m.mu_s, m.lambda_s, m.vbar]
    for i in range(3):
        vals = []
        for sgn in (1, -1):
            p = list(base)
            p[i] += sgn * 1e-4 * base[i]
            ctx.fsi_set_material(*p)
            vals.append(ctx.fsi_adjoint(U0, 0.25, M)[0])
        ctx.fsi_set_material(*base)
        fd = (vals[0] - vals[1]) / (2e-4 * base[i])
        assert abs(g[i] - fd) <= 1e-6 * abs(fd), (i, g[i], fd)
