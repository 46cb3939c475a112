"""Pins of the FP64 oracle's ALE-FSI step against facts the paper and the
mathematics fix (CPU only). Each test names what a plausible mistake would
break: a dropped term, a wrong sign, a transposed operand or a wrong index.
"""
import numpy as np
import pytest

from oracle import fsi as of
from paper_1907_01252_gb300 import workloads as wl

MAT = wl.Material()


# ---------------------------------------------------------------------------
# Independent Q2 basis for the checks (Vandermonde inversion on {0, 1/2, 1},
# Gauss-Legendre points from numpy), no code shared with the oracle.
# ---------------------------------------------------------------------------
_NODES = np.array([0.0, 0.5, 1.0])
_COEF = np.linalg.inv(np.vander(_NODES, 3, increasing=True))   # columns: basis a


def basis1d(s):
    V = np.vander(np.atleast_1d(s), 3, increasing=True)
    return V @ _COEF


def dbasis1d(s):
    s = np.atleast_1d(s)
    dV = np.stack([np.zeros_like(s), np.ones_like(s), 2 * s], axis=-1)
    return dV @ _COEF


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def test_q2_basis_partition_of_unity_and_nodality():
    s = np.linspace(0, 1, 7)
    L = of.lagrange2(s)
    dL = of.lagrange2_deriv(s)
    assert np.allclose(L.sum(-1), 1.0, atol=1e-15)
    assert np.allclose(dL.sum(-1), 0.0, atol=1e-14)
    assert np.allclose(of.lagrange2(_NODES), np.eye(3), atol=1e-15)
    assert np.allclose(L, basis1d(s), atol=1e-14)
    assert np.allclose(dL, dbasis1d(s), atol=1e-13)


def test_gauss3_exact_to_degree5():
    for p in range(6):
        q = np.sum(of.GAUSS_WEIGHTS * of.GAUSS_POINTS ** p)
        assert abs(q - 1.0 / (p + 1)) < 1e-15
    assert abs(np.sum(of.GAUSS_WEIGHTS * of.GAUSS_POINTS ** 6) - 1 / 7) > 1e-6


# ---------------------------------------------------------------------------
# Helpers: small meshes and element evaluation
# ---------------------------------------------------------------------------
def channel_mesh(nx, ny, solid=True, H=0.41):
    nxs = wl.cells_per_segment(wl.X_BREAKS, nx)
    nys = wl.cells_per_segment((0.0, 0.2, H), ny)
    return of.make_mesh(wl.X_BREAKS, (0.0, 0.2, H), nxs, nys, wl.SOLID_BOX if solid else None)


def nodal(mesh, f):
    """Nodal values [n_nodes, 5] of f(x, y) -> 5 components."""
    return np.stack(f(mesh.node_x, mesh.node_y), axis=-1).astype(float)


def elem(mesh, U, Uo, k=1e-2, theta=0.6, alpha=None, mat=MAT):
    tab = of.CellTables(mesh)
    if alpha is None:
        alpha = np.zeros(mesh.n_cells)
    return of.element_residual(mesh, tab, mat, U[mesh.cell_nodes], Uo[mesh.cell_nodes], k, theta, alpha)


def assemble(mesh, Re, comps=slice(None)):
    R = np.zeros((mesh.n_nodes, 5))
    np.add.at(R, mesh.cell_nodes, Re)
    return R


def plain_ns_cell_residual(mesh, U, Uo, k, theta, mat=MAT):
    """Textbook Galerkin Navier-Stokes theta-step residual on a fixed mesh
    (u = 0): rho(v - vo) + k theta rho (grad v) v + k (1-theta) rho (grad vo) vo
    tested with phi, plus the symmetric viscous stress and the pressure p_n,
    the do-nothing correction on x = x_max, and k div v tested with xi.
    Written with an independent basis and quadrature."""
    pts, wts = gauss01(3)          # the method integrates with 3x3 Gauss points
    rho, nu = mat.rho_f, mat.nu_f
    out = np.zeros((mesh.n_cells, 9, 5))
    for c in range(mesh.n_cells):
        if mesh.cell_solid[c]:
            continue
        hx, hy = mesh.hx[c], mesh.hy[c]
        Ue, Uoe = U[mesh.cell_nodes[c]], Uo[mesh.cell_nodes[c]]
        for sq, ws in zip(pts, wts):
            for tq, wt in zip(pts, wts):
                Bs, Bt = basis1d(sq)[0], basis1d(tq)[0]
                dBs, dBt = dbasis1d(sq)[0], dbasis1d(tq)[0]
                phi = np.outer(Bt, Bs).ravel()
                gx = np.outer(Bt, dBs).ravel() / hx
                gy = np.outer(dBt, Bs).ravel() / hy
                w = ws * wt * hx * hy
                def fields(X):
                    v = X[:, :2].T @ phi
                    G = np.stack([X[:, :2].T @ gx, X[:, :2].T @ gy], axis=1)   # G[i, j] = d v_i / d x_j
                    return v, G, X[:, 4] @ phi
                v, G, p = fields(Ue)
                vo, Go, _ = fields(Uoe)
                fv = rho * (v - vo) + k * theta * rho * G @ v + k * (1 - theta) * rho * Go @ vo
                S = k * theta * rho * nu * (G + G.T) + k * (1 - theta) * rho * nu * (Go + Go.T) - k * p * np.eye(2)
                for l in range(9):
                    out[c, l, :2] += w * (fv * phi[l] + S @ np.array([gx[l], gy[l]]))
                    out[c, l, 4] += w * k * np.trace(G) * phi[l]
        if mesh.cell_ix[c] == mesh.nx - 1:       # outflow edge s = 1
            for tq, wt in zip(pts, wts):
                Bs, Bt = basis1d(1.0)[0], basis1d(tq)[0]
                dBs, dBt = dbasis1d(1.0)[0], dbasis1d(tq)[0]
                phi = np.outer(Bt, Bs).ravel()
                gx = np.outer(Bt, dBs).ravel() / hx
                gy = np.outer(dBt, Bs).ravel() / hy
                for X, wk in ((Ue, k * theta), (Uoe, k * (1 - theta))):
                    G = np.stack([X[:, :2].T @ gx, X[:, :2].T @ gy], axis=1)
                    tv = -wk * rho * nu * G.T @ np.array([1.0, 0.0])
                    for l in range(9):
                        out[c, l, :2] += wt * hy * tv * phi[l]
    return out


# ---------------------------------------------------------------------------
# ALE kinematics
# ---------------------------------------------------------------------------
def test_zero_displacement_is_plain_navier_stokes():
    """u = 0 gives F = I, J = 1: the ALE residual is the plain NS residual."""
    mesh = channel_mesh(8, 2)
    rng = np.random.default_rng(0)
    U = rng.standard_normal((mesh.n_nodes, 5))
    Uo = rng.standard_normal((mesh.n_nodes, 5))
    U[:, 2:4] = 0.0
    Uo[:, 2:4] = 0.0
    U[:, 4] *= 50
    k, th = 1e-2, 0.6
    Re = elem(mesh, U, Uo, k, th)
    ref = plain_ns_cell_residual(mesh, U, Uo, k, th)
    fl = ~mesh.cell_solid
    scale = np.abs(ref[fl]).max()
    assert np.abs(Re[fl][..., [0, 1, 4]] - ref[fl][..., [0, 1, 4]]).max() <= 1e-12 * scale


@pytest.mark.parametrize("eps", [0.05, -0.03])
def test_uniform_stretch_gives_closed_form_J(eps):
    """u = (0, eps*y): F = diag(1, 1 + eps), J = 1 + eps. Summing the
    divergence rows (partition of unity) integrates J tr(grad v F^{-1}):
    v = (x, 0) gives k (1 + eps) |Omega_f|, v = (0, y) gives k |Omega_f|."""
    mesh = channel_mesh(8, 2, solid=False)
    k = 0.1
    area = (mesh.xv[-1] - mesh.xv[0]) * mesh.H
    U = nodal(mesh, lambda x, y: (x, 0 * x, 0 * x, eps * y, 0 * x))
    total = elem(mesh, U, U, k)[..., 4].sum()
    assert abs(total - k * (1 + eps) * area) < 1e-12 * area
    U = nodal(mesh, lambda x, y: (0 * x, y, 0 * x, eps * y, 0 * x))
    total = elem(mesh, U, U, k)[..., 4].sum()
    assert abs(total - k * area) < 1e-12 * area


def test_shear_divergence_catches_transposed_inverse():
    """u = (gamma*y, 0): F = [[1, gamma], [0, 1]], J = 1, v = (0, x):
    tr(grad v F^{-1}) = -gamma, while a transposed inverse would give 0."""
    mesh = channel_mesh(8, 2, solid=False)
    k, gamma = 0.1, 0.2
    area = (mesh.xv[-1] - mesh.xv[0]) * mesh.H
    U = nodal(mesh, lambda x, y: (0 * x, x, gamma * y, 0 * x, 0 * x))
    total = elem(mesh, U, U, k)[..., 4].sum()
    assert abs(total - (-gamma) * k * area) < 1e-12 * area


def test_rigid_translation_ale_mass_term_vanishes():
    """Mesh moving rigidly (u = c(t), F = I) under a steady quadratic Eulerian
    field w: v_n(x) = w(x + c_n). The ALE mass term
    (v_n - v_{n-1}) - grad v_{n-1/2} F^{-1}_{n-1/2} (u_n - u_{n-1}) vanishes
    exactly (trapezoidal rule is exact for the linear gradient of a quadratic),
    so the residual equals the plain NS residual without time derivative."""
    mesh = channel_mesh(8, 2, solid=False)
    c_new, c_old = np.array([0.013, -0.007]), np.array([-0.004, 0.002])
    def w(x, y):
        return (0.3 + 0.5 * x * y - 0.2 * y ** 2, -0.1 + 0.4 * x ** 2 - 0.25 * x * y)
    def state(c):
        wx, wy = w(mesh.node_x + c[0], mesh.node_y + c[1])
        return np.stack([wx, wy, c[0] + 0 * wx, c[1] + 0 * wx, 40 * mesh.node_x], -1)
    U, Uo = state(c_new), state(c_old)
    k, th = 2e-2, 0.55
    Re = elem(mesh, U, Uo, k, th)
    # plain NS with the same fields at fixed mesh and no mass term
    U0, Uo0 = U.copy(), Uo.copy()
    U0[:, 2:4] = Uo0[:, 2:4] = 0
    # plain residual minus its (v_n - v_{n-1}) mass part (the k = 0 evaluation)
    ref = plain_ns_cell_residual(mesh, U0, Uo0, k, th) - plain_ns_cell_residual(mesh, U0, Uo0, 0.0, th)
    scale = np.abs(ref[..., :2]).max()
    assert np.abs(Re[..., :2] - ref[..., :2]).max() <= 1e-11 * scale


def test_affine_divergence_free_field_has_zero_divergence_rows():
    """u = B x (affine), Eulerian v(x) = A x with tr A = 0 pulled back:
    v_hat = A (I + B) x_hat. Then J F^{-1} : grad v_hat^T = J tr(A) = 0 pointwise."""
    mesh = channel_mesh(8, 2, solid=False)
    B = np.array([[0.04, -0.03], [0.02, 0.05]])
    A = np.array([[0.7, 1.3], [-0.4, -0.7]])
    M = A @ (np.eye(2) + B)
    U = nodal(mesh, lambda x, y: (M[0, 0] * x + M[0, 1] * y, M[1, 0] * x + M[1, 1] * y,
                                  B[0, 0] * x + B[0, 1] * y, B[1, 0] * x + B[1, 1] * y, 0 * x))
    Re = elem(mesh, U, U, 0.1)
    assert np.abs(Re[..., 4]).max() < 1e-14


# ---------------------------------------------------------------------------
# Fluid: steady Poiseuille flow is a discrete solution (Q2 reproduces the
# parabola, the pressure is linear, LPS vanishes on Q1, the do-nothing
# correction removes the symmetric-gradient traction).
# ---------------------------------------------------------------------------
def poiseuille_state(mesh, mat=MAT):
    H = mesh.H
    vmax = 1.5 * mat.vbar
    y = mesh.node_y
    vx = vmax * 4 * y * (H - y) / H ** 2
    G = 8 * mat.rho_f * mat.nu_f * vmax / H ** 2
    p = G * (mesh.xv[-1] - mesh.node_x)
    return np.stack([vx, 0 * y, 0 * y, 0 * y, p], -1)


def test_poiseuille_is_exact_discrete_steady_state():
    mesh = channel_mesh(16, 4, solid=False)
    U = poiseuille_state(mesh)
    t = 1.0
    prob = of.StepProblem(mesh, MAT, U, t, 1e-2, 0.5 + 1e-2)
    R = prob.residual(U)
    scale = np.abs(elem(mesh, U, U * 0, 1e-2)).max()
    assert np.abs(R).max() <= 1e-12 * scale
    Un, info = of.newton_solve(prob, U)
    assert info.converged
    assert np.abs(Un - U).max() <= 1e-10 * np.abs(U).max()


def test_outflow_correction_is_needed_for_poiseuille():
    """Without the do-nothing correction the residual would not vanish: check the
    outflow rows carry exactly the correction rho nu (grad v)^T n."""
    mesh = channel_mesh(8, 2, solid=False)
    U = poiseuille_state(mesh)
    Re = elem(mesh, U, U, 1e-2)
    R = assemble(mesh, Re)
    interior_out = (mesh.node_i == mesh.nnx - 1) & ~mesh.dir_v
    assert np.abs(R[interior_out, :2]).max() < 1e-12 * np.abs(Re).max()


# ---------------------------------------------------------------------------
# Local projection stabilisation
# ---------------------------------------------------------------------------
def test_lps_kernel_is_q1_and_positive():
    mesh = channel_mesh(8, 2, solid=False)
    tab = of.CellTables(mesh)
    a = np.tile(np.arange(3), 3)
    b = np.repeat(np.arange(3), 3)
    for S in tab.S_lps[:3]:
        for q1 in (np.ones(9), a / 2.0, b / 2.0, a * b / 4.0):
            assert np.abs(S @ q1).max() < 1e-13 * np.abs(S).max()
        ev = np.linalg.eigvalsh(0.5 * (S + S.T))
        assert ev.min() > -1e-13 * ev.max()
        assert np.sum(ev > 1e-10 * ev.max()) == 5        # Q2 / Q1 has dimension 9 - 4
    bubble = (a * (2 - a) * b * (2 - b)).astype(float)
    assert bubble @ tab.S_lps[0] @ bubble > 0


# ---------------------------------------------------------------------------
# Solid: St. Venant-Kirchhoff
# ---------------------------------------------------------------------------
def solid_block_mesh():
    return of.make_mesh((0.0, 1.0), (0.0, 0.5), (4,), (2,), ((-1, 2), (-1, 2)))


def test_stvk_uniaxial_patch_test():
    """Homogeneous stretch u = (eps x, 0) of an all-solid block: constant first
    Piola stress, so interior momentum rows vanish and the right-edge rows sum to
    k * P11 * height with the uniaxial StVK response
    P11 = (2 mu + lambda) (1 + eps) eps (1 + eps / 2)."""
    mesh = solid_block_mesh()
    eps, k = 0.02, 0.1
    U = nodal(mesh, lambda x, y: (0 * x, 0 * x, eps * x, 0 * x, 0 * x))
    R = assemble(mesh, elem(mesh, U, U, k, 0.7))
    mu, lam = MAT.mu_s, MAT.lambda_s
    P11 = (2 * mu + lam) * (1 + eps) * eps * (1 + eps / 2)
    interior = (mesh.node_i > 0) & (mesh.node_i < mesh.nnx - 1) & (mesh.node_j > 0) & (mesh.node_j < mesh.nny - 1)
    assert np.abs(R[interior, :2]).max() < 1e-9 * k * P11
    right = mesh.node_i == mesh.nnx - 1
    height = mesh.yv[-1] - mesh.yv[0]
    assert abs(R[right, 0].sum() - k * P11 * height) < 1e-12 * k * P11
    assert abs(R[right, 1].sum()) < 1e-9 * k * P11


def test_stvk_rigid_motion_has_zero_stress():
    """Rigid rotation plus translation: E = 0, so the elastic rows vanish."""
    mesh = solid_block_mesh()
    a = 0.3
    Rm = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    D = Rm - np.eye(2)
    U = nodal(mesh, lambda x, y: (0 * x, 0 * x, D[0, 0] * x + D[0, 1] * y + 0.1, D[1, 0] * x + D[1, 1] * y - 0.2, 0 * x))
    Re = elem(mesh, U, U, 0.1)
    assert np.abs(Re[..., :2]).max() < 1e-7          # vs stresses ~ mu_s * k = 5e4


# ---------------------------------------------------------------------------
# Jacobian, Newton, time order
# ---------------------------------------------------------------------------
def test_jacobian_matches_central_differences():
    mesh = channel_mesh(8, 2)
    rng = np.random.default_rng(5)
    Uo = wl.random_state(mesh.n_nodes, 11, u_scale=1e-3)
    prob = of.StepProblem(mesh, MAT, Uo, 0.05, 1e-2, 0.51)
    U = prob.apply_dirichlet(wl.random_state(mesh.n_nodes, 12, u_scale=1e-3))
    A = prob.jacobian(U).toarray()
    n = mesh.n_dofs
    cols = rng.choice(n, 40, replace=False)
    for j in cols:
        scale = max(abs(U.ravel()[j]), 1e-3)
        h = 1e-6 * scale
        e = np.zeros(n)
        e[j] = h
        fd = (prob.residual(U.ravel() + e) - prob.residual(U.ravel() - e)).ravel() / (2 * h)
        err = np.abs(fd - A[:, j]).max()
        noise = 1e-13 * np.abs(prob.residual(U)).max() / h        # round-off of the difference quotient
        assert err <= 2e-5 * np.abs(A[:, j]).max() + noise, (j, err)


def test_newton_converges_quadratically():
    mesh = channel_mesh(16, 4)
    model = of.FSIModel(mesh, MAT)
    U = np.zeros((mesh.n_nodes, 5))
    k = 1 / 64
    for n in range(6):
        prob = of.StepProblem(mesh, MAT, U, (n + 1) * k, k, model.theta_fine(k), model.tab)
        U, info = of.newton_solve(prob, U)
    r = info.residual_norms
    assert info.converged and len(r) >= 3
    for a, b in zip(r[:-1], r[1:]):
        if a > 1e-9 * r[0]:
            assert b <= 10 * a ** 2 / r[0] + 1e-12 * r[0]


def test_shifted_crank_nicolson_is_second_order():
    """theta = 1/2 + k differs from Crank-Nicolson by O(k), so the step is
    second order: velocity of the pure channel flow and displacement of the
    coupled problem converge like k^2 (the pressure, a multiplier taken at t_n
    in both theta terms, is only first order and is not checked here)."""
    T = 0.08
    def rates(mesh, ms, m_ref, comp):
        model = of.FSIModel(mesh, MAT, newton_tol=1e-13)
        run = lambda m: model.propagate(np.zeros((mesh.n_nodes, 5)), 0.0, T, m)
        ref = run(m_ref)
        errs = [np.linalg.norm((run(m) - ref)[:, comp]) for m in ms]
        return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    r = rates(channel_mesh(8, 2, solid=False), (8, 16, 32), 256, slice(0, 2))
    assert np.all(r > 1.9) and np.all(r < 2.15), r
    r = rates(channel_mesh(8, 2, solid=True), (16, 32, 64), 512, slice(2, 4))
    assert np.all(r > 1.9) and np.all(r < 2.2), r


def test_implicit_euler_coarse_step_is_first_order_towards_the_fine_solution():
    """The coarse propagator is the same step equation at theta = 1 (Sec. 3: implicit
    Euler, with the n-1/2 means of the ALE mass term kept). It must converge to the
    solution of the fine scheme at first order: theta = 1 steps of decreasing size
    against a shifted Crank-Nicolson run with many steps (second order, so its own
    error is negligible). A wrong weight between the old and new terms at theta = 1
    would change the limit or the order."""
    T = 0.08
    for mesh, comp, ms in ((channel_mesh(8, 2, solid=False), slice(0, 2), (8, 16, 32)),
                           (channel_mesh(8, 2, solid=True), slice(2, 4), (16, 32, 64))):
        model = of.FSIModel(mesh, MAT, newton_tol=1e-13)
        U0 = np.zeros((mesh.n_nodes, 5))
        ref = model.propagate(U0, 0.0, T, 512)
        errs = [np.linalg.norm((model.propagate(U0, 0.0, T, m, theta=1.0) - ref)[:, comp]) for m in ms]
        r = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all(r > 0.85) and np.all(r < 1.2), (r, errs)
