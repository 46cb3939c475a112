"""Manufactured-solution pins of the FP64 oracle (CPU only).

The oracle's element residual (Sec. 2.3 with the forms of Eq. (semiforms)) is
evaluated at U_n = U_{n-1} = U, where the discrete time derivative and the ALE
mass term vanish and the theta-weighted terms add up to the steady operator:
the momentum rows become the weak form of the steady Navier-Stokes equations
in ALE coordinates (Eq. (ALE), fluid stress Eq. (ALE:stress)), the pressure rows
the divergence constraint plus the local projection stabilisation. A known
smooth solution (v*, p*) with its forcing f = rho (v*.grad) v* - div sigma(v*, p*)
then has to be approached at the rates of equal-order Q2 elements: velocity
L2 error O(h^3), pressure L2 error O(h^2).

Two cases: the identity ALE map (u = 0, the plain Navier-Stokes limit), and a
fixed smooth mesh deformation u* (zero on the boundary, so the physical domain
is still the unit square) under which the same physical solution is sought on
the deformed mesh. The second exercises F = I + grad u, J = det F and F^{-1}
in every term through the convergence rates.

Everything but the element residual is written here: the load vector, the
boundary rows, the steady Newton solve (complex-step Jacobian of the map U ->
R(U, U)), the Q2 evaluation for the errors.
"""
import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fsi as of


@dataclasses.dataclass(frozen=True)
class Fluid:
    rho_f: float = 100.0
    nu_f: float = 1.0
    rho_s: float = 100.0
    mu_s: float = 1.0
    lambda_s: float = 1.0
    vbar: float = 1.0
    ramp_t: float = 0.2
    theta0: float = 1.0
    alpha0: float = 0.1


A_V, B_P = 1.0, 100.0   # velocity and pressure amplitudes of the manufactured solution


def v_exact(x, y):
    """Divergence-free: v = A (sin(pi x) cos(pi y), -cos(pi x) sin(pi y))."""
    X, Y = np.pi * x, np.pi * y
    return A_V * np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)], -1)


def p_exact(x, y):
    return B_P * np.cos(np.pi * x) * np.cos(np.pi * y)


def forcing(x, y, m):
    """f = rho (v.grad) v - rho nu lap v + grad p for the fields above:
    (v.grad) v = A^2 pi/2 (sin 2 pi x, sin 2 pi y), lap v = -2 pi^2 v."""
    X, Y = np.pi * x, np.pi * y
    r, nu = m.rho_f, m.nu_f
    conv = A_V ** 2 * np.pi / 2 * np.stack([np.sin(2 * X), np.sin(2 * Y)], -1)
    grad_p = -B_P * np.pi * np.stack([np.sin(X) * np.cos(Y), np.cos(X) * np.sin(Y)], -1)
    return r * conv + 2 * np.pi ** 2 * r * nu * v_exact(x, y) + grad_p


def u_mesh(x, y, eps):
    """Smooth mesh displacement, zero on the boundary of the unit square."""
    s = eps * np.sin(np.pi * x) * np.sin(np.pi * y)
    return np.stack([s, 0.5 * s * np.sin(2 * np.pi * x)], -1)


def q2_1d(s):
    """Quadratic Lagrange basis on [0, 1] with nodes 0, 1/2, 1, and its derivative."""
    val = np.stack([2 * (s - 0.5) * (s - 1), -4 * s * (s - 1), 2 * s * (s - 0.5)], -1)
    der = np.stack([4 * s - 3, 4 - 8 * s, 4 * s - 1], -1)
    return val, der


GQ, GW = np.polynomial.legendre.leggauss(6)
GQ, GW = 0.5 * (GQ + 1), 0.5 * GW
_L, _D = q2_1d(GQ)
PHI = np.einsum("pb,qa->pqba", _L, _L).reshape(36, 9)      # point (p = t index, q = s index), node b*3+a
DPS = np.einsum("pb,qa->pqba", _L, _D).reshape(36, 9)
DPT = np.einsum("pb,qa->pqba", _D, _L).reshape(36, 9)
WQ = np.outer(GW, GW).ravel()


def cell_points(mesh, c):
    x0, y0 = mesh.xv[mesh.cell_ix[c]], mesh.yv[mesh.cell_iy[c]]
    hx, hy = mesh.hx[c], mesh.hy[c]
    T, S = np.meshgrid(GQ, GQ, indexing="ij")
    return x0 + hx * S.ravel(), y0 + hy * T.ravel(), hx, hy


def deformed(mesh, c, Uc):
    """Physical points x_h = X + u_h(X) at the cell's quadrature points and J_h = det(I + grad u_h)."""
    X, Y, hx, hy = cell_points(mesh, c)
    u = PHI @ Uc[:, 2:4]
    gs, gt = DPS @ Uc[:, 2:4] / hx, DPT @ Uc[:, 2:4] / hy
    J = (1 + gs[:, 0]) * (1 + gt[:, 1]) - gt[:, 0] * gs[:, 1]
    return X + u[:, 0], Y + u[:, 1], J * WQ * hx * hy


def steady_solve(nc, m, eps=0.0, alpha_fn=None):
    """Discrete steady solution on an nc x nc mesh of the unit square with the
    mesh displacement fixed to the Q2 interpolant of u_mesh(eps). Returns the
    L2 errors of v and of p (mean removed) on the deformed domain."""
    mesh = of.make_mesh((0.0, 1.0), (0.0, 1.0), (nc,), (nc,), None)
    tab = of.CellTables(mesh)
    cn = mesh.cell_nodes
    U0 = np.zeros((mesh.n_nodes, 5))
    U0[:, 2:4] = u_mesh(mesh.node_x, mesh.node_y, eps)
    xp, yp = mesh.node_x + U0[:, 2], mesh.node_y + U0[:, 3]      # physical node positions
    U0[:, 0:2] = v_exact(xp, yp)
    U0[:, 4] = p_exact(xp, yp)
    alpha = (alpha_fn or of.stabilisation_weights)(mesh, tab, m, U0)
    F = np.zeros((mesh.n_nodes, 5))
    for c in range(mesh.n_cells):
        x, y, wj = deformed(mesh, c, U0[cn[c]])
        F[cn[c], 0:2] += PHI.T @ (wj[:, None] * forcing(x, y, m))
    bnd = (mesh.node_i == 0) | (mesh.node_i == mesh.nnx - 1) | (mesh.node_j == 0) | (mesh.node_j == mesh.nny - 1)
    ident = np.zeros((mesh.n_nodes, 5), dtype=bool)
    ident[bnd, 0:2] = True
    ident[:, 2:4] = True                                        # the mesh motion is given
    pin = mesh.n_nodes // 2                                    # the pressure constant
    ident[pin, 4] = True
    target = np.where(ident, U0, 0.0)

    def elem(Ue):
        return of.element_residual(mesh, tab, m, Ue, Ue, 1.0, 1.0, alpha)

    def resid(U):
        R = np.zeros((mesh.n_nodes, 5))
        np.add.at(R, cn, elem(U[cn]))
        R -= F
        R[ident] = (U - target)[ident]
        return R

    dof = 5 * cn[:, :, None] + np.arange(5)
    eye = np.eye(45).reshape(45, 9, 5)

    def jacobian(U):
        h = 1e-30
        Ke = np.moveaxis(elem(U[cn][None] + 1j * h * eye[:, None]).imag / h, 0, -1).reshape(-1, 9, 5, 9, 5)
        rows = np.broadcast_to(dof[:, :, :, None, None], Ke.shape).ravel()
        cols = np.broadcast_to(dof[:, None, None, :, :], Ke.shape).ravel()
        keep = ~ident.ravel()[rows]
        idd = np.nonzero(ident.ravel())[0]
        return sp.coo_matrix((np.concatenate([Ke.ravel()[keep], np.ones(len(idd))]),
                              (np.concatenate([rows[keep], idd]), np.concatenate([cols[keep], idd]))),
                             shape=(mesh.n_dofs, mesh.n_dofs)).tocsc()

    U = np.where(ident, U0, 0.0)
    r0 = None
    for _ in range(15):
        R = resid(U)
        nr = np.linalg.norm(R)
        r0 = nr if r0 is None else r0
        if nr <= 1e-11 * max(r0, 1.0):
            break
        U = U + spla.spsolve(jacobian(U), -R.ravel()).reshape(U.shape)
    else:
        raise AssertionError("steady Newton did not converge")
    ev, dp = 0.0, []
    for c in range(mesh.n_cells):
        Uc = U[cn[c]]
        x, y, wj = deformed(mesh, c, Uc)
        ev += (wj[:, None] * (PHI @ Uc[:, 0:2] - v_exact(x, y)) ** 2).sum()
        dp.append((wj, PHI @ Uc[:, 4] - p_exact(x, y)))
    area = sum(w.sum() for w, _ in dp)
    mean = sum((w * d).sum() for w, d in dp) / area
    ep = sum((w * (d - mean) ** 2).sum() for w, d in dp)
    return np.sqrt(ev), np.sqrt(ep)


def rates(errs):
    e = np.array(errs)
    return np.log2(e[:-1] / e[1:])


def test_navier_stokes_limit_converges_at_q2_rates():
    """u = 0 (identity ALE map): velocity L2 rate 3, pressure L2 rate 2."""
    m = Fluid()
    res = [steady_solve(nc, m) for nc in (4, 8, 16, 32)]
    rv, rp = rates([r[0] for r in res]), rates([r[1] for r in res])
    assert np.all(rv[1:] > 2.9), rv
    assert np.all(rp[1:] > 1.9), rp


def test_convective_navier_stokes_limit_converges():
    """Reynolds number 100 (nu = 0.01): the convective term and the velocity-
    dependent stabilisation weight matter; the rates hold on the finer meshes."""
    m = Fluid(nu_f=0.01)
    res = [steady_solve(nc, m) for nc in (8, 16, 32)]
    rv, rp = rates([r[0] for r in res]), rates([r[1] for r in res])
    assert rv[-1] > 2.8, rv
    assert rp[-1] > 1.8, rp


def test_deformed_ale_mesh_converges_at_q2_rates():
    """The same physical solution sought on a mesh moved by a smooth u*
    (max |u*| = 0.08 of the unit square): every ALE factor (F, J, F^{-1}, the
    Piola stress, the ALE convection and divergence) enters; the rates of the
    identity map are kept, and the errors stay close to its errors."""
    m = Fluid()
    res = [steady_solve(nc, m, eps=0.08) for nc in (4, 8, 16, 32)]
    rv, rp = rates([r[0] for r in res]), rates([r[1] for r in res])
    assert np.all(rv[1:] > 2.9), rv
    assert np.all(rp[1:] > 1.9), rp
    flat = steady_solve(16, m)
    assert res[2][0] < 3 * flat[0] and res[2][1] < 3 * flat[1]
