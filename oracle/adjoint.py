"""FP64 CPU oracle: discrete adjoint of the theta-step trajectory (test infrastructure only).

The fine propagator of Sec. 3 is a sequence of steps R_n(U_n, U_{n-1}; p) = 0
(the step equation of Sec. 2.3). For the tip functional

    J = sum_{n=0}^{M} w_n |u(x_tip, t_n)|^2,   w_0 = w_M = k/2, w_n = k otherwise,

the discrete adjoint runs backward:

    (dR_n/dU_n)^T lam_n = -w_n dg/dU_n - (dR_{n+1}/dU_n)^T lam_{n+1},
    dJ/dp = sum_{n=1}^{M} lam_n^T dR_n/dp,

with p = (mu_s, lambda_s, vbar) (St. Venant-Kirchhoff Lame parameters of
Eq. (stress) and the mean inflow velocity of the Dirichlet data). Every
derivative here is a complex-step derivative of the oracle residual, so it
shares no derivation with the CUDA tangents.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fsi as of


def tip_node(mesh: of.Mesh, solid_box):
    """Node at the top centre of the solid box."""
    (x0, x1), (_, y1) = solid_box
    d = (mesh.node_x - 0.5 * (x0 + x1)) ** 2 + (mesh.node_y - y1) ** 2
    i = int(np.argmin(d))
    if d[i] > 1e-20:
        raise ValueError("no mesh node at the bar tip")
    return i


def _alpha_from_old(tab, mat, Uoe):
    """Stabilisation weights from cell-local old states [..., cell, 9, 5] (complex-safe)."""
    vq = np.matmul(tab.phi, Uoe[..., 0:2])
    vbar = (tab.W[:, :, None] * vq).sum(axis=-2) / tab.W.sum(axis=1)[:, None]
    speed = np.sqrt((vbar ** 2).sum(axis=-1))
    h = tab.h_cell
    return mat.alpha0 * h ** 2 / (mat.rho_f * mat.nu_f + mat.rho_f * speed * h)


class _CMat:
    """A material whose fields may be complex (for parameter derivatives)."""

    def __init__(self, mat, **kw):
        for f in dataclasses.fields(mat):
            setattr(self, f.name, kw.get(f.name, getattr(mat, f.name)))


def _element_general(mesh, tab, mat, Ue, Uoe, k, theta):
    """Cell residuals with the stabilisation weight taken from the old cell state."""
    return of.element_residual(mesh, tab, mat, Ue, Uoe, k, theta, _alpha_from_old(tab, mat, Uoe))


def old_state_jacobian(mesh, tab, mat, U, Uold, t_new, k, theta, h=1e-30):
    """dR/dU_old (CSR): complex steps over the 45 old values of every cell,
    assembled with the same row selection as the residual (identity rows give 0)."""
    prob = of.StepProblem(mesh, mat, Uold, t_new, k, theta, tab)
    Ue = np.asarray(U, dtype=float)[mesh.cell_nodes]
    Uoe = np.asarray(Uold, dtype=float)[mesh.cell_nodes]
    eye = np.eye(45).reshape(45, 9, 5)
    pert = Uoe[None] + 1j * h * eye[:, None]
    Re = _element_general(mesh, tab, mat, np.broadcast_to(Ue[None], pert.shape).astype(complex), pert, k, theta)
    Ke = np.moveaxis(Re.imag / h, 0, -1).reshape(-1, 9, 5, 9, 5) * prob.keep[:, :, :, None, None]
    dof = 5 * mesh.cell_nodes[:, :, None] + np.arange(5)[None, None, :]
    rows = np.broadcast_to(dof[:, :, :, None, None], Ke.shape).ravel()
    cols = np.broadcast_to(dof[:, None, None, :, :], Ke.shape).ravel()
    B = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(mesh.n_dofs, mesh.n_dofs)).tocsr()
    B.sum_duplicates()
    return B


def residual_parameter_derivatives(mesh, tab, mat, U, Uold, t_new, k, theta, h=1e-30):
    """dR/d(mu_s, lambda_s, vbar) as three vectors (complex steps on the parameters)."""
    prob = of.StepProblem(mesh, mat, Uold, t_new, k, theta, tab)
    Ue = np.asarray(U, dtype=float)[mesh.cell_nodes].astype(complex)
    Uoe = np.asarray(Uold, dtype=float)[mesh.cell_nodes].astype(complex)
    y = mesh.node_y - mesh.yv[0]
    H = mesh.H
    out = []
    for name in ("mu_s", "lambda_s", "vbar"):
        cm = _CMat(mat, **{name: getattr(mat, name) + 1j * h})
        Re = _element_general(mesh, tab, cm, Ue, Uoe, k, theta) * prob.keep
        R = np.zeros((mesh.n_nodes, 5), dtype=complex)
        np.add.at(R, mesh.cell_nodes, Re)
        # identity rows carry U - g(t): only the inflow profile depends on a parameter (vbar)
        g = np.zeros((mesh.n_nodes, 5), dtype=complex)
        prof = of.inflow_ramp(t_new, mat.ramp_t) * 1.5 * cm.vbar * 4.0 * y * (H - y) / H ** 2
        g[mesh.on_inflow, 0] = prof[mesh.on_inflow]
        R[prob.ident] = -g[prob.ident]
        out.append(R.imag.ravel() / h)
    return out


def trajectory(model: of.FSIModel, U0, t0, k, M):
    theta = model.theta_fine(k)
    Us = [np.asarray(U0, dtype=float).reshape(model.mesh.n_nodes, 5)]
    for n in range(M):
        Us.append(model.step(Us[-1], t0 + n * k, k, theta))
    return Us


def tip_functional(Us, k, tip):
    M = len(Us) - 1
    w = np.full(M + 1, k)
    w[0] = w[-1] = 0.5 * k
    return float(sum(w[n] * np.sum(Us[n][tip, 2:4] ** 2) for n in range(M + 1)))


def adjoint_gradient(model: of.FSIModel, U0, t0, k, M, tip):
    """J and dJ/d(mu_s, lambda_s, vbar) of the M-step fine trajectory from U0 at t0."""
    mesh, tab, mat = model.mesh, model.tab, model.mat
    theta = model.theta_fine(k)
    Us = trajectory(model, U0, t0, k, M)
    J = tip_functional(Us, k, tip)
    w = np.full(M + 1, k)
    w[0] = w[-1] = 0.5 * k
    grad = np.zeros(3)
    lam_next = None
    for n in range(M, 0, -1):
        rhs = np.zeros(mesh.n_dofs)
        rhs[5 * tip + 2:5 * tip + 4] = -w[n] * 2.0 * Us[n][tip, 2:4]
        if lam_next is not None:
            B = old_state_jacobian(mesh, tab, mat, Us[n + 1], Us[n], t0 + (n + 1) * k, k, theta)
            rhs -= B.T @ lam_next
        prob = of.StepProblem(mesh, mat, Us[n - 1], t0 + n * k, k, theta, tab)
        A = prob.jacobian(Us[n])
        lam = spla.spsolve(A.T.tocsc(), rhs)
        dR = residual_parameter_derivatives(mesh, tab, mat, Us[n], Us[n - 1], t0 + n * k, k, theta)
        grad += np.array([lam @ d for d in dR])
        lam_next = lam
    return J, grad
