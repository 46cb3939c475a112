"""FP64 CPU oracle: monolithic ALE fluid-structure time step (test infrastructure only).

Follows Sec. 2 of Margenberg & Richter, "Parallel time-stepping for
fluid-structure interactions":
  * ALE system, Eq. (ALE) and the ALE fluid stress, Eq. (ALE:stress);
  * St. Venant-Kirchhoff solid, Eq. (stress);
  * monolithic variational form, Eq. (variational) with test spaces Eq. (test);
  * equal-order iso-parametric Q2 elements on an interface-fitted quad mesh
    (Sec. 2.2; on axis-aligned rectangles the iso-parametric map is affine);
  * shifted Crank-Nicolson step, Sec. 2.3, with the semi-linear forms of
    Eq. (semiforms) and theta = 1/2 + theta0 * k.

Readings of places where the paper is silent or garbled (the same readings are
used by the CUDA library):
  R1  midpoint means: v_{n-1/2}, F_{n-1/2} = I + grad u_{n-1/2},
      J_{n-1/2} = (J_{n-1} + J_n) / 2 (mean of the determinants).
  R2  the old-time A_NS term is evaluated at (v_{n-1}, u_{n-1}, p_n) as printed;
      A_div is taken at t_n only; the kinematic row is
      (u_n - u_{n-1}, psi_s) - k (theta v_n + (1 - theta) v_{n-1}, psi_s).
  R3  the ALE mass term keeps the n-1/2 means for every theta (also theta = 1).
  R4  pressure stabilisation: one-level local projection on fluid cells,
      k * alpha_K (grad(p - pi1 p), grad(xi - pi1 xi))_K, pi1 = Q1 vertex
      interpolation on the cell, alpha_K = alpha0 h_K^2 / (rho_f nu_f +
      rho_f |vbar_K| h_K), vbar_K the cell mean of v_{n-1}, h_K the cell
      diameter, reference-frame gradients.
  R5  pressure rows: nodes touching a fluid cell carry the fluid divergence +
      stabilisation rows (fluid cells only); other pressure dofs get p = 0.
  R6  displacement rows: nodes in the closure of the solid carry the kinematic
      row (solid cells only); other interior nodes the harmonic extension row
      (fluid cells only); u = 0 on the whole outer boundary.
  R7  velocity Dirichlet data: parabolic inflow on x = 0 with the smooth ramp
      s(t) = (1 - cos(pi t / ramp_t)) / 2 for t < ramp_t, 1 afterwards;
      v = 0 on the walls y = 0 and y = H; do-nothing outflow on x = x_max with
      the correction term of Eq. (variational).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# --------------------------------------------------------------------------
# Reference element: 1D quadratic Lagrange basis on [0, 1] (nodes 0, 1/2, 1)
# and the 3-point Gauss rule.  Q2 = tensor products (Sec. 2.2, V_h^(2)).
# --------------------------------------------------------------------------
GAUSS_POINTS = 0.5 + np.array([-1.0, 0.0, 1.0]) * np.sqrt(0.15)
GAUSS_WEIGHTS = np.array([5.0, 8.0, 5.0]) / 18.0


def lagrange2(s):
    s = np.asarray(s, dtype=float)
    return np.stack([(1 - s) * (1 - 2 * s), 4 * s * (1 - s), s * (2 * s - 1)], axis=-1)


def lagrange2_deriv(s):
    s = np.asarray(s, dtype=float)
    return np.stack([4 * s - 3, 4 - 8 * s, 4 * s - 1], axis=-1)


def lagrange1(s):
    s = np.asarray(s, dtype=float)
    return np.stack([1 - s, s], axis=-1)


def lagrange1_deriv(s):
    s = np.asarray(s, dtype=float)
    return np.stack([-np.ones_like(s), np.ones_like(s)], axis=-1)


# --------------------------------------------------------------------------
# Mesh: interface-fitted tensor-product mesh, Q2 node grid (2nx+1) x (2ny+1).
# Node id = j * (2nx+1) + i; cell id = cy * nx + cx; local node l = b*3 + a.
# Nodal unknowns (v_x, v_y, u_x, u_y, p), dof = 5 * node + component.
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Mesh:
    xv: np.ndarray          # vertex x coordinates (nx+1)
    yv: np.ndarray          # vertex y coordinates (ny+1)
    solid_box: tuple | None

    def __post_init__(self):
        self.nx = len(self.xv) - 1
        self.ny = len(self.yv) - 1
        self.nnx = 2 * self.nx + 1
        self.nny = 2 * self.ny + 1
        self.n_nodes = self.nnx * self.nny
        self.n_cells = self.nx * self.ny
        self.xn = np.empty(self.nnx)
        self.xn[0::2] = self.xv
        self.xn[1::2] = 0.5 * (self.xv[:-1] + self.xv[1:])
        self.yn = np.empty(self.nny)
        self.yn[0::2] = self.yv
        self.yn[1::2] = 0.5 * (self.yv[:-1] + self.yv[1:])
        cx, cy = np.meshgrid(np.arange(self.nx), np.arange(self.ny), indexing="xy")
        cx, cy = cx.ravel(), cy.ravel()               # cell id = cy*nx + cx
        self.cell_ix = cx
        self.cell_iy = cy
        a = np.tile(np.arange(3), 3)
        b = np.repeat(np.arange(3), 3)
        self.cell_nodes = (2 * cy[:, None] + b[None, :]) * self.nnx + (2 * cx[:, None] + a[None, :])
        self.hx = self.xv[cx + 1] - self.xv[cx]
        self.hy = self.yv[cy + 1] - self.yv[cy]
        xc = 0.5 * (self.xv[cx] + self.xv[cx + 1])
        yc = 0.5 * (self.yv[cy] + self.yv[cy + 1])
        if self.solid_box is None:
            self.cell_solid = np.zeros(self.n_cells, dtype=bool)
        else:
            (x0, x1), (y0, y1) = self.solid_box
            self.cell_solid = (xc > x0) & (xc < x1) & (yc > y0) & (yc < y1)
        node_in_solid = np.zeros(self.n_nodes, dtype=bool)
        node_in_fluid = np.zeros(self.n_nodes, dtype=bool)
        node_in_solid[self.cell_nodes[self.cell_solid].ravel()] = True
        node_in_fluid[self.cell_nodes[~self.cell_solid].ravel()] = True
        self.node_in_solid = node_in_solid          # closure of the solid
        self.node_in_fluid = node_in_fluid          # touches a fluid cell
        ni = np.tile(np.arange(self.nnx), self.nny)
        nj = np.repeat(np.arange(self.nny), self.nnx)
        self.node_i, self.node_j = ni, nj
        self.node_x = self.xn[ni]
        self.node_y = self.yn[nj]
        on_in = ni == 0
        on_out = ni == self.nnx - 1
        on_wall = (nj == 0) | (nj == self.nny - 1)
        self.on_inflow = on_in
        self.dir_v = on_in | on_wall                 # velocity Dirichlet nodes
        self.dir_u = on_in | on_out | on_wall        # u = 0 on the outer boundary
        self.p_identity = ~node_in_fluid             # pressure dofs with p = 0
        self.H = self.yv[-1] - self.yv[0]
        self.outflow_cells = np.nonzero(cx == self.nx - 1)[0]

    @property
    def n_dofs(self):
        return 5 * self.n_nodes


def make_mesh(x_breaks, y_breaks, nx_seg, ny_seg, solid_box=None):
    """Tensor mesh with uniform spacing inside each segment between break points."""
    def axis(breaks, counts):
        pts = [np.array([breaks[0]])]
        for a, b, n in zip(breaks[:-1], breaks[1:], counts):
            pts.append(np.linspace(a, b, n + 1)[1:])
        return np.concatenate(pts)
    return Mesh(axis(x_breaks, nx_seg), axis(y_breaks, ny_seg), solid_box)


# --------------------------------------------------------------------------
# Per-cell quadrature tables (3x3 Gauss, affine rectangles).
# --------------------------------------------------------------------------
class CellTables:
    def __init__(self, mesh: Mesh):
        L = lagrange2(GAUSS_POINTS)          # [q1, a]
        dL = lagrange2_deriv(GAUSS_POINTS)
        # q = q2*3 + q1, l = b*3 + a
        self.phi = np.einsum("pb,qa->pqba", L, L).reshape(9, 9)
        dphids = np.einsum("pb,qa->pqba", L, dL).reshape(9, 9)
        dphidt = np.einsum("pb,qa->pqba", dL, L).reshape(9, 9)
        hx, hy = mesh.hx, mesh.hy
        self.dphi = np.stack([dphids[None] / hx[:, None, None], dphidt[None] / hy[:, None, None]], axis=-1)
        w2 = np.outer(GAUSS_WEIGHTS, GAUSS_WEIGHTS).ravel()        # [q2*3+q1]
        self.W = w2[None, :] * (hx * hy)[:, None]                  # [cell, q]
        # Outflow edge s = 1: edge points t = Gauss, ds = hy * w
        Le = lagrange2(np.array(1.0))                                # [a]
        dLe = lagrange2_deriv(np.array(1.0))
        self.phi_e = np.einsum("pb,a->pba", L, Le).reshape(3, 9)
        dphids_e = np.einsum("pb,a->pba", L, dLe).reshape(3, 9)
        dphidt_e = np.einsum("pb,a->pba", dL, Le).reshape(3, 9)
        oc = mesh.outflow_cells
        self.dphi_e = np.stack([dphids_e[None] / hx[oc, None, None], dphidt_e[None] / hy[oc, None, None]], axis=-1)
        self.W_e = GAUSS_WEIGHTS[None, :] * hy[oc, None]
        # Local projection: kappa(phi_l) = phi_l - pi1(phi_l); pi1 phi_l is the
        # Q1 vertex function for vertex nodes (a, b in {0, 2}), zero otherwise.
        L1 = lagrange1(GAUSS_POINTS)
        dL1 = lagrange1_deriv(GAUSS_POINTS)
        q1s = np.zeros((9, 9))
        q1t = np.zeros((9, 9))
        for bb, b in enumerate((0, 2)):
            for aa, a in enumerate((0, 2)):
                l = b * 3 + a
                q1s[:, l] = np.einsum("p,q->pq", L1[:, bb], dL1[:, aa]).ravel()
                q1t[:, l] = np.einsum("p,q->pq", dL1[:, bb], L1[:, aa]).ravel()
        dks = dphids - q1s
        dkt = dphidt - q1t
        gk = np.stack([dks[None] / hx[:, None, None], dkt[None] / hy[:, None, None]], axis=-1)
        self.S_lps = np.einsum("cq,cqld,cqmd->clm", self.W, gk, gk)  # [cell, 9, 9]
        self.h_cell = np.sqrt(hx ** 2 + hy ** 2)


# --------------------------------------------------------------------------
# Small 2x2 tensor helpers on trailing axes (analytic: safe for complex step).
# Convention: (grad v)_{ij} = d v_i / d x_j,  F = I + grad u.
# --------------------------------------------------------------------------
def det2(A):
    return A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]


def inv2(A):
    d = det2(A)
    out = np.empty_like(A)
    out[..., 0, 0] = A[..., 1, 1] / d
    out[..., 0, 1] = -A[..., 0, 1] / d
    out[..., 1, 0] = -A[..., 1, 0] / d
    out[..., 1, 1] = A[..., 0, 0] / d
    return out


def tr(A):
    return np.swapaxes(A, -1, -2)


def mm(A, B):
    shape = np.broadcast_shapes(A.shape, B.shape)
    C = np.empty(shape, dtype=np.result_type(A, B))
    for i in range(2):
        for j in range(2):
            C[..., i, j] = A[..., i, 0] * B[..., 0, j] + A[..., i, 1] * B[..., 1, j]
    return C


def mv(A, x):
    return np.stack([A[..., i, 0] * x[..., 0] + A[..., i, 1] * x[..., 1] for i in range(2)], axis=-1)


EYE2 = np.eye(2)


def inflow_ramp(t, ramp_t):
    """Smooth start of the inflow: (1 - cos(pi t / ramp_t)) / 2 for t < ramp_t, else 1."""
    return 0.5 * (1.0 - np.cos(np.pi * t / ramp_t)) if t < ramp_t else 1.0


def dirichlet_values(mesh: Mesh, mat, t):
    """Boundary data g(t): parabolic inflow with mean vbar (Sec. 4 profile), zero elsewhere."""
    g = np.zeros((mesh.n_nodes, 5))
    y = mesh.node_y - mesh.yv[0]
    H = mesh.H
    prof = inflow_ramp(t, mat.ramp_t) * 1.5 * mat.vbar * 4.0 * y * (H - y) / H ** 2
    g[mesh.on_inflow, 0] = prof[mesh.on_inflow]
    return g


# --------------------------------------------------------------------------
# Element residual of one theta step (Sec. 2.3), all cells at once.
# --------------------------------------------------------------------------
def element_residual(mesh: Mesh, tab: CellTables, mat, Ue, Uo, k, theta, alpha):
    """Cell contributions of the step residual.

    Ue : [..., n_cells, 9, 5] unknown state at t_n on the cell nodes (real or complex)
    Uo : [n_cells, 9, 5]      state at t_{n-1}
    alpha : [n_cells]         stabilisation weights alpha_K (from the old state)
    Returns [..., n_cells, 9, 5]: columns 0-1 momentum rows (test phi), columns
    2-3 displacement rows (kinematic on solid cells, harmonic on fluid cells),
    column 4 the divergence + stabilisation rows (fluid cells).
    """
    rf, nu, rs, mu, lam = mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s
    phi, dphi, W = tab.phi, tab.dphi, tab.W
    solid = mesh.cell_solid.astype(float)
    fluid = 1.0 - solid

    def at_qp(U):
        val = np.matmul(phi, U)                                       # [..., c, q, f]
        grad = np.stack([np.matmul(dphi[..., d], U) for d in range(2)], axis=-1)
        return val, grad

    def test_value(f):      # sum_q W phi_l(q) f(q)      -> [..., c, l, f]
        return np.matmul(phi.T, W[:, :, None] * f)

    def test_grad(g):       # sum_q W grad phi_l(q) . g  -> [..., c, l, f]
        Wg = W[:, :, None, None] * g
        return sum(np.matmul(np.swapaxes(dphi[..., d], -1, -2), Wg[..., d]) for d in range(2))

    val, grad = at_qp(Ue)
    valo, grado = at_qp(Uo)
    v, u, p = val[..., 0:2], val[..., 2:4], val[..., 4]
    Gv, Gu = grad[..., 0:2, :], grad[..., 2:4, :]
    vo, uo = valo[..., 0:2], valo[..., 2:4]
    Gvo, Guo = grado[..., 0:2, :], grado[..., 2:4, :]

    F = EYE2 + Gu
    Fo = EYE2 + Guo
    J, Jo = det2(F), det2(Fo)
    Fi, Foi = inv2(F), inv2(Fo)
    # midpoint quantities (R1)
    Gvh = 0.5 * (Gv + Gvo)
    Fh = EYE2 + 0.5 * (Gu + Guo)
    Jh = 0.5 * (J + Jo)
    Fhi = inv2(Fh)

    # ---- fluid momentum (Eq. semiforms: A_NS; step equation of Sec. 2.3) ----
    mass_f = rf * Jh[..., None] * ((v - vo) - mv(mm(Gvh, Fhi), u - uo))
    conv = rf * J[..., None] * mv(mm(Gv, Fi), v)
    conv_o = rf * Jo[..., None] * mv(mm(Gvo, Foi), vo)

    def piola_fluid_stress(Gv_, Fi_, J_, p_):
        sigma = rf * nu * (mm(Gv_, Fi_) + mm(tr(Fi_), tr(Gv_))) - p_[..., None, None] * EYE2
        return J_[..., None, None] * mm(sigma, tr(Fi_))

    st = piola_fluid_stress(Gv, Fi, J, p)
    st_o = piola_fluid_stress(Gvo, Foi, Jo, p)          # old geometry, new pressure (R2)
    fv_f = mass_f + k * theta * conv + k * (1 - theta) * conv_o
    fg_f = k * theta * st + k * (1 - theta) * st_o

    # ---- solid momentum (A_ES with St. Venant-Kirchhoff, Eq. stress) ----
    def first_piola(F_):
        E = 0.5 * (mm(tr(F_), F_) - EYE2)
        trE = E[..., 0, 0] + E[..., 1, 1]
        Sig = 2 * mu * E + lam * trE[..., None, None] * EYE2
        return mm(F_, Sig)

    fv_s = rs * (v - vo)
    fg_s = k * theta * first_piola(F) + k * (1 - theta) * first_piola(Fo)

    sf = solid[:, None, None]
    ff = fluid[:, None, None]
    fv = ff * fv_f + sf * fv_s
    fg = ff[..., None] * fg_f + sf[..., None] * fg_s

    # ---- displacement rows ----
    kin = (u - uo) - k * (theta * v + (1 - theta) * vo)        # solid cells (psi_s)
    harm = k * theta * Gu + k * (1 - theta) * Guo               # fluid cells (psi_f)
    # ---- divergence row (A_div at t_n) ----
    div = k * J * np.einsum("...ij,...ji->...", Gv, Fi)       # J F^{-1} : grad v^T

    out_shape = Ue.shape
    R = np.zeros(out_shape, dtype=np.result_type(Ue, float))
    R[..., 0:2] = test_value(fv) + test_grad(fg)
    R[..., 2:4] = sf * test_value(kin) + ff * test_grad(harm)
    R[..., 4] = fluid[:, None] * test_value(div[..., None])[..., 0]
    # local projection stabilisation (R4), constant in the unknowns apart from p
    R[..., 4] += (fluid * k * alpha)[..., :, None] * np.einsum("clm,...cm->...cl", tab.S_lps, Ue[..., 4])

    # ---- do-nothing correction on the outflow boundary (Eq. variational) ----
    oc = mesh.outflow_cells
    if len(oc):
        Ue_o = Ue[..., oc, :, :]
        Uo_o = Uo[..., oc, :, :]
        ge = np.einsum("cqld,...clf->...cqfd", tab.dphi_e, Ue_o)
        geo = np.einsum("cqld,...clf->...cqfd", tab.dphi_e, Uo_o)
        n = np.array([1.0, 0.0])

        def outflow_term(g):
            Gv_, Gu_ = g[..., 0:2, :], g[..., 2:4, :]
            F_ = EYE2 + Gu_
            J_ = det2(F_)
            FiT = tr(inv2(F_))
            return rf * nu * J_[..., None] * mv(mm(mm(FiT, tr(Gv_)), FiT), n)

        tv = -(k * theta * outflow_term(ge) + k * (1 - theta) * outflow_term(geo))
        tv = tv * fluid[oc][:, None, None]
        R[..., oc, :, 0:2] += np.einsum("cq,ql,...cqf->...clf", tab.W_e, tab.phi_e, tv)
    return R


def stabilisation_weights(mesh: Mesh, tab: CellTables, mat, U_old):
    """alpha_K = alpha0 h_K^2 / (rho_f nu_f + rho_f |vbar_K| h_K), vbar_K = cell mean of v_{n-1} (R4)."""
    Uo = U_old[mesh.cell_nodes]
    vq = np.einsum("ql,clf->cqf", tab.phi, Uo[..., 0:2])
    vbar = np.einsum("cq,cqf->cf", tab.W, vq) / tab.W.sum(axis=1)[:, None]
    speed = np.sqrt((vbar ** 2).sum(axis=1))
    h = tab.h_cell
    return mat.alpha0 * h ** 2 / (mat.rho_f * mat.nu_f + mat.rho_f * speed * h)


# --------------------------------------------------------------------------
# Global residual and Jacobian
# --------------------------------------------------------------------------
class StepProblem:
    """One theta step t_{n-1} -> t_n = t_{n-1} + k with fixed old state."""

    def __init__(self, mesh: Mesh, mat, U_old, t_new, k, theta, tab: CellTables | None = None):
        self.mesh = mesh
        self.mat = mat
        self.tab = tab if tab is not None else CellTables(mesh)
        self.U_old = np.asarray(U_old, dtype=float).reshape(mesh.n_nodes, 5)
        self.t_new = t_new
        self.k = k
        self.theta = theta
        self.g = dirichlet_values(mesh, mat, t_new)
        self.alpha = stabilisation_weights(mesh, self.tab, mat, self.U_old)
        m = mesh
        cn = m.cell_nodes
        # which cell contributions enter which rows (R5, R6)
        keep = np.ones((m.n_cells, 9, 5), dtype=bool)
        keep[:, :, 2] = keep[:, :, 3] = (m.cell_solid[:, None] == m.node_in_solid[cn])
        keep[:, :, 4] = ~m.cell_solid[:, None]
        ident = np.zeros((m.n_nodes, 5), dtype=bool)
        ident[m.dir_v, 0:2] = True
        ident[m.dir_u, 2:4] = True
        ident[m.p_identity, 4] = True
        keep &= ~ident[cn]
        self.keep = keep
        self.ident = ident

    def apply_dirichlet(self, U):
        U = U.reshape(self.mesh.n_nodes, 5).copy()
        U[self.mesh.dir_v, 0:2] = self.g[self.mesh.dir_v, 0:2]
        U[self.mesh.dir_u, 2:4] = 0.0
        return U

    def _element(self, Ue):
        return element_residual(self.mesh, self.tab, self.mat, Ue, self.U_old[self.mesh.cell_nodes],
                                self.k, self.theta, self.alpha)

    def residual(self, U):
        """Global residual; identity rows carry U - g (Dirichlet) or p (solid pressure)."""
        m = self.mesh
        U = np.asarray(U).reshape(m.n_nodes, 5)
        Re = self._element(U[m.cell_nodes]) * self.keep
        R = np.zeros((m.n_nodes, 5), dtype=Re.dtype)
        np.add.at(R, m.cell_nodes, Re)
        target = self.g.copy()
        target[:, 4] = 0.0
        R[self.ident] = (U - target)[self.ident]
        return R

    def element_jacobians(self, U, h=1e-30, chunk=256):
        """Element matrices dRe/dUe by the complex-step derivative, [cell, 9, 5, 9, 5]."""
        m = self.mesh
        U = np.asarray(U, dtype=float).reshape(m.n_nodes, 5)
        Ue = U[m.cell_nodes]
        Ke = np.empty((m.n_cells, 9, 5, 9, 5))
        eye = np.eye(45).reshape(45, 9, 5)
        Uo_all = self.U_old[m.cell_nodes]
        for c0 in range(0, m.n_cells, chunk):
            cs = slice(c0, min(c0 + chunk, m.n_cells))
            sub = _SubMesh(m, cs)
            pert = Ue[cs][None] + 1j * h * eye[:, None]
            Re = element_residual(sub, _SubTables(self.tab, cs, sub), self.mat, pert, Uo_all[cs],
                                  self.k, self.theta, self.alpha[cs])
            Ke[cs] = np.moveaxis(Re.imag / h, 0, -1).reshape(-1, 9, 5, 9, 5)
        return Ke

    def jacobian(self, U):
        """Global sparse Jacobian dR/dU (CSR), identity rows as in residual()."""
        m = self.mesh
        Ke = self.element_jacobians(U) * self.keep[:, :, :, None, None]
        dof = 5 * m.cell_nodes[:, :, None] + np.arange(5)[None, None, :]     # [cell, 9, 5]
        rows = np.broadcast_to(dof[:, :, :, None, None], Ke.shape).ravel()
        cols = np.broadcast_to(dof[:, None, None, :, :], Ke.shape).ravel()
        vals = Ke.ravel()
        idd = np.nonzero(self.ident.ravel())[0]
        rows = np.concatenate([rows, idd])
        cols = np.concatenate([cols, idd])
        vals = np.concatenate([vals, np.ones(len(idd))])
        A = sp.coo_matrix((vals, (rows, cols)), shape=(m.n_dofs, m.n_dofs)).tocsr()
        A.sum_duplicates()
        return A


class _SubMesh:
    """View of a cell range of a mesh (for chunked element evaluation)."""

    def __init__(self, mesh: Mesh, cs: slice):
        self.cell_solid = mesh.cell_solid[cs]
        ids = np.arange(mesh.n_cells)[cs]
        sel = np.isin(ids, mesh.outflow_cells)
        self.outflow_cells = np.nonzero(sel)[0]
        self._global_outflow_index = np.searchsorted(mesh.outflow_cells, ids[sel])


class _SubTables:
    def __init__(self, tab: CellTables, cs: slice, sub: _SubMesh):
        self.phi = tab.phi
        self.dphi = tab.dphi[cs]
        self.W = tab.W[cs]
        self.S_lps = tab.S_lps[cs]
        self.phi_e = tab.phi_e
        gi = sub._global_outflow_index
        self.dphi_e = tab.dphi_e[gi]
        self.W_e = tab.W_e[gi]


# --------------------------------------------------------------------------
# Newton's method for one step (Sec. 1 / Sec. 4: nonlinear systems by Newton).
# --------------------------------------------------------------------------
@dataclasses.dataclass
class NewtonInfo:
    iterations: int
    residual_norms: list
    converged: bool


def newton_solve(prob: StepProblem, U0, tol=1e-10, maxit=20, step_tol=0.0, min_iter=1):
    """Full Newton with exact Jacobian and a direct sparse solve, no damping.

    Stops after iteration m when ||R(U_m)||_2 <= tol * max(||R(U_0)||_2, 1)
    and the last correction satisfies ||delta||_2 <= step_tol * ||U||_2.
    """
    U = prob.apply_dirichlet(U0)
    norms = []
    r0 = None
    last_step_ok = step_tol <= 0.0
    for it in range(maxit + 1):
        R = prob.residual(U)
        nr = float(np.linalg.norm(R))
        norms.append(nr)
        if r0 is None:
            r0 = nr
        if it >= min_iter and nr <= tol * max(r0, 1.0) and last_step_ok:
            return U, NewtonInfo(it, norms, True)
        if it == maxit:
            break
        A = prob.jacobian(U)
        delta = spla.spsolve(A.tocsc(), -R.ravel()).reshape(U.shape)
        U = U + delta
        last_step_ok = step_tol <= 0.0 or np.linalg.norm(delta) <= step_tol * np.linalg.norm(U)
    return U, NewtonInfo(maxit, norms, False)


# --------------------------------------------------------------------------
# Propagators (Sec. 3): m theta steps over one slice.
# --------------------------------------------------------------------------
class FSIModel:
    def __init__(self, mesh: Mesh, mat, newton_tol=1e-10, newton_maxit=20, step_tol=0.0):
        self.mesh = mesh
        self.mat = mat
        self.tab = CellTables(mesh)
        self.newton_tol = newton_tol
        self.newton_maxit = newton_maxit
        self.step_tol = step_tol
        self.newton_counts = []

    def theta_fine(self, k):
        """Shifted Crank-Nicolson, theta = 1/2 + theta0 * k (Sec. 2.3)."""
        return 0.5 + self.mat.theta0 * k

    def step(self, U, t_old, k, theta):
        prob = StepProblem(self.mesh, self.mat, U, t_old + k, k, theta, self.tab)
        Un, info = newton_solve(prob, U, self.newton_tol, self.newton_maxit, self.step_tol)
        self.newton_counts.append(info.iterations)
        if not info.converged:
            raise RuntimeError(f"Newton did not converge at t={t_old + k}: {info.residual_norms}")
        return Un

    def propagate(self, U, t0, t1, m, theta=None):
        """m equal steps from t0 to t1; theta None = shifted CN of the step size."""
        k = (t1 - t0) / m
        th = self.theta_fine(k) if theta is None else theta
        U = np.asarray(U, dtype=float).reshape(self.mesh.n_nodes, 5)
        for j in range(m):
            U = self.step(U, t0 + j * k, k, th)
        return U


def mesh_for(workload, x_breaks, y_breaks, solid_box):
    return make_mesh(x_breaks, y_breaks, workload.nx_seg, workload.ny_seg,
                     solid_box if workload.with_solid else None)
