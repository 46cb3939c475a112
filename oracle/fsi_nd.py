"""FP64 CPU oracle for the ALE-FSI step in d = 2 or 3 dimensions (test infrastructure only).

The discrete system of oracle/fsi.py (Sec. 2 of Margenberg & Richter, "Parallel
time-stepping for fluid-structure interactions": Eq. (ALE), (ALE:stress),
(stress), (variational), (test); the shifted Crank-Nicolson step of Sec. 2.3
with the forms of Eq. (semiforms)), written once for any space dimension d:
equal-order Q2 on axis-aligned boxes (9-node quadrilaterals, 27-node
hexahedra), 3^d Gauss points, per node the unknowns (v_1..v_d, u_1..u_d, p).
The readings R1-R7 of oracle/fsi.py hold unchanged; in 3D:

  R13 inflow on x = x_min: v_x = s(t) * 36 vbar (y - y0)(y1 - y)(z - z0)(z1 - z)
      / ((y1 - y0)^2 (z1 - z0)^2), whose mean over the cross-section is vbar;
      no-slip on the four lateral walls; do-nothing outflow on x = x_max with
      the correction term of Eq. (variational); u = 0 on the whole boundary.
  R14 local projection stabilisation: pi1 = Q1 (trilinear) vertex interpolation
      on the cell, h_K the cell diameter.

At d = 2 this module and oracle/fsi.py are independent writings of the same
formulas (a test compares them).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fsi import GAUSS_POINTS, GAUSS_WEIGHTS, inflow_ramp, lagrange1, lagrange1_deriv, lagrange2, \
    lagrange2_deriv, newton_solve


# --------------------------------------------------------------------------
# d x d tensor helpers on trailing axes (analytic, so complex steps pass through).
# Convention: (grad v)_{ij} = d v_i / d x_j, F = I + grad u.
# --------------------------------------------------------------------------
def det(A):
    if A.shape[-1] == 2:
        return A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    return (A[..., 0, 0] * (A[..., 1, 1] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 1])
            - A[..., 0, 1] * (A[..., 1, 0] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 0])
            + A[..., 0, 2] * (A[..., 1, 0] * A[..., 2, 1] - A[..., 1, 1] * A[..., 2, 0]))


def adjugate(A):
    """adj(A), with A adj(A) = det(A) I (transpose of the cofactor matrix)."""
    d = A.shape[-1]
    out = np.empty_like(A)
    if d == 2:
        out[..., 0, 0] = A[..., 1, 1]
        out[..., 0, 1] = -A[..., 0, 1]
        out[..., 1, 0] = -A[..., 1, 0]
        out[..., 1, 1] = A[..., 0, 0]
        return out
    for i in range(3):
        for j in range(3):
            # cofactor C_ji: minor of A without row j and column i
            r = [x for x in range(3) if x != j]
            c = [x for x in range(3) if x != i]
            minor = A[..., r[0], c[0]] * A[..., r[1], c[1]] - A[..., r[0], c[1]] * A[..., r[1], c[0]]
            out[..., i, j] = (-1) ** (i + j) * minor
    return out


def inv(A):
    return adjugate(A) / det(A)[..., None, None]


def tr(A):
    return np.swapaxes(A, -1, -2)


def mm(A, B):
    return np.einsum("...ij,...jk->...ik", A, B)


def mv(A, x):
    return np.einsum("...ij,...j->...i", A, x)


def trace(A):
    return np.einsum("...ii->...", A)


# --------------------------------------------------------------------------
# Mesh: tensor mesh of axis-aligned boxes, Q2 node grid (2 n_a + 1) per axis.
# Node id: x fastest, then y, then z; cell id likewise; local node: x fastest.
# --------------------------------------------------------------------------
class MeshND:
    def __init__(self, axes, solid_box=None):
        self.axes = [np.asarray(a, dtype=float) for a in axes]
        d = self.d = len(self.axes)
        self.ncell = [len(a) - 1 for a in self.axes]
        self.nnode = [2 * n + 1 for n in self.ncell]
        self.n_nodes = int(np.prod(self.nnode))
        self.n_cells = int(np.prod(self.ncell))
        self.nc = 2 * d + 1
        self.node_coord = []
        for a, n in zip(self.axes, self.ncell):
            xn = np.empty(2 * n + 1)
            xn[0::2] = a
            xn[1::2] = 0.5 * (a[:-1] + a[1:])
            self.node_coord.append(xn)
        # node multi-indices (x fastest)
        idx = np.indices(self.nnode[::-1]).reshape(d, -1)[::-1]      # idx[a] = index along axis a
        self.node_idx = idx
        self.node_xyz = np.stack([self.node_coord[a][idx[a]] for a in range(d)], axis=-1)
        cidx = np.indices(self.ncell[::-1]).reshape(d, -1)[::-1]
        self.cell_idx = cidx
        lidx = np.indices((3,) * d).reshape(d, -1)[::-1]             # local node multi-index, x fastest
        self.local_idx = lidx
        strides = np.cumprod([1] + self.nnode[:-1])
        self.cell_nodes = sum(((2 * cidx[a])[:, None] + lidx[a][None, :]) * strides[a] for a in range(d))
        self.h = np.stack([self.axes[a][cidx[a] + 1] - self.axes[a][cidx[a]] for a in range(d)], axis=-1)
        centre = np.stack([0.5 * (self.axes[a][cidx[a]] + self.axes[a][cidx[a] + 1]) for a in range(d)], axis=-1)
        if solid_box is None:
            self.cell_solid = np.zeros(self.n_cells, dtype=bool)
        else:
            self.cell_solid = np.all([(centre[:, a] > solid_box[a][0]) & (centre[:, a] < solid_box[a][1])
                                      for a in range(d)], axis=0)
        self.node_in_solid = np.zeros(self.n_nodes, dtype=bool)
        self.node_in_fluid = np.zeros(self.n_nodes, dtype=bool)
        self.node_in_solid[self.cell_nodes[self.cell_solid].ravel()] = True
        self.node_in_fluid[self.cell_nodes[~self.cell_solid].ravel()] = True
        on_in = idx[0] == 0
        on_out = idx[0] == self.nnode[0] - 1
        on_wall = np.zeros(self.n_nodes, dtype=bool)
        for a in range(1, d):
            on_wall |= (idx[a] == 0) | (idx[a] == self.nnode[a] - 1)
        self.on_inflow = on_in
        self.dir_v = on_in | on_wall
        self.dir_u = on_in | on_out | on_wall
        self.p_identity = ~self.node_in_fluid
        self.outflow_cells = np.nonzero(cidx[0] == self.ncell[0] - 1)[0]

    @property
    def n_dofs(self):
        return self.nc * self.n_nodes


def make_mesh_nd(breaks, counts, solid_box=None):
    """Tensor mesh with uniform spacing inside each segment between break points, per axis."""
    axes = []
    for br, cnt in zip(breaks, counts):
        pts = [np.array([br[0]])]
        for a, b, n in zip(br[:-1], br[1:], cnt):
            pts.append(np.linspace(a, b, n + 1)[1:])
        axes.append(np.concatenate(pts))
    return MeshND(axes, solid_box)


# --------------------------------------------------------------------------
# Per-cell quadrature tables: 3^d Gauss points, affine boxes.
# --------------------------------------------------------------------------
class CellTablesND:
    def __init__(self, mesh: MeshND):
        d = mesh.d
        L = lagrange2(GAUSS_POINTS)          # [point, node]
        dL = lagrange2_deriv(GAUSS_POINTS)
        qidx = np.indices((3,) * d).reshape(d, -1)[::-1]             # quadrature multi-index, x fastest
        lidx = mesh.local_idx
        nq, nl = qidx.shape[1], lidx.shape[1]
        # phi[q, l] = prod_a L(q_a, l_a); dref[q, l, a] = derivative along axis a on the unit box
        self.phi = np.ones((nq, nl))
        for a in range(d):
            self.phi *= L[qidx[a]][:, lidx[a]]
        dref = np.ones((nq, nl, d))
        for a in range(d):
            for b in range(d):
                dref[:, :, a] *= (dL if a == b else L)[qidx[b]][:, lidx[b]]
        h = mesh.h
        self.dphi = dref[None] / h[:, None, None, :]                 # [cell, q, l, d]
        w = np.ones(nq)
        for a in range(d):
            w *= GAUSS_WEIGHTS[qidx[a]]
        self.W = w[None, :] * np.prod(h, axis=1)[:, None]             # [cell, q]
        # outflow face x = x_max: reference s_x = 1, Gauss points on the other axes
        fidx = np.indices((3,) * (d - 1)).reshape(d - 1, -1)[::-1]
        nf = fidx.shape[1]
        Le, dLe = lagrange2(np.array([1.0])), lagrange2_deriv(np.array([1.0]))
        self.phi_e = np.ones((nf, nl))
        dref_e = np.ones((nf, nl, d))
        for a in range(d):
            if a == 0:
                self.phi_e *= Le[np.zeros(nf, dtype=int)][:, lidx[0]]
                for b in range(d):
                    dref_e[:, :, b] *= (dLe if b == 0 else Le)[np.zeros(nf, dtype=int)][:, lidx[0]]
            else:
                self.phi_e *= L[fidx[a - 1]][:, lidx[a]]
                for b in range(d):
                    dref_e[:, :, b] *= (dL if b == a else L)[fidx[a - 1]][:, lidx[a]]
        oc = mesh.outflow_cells
        self.dphi_e = dref_e[None] / h[oc][:, None, None, :]
        wf = np.ones(nf)
        for a in range(1, d):
            wf *= GAUSS_WEIGHTS[fidx[a - 1]]
        self.W_e = wf[None, :] * np.prod(h[oc][:, 1:], axis=1)[:, None]
        # local projection: kappa(phi_l) = phi_l - pi1(phi_l); pi1 phi_l is the Q1
        # vertex function of l for vertex nodes (every l_a in {0, 2}), zero otherwise
        L1, dL1 = lagrange1(GAUSS_POINTS), lagrange1_deriv(GAUSS_POINTS)
        dq1 = np.zeros((nq, nl, d))
        for l in range(nl):
            if np.all((lidx[:, l] == 0) | (lidx[:, l] == 2)):
                vert = lidx[:, l] // 2
                for a in range(d):
                    f = np.ones(nq)
                    for b in range(d):
                        f = f * (dL1 if b == a else L1)[qidx[b], vert[b]]
                    dq1[:, l, a] = f
        gk = (dref - dq1)[None] / h[:, None, None, :]
        self.S_lps = np.einsum("cq,cqla,cqma->clm", self.W, gk, gk)
        self.h_cell = np.sqrt((h ** 2).sum(axis=1))


def dirichlet_values_nd(mesh: MeshND, mat, t):
    """Boundary data g(t): the inflow profile of R7 (2D) or R13 (3D), zero elsewhere."""
    d = mesh.d
    g = np.zeros((mesh.n_nodes, mesh.nc))
    s = inflow_ramp(t, mat.ramp_t)
    if d == 2:
        y0, y1 = mesh.axes[1][0], mesh.axes[1][-1]
        y = mesh.node_xyz[:, 1]
        prof = 1.5 * mat.vbar * 4.0 * (y - y0) * (y1 - y) / (y1 - y0) ** 2
    else:
        y0, y1 = mesh.axes[1][0], mesh.axes[1][-1]
        z0, z1 = mesh.axes[2][0], mesh.axes[2][-1]
        y, z = mesh.node_xyz[:, 1], mesh.node_xyz[:, 2]
        prof = 36.0 * mat.vbar * (y - y0) * (y1 - y) * (z - z0) * (z1 - z) / ((y1 - y0) ** 2 * (z1 - z0) ** 2)
    g[mesh.on_inflow, 0] = s * prof[mesh.on_inflow]
    return g


def element_residual_nd(mesh: MeshND, tab: CellTablesND, mat, Ue, Uo, k, theta, alpha, cells=None):
    """Cell contributions of the step residual, [..., cells, 3^d, 2d+1].

    Columns 0..d-1: momentum rows; d..2d-1: displacement rows (kinematic on
    solid cells, harmonic extension on fluid cells); 2d: divergence and
    stabilisation rows (fluid cells). cells: optional index array selecting
    the cells Ue, Uo and alpha belong to (default all)."""
    d = mesh.d
    cells = np.arange(mesh.n_cells) if cells is None else np.asarray(cells)
    I = np.eye(d)
    rf, nu, rs, mu, lam = mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s
    phi, dphi, W = tab.phi, tab.dphi[cells], tab.W[cells]
    solid = mesh.cell_solid[cells].astype(float)
    fluid = 1.0 - solid

    def at_qp(U):
        val = np.einsum("ql,...clf->...cqf", phi, U)
        grad = np.einsum("cqla,...clf->...cqfa", dphi, U)
        return val, grad

    def test_value(f):     # sum_q W phi_l f
        return np.einsum("cq,ql,...cqf->...clf", W, phi, f)

    def test_grad(g):      # sum_q W grad phi_l . g (rows of g)
        return np.einsum("cq,cqla,...cqfa->...clf", W, dphi, g)

    val, grad = at_qp(Ue)
    valo, grado = at_qp(Uo)
    v, u, p = val[..., 0:d], val[..., d:2 * d], val[..., 2 * d]
    Gv, Gu = grad[..., 0:d, :], grad[..., d:2 * d, :]
    vo, uo = valo[..., 0:d], valo[..., d:2 * d]
    Gvo, Guo = grado[..., 0:d, :], grado[..., d:2 * d, :]
    F, Fo = I + Gu, I + Guo
    J, Jo = det(F), det(Fo)
    Fi, Foi = inv(F), inv(Fo)
    Gvh = 0.5 * (Gv + Gvo)                      # R1 midpoint means
    Fhi = inv(I + 0.5 * (Gu + Guo))
    Jh = 0.5 * (J + Jo)

    mass_f = rf * Jh[..., None] * ((v - vo) - mv(mm(Gvh, Fhi), u - uo))
    conv = rf * J[..., None] * mv(mm(Gv, Fi), v)
    conv_o = rf * Jo[..., None] * mv(mm(Gvo, Foi), vo)

    def fluid_piola(Gv_, Fi_, J_, p_):
        sigma = rf * nu * (mm(Gv_, Fi_) + mm(tr(Fi_), tr(Gv_))) - p_[..., None, None] * I
        return J_[..., None, None] * mm(sigma, tr(Fi_))

    fv_f = mass_f + k * theta * conv + k * (1 - theta) * conv_o
    fg_f = k * theta * fluid_piola(Gv, Fi, J, p) + k * (1 - theta) * fluid_piola(Gvo, Foi, Jo, p)   # R2

    def svk_piola(F_):
        E = 0.5 * (mm(tr(F_), F_) - I)
        return mm(F_, 2 * mu * E + lam * trace(E)[..., None, None] * I)

    fv_s = rs * (v - vo)
    fg_s = k * theta * svk_piola(F) + k * (1 - theta) * svk_piola(Fo)
    sf, ff = solid[:, None, None], fluid[:, None, None]
    fv = ff * fv_f + sf * fv_s
    fg = ff[..., None] * fg_f + sf[..., None] * fg_s

    kin = (u - uo) - k * (theta * v + (1 - theta) * vo)
    harm = k * theta * Gu + k * (1 - theta) * Guo
    div = k * J * trace(mm(Gv, Fi))

    R = np.zeros(Ue.shape, dtype=np.result_type(Ue, float))
    R[..., 0:d] = test_value(fv) + test_grad(fg)
    R[..., d:2 * d] = sf * test_value(kin) + ff * test_grad(harm)
    R[..., 2 * d] = fluid[:, None] * test_value(div[..., None])[..., 0]
    R[..., 2 * d] += (fluid * k * alpha)[:, None] * np.einsum("clm,...cm->...cl", tab.S_lps[cells], Ue[..., 2 * d])

    # do-nothing correction on x = x_max (Eq. variational), momentum rows
    pos = {c: i for i, c in enumerate(mesh.outflow_cells)}
    sel = [j for j, c in enumerate(cells) if c in pos]
    if sel:
        gi = np.array([pos[cells[j]] for j in sel])
        n = np.zeros(d)
        n[0] = 1.0

        def term(Uc):
            g = np.einsum("cqla,...clf->...cqfa", tab.dphi_e[gi], Uc)
            Gv_, Gu_ = g[..., 0:d, :], g[..., d:2 * d, :]
            F_ = I + Gu_
            FiT = tr(inv(F_))
            return rf * nu * det(F_)[..., None] * mv(mm(mm(FiT, tr(Gv_)), FiT), n)

        sel = np.array(sel)
        tv = -(k * theta * term(Ue[..., sel, :, :]) + k * (1 - theta) * term(Uo[..., sel, :, :]))
        tv = tv * fluid[sel][:, None, None]
        R[..., sel, :, 0:d] += np.einsum("cq,ql,...cqf->...clf", tab.W_e[gi], tab.phi_e, tv)
    return R


def stabilisation_weights_nd(mesh: MeshND, tab: CellTablesND, mat, U_old):
    """alpha_K = alpha0 h_K^2 / (rho_f nu_f + rho_f |vbar_K| h_K), vbar_K the cell mean of v_{n-1}."""
    d = mesh.d
    Uo = U_old[mesh.cell_nodes]
    vq = np.einsum("ql,clf->cqf", tab.phi, Uo[..., 0:d])
    vbar = np.einsum("cq,cqf->cf", tab.W, vq) / tab.W.sum(axis=1)[:, None]
    speed = np.sqrt((vbar ** 2).sum(axis=1))
    h = tab.h_cell
    return mat.alpha0 * h ** 2 / (mat.rho_f * mat.nu_f + mat.rho_f * speed * h)


class StepProblemND:
    """One theta step t_{n-1} -> t_n with fixed old state; rows selected as in R5, R6."""

    def __init__(self, mesh: MeshND, mat, U_old, t_new, k, theta, tab: CellTablesND | None = None):
        self.mesh, self.mat, self.k, self.theta, self.t_new = mesh, mat, k, theta, t_new
        self.tab = tab if tab is not None else CellTablesND(mesh)
        d, nc = mesh.d, mesh.nc
        self.U_old = np.asarray(U_old, dtype=float).reshape(mesh.n_nodes, nc)
        self.g = dirichlet_values_nd(mesh, mat, t_new)
        self.alpha = stabilisation_weights_nd(mesh, self.tab, mat, self.U_old)
        cn = mesh.cell_nodes
        keep = np.ones((mesh.n_cells, cn.shape[1], nc), dtype=bool)
        keep[:, :, d:2 * d] = (mesh.cell_solid[:, None] == mesh.node_in_solid[cn])[:, :, None]
        keep[:, :, 2 * d] = ~mesh.cell_solid[:, None]
        ident = np.zeros((mesh.n_nodes, nc), dtype=bool)
        ident[mesh.dir_v, 0:d] = True
        ident[mesh.dir_u, d:2 * d] = True
        ident[mesh.p_identity, 2 * d] = True
        self.keep = keep & ~ident[cn]
        self.ident = ident

    def apply_dirichlet(self, U):
        d = self.mesh.d
        U = np.asarray(U).reshape(self.mesh.n_nodes, self.mesh.nc).copy()
        U[self.mesh.dir_v, 0:d] = self.g[self.mesh.dir_v, 0:d]
        U[self.mesh.dir_u, d:2 * d] = 0.0
        return U

    def residual(self, U):
        m = self.mesh
        U = np.asarray(U).reshape(m.n_nodes, m.nc)
        Re = element_residual_nd(m, self.tab, self.mat, U[m.cell_nodes], self.U_old[m.cell_nodes],
                                 self.k, self.theta, self.alpha) * self.keep
        R = np.zeros((m.n_nodes, m.nc), dtype=Re.dtype)
        np.add.at(R, m.cell_nodes, Re)
        target = self.g.copy()
        target[:, 2 * m.d] = 0.0
        R[self.ident] = (U - target)[self.ident]
        return R

    def element_jacobians(self, U, h=1e-30, chunk=32):
        """dRe/dUe by the complex-step derivative, [cell, nl, nc, nl, nc]."""
        m = self.mesh
        nl, nc = m.cell_nodes.shape[1], m.nc
        U = np.asarray(U, dtype=float).reshape(m.n_nodes, nc)
        Ue, Uo = U[m.cell_nodes], self.U_old[m.cell_nodes]
        Ke = np.empty((m.n_cells, nl, nc, nl, nc))
        eye = np.eye(nl * nc).reshape(nl * nc, nl, nc)
        for c0 in range(0, m.n_cells, chunk):
            cs = np.arange(c0, min(c0 + chunk, m.n_cells))
            pert = Ue[cs][None] + 1j * h * eye[:, None]
            Re = element_residual_nd(m, self.tab, self.mat, pert, Uo[cs], self.k, self.theta, self.alpha[cs], cs)
            Ke[cs] = np.moveaxis(Re.imag / h, 0, -1).reshape(-1, nl, nc, nl, nc)
        return Ke

    def jacobian(self, U):
        m = self.mesh
        nc = m.nc
        Ke = self.element_jacobians(U) * self.keep[:, :, :, None, None]
        dof = nc * m.cell_nodes[:, :, None] + np.arange(nc)[None, None, :]
        rows = np.broadcast_to(dof[:, :, :, None, None], Ke.shape).ravel()
        cols = np.broadcast_to(dof[:, None, None, :, :], Ke.shape).ravel()
        idd = np.nonzero(self.ident.ravel())[0]
        A = sp.coo_matrix((np.concatenate([Ke.ravel(), np.ones(len(idd))]),
                           (np.concatenate([rows, idd]), np.concatenate([cols, idd]))),
                          shape=(m.n_dofs, m.n_dofs)).tocsr()
        A.sum_duplicates()
        return A


class FSIModelND:
    """theta steps of the d-dimensional system, each solved by full Newton with direct solves."""

    def __init__(self, mesh: MeshND, mat, newton_tol=1e-10, newton_maxit=20):
        self.mesh, self.mat = mesh, mat
        self.tab = CellTablesND(mesh)
        self.newton_tol, self.newton_maxit = newton_tol, newton_maxit
        self.newton_counts = []

    def theta_fine(self, k):
        return 0.5 + self.mat.theta0 * k

    def step(self, U, t_old, k, theta):
        prob = StepProblemND(self.mesh, self.mat, U, t_old + k, k, theta, self.tab)
        Un, info = newton_solve(prob, U, self.newton_tol, self.newton_maxit)
        self.newton_counts.append(info.iterations)
        if not info.converged:
            raise RuntimeError(f"Newton did not converge at t={t_old + k}: {info.residual_norms}")
        return Un

    def propagate(self, U, t0, t1, m, theta=None):
        k = (t1 - t0) / m
        th = self.theta_fine(k) if theta is None else theta
        U = np.asarray(U, dtype=float).reshape(self.mesh.n_nodes, self.mesh.nc)
        for j in range(m):
            U = self.step(U, t0 + j * k, k, th)
        return U
