"""Pins of the FP64 oracle that need no solve (CPU only).

1. A change of units. The step residual of Sec. 2.3 (forms of Eq. (semiforms),
   materials of Eq. (stress)) is a sum of physical terms, so measuring lengths,
   times and masses in other units (factors L, T, M) must scale every row of
   one kind by one factor: momentum rows by M/T, kinematic rows by L^3,
   harmonic-extension rows by T L, divergence rows by L^2, identity rows like
   their unknown. Any term with the wrong dimensions breaks this: a missing
   density, a viscosity without its density, a power of h or of k too many or
   too few. That includes the stabilisation weight of the local projection
   term, whose form the paper leaves open (the reading alpha_K = alpha0 h^2 /
   (rho_f nu_f + rho_f |vbar_K| h) has the dimensions the divergence row
   needs); the test plants two wrong weights in the oracle and checks that
   the pin catches both.
2. The mass terms use the density of their own material: with u = p = 0 and
   a spatially constant velocity change c, every term but the mass terms
   vanishes, and a momentum row equals c times the density-weighted integral
   of its basis function over the fluid and solid cells, which for Q2 on
   rectangles is hx hy w_a w_b with the Simpson weights w = (1/6, 2/3, 1/6).
"""
import dataclasses

import numpy as np
import pytest

from oracle import fsi as of
from paper_1907_01252_gb300 import workloads as wl

L_F, T_F, M_F = 10.0, 3.0, 7.0   # new unit of length, time and mass, in the old units


def scaled_material(m):
    return dataclasses.replace(
        m, rho_f=m.rho_f * M_F / L_F ** 3, rho_s=m.rho_s * M_F / L_F ** 3, nu_f=m.nu_f * L_F ** 2 / T_F,
        mu_s=m.mu_s * M_F / (L_F * T_F ** 2), lambda_s=m.lambda_s * M_F / (L_F * T_F ** 2),
        vbar=m.vbar * L_F / T_F, ramp_t=m.ramp_t * T_F)


def state_scale():
    return np.array([L_F / T_F, L_F / T_F, L_F, L_F, M_F / (L_F * T_F ** 2)])


def residual_pair(w, seed=5):
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    (x0, x1), (y0, y1) = wl.SOLID_BOX
    box = ((x0 * L_F, x1 * L_F), (y0 * L_F, y1 * L_F))
    mesh2 = of.make_mesh(tuple(b * L_F for b in wl.X_BREAKS), tuple(b * L_F for b in wl.Y_BREAKS),
                         w.nx_seg, w.ny_seg, box)
    U = wl.random_state(mesh.n_nodes, seed)
    Uo = wl.random_state(mesh.n_nodes, seed + 1)
    t_new, k, theta = 0.1, 1e-2, 0.6          # t_new inside the inflow ramp
    m = w.material
    R = of.StepProblem(mesh, m, Uo, t_new, k, theta).residual(U)
    prob2 = of.StepProblem(mesh2, scaled_material(m), Uo * state_scale(), t_new * T_F, k * T_F, theta)
    R2 = prob2.residual(U * state_scale())
    # expected factor per row
    D = np.empty((mesh.n_nodes, 5))
    D[:, 0:2] = M_F / T_F
    D[:, 2:4] = np.where(mesh.node_in_solid, L_F ** 3, T_F * L_F)[:, None]
    D[:, 4] = L_F ** 2
    ident = prob2.ident
    D[ident] = np.broadcast_to(state_scale(), D.shape)[ident]
    return R, R2, D, ident


def invariance_defect(w):
    """Largest relative deviation from the unit scaling, per row kind."""
    R, R2, D, ident = residual_pair(w)
    out = {}
    for name, cols in (("momentum", slice(0, 2)), ("displacement", slice(2, 4)), ("pressure", slice(4, 5))):
        want, got = (D * R)[:, cols], R2[:, cols]
        sel = ~ident[:, cols]
        out[name] = np.abs(got - want)[sel].max() / np.abs(want[sel]).max()
    return out


def test_residual_is_invariant_under_a_change_of_units():
    d = invariance_defect(wl.Workload("units", nx=16, ny=4, T=1.0, n_slices=4, m_fine=4))
    assert max(d.values()) <= 1e-12, d


@pytest.mark.parametrize("wrong", ["h instead of h^2", "rho_f dropped"])
def test_units_pin_catches_a_wrong_stabilisation_weight(monkeypatch, wrong):
    right = of.stabilisation_weights

    def alpha(mesh, tab, mat, U_old):
        a = right(mesh, tab, mat, U_old)
        return a / tab.h_cell if wrong == "h instead of h^2" else a * mat.rho_f
    monkeypatch.setattr(of, "stabilisation_weights", alpha)
    d = invariance_defect(wl.Workload("units", nx=16, ny=4, T=1.0, n_slices=4, m_fine=4))
    assert d["pressure"] > 1e-6, d
    assert d["momentum"] <= 1e-12 and d["displacement"] <= 1e-12, d


def test_mass_terms_use_the_density_of_their_material():
    mat = dataclasses.replace(wl.Material(), rho_s=2500.0)
    w = wl.Workload("mass", nx=16, ny=4, T=1.0, n_slices=4, m_fine=4, material=mat)
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    c = np.array([0.3, -0.7])
    k, theta = 1e-2, 0.6
    U = np.zeros((mesh.n_nodes, 5))
    U[:, 0:2] = c
    prob = of.StepProblem(mesh, mat, np.zeros((mesh.n_nodes, 5)), 0.5, k, theta)
    R = prob.residual(U)
    # closed form: sum over the node's cells of rho_K hx hy w_a w_b (Simpson weights)
    simpson = np.array([1.0, 4.0, 1.0]) / 6.0
    mass = np.zeros(mesh.n_nodes)
    kin = np.zeros(mesh.n_nodes)
    for cell in range(mesh.n_cells):
        rho = mat.rho_s if mesh.cell_solid[cell] else mat.rho_f
        area = mesh.hx[cell] * mesh.hy[cell]
        for l in range(9):
            node = mesh.cell_nodes[cell, l]
            wgt = area * simpson[l % 3] * simpson[l // 3]
            mass[node] += rho * wgt
            if mesh.cell_solid[cell]:
                kin[node] += wgt
    free_v = ~prob.ident[:, 0]
    np.testing.assert_allclose(R[free_v, 0:2], mass[free_v, None] * c, rtol=1e-13, atol=0)
    # kinematic rows: (u_n - u_{n-1}) - k (theta v_n + (1 - theta) v_{n-1}) = -k theta c on the solid
    kin_rows = mesh.node_in_solid & ~prob.ident[:, 2]
    assert kin_rows.sum() > 0
    np.testing.assert_allclose(R[kin_rows, 2:4], -k * theta * kin[kin_rows, None] * c, rtol=1e-13, atol=0)
    # nodes whose cells are all solid see rho_s only, all fluid rho_f only
    only_s = free_v & (mass > 0) & np.isclose(mass, mat.rho_s * kin)
    only_f = free_v & ~mesh.node_in_solid
    assert only_s.sum() > 0 and only_f.sum() > 0
    ratio_s = R[only_s, 0] / (c[0] * kin[only_s])
    np.testing.assert_allclose(ratio_s, mat.rho_s, rtol=1e-13)
    # the rest of the residual vanishes
    assert np.abs(R[~mesh.node_in_solid & ~prob.ident[:, 2], 2:4]).max() <= 1e-12
    assert np.abs(R[~prob.ident[:, 4], 4]).max() <= 1e-12
