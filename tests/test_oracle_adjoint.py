"""Pins of the oracle's discrete adjoint (CPU only): the old-state Jacobian
against central differences, and the adjoint gradient of the bar-tip
functional against central differences of the functional itself."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import fsi as of
from paper_1907_01252_gb300 import workloads as wl

MAT = wl.Material()


@pytest.fixture(scope="module")
def setup():
    mesh = of.make_mesh(wl.X_BREAKS, wl.Y_BREAKS, wl.cells_per_segment(wl.X_BREAKS, 8),
                        wl.cells_per_segment(wl.Y_BREAKS, 2), wl.SOLID_BOX)
    model = of.FSIModel(mesh, MAT, newton_tol=1e-13)
    k = 1 / 200
    Us = oa.trajectory(model, np.zeros((mesh.n_nodes, 5)), 0.0, k, 6)
    return mesh, model, k, Us


def test_old_state_jacobian_matches_central_differences(setup):
    mesh, model, k, Us = setup
    U, Uo = Us[6], Us[5]
    B = oa.old_state_jacobian(mesh, model.tab, MAT, U, Uo, 6 * k, k, 0.5 + k).toarray()

    def R_of_old(Uold):
        return of.StepProblem(mesh, MAT, Uold, 6 * k, k, 0.5 + k, model.tab).residual(U).ravel()

    rng = np.random.default_rng(0)
    for j in rng.choice(mesh.n_dofs, 30, replace=False):
        h = 1e-6 * max(abs(Uo.ravel()[j]), 1e-3)
        e = np.zeros(mesh.n_dofs)
        e[j] = h
        fd = (R_of_old((Uo.ravel() + e).reshape(-1, 5)) - R_of_old((Uo.ravel() - e).reshape(-1, 5))) / (2 * h)
        noise = 1e-13 * np.abs(R_of_old(Uo)).max() / h
        assert np.abs(fd - B[:, j]).max() <= 1e-5 * np.abs(B[:, j]).max() + noise


def test_adjoint_gradient_matches_central_differences(setup):
    mesh, model, k, Us = setup
    tip = oa.tip_node(mesh, wl.SOLID_BOX)
    J, grad = oa.adjoint_gradient(model, Us[3], 3 * k, k, 5, tip)

    def J_of(**kw):
        mo = of.FSIModel(mesh, dataclasses.replace(MAT, **kw), newton_tol=1e-13)
        return oa.tip_functional(oa.trajectory(mo, Us[3], 3 * k, k, 5), k, tip)

    assert J == pytest.approx(J_of(), rel=1e-12)
    for i, name in enumerate(("mu_s", "lambda_s", "vbar")):
        v = getattr(MAT, name)
        h = 1e-4 * v
        fd = (J_of(**{name: v + h}) - J_of(**{name: v - h})) / (2 * h)
        assert abs(grad[i] - fd) <= 1e-5 * abs(fd), (name, grad[i], fd)
