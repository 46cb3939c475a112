"""Pins of the d-dimensional oracle (oracle/fsi_nd.py) on the CPU.

At d = 2 it must reproduce the 2D oracle (an independent writing of the same
formulas, itself pinned in test_oracle_fsi.py). At d = 3 the pins come from
facts that do not depend on its code:
  * z-independent fields on an extruded mesh reduce every row to the 2D row
    times the integral of the 1D quadratic basis function in z;
  * exchanging the y and z axes (mesh, data, state) permutes the residual;
  * tensor helpers against numpy.linalg, Jacobi's formula for d det;
  * divergence-free affine fields, rigid motions of the solid, the Q1 kernel
    of the stabilisation, the mean of the inflow profile;
  * the Jacobian against central differences, quadratic Newton convergence.
"""
import numpy as np
import pytest

from oracle import fsi as of
from oracle import fsi_nd as on
from paper_1907_01252_gb300 import workloads as wl

XB = (0.0, 0.6, 0.7, 2.0)
YB = (0.0, 0.2, 0.41)
ZB = (0.0, 0.15, 0.41)


def state_nd(mesh, seed, v=1.0, u=2e-3, p=100.0):
    rng = np.random.default_rng(seed)
    d = mesh.d
    U = np.empty((mesh.n_nodes, mesh.nc))
    U[:, 0:d] = v * rng.uniform(-1, 1, (mesh.n_nodes, d))
    U[:, d:2 * d] = u * rng.uniform(-1, 1, (mesh.n_nodes, d))
    U[:, 2 * d] = p * rng.uniform(-1, 1, mesh.n_nodes)
    return U


def test_generic_oracle_in_2d_equals_the_2d_oracle():
    w = wl.Workload("t", nx=16, ny=4, T=1.0, n_slices=2, m_fine=2)
    m2 = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    mn = on.make_mesh_nd([wl.X_BREAKS, wl.Y_BREAKS], [w.nx_seg, w.ny_seg], wl.SOLID_BOX)
    assert np.array_equal(mn.cell_nodes, m2.cell_nodes)
    U, Uo = wl.random_state(m2.n_nodes, 1), wl.random_state(m2.n_nodes, 2)
    mat, k, th = w.material, 0.01, 0.51
    p2 = of.StepProblem(m2, mat, Uo, 0.3, k, th)
    pn = on.StepProblemND(mn, mat, Uo, 0.3, k, th)
    R2, Rn = p2.residual(U), pn.residual(U)
    assert np.abs(R2 - Rn).max() <= 1e-13 * np.abs(R2).max()
    A2, An = p2.jacobian(U), pn.jacobian(U)
    assert abs(A2 - An).max() <= 1e-13 * abs(A2).max()
    # one Newton-solved step from rest
    Z = np.zeros((m2.n_nodes, 5))
    s2 = of.FSIModel(m2, mat).step(Z, 0.1, 0.05, 1.0)
    sn = on.FSIModelND(mn, mat).step(Z, 0.1, 0.05, 1.0)
    assert np.abs(s2 - sn).max() <= 1e-11 * np.abs(s2).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_3d_tensor_helpers_match_numpy_and_jacobi(seed):
    rng = np.random.default_rng(seed)
    A = np.eye(3) + 0.3 * rng.standard_normal((5, 3, 3))
    assert np.allclose(on.det(A), np.linalg.det(A), rtol=1e-14, atol=0)
    assert np.allclose(on.inv(A), np.linalg.inv(A), rtol=1e-12, atol=1e-14)
    assert np.allclose(np.einsum("...ij,...jk->...ik", A, on.adjugate(A)),
                       on.det(A)[:, None, None] * np.eye(3), atol=1e-13)
    # Jacobi: d det(A)[dA] = tr(adj(A) dA), against a complex step of det
    dA = rng.standard_normal((5, 3, 3))
    h = 1e-30
    cs = on.det(A + 1j * h * dA).imag / h
    assert np.allclose(cs, np.einsum("...ij,...ji->...", on.adjugate(A), dA), rtol=1e-13)


def test_3d_basis_partition_of_unity():
    mesh = on.make_mesh_nd([(0, 1), (0, 1), (0, 1)], [[2], [1], [1]])
    tab = on.CellTablesND(mesh)
    assert tab.phi.shape == (27, 27)
    assert np.allclose(tab.phi.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(tab.dphi.sum(axis=2), 0.0, atol=1e-12)
    assert np.isclose(tab.W.sum(), 1.0)


def extruded(nx, ny, nz, solid):
    counts = [wl.cells_per_segment(XB, nx), wl.cells_per_segment(YB, ny)]
    box2 = ((0.6, 0.7), (0.0, 0.2)) if solid else None
    m2 = on.make_mesh_nd([XB, YB], counts, box2)
    box3 = ((0.6, 0.7), (0.0, 0.2), (ZB[0], ZB[-1])) if solid else None
    m3 = on.make_mesh_nd([XB, YB, ZB], counts + [wl.cells_per_segment(ZB, nz)], box3)
    return m2, m3


def test_3d_extruded_z_independent_fields_reduce_to_2d_rows():
    m2, m3 = extruded(8, 2, 2, solid=True)
    mat = wl.Material(alpha0=0.0)          # the cell stabilisation is not a tensor product in z
    t2, t3 = on.CellTablesND(m2), on.CellTablesND(m3)
    U2, Uo2 = state_nd(m2, 3), state_nd(m2, 4)

    def lift(U):
        n2 = m2.n_nodes
        U3 = np.zeros((m3.n_nodes, 7))
        idx = np.arange(m3.n_nodes) % n2          # node (i, j, kz) -> (i, j)
        U3[:, [0, 1, 3, 4, 6]] = U[idx][:, [0, 1, 2, 3, 4]]
        return U3
    U3, Uo3 = lift(U2), lift(Uo2)
    k, th = 0.02, 0.6
    R2 = on.element_residual_nd(m2, t2, mat, U2[m2.cell_nodes], Uo2[m2.cell_nodes], k, th, np.zeros(m2.n_cells))
    R3 = on.element_residual_nd(m3, t3, mat, U3[m3.cell_nodes], Uo3[m3.cell_nodes], k, th, np.zeros(m3.n_cells))
    n2c = m2.n_cells
    scale = np.abs(R2).max(axis=(0, 1))
    for c3 in range(m3.n_cells):
        c2, cz = c3 % n2c, c3 // n2c
        hz = m3.h[c3, 2]
        for c in range(3):
            wz = hz * (1 / 6, 2 / 3, 1 / 6)[c]
            rows = R3[c3, 9 * c:9 * c + 9]
            for j3, j2 in ((0, 0), (1, 1), (3, 2), (4, 3), (6, 4)):
                assert np.all(np.abs(rows[:, j3] - wz * R2[c2, :, j2]) <= 1e-12 * scale[j2]), (c3, c, j3)
            assert np.all(np.abs(rows[:, 5]) <= 1e-15 * scale[2])            # u_z rows
        # z-momentum rows: only the z-derivative of the test function, summing to zero over the z-nodes
        vz = R3[c3].reshape(3, 9, 7)[:, :, 2].sum(axis=0)
        assert np.all(np.abs(vz) <= 1e-12 * scale[0])


def test_3d_residual_is_symmetric_under_y_z_exchange():
    ax = [np.array([0.0, 0.3, 0.6, 0.7, 1.0]), np.array([0.0, 0.1, 0.2, 0.3, 0.41])]
    mesh = on.MeshND([ax[0], ax[1], ax[1]], ((0.6, 0.7), (0.1, 0.3), (0.1, 0.3)))
    assert mesh.cell_solid.sum() == 4
    nx, ny = mesh.nnode[0], mesh.nnode[1]
    i, j, kz = mesh.node_idx
    swap = i + nx * (kz + ny * j)                  # node (i, j, k) <-> (i, k, j)
    comps = [0, 2, 1, 3, 5, 4, 6]
    U, Uo = state_nd(mesh, 5), state_nd(mesh, 6)
    Us, Uos = U[swap][:, comps], Uo[swap][:, comps]
    mat = wl.Material()
    k, th = 0.02, 0.55
    R = on.StepProblemND(mesh, mat, Uo, 0.1, k, th).residual(U)
    Rs = on.StepProblemND(mesh, mat, Uos, 0.1, k, th).residual(Us)
    assert np.abs(Rs - R[swap][:, comps]).max() <= 1e-12 * np.abs(R).max()


def test_3d_affine_divergence_free_velocity_has_zero_divergence_rows():
    mesh = on.make_mesh_nd([(0, 0.5, 1.0), (0, 0.4), (0, 0.3)], [[2, 1], [2], [1]])
    tab = on.CellTablesND(mesh)
    rng = np.random.default_rng(7)
    B = 0.02 * rng.standard_normal((3, 3))             # affine mesh displacement u = B x, F = I + B
    C = rng.standard_normal((3, 3))
    C -= np.trace(C) / 3 * np.eye(3)                   # tr C = 0, v = C F x: grad v F^{-1} = C
    X = mesh.node_xyz
    U = np.zeros((mesh.n_nodes, 7))
    U[:, 0:3] = X @ (C @ (np.eye(3) + B)).T
    U[:, 3:6] = X @ B.T
    U[:, 6] = rng.standard_normal(mesh.n_nodes)
    Re = on.element_residual_nd(mesh, tab, wl.Material(), U[mesh.cell_nodes], U[mesh.cell_nodes], 0.1, 0.5,
                                np.zeros(mesh.n_cells))
    assert np.abs(Re[..., 6]).max() <= 1e-13 * np.abs(Re[..., 0:3]).max()


def test_3d_rigid_motion_of_the_solid_has_zero_stress():
    mesh = on.MeshND([np.linspace(0, 1, 3), np.linspace(0, 1, 2), np.linspace(0, 1, 2)],
                     ((-1, 2), (-1, 2), (-1, 2)))
    assert mesh.cell_solid.all()
    tab = on.CellTablesND(mesh)
    a = 0.4
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    Q = Rz @ Rx                                     # finite rotation: F = Q, E = 0
    X = mesh.node_xyz
    U = np.zeros((mesh.n_nodes, 7))
    U[:, 0:3] = 0.3                                # v = v_old: no mass contribution
    U[:, 3:6] = X @ (Q - np.eye(3)).T + np.array([0.1, -0.2, 0.05])
    U[:, 6] = 0.0
    mat = wl.Material()
    k = 0.01
    Re = on.element_residual_nd(mesh, tab, mat, U[mesh.cell_nodes], U[mesh.cell_nodes], k, 0.5,
                                np.zeros(mesh.n_cells))
    scale = k * mat.mu_s * 0.4                     # stress scale of a comparable strain
    assert np.abs(Re[..., 0:3]).max() <= 1e-10 * scale


def test_3d_stabilisation_kernel_is_q1_and_rank_19():
    mesh = on.make_mesh_nd([(0, 0.3), (0, 0.2), (0, 0.25)], [[1], [1], [1]])
    tab = on.CellTablesND(mesh)
    S = tab.S_lps[0]
    X = mesh.node_xyz[mesh.cell_nodes[0]]
    for f in (np.ones(27), X[:, 0], X[:, 1] * X[:, 2], X[:, 0] * X[:, 1] * X[:, 2]):
        assert np.abs(S @ f).max() <= 1e-12 * np.abs(S).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev.min() >= -1e-12 * ev.max()
    assert int((ev > 1e-10 * ev.max()).sum()) == 27 - 8
    assert np.abs(S @ (X[:, 0] ** 2)).max() > 1e-6 * np.abs(S).max()


def test_3d_inflow_profile_has_mean_vbar():
    mesh = on.make_mesh_nd([(0, 1.5), (0, 0.41), (0, 0.41)], [[1], [2], [2]])
    mat = wl.Material(vbar=1.3, ramp_t=0.2)
    g = on.dirichlet_values_nd(mesh, mat, 1.0)
    # Q2 interpolation is exact for the biquadratic profile: integrate it over the inflow face
    face = mesh.on_inflow
    y, z = mesh.node_xyz[face, 1], mesh.node_xyz[face, 2]
    vals = g[face, 0]
    ny, nz = mesh.nnode[1], mesh.nnode[2]
    V = vals.reshape(nz, ny)
    yy, zz = np.unique(y), np.unique(z)
    # composite Simpson on the Q2 node grid (exact for quadratics in each variable)
    def simpson_w(x):
        w = np.zeros(len(x))
        for c in range(0, len(x) - 2, 2):
            h = x[c + 2] - x[c]
            w[c:c + 3] += h * np.array([1, 4, 1]) / 6
        return w
    integral = simpson_w(zz) @ V @ simpson_w(yy)
    assert integral / (0.41 * 0.41) == pytest.approx(1.3, rel=1e-13)
    assert np.abs(g[~face]).max() == 0.0


def small_3d():
    counts = [[2, 1, 2], [1, 1], [1, 1, 1]]
    return on.make_mesh_nd([(0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41)], counts,
                           ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355)))


def test_3d_jacobian_matches_central_differences():
    mesh = small_3d()
    assert mesh.cell_solid.sum() == 1
    U, Uo = state_nd(mesh, 8), state_nd(mesh, 9)
    prob = on.StepProblemND(mesh, wl.Material(), Uo, 0.15, 0.02, 0.52)
    A = prob.jacobian(U).toarray()
    rng = np.random.default_rng(10)
    for _ in range(3):
        dU = rng.standard_normal(U.shape) * np.array([1, 1, 1, 1e-3, 1e-3, 1e-3, 100.0])
        h = 1e-6
        fd = (prob.residual(U + h * dU) - prob.residual(U - h * dU)).ravel() / (2 * h)
        lin = A @ dU.ravel()
        assert np.abs(fd - lin).max() <= 2e-5 * np.abs(lin).max()


def test_3d_newton_converges_quadratically():
    """Fine steps from rest through the inflow ramp; the last step's residuals
    decay quadratically (relative to the first residual of the step)."""
    mesh = small_3d()
    model = on.FSIModelND(mesh, wl.Material())
    U = np.zeros((mesh.n_nodes, 7))
    k = 1 / 64
    for n in range(4):
        prob = on.StepProblemND(mesh, model.mat, U, (n + 1) * k, k, model.theta_fine(k), model.tab)
        U, info = of.newton_solve(prob, U)
    r = info.residual_norms
    assert info.converged and len(r) >= 3
    for a, b in zip(r[:-1], r[1:]):
        if a > 1e-9 * r[0]:
            assert b <= 10 * a ** 2 / r[0] + 1e-12 * r[0], r


def test_3d_channel_mesh_of_the_32x8x8_workload():
    """The 3D workload: 32 x 8 x 8 hexahedral Q2 cells, 18,785 nodes, 7 unknowns per node (131,495 dofs)."""
    counts = wl.cells_per_segment_3d(32, 8, 8)
    assert counts == ((9, 1, 22), (4, 4), (1, 6, 1))
    mesh = on.make_mesh_nd([wl.X3_BREAKS, wl.Y3_BREAKS, wl.Z3_BREAKS], counts, wl.SOLID_BOX_3D)
    assert mesh.n_nodes == 65 * 17 * 17 == 18785 and mesh.n_dofs == 131495
    assert mesh.cell_solid.sum() == 1 * 4 * 6                  # the plate is resolved by cell faces
    assert np.isclose(mesh.axes[0][9], 0.4) and np.isclose(mesh.axes[0][10], 0.45)


def test_library_3d_mesh_size_matches_the_oracle_mesh():
    """fsi3d_mesh_size (host code of the CUDA library) against the oracle mesh and the Q2 pattern count."""
    from paper_1907_01252_gb300 import build, fsi
    build.build_library()
    counts = wl.cells_per_segment_3d(32, 8, 8)
    nodes, dofs, nnzb = fsi.mesh3d_size([wl.X3_BREAKS, wl.Y3_BREAKS, wl.Z3_BREAKS], counts, wl.SOLID_BOX_3D)
    assert (nodes, dofs) == (18785, 131495)
    assert nnzb == (8 * 32 + 1) * (8 * 8 + 1) * (8 * 8 + 1) == 1085825
    small = ((2, 1, 2), (1, 1), (1, 1, 1))
    br = ((0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41))
    m = on.make_mesh_nd(br, small, ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355)))
    n, d, b = fsi.mesh3d_size(br, small)
    pairs = {(int(a), int(c)) for cell in m.cell_nodes for a in cell for c in cell}
    assert (n, d, b) == (m.n_nodes, m.n_dofs, len(pairs))
