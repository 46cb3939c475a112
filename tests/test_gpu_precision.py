"""Precision variants against the FP64 oracle through the C ABI.

precision = 1: the whole linear solver (FGMRES, multigrid, Vanka, operator) in
FP32 inside the FP64 Newton loop; precision = 2: FP64 FGMRES on the FP64
Jacobian with the multigrid preconditioner in FP32. The Newton residual stays
FP64 in both, so the converged step solves the same discrete equations: the
target is <= 1e-8 relative error in the bar-tip displacement (and per field);
mode 2 keeps the FP64 tolerances and is held to the FP64 parity bar (1e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi as of  # noqa: E402
from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

FIELDS = {"v": slice(0, 2), "u": slice(2, 4), "p": slice(4, 5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def rel(got, ref, sl):
    den = np.linalg.norm(ref[:, sl])
    return np.linalg.norm(got[:, sl] - ref[:, sl]) / (den if den > 0 else 1.0)


def tip_node(mesh):
    (x0, x1), (_, y1) = wl.SOLID_BOX
    d = (mesh.node_x - 0.5 * (x0 + x1)) ** 2 + (mesh.node_y - y1) ** 2
    i = int(np.argmin(d))
    assert d[i] < 1e-20
    return i


TOL = {1: 1e-8, 2: 1e-10}


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_solver_fine_propagator_matches_fp64_oracle(precision):
    from paper_1907_01252_gb300 import fsi
    w = wl.Workload("p32", nx=16, ny=4, T=0.5, n_slices=4, m_fine=4)
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    model = of.FSIModel(mesh, w.material)
    dt = w.T / w.n_slices
    U0 = np.zeros((2, mesh.n_nodes, 5))
    U0[1] = model.propagate(U0[0], 0.0, dt, 8)
    ctx = fsi.Context(w, max_batch=2, precision=precision)
    dev = torch.tensor(U0.reshape(2, -1), dtype=torch.float64, device="cuda:0")
    Uf, stats = ctx.fsi_fine(dev, [0.0, dt])
    got = Uf.cpu().numpy().reshape(2, -1, 5)
    tip = tip_node(mesh)
    for s in range(2):
        ref = model.propagate(U0[s], s * dt, (s + 1) * dt, w.m_fine)
        for name, sl in FIELDS.items():
            assert rel(got[s], ref, sl) <= TOL[precision], (s, name)
        assert np.linalg.norm(got[s][tip, 2:4] - ref[tip, 2:4]) <= TOL[precision] * np.linalg.norm(ref[tip, 2:4])
    # batched equals single-slice runs bit for bit in FP32 too
    Us, _ = ctx.fsi_fine(dev[1:2].contiguous(), [dt])
    assert torch.equal(Us[0], Uf[1])


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_solver_coarse_step_matches_fp64_oracle(precision):
    from paper_1907_01252_gb300 import fsi
    w = wl.SMALL_16x4
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    model = of.FSIModel(mesh, w.material)
    U0 = model.propagate(np.zeros((mesh.n_nodes, 5)), 0.0, 0.1, 4)
    K = w.k_coarse
    ctx = fsi.Context(w, max_batch=1, precision=precision)
    U1, stats = ctx.fsi_theta_step(torch.tensor(U0.reshape(1, -1), device="cuda:0"), [0.1], K, 1.0)
    got = U1.cpu().numpy().reshape(-1, 5)
    ref = model.step(U0, 0.1, K, 1.0)
    for name, sl in FIELDS.items():
        assert rel(got, ref, sl) <= TOL[precision], name
