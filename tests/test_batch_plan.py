"""Host side of the batch runner (no GPU): mesh sizes without a context, the
seeded uneven batch, and the longest-first schedule the runner follows."""
import numpy as np
import pytest

from oracle import fsi as of
from paper_1907_01252_gb300 import workloads as wl


@pytest.fixture(scope="module")
def fsi():
    from paper_1907_01252_gb300 import build, fsi as mod
    build.build_library()
    return mod


@pytest.mark.parametrize("nx,ny", [(16, 4), (64, 16), (128, 32), (7, 3)])
def test_mesh_size_matches_oracle_mesh_and_q2_pattern_count(fsi, nx, ny):
    w = wl.Workload("m", nx=nx, ny=ny, T=1.0, n_slices=1, m_fine=1)
    nodes, dofs, nnzb = fsi.mesh_size(w)
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    assert (nodes, dofs) == (mesh.n_nodes, mesh.n_dofs)
    # Q2 on a tensor grid of n cells couples 8n + 1 node pairs per axis
    # (interior vertices 5 partners, end vertices 3, edge midpoints 3)
    assert nnzb == (8 * nx + 1) * (8 * ny + 1)
    # and that is the number of node pairs sharing a cell in the oracle mesh
    pairs = set()
    for cell in mesh.cell_nodes:
        for a in cell:
            for b in cell:
                pairs.add((int(a), int(b)))
    assert nnzb == len(pairs)


def test_uneven_batch_is_seeded_and_in_range():
    a, b = wl.uneven_batch(), wl.uneven_batch()
    assert a == b and len(a) == 48
    assert wl.uneven_batch(seed=7) != a
    for w in a:
        assert 16 <= w.ny <= 48 and w.nx == 4 * w.ny
        assert 16 <= w.n_slices <= 32 and w.m_fine == 16 and w.T == 1.0
        m = w.material
        assert 2e5 <= m.mu_s <= 2e6 and m.lambda_s == pytest.approx(4 * m.mu_s, rel=1e-15)
        assert 0.5 <= m.vbar <= 1.5
    mus = np.log([w.material.mu_s for w in a])
    assert mus.min() < np.log(4e5) and mus.max() > np.log(1e6)   # spread over the range


def _plan(fsi, workloads, workers, max_iter=1):
    return fsi.Batch(workloads, max_iter=max_iter, device_states=False).plan(workers)


@pytest.mark.parametrize("workers", [1, 3, 8, 64])
def test_longest_first_schedule_obeys_the_list_scheduling_bounds(fsi, workers):
    ws = wl.uneven_batch()
    p = _plan(fsi, ws, workers)
    cost = np.array(p["cost"])
    assert sorted(p["order"]) == list(range(len(ws)))
    assert np.all(np.diff(cost[p["order"]]) <= 0)                 # longest first
    assert all(0 <= k < workers for k in p["worker"])
    load = np.zeros(workers)
    for i, k in enumerate(p["worker"]):
        load[k] += cost[i]
    assert p["makespan"] == pytest.approx(load.max(), rel=1e-12)
    total, biggest = cost.sum(), cost.max()
    assert p["makespan"] >= max(total / workers, biggest) * (1 - 1e-12)          # no schedule beats this
    assert p["makespan"] <= total / workers + (1 - 1 / workers) * biggest + 1e-6 * total   # greedy list bound
    if workers == 1:
        assert p["makespan"] == pytest.approx(total, rel=1e-12)
    if workers >= len(ws):
        assert p["makespan"] == pytest.approx(biggest, rel=1e-12)
        assert len(set(p["worker"])) == len(ws)


def test_cost_scales_with_dofs_and_fine_work(fsi):
    m = wl.Material()
    a = wl.Workload("a", nx=64, ny=16, T=1.0, n_slices=16, m_fine=16, material=m)
    b = wl.Workload("b", nx=128, ny=32, T=1.0, n_slices=16, m_fine=16, material=m)
    c = wl.Workload("c", nx=64, ny=16, T=1.0, n_slices=16, m_fine=32, material=m)
    p = _plan(fsi, [a, b, c], 2)
    ca, cb, cc = p["cost"]
    assert cb / ca == pytest.approx(fsi.mesh_size(b)[1] / fsi.mesh_size(a)[1], rel=1e-12)
    assert cc > ca
    # more Parareal iterations cost more
    assert _plan(fsi, [a], 1, max_iter=3)["cost"][0] > ca


def test_bad_plan_arguments_are_rejected(fsi):
    with pytest.raises(fsi.FsiError) as e:
        _plan(fsi, wl.uneven_batch(n=2), 0)
    assert e.value.code == fsi.FSI_EINVAL


@pytest.mark.parametrize("w", [wl.SMALL_16x4, wl.LARGE_128x32])
def test_tip_node_is_the_oracle_mesh_node_at_the_bar_tip(w):
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    t = wl.tip_node(w)
    assert abs(mesh.node_x[t] - 0.65) < 1e-12 and abs(mesh.node_y[t] - 0.2) < 1e-12


def test_argument_errors_are_reported_before_any_device_work(fsi):
    """These checks run on the host before any CUDA call, so they need no GPU."""
    import ctypes as C
    lib = fsi.load_library()
    ws = wl.uneven_batch(n=2)
    b = fsi.Batch(ws, max_iter=1, device_states=False)
    # workers < 1, negative count, null states
    assert lib.fsi_batch_parareal(b._inst, 2, 0, None) == fsi.FSI_EINVAL
    assert lib.fsi_batch_parareal(b._inst, -1, 1, None) == fsi.FSI_EINVAL
    assert lib.fsi_batch_parareal(b._inst, 2, 1, None) == fsi.FSI_EINVAL       # U pointers are NULL
    assert "null state" in lib.fsi_last_error().decode()
    assert lib.fsi_batch_parareal(b._inst, 0, 1, None) == fsi.FSI_OK           # nothing to do
    cand = (C.c_int * 2)(1, 0)
    secs = (C.c_double * 2)()
    best = C.c_int()
    assert lib.fsi_batch_autotune(b._inst, 2, cand, 2, secs, C.byref(best), None) == fsi.FSI_EINVAL
    assert lib.fsi_dense_invert(0, 5, None, None, 0, None) == fsi.FSI_EINVAL
    assert lib.fsi_dense_invert(1, 5, None, None, 2, None) == fsi.FSI_EINVAL
    nodes, dofs, nnzb = C.c_int(), C.c_int(), C.c_int()
    bad = fsi.fsi_mesh()
    assert lib.fsi_mesh_size(C.byref(bad), C.byref(nodes), C.byref(dofs), C.byref(nnzb)) == fsi.FSI_EINVAL
