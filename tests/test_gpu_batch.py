"""The batch runner on the GPU: independent problems of uneven meshes,
materials and slice counts run concurrently by worker threads; each result is
bit-identical to the problem run alone, one problem matches the FP64 oracle's
Parareal iterate, and a failing problem leaves the others untouched."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi as of  # noqa: E402
from oracle import parareal as opr  # noqa: E402
from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def small_uneven():
    """Four small problems: meshes 16x4 .. 32x8, different materials and slice counts."""
    out = []
    for i, (nx, ny, slices, mu, vbar) in enumerate([(16, 4, 3, 3e5, 0.8), (24, 6, 2, 1.2e6, 1.3),
                                                    (32, 8, 4, 5e5, 1.0), (20, 5, 3, 2e6, 0.6)]):
        out.append(wl.Workload("b%d" % i, nx=nx, ny=ny, T=0.03 * slices, n_slices=slices, m_fine=4,
                               material=wl.Material(mu_s=mu, lambda_s=4 * mu, vbar=vbar)))
    return out


def solo(w, max_iter):
    from paper_1907_01252_gb300 import fsi
    ctx = fsi.Context(w, max_batch=w.n_slices)
    U = torch.zeros((w.n_slices + 1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    U, st = ctx.parareal_iterate(U, max_iter, 0.0)
    return U, st


def test_batch_results_are_bitwise_solo_runs_and_match_the_oracle():
    from paper_1907_01252_gb300 import fsi
    ws = small_uneven()
    batch = fsi.Batch(ws, max_iter=2)
    res = batch.run(workers=3)
    assert all(r["status"] == 0 for r in res)
    assert {r["worker"] for r in res} <= {0, 1, 2}
    for w, U, r in zip(ws, batch.states, res):
        ref, st = solo(w, 2)
        assert torch.equal(U, ref), w.name
        assert r["stats"]["iterations"] == st["iterations"] == 2
        assert r["stats"]["fine"]["gmres_iters"] == st["fine"]["gmres_iters"]
    # the problem with a non-default material against the oracle's Parareal iterate
    w = ws[1]
    mesh = of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)
    model = of.FSIModel(mesh, w.material)
    dt = w.T / w.n_slices
    fine = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, w.m_fine)
    coarse = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, 1, theta=1.0)
    hist = opr.parareal(np.zeros((mesh.n_nodes, 5)), w.n_slices, coarse, fine, 2)
    got = batch.states[1].cpu().numpy().reshape(w.n_slices + 1, -1, 5)
    for n in range(1, w.n_slices + 1):
        for sl in (slice(0, 2), slice(2, 4), slice(4, 5)):
            ref = hist[2][n][:, sl]
            den = np.linalg.norm(ref)
            assert np.linalg.norm(got[n][:, sl] - ref) <= 1e-10 * (den if den > 0 else 1.0), (n, sl)


def test_failing_problem_reports_its_status_and_spares_the_others():
    from paper_1907_01252_gb300 import fsi
    ws = small_uneven()
    ws[2] = dataclasses.replace(ws[2], newton_maxit=1)     # a theta = 1 coarse step needs more than one iteration
    batch = fsi.Batch(ws, max_iter=1)
    with pytest.raises(fsi.FsiError) as e:
        batch.run(workers=2)
    assert e.value.code == fsi.FSI_ENEWTON
    res = batch.results()
    assert [r["status"] for r in res] == [0, 0, fsi.FSI_ENEWTON, 0]
    for i in (0, 1, 3):
        ref, _ = solo(ws[i], 1)
        assert torch.equal(batch.states[i], ref)


def test_autotuner_picks_a_candidate_and_keeps_the_results():
    from paper_1907_01252_gb300 import fsi
    ws = small_uneven()
    batch = fsi.Batch(ws, max_iter=1)
    best, secs = batch.autotune([1, 2, 4])
    assert best in (1, 2, 4)
    assert len(secs) == 3 and all(s > 0 for s in secs)
    assert secs[[1, 2, 4].index(best)] == min(secs)
    for w, U in zip(ws, batch.states):
        ref, _ = solo(w, 1)
        assert torch.equal(U, ref)


def test_bad_batch_arguments_are_rejected():
    from paper_1907_01252_gb300 import fsi
    batch = fsi.Batch(small_uneven()[:1], max_iter=1)
    with pytest.raises(fsi.FsiError) as e:
        batch.run(workers=0)
    assert e.value.code == fsi.FSI_EINVAL
