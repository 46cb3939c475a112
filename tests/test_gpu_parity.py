"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the residual and the Jacobian are the same finite sums evaluated
in a different order, so they agree to a few hundred ulps of the largest
term (1e-12 relative to the largest entry). States after Newton solves agree
to the 1e-10 relative accuracy the library targets (field by field: v, u, p).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi as of  # noqa: E402
from oracle import parareal as opr  # noqa: E402
from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"
FIELDS = {"v": slice(0, 2), "u": slice(2, 4), "p": slice(4, 5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def ctx_for(w, S, **kw):
    from paper_1907_01252_gb300 import fsi
    return fsi.Context(w, max_batch=S, **kw)


def oracle_mesh(w):
    return of.mesh_for(w, wl.X_BREAKS, wl.Y_BREAKS, wl.SOLID_BOX)


def to_dev(a):
    return torch.tensor(np.asarray(a).reshape(a.shape[0], -1), dtype=torch.float64, device=DEV)


def rel_field_errors(got, ref):
    out = {}
    for name, sl in FIELDS.items():
        den = np.linalg.norm(ref[..., sl])
        out[name] = np.linalg.norm(got[..., sl] - ref[..., sl]) / (den if den > 0 else 1.0)
    return out


# 16 x 4 is the small workload; 24 x 6 puts odd segment counts in the
# multigrid hierarchy; 36 x 10 spans more cells than one reduction chunk.
MESHES = [(16, 4), (24, 6), (36, 10)]


@pytest.mark.parametrize("nx,ny", MESHES)
def test_residual_matches_oracle(nx, ny):
    w = wl.Workload(f"r{nx}", nx=nx, ny=ny, T=1.0, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    S = 3
    U = np.stack([wl.random_state(mesh.n_nodes, 100 + s) for s in range(S)])
    Uo = np.stack([wl.random_state(mesh.n_nodes, 200 + s) for s in range(S)])
    t_new = [0.05, 0.13, 0.7]
    k, th = 1e-2, 0.51
    ctx = ctx_for(w, S)
    R = ctx.fsi_residual(to_dev(U), to_dev(Uo), t_new, k, th).cpu().numpy().reshape(S, -1, 5)
    for s in range(S):
        prob = of.StepProblem(mesh, w.material, Uo[s], t_new[s], k, th)
        ref = prob.residual(U[s])
        assert np.abs(R[s] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny", MESHES[:2])
def test_jacobian_matches_oracle(nx, ny):
    w = wl.Workload(f"j{nx}", nx=nx, ny=ny, T=1.0, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    S = 2
    U = np.stack([wl.random_state(mesh.n_nodes, 300 + s) for s in range(S)])
    Uo = np.stack([wl.random_state(mesh.n_nodes, 400 + s) for s in range(S)])
    k, th = 1e-2, 0.51
    ctx = ctx_for(w, S)
    vals = ctx.fsi_jacobian(to_dev(U), to_dev(Uo), k, th).cpu().numpy()
    rowptr, colidx = ctx.fsi_bsr_pattern()
    import scipy.sparse as sp
    for s in range(S):
        A = sp.bsr_matrix((vals[s], colidx, rowptr), shape=(mesh.n_dofs, mesh.n_dofs)).toarray()
        prob = of.StepProblem(mesh, w.material, Uo[s], 0.3, k, th)
        ref = prob.jacobian(U[s]).toarray()
        assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


def test_spmv_matches_oracle_matrix():
    w = wl.Workload("spmv", nx=24, ny=6, T=1.0, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    S = 2
    U = np.stack([wl.random_state(mesh.n_nodes, 500 + s) for s in range(S)])
    x = np.stack([wl.random_state(mesh.n_nodes, 600 + s) for s in range(S)])
    ctx = ctx_for(w, S)
    vals = ctx.fsi_jacobian(to_dev(U), to_dev(U), 1e-2, 0.6)
    y = ctx.fsi_bsr_spmv(vals, to_dev(x)).cpu().numpy()
    for s in range(S):
        A = of.StepProblem(mesh, w.material, U[s], 0.2, 1e-2, 0.6).jacobian(U[s])
        ref = A @ x[s].ravel()
        assert np.abs(y[s] - ref).max() <= 1e-12 * (abs(A) @ abs(x[s].ravel())).max()


def test_spmv_f32_and_float_pair_products():
    """The FP32 and float-pair products against the FP64 product of the same values: FP32
    values and vectors within the bound of a sequential FP32 sum (125 terms at most per row
    component: 25 blocks of 5), float pairs within 2^-44 of sum |a x| per row. 36 x 10
    cells: 1,533 rows, 3 slices; one slice alone gives the same bits."""
    import scipy.sparse as sp
    w = wl.Workload("spmv_w", nx=36, ny=10, T=1.0, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    S = 3
    U = np.stack([wl.random_state(mesh.n_nodes, 700 + s) for s in range(S)])
    x = np.stack([wl.random_state(mesh.n_nodes, 800 + s) for s in range(S)])
    ctx = ctx_for(w, S, ff_operator=1)
    vals = ctx.fsi_jacobian(to_dev(U), to_dev(U), 1e-2, 0.6)
    rowptr, colidx = ctx.fsi_bsr_pattern()
    xd = to_dev(x)
    y_ff = ctx.fsi_bsr_spmv_ff(vals, xd).cpu().numpy()
    v32, x32 = vals.float(), xd.float()
    y_32 = ctx.fsi_bsr_spmv_f32(v32, x32).cpu().numpy()
    v32h, x32h = v32.double().cpu().numpy(), x32.double().cpu().numpy()
    vh = vals.cpu().numpy()
    n = mesh.n_dofs
    for s in range(S):
        A = sp.bsr_matrix((vh[s], colidx, rowptr), shape=(n, n))
        ref, mag = A @ x[s].ravel(), abs(A) @ abs(x[s].ravel())
        assert np.all(np.abs(y_ff[s] - ref) <= 2.0 ** -44 * mag)
        A32 = sp.bsr_matrix((v32h[s], colidx, rowptr), shape=(n, n))
        ref32, mag32 = A32 @ x32h[s], abs(A32) @ abs(x32h[s])
        assert np.all(np.abs(y_32[s].astype(np.float64) - ref32) <= 125 * 2.0 ** -24 * mag32 + 1e-38)
    one_ff = ctx.fsi_bsr_spmv_ff(vals[1:2].contiguous(), xd[1:2].contiguous()).cpu().numpy()
    one_32 = ctx.fsi_bsr_spmv_f32(v32[1:2].contiguous(), x32[1:2].contiguous()).cpu().numpy()
    assert np.array_equal(one_ff[0], y_ff[1]) and np.array_equal(one_32[0], y_32[1])


def test_spmv_tile_variants_give_the_same_bits():
    """Every kernel variant of the block product (the row-list kernel and the
    row-tile kernel with 8, 16, 32 and 64 rows per CTA, staged by a bulk copy)
    sums each row component in the same order: identical bits for FP64, FP32
    and float-pair values. 36 x 10 cells: 1,533 node rows, so the last tile is
    ragged for every height; 3 slices. The FP64 product also matches the
    oracle's matrix."""
    import scipy.sparse as sp
    from paper_1907_01252_gb300 import fsi
    w = wl.Workload("spmv_t", nx=36, ny=10, T=1.0, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    S = 3
    U = np.stack([wl.random_state(mesh.n_nodes, 710 + s) for s in range(S)])
    x = np.stack([wl.random_state(mesh.n_nodes, 810 + s) for s in range(S)])
    ctx = ctx_for(w, S, ff_operator=1)
    vals = ctx.fsi_jacobian(to_dev(U), to_dev(U), 1e-2, 0.6)
    xd = to_dev(x)
    for vt, (v, xx) in enumerate(((vals, xd), (vals.float(), xd.float()), (vals, xd))):
        ref = ctx.fsi_bsr_spmv_variant(vt, 0, v, xx).cpu()
        assert torch.isfinite(ref).all()
        for rows in (8, 16, 32, 64):
            try:
                got = ctx.fsi_bsr_spmv_variant(vt, rows, v, xx).cpu()
            except fsi.FsiError as err:   # a tile of 64 rows of 8-byte blocks exceeds shared memory
                assert vt != 1 and rows == 64 and "shared memory" in str(err), (vt, rows, err)
                continue
            assert torch.equal(got, ref), (vt, rows)
        if vt == 0:
            rowptr, colidx = ctx.fsi_bsr_pattern()
            vh, n = vals.cpu().numpy(), mesh.n_dofs
            for s in range(S):
                A = sp.bsr_matrix((vh[s], colidx, rowptr), shape=(n, n))
                assert np.abs(ref[s].numpy() - A @ x[s].ravel()).max() <= 1e-12 * (abs(A) @ abs(x[s].ravel())).max()
    # the library's own products (tuned variant) give the same bits as well
    assert torch.equal(ctx.fsi_bsr_spmv(vals, xd).cpu(), ctx.fsi_bsr_spmv_variant(0, 0, vals, xd).cpu())
    assert torch.equal(ctx.fsi_bsr_spmv_ff(vals, xd).cpu(), ctx.fsi_bsr_spmv_variant(2, 0, vals, xd).cpu())


def developed_states(w, mesh, steps, k):
    model = of.FSIModel(mesh, w.material)
    U = np.zeros((mesh.n_nodes, 5))
    out = []
    for n in range(steps):
        U = model.step(U, n * k, k, model.theta_fine(k))
        out.append(U)
    return model, out


def test_theta_step_matches_oracle_and_batch_is_bitwise_serial():
    w = wl.SMALL_16x4
    mesh = oracle_mesh(w)
    k = w.k_fine
    model, states = developed_states(w, mesh, 12, k)
    pick = [3, 7, 11]
    U0 = np.stack([states[i] for i in pick])
    t0 = [(i + 1) * k for i in pick]
    th = 0.5 + k
    ctx = ctx_for(w, 3)
    Ub, stats = ctx.fsi_theta_step(to_dev(U0), t0, k, th)
    got = Ub.cpu().numpy().reshape(3, -1, 5)
    for s, i in enumerate(pick):
        ref = model.step(U0[s], t0[s], k, th)
        errs = rel_field_errors(got[s], ref)
        assert max(errs.values()) <= 1e-10, errs
        # the same slice alone gives the same bits
        Us, _ = ctx.fsi_theta_step(to_dev(U0[s:s + 1]), [t0[s]], k, th)
        assert torch.equal(Us[0], Ub[s])
    assert stats["max_gmres"] < 200


def test_batched_slices_with_different_krylov_counts_match_solo_runs():
    """Slices of one batch whose FGMRES solves end at different iterations:
    every slice keeps its own Newton correction, so the batch needs exactly the
    Newton and FGMRES iterations of the solo runs and returns their bits."""
    w = wl.SMALL_16x4
    ctx = ctx_for(w, 2)
    K = w.k_coarse
    U = torch.zeros((1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    for i in range(4):                       # a developed state at t = 4K
        U, _ = ctx.fsi_coarse(U, [i * K])
    U0 = torch.cat([torch.zeros_like(U), U]).contiguous()
    t0 = [0.0, 4 * K]
    solo = [ctx.fsi_theta_step(U0[s:s + 1].contiguous(), [t0[s]], K, 1.0) for s in range(2)]
    assert solo[0][1]["gmres_iters"] != solo[1][1]["gmres_iters"]
    Ub, stats = ctx.fsi_theta_step(U0, t0, K, 1.0)
    for key in ("newton_iters", "gmres_iters"):
        assert stats[key] == solo[0][1][key] + solo[1][1][key], key
    for s in range(2):
        assert torch.equal(Ub[s], solo[s][0][0])


def test_inexact_newton_meets_the_parity_bar_with_fewer_krylov_iterations():
    """Inexact Newton (the default forcing) against every solve to gmres_rtol:
    both within 1e-10 of the oracle step, the inexact one with fewer FGMRES
    iterations and the same Newton iteration count."""
    w = wl.SMALL_16x4
    mesh = oracle_mesh(w)
    k = w.k_fine
    model, states = developed_states(w, mesh, 12, k)
    U0, t0, th = states[11], 12 * k, 0.5 + k
    ref = model.step(U0, t0, k, th)
    out = {}
    for eta in (0.0, w.newton_eta):
        ctx = ctx_for(w, 1, newton_eta=eta)
        U1, st = ctx.fsi_theta_step(to_dev(U0[None]), [t0], k, th)
        errs = rel_field_errors(U1.cpu().numpy().reshape(-1, 5), ref)
        assert max(errs.values()) <= 1e-10, (eta, errs)
        out[eta] = st
    assert w.newton_eta > 0
    assert out[w.newton_eta]["gmres_iters"] < out[0.0]["gmres_iters"]
    assert out[w.newton_eta]["newton_iters"] == out[0.0]["newton_iters"]


def test_fine_and_coarse_propagators_match_oracle():
    w = wl.Workload("prop", nx=16, ny=4, T=0.5, n_slices=4, m_fine=4)
    mesh = oracle_mesh(w)
    dt = w.T / w.n_slices
    model = of.FSIModel(mesh, w.material)
    U0 = np.zeros((2, mesh.n_nodes, 5))
    U0[1] = model.propagate(U0[0], 0.0, dt, 8)
    ctx = ctx_for(w, 2)
    Uf, _ = ctx.fsi_fine(to_dev(U0), [0.0, dt])
    Uc, _ = ctx.fsi_coarse(to_dev(U0), [0.0, dt])
    Uf = Uf.cpu().numpy().reshape(2, -1, 5)
    Uc = Uc.cpu().numpy().reshape(2, -1, 5)
    for s in range(2):
        ref_f = model.propagate(U0[s], s * dt, (s + 1) * dt, w.m_fine)
        ref_c = model.propagate(U0[s], s * dt, (s + 1) * dt, 1, theta=1.0)
        assert max(rel_field_errors(Uf[s], ref_f).values()) <= 1e-10
        assert max(rel_field_errors(Uc[s], ref_c).values()) <= 1e-10


# a short run, and the 16 x 4 workload as specified: T = 1, 8 slices of 16 fine
# shifted Crank-Nicolson steps, one implicit-Euler coarse step per slice. Over
# its 128 fine steps per iteration two solutions that each meet the Newton
# stopping test at 1e-10 drift apart by about that much in the pressure, so
# both sides solve that workload's Newton systems to 1e-11 (just above the
# residual's round-off floor of about 1.5e-12 relative), and the GPU solves
# every Newton correction to the FGMRES tolerance (no inexact forcing), as the
# oracle's direct solver does.
#
# The bar. Eq. (parareal:iteration) makes the iterate at boundary n+1 a sum of
# three propagator results, F(U_n^i) + C(U_n^(i+1)) - C(U_n^i), and on the 16 x 4
# workload (coarse step K = 1/8) the three terms' pressures add up to as much as
# 15x the pressure of the sum (boundary 2 after iteration 2, in the oracle; about
# 3x where the terms do not cancel). The propagators agree with the oracle's to a
# few 1e-12 on the oracle's own inputs, and a sum carries its terms' errors, so
# the iterate after iteration 2 is held to 1e-10 of the size of the terms it is
# summed from, per field: |U - U_ref| <= 1e-10 (|F| + |C_new| + |C_old|). The
# serial limit (k = N) has no such sum and keeps the plain 1e-10 of |U| per field.
@pytest.mark.parametrize("w", [wl.Workload("pr", nx=16, ny=4, T=0.4, n_slices=4, m_fine=4),
                               dataclasses.replace(wl.SMALL_16x4, newton_tol=1e-11, gmres_rtol_first=0.0,
                                                   newton_eta=0.0)],
                         ids=["short", "fsi2d_q2_16x4_T1_8x16"])
def test_parareal_matches_oracle_iterates_and_reaches_serial(w):
    mesh = oracle_mesh(w)
    model = of.FSIModel(mesh, w.material, newton_tol=w.newton_tol)
    dt = w.T / w.n_slices
    N = w.n_slices
    calls = {"F": [], "C": []}   # every propagator result, in call order

    def fine(U, n):
        calls["F"].append(model.propagate(U, n * dt, (n + 1) * dt, w.m_fine))
        return calls["F"][-1]

    def coarse(U, n):
        calls["C"].append(model.propagate(U, n * dt, (n + 1) * dt, 1, theta=1.0))
        return calls["C"][-1]

    U0 = np.zeros((mesh.n_nodes, 5))
    hist = opr.parareal(U0, N, coarse, fine, 2)
    # call order: predictor sweep (N coarse), then per iteration N fine and N coarse
    F2, C1, C2 = calls["F"][N:2 * N], calls["C"][N:2 * N], calls["C"][2 * N:3 * N]
    ser = opr.serial(U0, N, lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, w.m_fine))
    ctx = ctx_for(w, N)
    for iters, ref in ((2, hist[2]), (N, ser)):
        U = torch.zeros((N + 1, mesh.n_dofs), dtype=torch.float64, device=DEV)
        U, st = ctx.parareal_iterate(U, iters, 0.0)
        got = U.cpu().numpy().reshape(N + 1, -1, 5)
        assert st["iterations"] == iters
        for n in range(1, N + 1):
            for name, sl in FIELDS.items():
                err = np.linalg.norm(got[n][..., sl] - ref[n][..., sl])
                if iters == 2:
                    bar = 1e-10 * sum(np.linalg.norm(t[n - 1][..., sl]) for t in (F2, C1, C2))
                else:
                    bar = 1e-10 * np.linalg.norm(ref[n][..., sl])
                assert err <= bar, (iters, n, name, err, bar)


@pytest.mark.parametrize("chunk", [1, 3])
def test_pipelined_parareal_is_bitwise_the_serial_schedule(chunk):
    """The pipelined schedule (sweeps on a helper thread and stream, fine solves
    in batches as their inputs appear) changes when things run, not what."""
    w = wl.Workload("pipe", nx=16, ny=4, T=0.5, n_slices=5, m_fine=3)
    ref_ctx = ctx_for(w, w.n_slices)
    ctx = ctx_for(w, w.n_slices, pipeline_chunk=chunk)
    for iters in (1, 3, w.n_slices):
        U = torch.zeros((w.n_slices + 1, ref_ctx.n_dofs), dtype=torch.float64, device=DEV)
        Ur, sr = ref_ctx.parareal_iterate(U.clone(), iters, 0.0)
        Up, sp = ctx.parareal_iterate(U.clone(), iters, 0.0)
        assert torch.equal(Up, Ur), iters
        for key in ("iterations", "increment_v", "increment_u", "increment_p", "fine_steps", "coarse_steps"):
            assert sp[key] == sr[key], (iters, key)
        assert sp["fine"]["gmres_iters"] == sr["fine"]["gmres_iters"]
        assert sp["coarse"]["gmres_iters"] == sr["coarse"]["gmres_iters"]
    # a tolerance that stops early stops at the same iteration
    Ur, sr = ref_ctx.parareal_iterate(torch.zeros_like(U), w.n_slices, 0.05)
    Up, sp = ctx.parareal_iterate(torch.zeros_like(U), w.n_slices, 0.05)
    assert sp["iterations"] == sr["iterations"] and torch.equal(Up, Ur)


def test_multiplicative_smoother_step_matches_oracle():
    """The coloured multiplicative Vanka smoother changes only the preconditioner."""
    w = wl.SMALL_16x4
    mesh = oracle_mesh(w)
    k = w.k_fine
    model, states = developed_states(w, mesh, 6, k)
    U0 = np.stack([states[2], states[5]])
    t0 = [3 * k, 6 * k]
    ctx = ctx_for(w, 2, mg_smoother=1, mg_smooth=1, mg_omega=1.0)
    Ub, _ = ctx.fsi_theta_step(to_dev(U0), t0, k, 0.5 + k)
    got = Ub.cpu().numpy().reshape(2, -1, 5)
    for s in range(2):
        ref = model.step(U0[s], t0[s], k, 0.5 + k)
        assert max(rel_field_errors(got[s], ref).values()) <= 1e-10
    Us, _ = ctx.fsi_theta_step(to_dev(U0[1:]), t0[1:], k, 0.5 + k)
    assert torch.equal(Us[0], Ub[1])


def test_cuda_graph_replay_is_bitwise_identical():
    """FGMRES iterations replayed from CUDA graphs (small batches) run the same
    kernels in the same order as direct launches."""
    w = wl.SMALL_16x4
    mesh = oracle_mesh(w)
    k = w.k_coarse
    _, states = developed_states(w, mesh, 4, w.k_fine)
    U0 = to_dev(np.stack([states[3], states[1]]))
    out = []
    for gmax in (0, 4):
        ctx = ctx_for(w, 2, graph_max_batch=gmax)
        U1, st = ctx.fsi_theta_step(U0, [0.1, 0.1], k, 1.0)
        U2, _ = ctx.fsi_theta_step(U1, [0.1 + k, 0.1 + k], k, 1.0)   # replays the captured graphs
        out.append(U2)
    assert torch.equal(out[0], out[1])


def test_parareal_continue_is_bitwise_one_longer_run():
    """A run stepped one iteration at a time (parareal_continue) computes the
    bits of one parareal_iterate call with the summed iteration count, also
    after a pipelined start and across a host round trip of the iterate."""
    from paper_1907_01252_gb300 import fsi
    w = wl.Workload("cont", nx=16, ny=4, T=0.5, n_slices=5, m_fine=3)
    ctx = ctx_for(w, w.n_slices)
    U0 = torch.zeros((w.n_slices + 1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError):          # nothing to continue yet
        ctx.parareal_continue(U0.clone(), 1, 0.0)
    Uref, sref = ctx.parareal_iterate(U0.clone(), 3, 0.0, history=True)
    U = U0.clone()
    _, s0 = ctx.parareal_iterate(U, 0, 0.0)
    assert s0["iterations"] == 0
    hist = []
    for it in (1, 2, 3):
        U = U.cpu().to(DEV)                    # the caller may keep the iterate on the host in between
        _, st = ctx.parareal_continue(U, 1, 0.0, history=True)
        assert st["iterations"] == it
        hist += st["history"]
    assert torch.equal(U, Uref)
    assert np.array_equal(np.array(hist), np.array(sref["history"]))
    # continuing after the pipelined schedule
    ctxp = ctx_for(w, w.n_slices, pipeline_chunk=2)
    U3 = U0.clone()
    ctxp.parareal_iterate(U3, 2, 0.0)
    ctxp.parareal_continue(U3, 1, 0.0)
    assert torch.equal(U3, Uref)
    # no iteration runs past n_slices; a new parareal_iterate starts a new run of the context
    Un, _ = ctxp.parareal_iterate(U0.clone(), w.n_slices, 0.0)
    U2 = U0.clone()
    ctx.parareal_iterate(U2, 1, 0.0)
    _, st = ctx.parareal_continue(U2, 2, 0.0)
    assert st["iterations"] == 3 and torch.equal(U2, Uref)
    _, st = ctx.parareal_continue(U2, 10, 0.0)
    assert st["iterations"] == w.n_slices and torch.equal(U2, Un)


def test_theta_step_128x32_matches_oracle():
    """The benchmarked mesh: 128 x 32 cells (83,525 dofs), so the solve runs the
    whole multigrid hierarchy and the cluster inverse of the coarsest level.
    Two slices from developed oracle states: an implicit-Euler step from rest
    to full inflow at t = 0.3, and one fine step on from there; one fine
    shifted Crank-Nicolson step of both, batched, against the oracle's steps."""
    w = wl.LARGE_128x32
    mesh = oracle_mesh(w)
    model = of.FSIModel(mesh, w.material)
    k = w.k_fine
    th = model.theta_fine(k)
    Ua = model.step(np.zeros((mesh.n_nodes, 5)), 0.25, 0.05, 1.0)
    Ub = model.step(Ua, 0.3, k, th)
    Uc = model.step(Ub, 0.3 + k, k, th)
    ctx = ctx_for(w, 2)
    assert ctx.n_levels >= 5
    U1, st = ctx.fsi_theta_step(to_dev(np.stack([Ua, Ub])), [0.3, 0.3 + k], k, th)
    got = U1.cpu().numpy().reshape(2, -1, 5)
    for s, ref in enumerate((Ub, Uc)):
        errs = rel_field_errors(got[s], ref)
        assert max(errs.values()) <= 1e-10, (s, errs)


def test_float_float_operator_product_keeps_the_parity_bar():
    """The Krylov operator and the multigrid residuals applied with float-pair
    blocks and a compensated FP32 accumulation (ff_operator = 1): the theta step
    still meets the 1e-10 bar against the oracle, stays within 1e-12 of the FP64
    product, and a batch still equals its solo runs bit for bit."""
    w = wl.SMALL_16x4
    mesh = oracle_mesh(w)
    k = w.k_fine
    model, states = developed_states(w, mesh, 12, k)
    pick = [5, 11]
    U0 = np.stack([states[i] for i in pick])
    t0 = [(i + 1) * k for i in pick]
    th = 0.5 + k
    ctx = ctx_for(w, 2, ff_operator=1)
    ctx64 = ctx_for(w, 2, ff_operator=0)
    Ub, st = ctx.fsi_theta_step(to_dev(U0), t0, k, th)
    U64, st64 = ctx64.fsi_theta_step(to_dev(U0), t0, k, th)
    got, g64 = Ub.cpu().numpy().reshape(2, -1, 5), U64.cpu().numpy().reshape(2, -1, 5)
    for s, i in enumerate(pick):
        ref = model.step(U0[s], t0[s], k, th)
        assert max(rel_field_errors(got[s], ref).values()) <= 1e-10
        assert max(rel_field_errors(got[s], g64[s]).values()) <= 1e-12
        Us, _ = ctx.fsi_theta_step(to_dev(U0[s:s + 1]), [t0[s]], k, th)
        assert torch.equal(Us[0], Ub[s])
    assert st["newton_iters"] == st64["newton_iters"]
