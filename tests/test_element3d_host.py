"""The 3D code of the CUDA library (csrc/fsi_element3d.cuh, fsi_mesh3d.h, fsi_mg3d.h,
fsi_vanka3.h: the per-entry __host__ __device__ functions the kernels run), compiled for
the host with the system C++ compiler and run in host loops, against the 3D oracle:
element residuals and Jacobians, the assembled system, multigrid transfers, the block
Vanka solves, and a whole theta step (Newton, FGMRES, V-cycle)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fsi_nd as on
from paper_1907_01252_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def host_lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("el3") / "libel3.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "native", "element3d_host.cpp"),
                    os.path.join(HERE, "native", "solver3d_host.cpp")], check=True)
    lib = C.CDLL(out)
    P = C.POINTER(C.c_double)
    lib.fsi3_cell_residual_host.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P]
    return lib


def ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def state(mesh, seed):
    rng = np.random.default_rng(seed)
    U = np.empty((mesh.n_nodes, 7))
    U[:, 0:3] = rng.uniform(-1, 1, (mesh.n_nodes, 3))
    U[:, 3:6] = 2e-3 * rng.uniform(-1, 1, (mesh.n_nodes, 3))
    U[:, 6] = 100 * rng.uniform(-1, 1, mesh.n_nodes)
    return U


@pytest.mark.parametrize("seed,k,theta", [(1, 0.02, 0.52), (2, 1 / 16, 1.0)])
def test_cell_residual_matches_the_3d_oracle(host_lib, seed, k, theta):
    mesh = on.make_mesh_nd([(0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41)],
                           [[2, 1, 2], [1, 1], [1, 1, 1]], ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355)))
    assert mesh.cell_solid.sum() == 1 and len(mesh.outflow_cells) > 0
    mat = wl.Material()
    tab = on.CellTablesND(mesh)
    U, Uo = state(mesh, seed), state(mesh, seed + 10)
    alpha = on.stabilisation_weights_nd(mesh, tab, mat, Uo)
    ref = on.element_residual_nd(mesh, tab, mat, U[mesh.cell_nodes], Uo[mesh.cell_nodes], k, theta, alpha)
    phys = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s])
    outflow = np.zeros(mesh.n_cells, dtype=bool)
    outflow[mesh.outflow_cells] = True
    scale = np.abs(ref).max(axis=(0, 1))
    for c in range(mesh.n_cells):
        Ue = np.ascontiguousarray(U[mesh.cell_nodes[c]])
        Uoe = np.ascontiguousarray(Uo[mesh.cell_nodes[c]])
        h = np.ascontiguousarray(mesh.h[c])
        Re = np.zeros((27, 7))
        host_lib.fsi3_cell_residual_host(ptr(phys), ptr(Ue), ptr(Uoe), ptr(h), int(mesh.cell_solid[c]),
                                         int(outflow[c]), k, theta, float(alpha[c]), ptr(Re))
        err = np.abs(Re - ref[c]).max(axis=0)
        assert np.all(err <= 1e-12 * scale), (c, err / scale)


@pytest.mark.parametrize("seed,k,theta", [(3, 0.02, 0.52), (4, 1 / 16, 1.0)])
def test_cell_jacobian_matches_the_3d_oracle_complex_step(host_lib, seed, k, theta):
    """Hand-derived 3D tangent and contraction against the oracle's complex-step element matrices."""
    P = C.POINTER(C.c_double)
    host_lib.fsi3_cell_jacobian_host.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P]
    mesh = on.make_mesh_nd([(0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41)],
                           [[2, 1, 2], [1, 1], [1, 1, 1]], ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355)))
    mat = wl.Material()
    U, Uo = state(mesh, seed), state(mesh, seed + 10)
    prob = on.StepProblemND(mesh, mat, Uo, 0.2, k, theta)
    ref = prob.element_jacobians(U)                                 # [cell, 27, 7, 27, 7]
    phys = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s])
    outflow = np.zeros(mesh.n_cells, dtype=bool)
    outflow[mesh.outflow_cells] = True
    cells = [int(np.argmax(mesh.cell_solid)), int(mesh.outflow_cells[0]), 0]
    for c in cells:
        Ue = np.ascontiguousarray(U[mesh.cell_nodes[c]])
        Uoe = np.ascontiguousarray(Uo[mesh.cell_nodes[c]])
        h = np.ascontiguousarray(mesh.h[c])
        Ke = np.zeros((189, 189))
        host_lib.fsi3_cell_jacobian_host(ptr(phys), ptr(Ue), ptr(Uoe), ptr(h), int(mesh.cell_solid[c]),
                                         int(outflow[c]), k, theta, float(prob.alpha[c]), ptr(Ke))
        R = ref[c].reshape(189, 189)
        # per field block: errors relative to the block's largest entry
        for ci in range(7):
            for cj in range(7):
                blk_ref = R[ci::7, cj::7]
                blk = Ke[ci::7, cj::7]
                sc = max(np.abs(blk_ref).max(), 1e-300)
                assert np.abs(blk - blk_ref).max() <= 1e-10 * max(sc, 1e-12 * np.abs(R).max()), (c, ci, cj)


BREAKS3 = ((0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41))
COUNTS3 = ((2, 1, 2), (1, 1), (1, 1, 1))
BOX3 = ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355))


def mesh_args(breaks=BREAKS3, counts=COUNTS3, box=BOX3):
    keep = []
    args = []
    for br, cn in zip(breaks, counts):
        b = np.ascontiguousarray(br, dtype=float)
        c = np.ascontiguousarray(cn, dtype=np.int32)
        keep += [b, c]
        args += [ptr(b), c.ctypes.data_as(C.POINTER(C.c_int)), len(cn)]
    bx = np.ascontiguousarray(np.ravel(box), dtype=float) if box is not None else None
    keep.append(bx)
    args.append(ptr(bx) if bx is not None else None)
    return args, keep


def test_3d_mesh_tables_match_the_oracle_mesh(host_lib):
    oracle_mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    args, keep = mesh_args()
    sizes = np.zeros(3, dtype=np.int32)
    cn = np.zeros((oracle_mesh.n_cells, 27), dtype=np.int32)
    nf = np.zeros(oracle_mesh.n_nodes, dtype=np.uint8)
    cf = np.zeros(oracle_mesh.n_cells, dtype=np.uint8)
    ip = lambda a: a.ctypes.data_as(C.c_void_p)
    host_lib.fsi3_mesh_host(*args, ip(sizes), ip(cn), ip(nf), ip(cf))
    nx, ny, nz = (sum(c) for c in COUNTS3)
    assert sizes[0] == oracle_mesh.n_nodes and sizes[1] == oracle_mesh.n_cells
    assert sizes[2] == (8 * nx + 1) * (8 * ny + 1) * (8 * nz + 1)          # Q2 pattern count per axis 8n + 1
    assert np.array_equal(cn, oracle_mesh.cell_nodes)
    assert np.array_equal((cf & 1).astype(bool), oracle_mesh.cell_solid)
    assert np.array_equal((nf & 1).astype(bool), oracle_mesh.dir_v)
    assert np.array_equal((nf & 2).astype(bool), oracle_mesh.dir_u)
    assert np.array_equal((nf & 4).astype(bool), oracle_mesh.p_identity)
    assert np.array_equal((nf & 8).astype(bool), oracle_mesh.node_in_solid)
    assert np.array_equal((nf & 16).astype(bool), oracle_mesh.on_inflow)


@pytest.mark.parametrize("seed,t_new,k,theta", [(5, 0.13, 0.02, 0.52), (6, 0.3, 1 / 16, 1.0)])
def test_assembled_3d_residual_matches_the_oracle(host_lib, seed, t_new, k, theta):
    """Per-cell residuals (with the stabilisation weights) and the fixed-order row gather,
    run in host loops, against the oracle's assembled residual (identity rows included)."""
    P = C.POINTER(C.c_double)
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material(vbar=1.2)
    U, Uo = state(mesh, seed), state(mesh, seed + 20)
    ref = on.StepProblemND(mesh, mat, Uo, t_new, k, theta).residual(U)
    args, keep = mesh_args()
    m = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s, mat.vbar, mat.ramp_t, mat.alpha0])
    R = np.zeros((mesh.n_nodes, 7))
    host_lib.fsi3_residual_host(*args, ptr(m), ptr(np.ascontiguousarray(U)), ptr(np.ascontiguousarray(Uo)),
                                C.c_double(t_new), C.c_double(k), C.c_double(theta), ptr(R))
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(R - ref).max(axis=0) <= 1e-12 * scale), np.abs(R - ref).max(axis=0) / scale


def test_assembled_3d_jacobian_matches_the_oracle(host_lib):
    """Element matrices and the fixed-order block gather (7 x 7 blocks, identity rows)
    against the oracle's complex-step global Jacobian, per field block."""
    import scipy.sparse as sp
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material()
    U, Uo = state(mesh, 7), state(mesh, 27)
    k, theta = 0.02, 0.52
    ref = on.StepProblemND(mesh, mat, Uo, 0.2, k, theta).jacobian(U).toarray()
    args, keep = mesh_args()
    sizes = np.zeros(3, dtype=np.int32)
    host_lib.fsi3_mesh_host(*args, sizes.ctypes.data_as(C.c_void_p), None, None, None)
    n_nodes, nnzb = int(sizes[0]), int(sizes[2])
    rowptr = np.zeros(n_nodes + 1, dtype=np.int32)
    colidx = np.zeros(nnzb, dtype=np.int32)
    vals = np.zeros((nnzb, 7, 7))
    m = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s, mat.vbar, mat.ramp_t, mat.alpha0])
    host_lib.fsi3_jacobian_host(*args, ptr(m), ptr(np.ascontiguousarray(U)), ptr(np.ascontiguousarray(Uo)),
                                C.c_double(k), C.c_double(theta), rowptr.ctypes.data_as(C.c_void_p),
                                colidx.ctypes.data_as(C.c_void_p), ptr(vals))
    A = sp.bsr_matrix((vals, colidx, rowptr), shape=(mesh.n_dofs, mesh.n_dofs)).toarray()
    for ci in range(7):
        for cj in range(7):
            blk_ref, blk = ref[ci::7, cj::7], A[ci::7, cj::7]
            sc = max(np.abs(blk_ref).max(), 1e-12 * np.abs(ref).max())
            assert np.abs(blk - blk_ref).max() <= 1e-10 * sc, (ci, cj)


# A finer mesh whose segments have odd and even cell counts, so the coarsening
# pairs cells in some segments and keeps a single cell at the end of others.
COUNTS3_FINE = ((4, 1, 3), (2, 3), (2, 2, 1))


def coarse_counts(counts):
    return tuple(tuple((n + 1) // 2 for n in seg) for seg in counts)


def q2_axis(breaks, counts, paired=False):
    """Q2 node coordinates of one axis: uniform cells per segment, a midpoint per cell.
    paired: the coarsening of that axis instead (every second vertex of a segment, plus
    its end when the count is odd, so the last coarse cell is one fine cell)."""
    v = [breaks[0]]
    for s, n in enumerate(counts):
        keep = list(range(2, n + 1, 2)) + ([n] if n % 2 else []) if paired else range(1, n + 1)
        v += [breaks[s] + (breaks[s + 1] - breaks[s]) * i / n for i in keep]
    v = np.array(v)
    x = np.empty(2 * len(v) - 1)
    x[0::2], x[1::2] = v, 0.5 * (v[:-1] + v[1:])
    return x


def transfer(host_lib, mode, inp, n_out):
    P = C.POINTER(C.c_double)
    host_lib.fsi3_transfer_host.argtypes = [P, C.c_void_p, C.c_int] * 3 + [P, C.c_int, P, P, C.c_void_p, P,
                                                                           C.c_void_p]
    args, keep = mesh_args(counts=COUNTS3_FINE)
    sizes = np.zeros(6, dtype=np.int32)
    out = np.zeros((n_out, 7))
    inp = np.ascontiguousarray(inp, dtype=float) if inp is not None else np.zeros(1)
    coords = np.zeros(sum(2 * sum(c) + 1 for c in COUNTS3_FINE) +
                      sum(2 * sum(c) + 1 for c in coarse_counts(COUNTS3_FINE)))
    fine = on.make_mesh_nd(BREAKS3, COUNTS3_FINE, BOX3)
    coarse = on.make_mesh_nd(BREAKS3, coarse_counts(COUNTS3_FINE), BOX3)
    flags = np.zeros(fine.n_nodes + coarse.n_nodes, dtype=np.uint8)
    host_lib.fsi3_transfer_host(*args, mode, ptr(inp), ptr(out), sizes.ctypes.data_as(C.c_void_p), ptr(coords),
                                flags.ctypes.data_as(C.c_void_p))
    return out, sizes, coords, flags, fine, coarse


def identity_mask(mesh):
    """[node][7] True on identity rows: Dirichlet velocity, Dirichlet displacement, p = 0."""
    return np.concatenate([np.repeat(mesh.dir_v[:, None], 3, 1), np.repeat(mesh.dir_u[:, None], 3, 1),
                           mesh.p_identity[:, None]], axis=1)


def node_points(xs):
    """[node][3] coordinates of the tensor node grid with x fastest."""
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    return np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)


def triquadratic(pts, seed, cubic=False):
    """A random field of degree <= 2 in each coordinate per component (plus x^3 if cubic)."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(3, 3, 3, 7))
    x, y, z = pts[:, 0:1], pts[:, 1:2], pts[:, 2:3]
    f = sum(coef[a, b, c] * x ** a * y ** b * z ** c for a in range(3) for b in range(3) for c in range(3))
    return f + (x ** 3 if cubic else 0.0)


def test_3d_coarse_level_and_node_flags(host_lib):
    """The coarsened level pairs cells per segment (odd counts keep one cell) and takes
    the oracle's node flags on both levels (flags depend on the topology alone)."""
    _, sizes, coords, flags, fine, coarse = transfer(host_lib, 0, None, 1)
    xs_f = [q2_axis(b, c) for b, c in zip(BREAKS3, COUNTS3_FINE)]
    xs_c = [q2_axis(b, c, paired=True) for b, c in zip(BREAKS3, COUNTS3_FINE)]
    assert list(sizes) == [len(x) for x in xs_f + xs_c]
    assert np.allclose(coords, np.concatenate(xs_f + xs_c), rtol=0, atol=1e-15)
    ff, fc = flags[:fine.n_nodes], flags[fine.n_nodes:]
    for m, fl in ((fine, ff), (coarse, fc)):
        assert np.array_equal((fl & 1).astype(bool), m.dir_v)
        assert np.array_equal((fl & 2).astype(bool), m.dir_u)
        assert np.array_equal((fl & 4).astype(bool), m.p_identity)


def test_3d_prolongation_reproduces_triquadratics(host_lib):
    """Q2 interpolation from the coarse level is exact for fields of degree <= 2 in each
    coordinate (zero on the fine identity rows), and not for a cubic."""
    _, sizes, coords, _, fine, coarse = transfer(host_lib, 0, None, 1)
    split = np.cumsum(sizes)[:-1]
    xs = np.split(coords, split)
    pf, pc = node_points(xs[:3]), node_points(xs[3:])
    for seed, cubic in ((1, False), (2, False), (3, True)):
        Pf, _, _, _, _, _ = transfer(host_lib, 1, triquadratic(pc, seed, cubic), fine.n_nodes)
        want = np.where(identity_mask(fine), 0.0, triquadratic(pf, seed, cubic))
        err = np.abs(Pf - want).max() / np.abs(want).max()
        assert (err > 1e-4) if cubic else (err < 1e-13), (seed, err)


def test_3d_state_interpolation_is_exact_and_injects(host_lib):
    """The fine state at the coarse nodes: exact for tri-quadratics and, the levels being
    nested, a plain injection of the fine values at the coinciding nodes (bit-exact)."""
    _, sizes, coords, _, fine, coarse = transfer(host_lib, 0, None, 1)
    xs = np.split(coords, np.cumsum(sizes)[:-1])
    pf, pc = node_points(xs[:3]), node_points(xs[3:])
    f = triquadratic(pf, 4)
    Uc, _, _, _, _, _ = transfer(host_lib, 3, f, coarse.n_nodes)
    assert np.abs(Uc - triquadratic(pc, 4)).max() <= 1e-13 * np.abs(f).max()
    rng = np.random.default_rng(5)
    Uf = rng.normal(size=(fine.n_nodes, 7))
    Uc, _, _, _, _, _ = transfer(host_lib, 3, Uf, coarse.n_nodes)
    idx = [np.searchsorted(xs[a], xs[3 + a]) for a in range(3)]
    for a in range(3):
        assert np.array_equal(xs[a][idx[a]], xs[3 + a])
    I, J, K = np.meshgrid(*idx, indexing="ij")
    inj = (I + sizes[0] * (J + sizes[1] * K)).ravel(order="F")
    assert np.array_equal(Uc, Uf[inj])


def test_3d_restriction_is_the_masked_transpose(host_lib):
    """<R r, x> = <r, P (x on the free coarse rows)> for random vectors; R is zero on the
    coarse identity rows and ignores the fine identity rows."""
    _, _, _, _, fine, coarse = transfer(host_lib, 0, None, 1)
    rng = np.random.default_rng(6)
    r = rng.normal(size=(fine.n_nodes, 7))
    x = rng.normal(size=(coarse.n_nodes, 7))
    Rr, _, _, _, _, _ = transfer(host_lib, 2, r, coarse.n_nodes)
    Px, _, _, _, _, _ = transfer(host_lib, 1, np.where(identity_mask(coarse), 0.0, x), fine.n_nodes)
    lhs, rhs = np.sum(Rr * x), np.sum(r * Px)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(Rr ** 2) * np.sum(x ** 2)), (lhs, rhs)
    assert np.all(Rr[identity_mask(coarse)] == 0.0)
    r2 = np.where(identity_mask(fine), 1e6 * rng.normal(size=r.shape), r)
    Rr2, _, _, _, _, _ = transfer(host_lib, 2, r2, coarse.n_nodes)
    assert np.array_equal(Rr, Rr2)


def oracle_blocks(host_lib, mesh, J):
    """The oracle's global Jacobian J (dense) cut into the library's 7 x 7 block pattern
    (rowptr, colidx from the host assembly), and that pattern."""
    args, keep = mesh_args()
    sizes = np.zeros(3, dtype=np.int32)
    host_lib.fsi3_mesh_host(*args, sizes.ctypes.data_as(C.c_void_p), None, None, None)
    n_nodes, nnzb = int(sizes[0]), int(sizes[2])
    rowptr = np.zeros(n_nodes + 1, dtype=np.int32)
    colidx = np.zeros(nnzb, dtype=np.int32)
    scratch = np.zeros((nnzb, 7, 7))
    mat = wl.Material()
    m = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s, mat.vbar, mat.ramp_t, mat.alpha0])
    U0 = np.zeros((n_nodes, 7))
    host_lib.fsi3_jacobian_host(*args, ptr(m), ptr(U0), ptr(U0), C.c_double(0.02), C.c_double(0.52),
                                rowptr.ctypes.data_as(C.c_void_p), colidx.ctypes.data_as(C.c_void_p), ptr(scratch))
    rows = np.repeat(np.arange(n_nodes), np.diff(rowptr))
    blocks = np.stack([J[7 * i:7 * i + 7, 7 * j:7 * j + 7] for i, j in zip(rows, colidx)])
    # every nonzero of J lies in the pattern
    Jp = np.zeros_like(J)
    for b, (i, j) in enumerate(zip(rows, colidx)):
        Jp[7 * i:7 * i + 7, 7 * j:7 * j + 7] = blocks[b]
    assert np.array_equal(Jp, J)
    return np.ascontiguousarray(blocks)


@pytest.fixture(scope="module")
def oracle_jacobian_3d():
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material()
    U, Uo = state(mesh, 8), state(mesh, 28)
    J = on.StepProblemND(mesh, mat, Uo, 0.2, 0.02, 0.52).jacobian(U).toarray()
    return mesh, J


def vanka(host_lib, blocks, r, precision, omega=0.8):
    P = C.POINTER(C.c_double)
    host_lib.fsi3_vanka_host.argtypes = [P, C.c_void_p, C.c_int] * 3 + [P, P, P, C.c_int, C.c_double, P, P,
                                                                        C.c_void_p]
    args, keep = mesh_args()
    n_nodes = r.shape[0]
    n_cells = (blocks.shape[0] and sum(COUNTS3[0]) * sum(COUNTS3[1]) * sum(COUNTS3[2]))
    zc = np.zeros((n_cells, 189))
    x = np.zeros((n_nodes, 7))
    cf = np.zeros(n_cells, dtype=np.uint8)
    rc = host_lib.fsi3_vanka_host(*args, ptr(blocks), ptr(np.ascontiguousarray(r)), precision, omega, ptr(zc),
                                  ptr(x), cf.ctypes.data_as(C.c_void_p))
    assert rc == 0
    return zc, x, cf


def test_3d_vanka_block_elimination_solves_the_local_systems(host_lib, oracle_jacobian_3d):
    """Per cell, the block elimination (A11, Schur complement S; or the decoupled
    displacement blocks) equals a dense solve with the cell's local matrix cut from the
    oracle's Jacobian; the node update is the damped average over the node's cells."""
    mesh, J = oracle_jacobian_3d
    blocks = oracle_blocks(host_lib, mesh, J)
    r = np.random.default_rng(9).normal(size=(mesh.n_nodes, 7))
    zc, x, cf = vanka(host_lib, blocks, r, 0)
    dec = (cf & 4).astype(bool)
    assert 0 < dec.sum() < mesh.n_cells
    worst = 0.0
    for c in range(mesh.n_cells):
        dofs = (7 * mesh.cell_nodes[c][:, None] + np.arange(7)).ravel()
        A = J[np.ix_(dofs, dofs)]
        z = np.linalg.solve(A, r.ravel()[dofs])
        worst = max(worst, np.abs(zc[c] - z).max() / (np.abs(z).max() * np.linalg.cond(A) * 1e-16))
        if dec[c]:
            # the structure the decoupled path relies on: displacement rows see only their own component
            for q in range(3):
                rows = 7 * np.arange(27) + 3 + q
                other = [d for d in range(189) if d % 7 != 3 + q]
                assert np.all(A[np.ix_(rows, other)] == 0.0)
    assert worst < 100.0, worst
    cnt = np.zeros(mesh.n_nodes)
    acc = np.zeros((mesh.n_nodes, 7))
    for c in range(mesh.n_cells):
        np.add.at(acc, mesh.cell_nodes[c], zc[c].reshape(27, 7))
        np.add.at(cnt, mesh.cell_nodes[c], 1.0)
    assert np.allclose(x, 0.8 * acc / cnt[:, None], rtol=1e-14, atol=0)


def test_3d_vanka_fp32_block_elimination(host_lib, oracle_jacobian_3d):
    """The same local solves with FP32 factors and FP32 application. The local matrices
    have condition numbers up to ~1e14 (stiff solid, pressure scaling), so FP32 gives
    a rough local solve: within 5e-3 of the FP64 one on every cell (~5e-4 seen on the
    solid cell, ~1e-6 on most), a smoother's accuracy, not a solver's."""
    mesh, J = oracle_jacobian_3d
    blocks = oracle_blocks(host_lib, mesh, J)
    r = np.random.default_rng(10).normal(size=(mesh.n_nodes, 7))
    z64, _, _ = vanka(host_lib, blocks, r, 0)
    z32, _, _ = vanka(host_lib, blocks, r, 1)
    err = np.abs(z32 - z64).max(axis=1) / np.abs(z64).max(axis=1)
    assert err.max() <= 5e-3 and np.median(err) <= 1e-5, (err.max(), np.median(err))


@pytest.fixture(scope="module")
def oracle_step_3d():
    """The oracle's theta step from rest to t = 0.52 at full inflow (a hard Newton start:
    the inflow profile against a fluid at rest), exact Newton with sparse direct solves."""
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material()
    Uo = np.zeros((mesh.n_nodes, 7))
    model = on.FSIModelND(mesh, mat, newton_tol=1e-12)
    return mesh, mat, Uo, model.step(Uo, 0.5, 0.02, 0.52)


@pytest.mark.parametrize("precision,smoother,coarse_sweeps", [(0, 0, 0), (1, 1, 0), (1, 1, 8)])
def test_3d_theta_step_matches_the_oracle(host_lib, oracle_step_3d, precision, smoother, coarse_sweeps):
    """One theta step solved the library's way (inexact Newton, FGMRES(50) + V-cycle with
    the block Vanka smoother over 2695 -> 1715 dofs, dense coarsest) equals the oracle's
    Newton step to 1e-9 per field; FP32 multigrid inside FP64 FGMRES reaches the same
    root. smoother 1 is the coloured multiplicative sweep; coarse_sweeps > 0 replaces the
    coarsest solve by that many sweeps."""
    mesh, mat, Uo, ref = oracle_step_3d
    P = C.POINTER(C.c_double)
    host_lib.fsi3_theta_step_host.argtypes = [P, C.c_void_p, C.c_int] * 3 + [P, P, P, C.c_int, P, C.c_double,
                                                                             C.c_double, C.c_double, P, C.c_void_p]
    args, keep = mesh_args()
    m = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s, mat.vbar, mat.ramp_t, mat.alpha0])
    #              newton_tol maxit restart gmres_maxit rtol rtol_first eta coarsest smooth omega lps smoother
    #              coarse_sweeps reuse
    prm = np.array([1e-10, 20, 50, 2000, 1e-12, 1e-6, 1e-3, 2000, 2 - smoother, 0.6 + 0.4 * smoother, 0.5,
                    smoother, coarse_sweeps, 2], dtype=float)
    U = np.zeros_like(Uo)
    stats = np.zeros(4, dtype=np.int32)
    rc = host_lib.fsi3_theta_step_host(*args, ptr(m), ptr(prm), precision, ptr(Uo), 0.52, 0.02, 0.52, ptr(U),
                                       stats.ctypes.data_as(C.c_void_p))
    assert rc == 0
    n_newton, n_krylov, levels, coarsest = stats
    assert levels == 2 and coarsest == 1715 and 3 <= n_newton <= 8
    # with sweeps in place of the coarsest solve the two-level toy hierarchy converges ~2.5x slower
    # (on three levels the two are alike); the bound only catches a broken preconditioner
    assert n_krylov <= (120 if coarse_sweeps == 0 else 300) * n_newton, n_krylov
    scale = np.abs(ref).max(axis=0)
    err = np.abs(U - ref).max(axis=0) / scale
    assert np.all(err <= 1e-9), err


@pytest.mark.parametrize("seed,k,theta", [(1, 0.02, 0.52), (2, 1 / 16, 1.0)])
def test_cooperative_cell_jacobian_matches_the_serial_one(host_lib, seed, k, theta):
    """The element matrix routine of the kernel (work spread over a thread group, the
    contraction over the Gauss points sum-factorised; run here as one host thread)
    equals the serial routine up to rounding on fluid, solid and outflow cells: every
    (test, trial) block within 1e-13 of its largest entry, zero blocks exactly zero,
    every entry written."""
    P = C.POINTER(C.c_double)
    for name in ("fsi3_cell_jacobian_host", "fsi3_cell_jacobian_cta_host"):
        getattr(host_lib, name).argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P]
    mesh = on.make_mesh_nd([(0.0, 0.4, 0.45, 0.9), (0.0, 0.2, 0.41), (0.0, 0.055, 0.355, 0.41)],
                           [[2, 1, 2], [1, 1], [1, 1, 1]], ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355)))
    mat = wl.Material()
    U, Uo = state(mesh, seed), state(mesh, seed + 30)
    phys = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s])
    outflow = np.zeros(mesh.n_cells, dtype=bool)
    outflow[mesh.outflow_cells] = True
    h = np.array([0.2, 0.2, 0.055])
    kinds = set()
    for c in range(mesh.n_cells):
        Ue = np.ascontiguousarray(U[mesh.cell_nodes[c]])
        Uoe = np.ascontiguousarray(Uo[mesh.cell_nodes[c]])
        args = (ptr(phys), ptr(Ue), ptr(Uoe), ptr(h), int(mesh.cell_solid[c]), int(outflow[c]), k, theta, 3e-4)
        K1, K2 = np.zeros(189 * 189), np.zeros(189 * 189)
        host_lib.fsi3_cell_jacobian_host(*args, ptr(K1))
        host_lib.fsi3_cell_jacobian_cta_host(*args, ptr(K2))
        A1, A2 = K1.reshape(27, 7, 27, 7), K2.reshape(27, 7, 27, 7)
        for ci in range(7):
            for cj in range(7):
                b1, b2 = A1[:, ci, :, cj], A2[:, ci, :, cj]
                sc = np.abs(b1).max()
                if sc == 0.0:
                    assert np.all(b2 == 0.0), (c, ci, cj)
                else:
                    assert np.abs(b2 - b1).max() <= 1e-13 * sc, (c, ci, cj, np.abs(b2 - b1).max() / sc)
        kinds.add((bool(mesh.cell_solid[c]), bool(outflow[c])))
    assert kinds == {(False, False), (True, False), (False, True)}


def test_3d_cell_colours_share_no_node():
    """The coloured sweep adds each colour's corrections without atomics: cells of one
    colour (the parities of the three cell indices) must share no node, and the eight
    colours must cover every cell once."""
    counts = ((4, 1, 3), (2, 3), (2, 2, 1))
    mesh = on.make_mesh_nd(BREAKS3, counts, BOX3)
    nx, ny, nz = (sum(c) for c in counts)
    cells = np.arange(mesh.n_cells)
    cx, cy, cz = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    colour = (cx & 1) + 2 * (cy & 1) + 4 * (cz & 1)
    assert np.all(np.bincount(colour, minlength=8) > 0)
    for k in range(8):
        nodes = mesh.cell_nodes[colour == k].ravel()
        assert len(np.unique(nodes)) == len(nodes), k


@pytest.mark.parametrize("solid", [0, 1])
def test_unit_direction_tangent_matches_the_general_one(host_lib, solid):
    """The tangent specialised to unit directions (rank-one forms for the velocity,
    velocity-gradient, displacement and pressure directions) equals the general
    linearisation at every Gauss point and direction, on random states, to 1e-13 of
    the largest entry of that point's tangent."""
    P = C.POINTER(C.c_double)
    host_lib.fsi3_tangents_host.argtypes = [P, P, P, P, C.c_int, C.c_double, C.c_double, P, P]
    mat = wl.Material()
    phys = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s])
    rng = np.random.default_rng(40 + solid)
    for trial in range(3):
        Ue = np.empty((27, 7))
        Ue[:, :3], Ue[:, 3:6], Ue[:, 6] = rng.normal(size=(27, 3)), 0.05 * rng.normal(size=(27, 3)), rng.normal(size=27)
        Uo = Ue + 0.01 * rng.normal(size=Ue.shape)
        h = rng.uniform(0.05, 0.2, 3)
        Dg, Du = np.zeros(27 * 28 * 28), np.zeros(27 * 28 * 28)
        host_lib.fsi3_tangents_host(ptr(phys), ptr(np.ascontiguousarray(Ue)), ptr(np.ascontiguousarray(Uo)), ptr(h),
                                    solid, 0.02, 0.52, ptr(Dg), ptr(Du))
        Dg, Du = Dg.reshape(27, 28, 28), Du.reshape(27, 28, 28)
        scale = np.abs(Dg).max(axis=(1, 2))
        assert np.all(np.abs(Du - Dg).max(axis=(1, 2)) <= 1e-13 * scale), np.max(np.abs(Du - Dg).max(axis=(1, 2)) / scale)


def test_3d_coarse_theta_step_matches_the_oracle(host_lib):
    """The coarse propagator's step (theta = 1, implicit Euler, k = 0.04: twice the fine
    step; on this 5 x 2 x 3 toy mesh undamped Newton from the old state diverges at
    k = 1/16, in the oracle as well) from a state with flow and displacement, run the library's way on the host (FP32
    multigrid, coloured sweeps, swept coarsest level, hierarchy rebuilt per iterate),
    equals the oracle's exact-Newton step to 1e-9 per field."""
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material()
    model = on.FSIModelND(mesh, mat, newton_tol=1e-12)
    U0 = model.step(np.zeros((mesh.n_nodes, 7)), 0.1, 0.02, 0.52)   # a state with flow and displacement
    ref = model.step(U0, 0.12, 0.04, 1.0)
    P = C.POINTER(C.c_double)
    host_lib.fsi3_theta_step_host.argtypes = [P, C.c_void_p, C.c_int] * 3 + [P, P, P, C.c_int, P, C.c_double,
                                                                             C.c_double, C.c_double, P, C.c_void_p]
    args, keep = mesh_args()
    m = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s, mat.vbar, mat.ramp_t, mat.alpha0])
    prm = np.array([1e-10, 20, 50, 2000, 1e-12, 1e-6, 1e-3, 2000, 1, 1.0, 0.25, 1, 8, 0], dtype=float)
    U = np.zeros_like(U0)
    stats = np.zeros(4, dtype=np.int32)
    rc = host_lib.fsi3_theta_step_host(*args, ptr(m), ptr(prm), 1, ptr(np.ascontiguousarray(U0)), 0.16, 0.04, 1.0,
                                       ptr(U), stats.ctypes.data_as(C.c_void_p))
    assert rc == 0 and stats[0] >= 2
    err = np.abs(U - ref).max(axis=0) / np.abs(ref).max(axis=0)
    assert np.all(err <= 1e-9), err


@pytest.mark.parametrize("seed,k,theta", [(3, 0.02, 0.52), (4, 1 / 16, 1.0)])
def test_cooperative_cell_residual_is_bitwise_the_serial_one(host_lib, seed, k, theta):
    """The cell residual routine of the kernel (point and face fluxes in parallel, one
    thread per entry; run here as one host thread) performs the serial routine's
    arithmetic in the same order: identical bits on fluid, solid and outflow cells."""
    P = C.POINTER(C.c_double)
    for name in ("fsi3_cell_residual_host", "fsi3_cell_residual_cta_host"):
        getattr(host_lib, name).argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, P]
    mesh = on.make_mesh_nd(BREAKS3, COUNTS3, BOX3)
    mat = wl.Material()
    U, Uo = state(mesh, seed), state(mesh, seed + 30)
    phys = np.array([mat.rho_f, mat.nu_f, mat.rho_s, mat.mu_s, mat.lambda_s])
    outflow = np.zeros(mesh.n_cells, dtype=bool)
    outflow[mesh.outflow_cells] = True
    h = np.array([0.2, 0.2, 0.055])
    for c in range(mesh.n_cells):
        Ue = np.ascontiguousarray(U[mesh.cell_nodes[c]])
        Uoe = np.ascontiguousarray(Uo[mesh.cell_nodes[c]])
        args = (ptr(phys), ptr(Ue), ptr(Uoe), ptr(h), int(mesh.cell_solid[c]), int(outflow[c]), k, theta, 3e-4)
        R1, R2 = np.zeros(189), np.zeros(189)
        host_lib.fsi3_cell_residual_host(*args, ptr(R1))
        host_lib.fsi3_cell_residual_cta_host(*args, ptr(R2))
        assert np.array_equal(R1, R2), c
