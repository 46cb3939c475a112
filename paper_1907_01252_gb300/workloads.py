"""Seeded synthetic workloads for the channel-with-elastic-bar FSI problem.

This module describes INPUTS only: geometry break points, cells per segment,
material constants, time windows and seeded random states. It holds none of
the method's arithmetic and imports nothing from the rest of the package, so
both the CUDA path and the FP64 oracle may take their inputs from it.

Geometry (reference configuration, Sec. 4 setting re-sized to the workloads
used here): channel [0, 2] x [0, 0.41], an elastic bar x in [0.6, 0.7],
y in [0, 0.2] attached to the bottom wall. Break points at the bar edges make
the tensor mesh interface-fitted (Sec. 2.2, the mesh resolves the interface).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

X_BREAKS = (0.0, 0.6, 0.7, 2.0)
Y_BREAKS = (0.0, 0.2, 0.41)
SOLID_BOX = ((0.6, 0.7), (0.0, 0.2))


def cells_per_segment(breaks, n_cells):
    """Split n_cells over the segments of `breaks` in proportion to length.

    Each segment gets round(n * len / total) cells, at least one; the longest
    segment absorbs the difference so that the counts sum to n_cells.
    (16 -> 5/1/10 and 128 -> 38/6/84 in x; 4 -> 2/2 and 32 -> 16/16 in y.)
    """
    lengths = [b - a for a, b in zip(breaks[:-1], breaks[1:])]
    total = breaks[-1] - breaks[0]
    counts = [max(1, int(math.floor(n_cells * L / total + 0.5))) for L in lengths]
    longest = int(np.argmax(lengths))
    counts[longest] += n_cells - sum(counts)
    if counts[longest] < 1:
        raise ValueError("too few cells for the break points")
    return tuple(counts)


@dataclasses.dataclass(frozen=True)
class Material:
    rho_f: float = 1000.0     # fluid density
    nu_f: float = 1e-3        # kinematic viscosity
    rho_s: float = 1000.0     # solid density
    mu_s: float = 5e5         # shear modulus
    lambda_s: float = 2e6     # first Lame parameter (Poisson ratio 0.4)
    vbar: float = 1.0         # mean inflow velocity
    ramp_t: float = 0.2       # inflow ramp duration
    theta0: float = 1.0       # shifted CN: theta = 1/2 + theta0 * k
    alpha0: float = 0.1       # local-projection stabilisation constant


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    T: float
    n_slices: int
    m_fine: int
    m_coarse: int = 1
    newton_tol: float = 1e-10
    newton_maxit: int = 20
    gmres_restart: int = 50
    gmres_maxit: int = 2000
    gmres_rtol: float = 1e-12
    # inexact Newton: first correction of a step to 1e-6, later ones until the
    # linear residual is 1e-3 x the Newton target (0 disables: every solve to gmres_rtol)
    gmres_rtol_first: float = 1e-6
    newton_eta: float = 1e-3
    parareal_tol: float = 1e-8
    material: Material = Material()
    with_solid: bool = True

    @property
    def nx_seg(self):
        return cells_per_segment(X_BREAKS, self.nx)

    @property
    def ny_seg(self):
        return cells_per_segment(Y_BREAKS, self.ny)

    @property
    def n_nodes(self):
        return (2 * self.nx + 1) * (2 * self.ny + 1)

    @property
    def n_dofs(self):
        return 5 * self.n_nodes

    @property
    def k_fine(self):
        return self.T / self.n_slices / self.m_fine

    @property
    def k_coarse(self):
        return self.T / self.n_slices / self.m_coarse


# 2D monolithic ALE FSI, FP64, 16 x 4 Q2 cells, T = 1, 8 slices x 16 fine CN steps.
SMALL_16x4 = Workload("fsi2d_q2_16x4_T1_8x16", nx=16, ny=4, T=1.0, n_slices=8, m_fine=16)
# Same problem at scale: 128 x 32 Q2 cells (83,525 dofs), T = 2, 64 slices x 32 fine CN steps.
LARGE_128x32 = Workload("fsi2d_q2_128x32_T2_64x32", nx=128, ny=32, T=2.0, n_slices=64, m_fine=32)

WORKLOADS = {w.name: w for w in (SMALL_16x4, LARGE_128x32)}


# 3D channel with an elastic plate on the bottom wall: channel [0, 1.5] x [0, 0.41] x [0, 0.41], plate
# 0.05 x 0.2 x 0.3 at x in [0.4, 0.45] (the x position is not given; this is a reading), centred in z.
X3_BREAKS = (0.0, 0.4, 0.45, 1.5)
Y3_BREAKS = (0.0, 0.2, 0.41)
Z3_BREAKS = (0.0, 0.055, 0.355, 0.41)
SOLID_BOX_3D = ((0.4, 0.45), (0.0, 0.2), (0.055, 0.355))


def cells_per_segment_3d(nx, ny, nz):
    """Cells per segment on the three axes of the 3D channel (32 x 8 x 8 -> 9/1/22, 4/4, 1/6/1)."""
    return (cells_per_segment(X3_BREAKS, nx), cells_per_segment(Y3_BREAKS, ny), cells_per_segment(Z3_BREAKS, nz))


@dataclasses.dataclass(frozen=True)
class Workload3D:
    """The 3D channel with the plate: nx x ny x nz hexahedral Q2 cells split over the
    segments of X3/Y3/Z3_BREAKS, interval T cut into n_slices slices of m_fine fine and
    m_coarse coarse steps, solver settings as for Workload."""
    name: str
    nx: int
    ny: int
    nz: int
    T: float
    n_slices: int
    m_fine: int
    m_coarse: int = 1
    newton_tol: float = 1e-10
    newton_maxit: int = 20
    gmres_restart: int = 50
    gmres_maxit: int = 2000
    gmres_rtol: float = 1e-12
    gmres_rtol_first: float = 1e-6
    newton_eta: float = 1e-3
    parareal_tol: float = 1e-8
    material: Material = Material()
    with_solid: bool = True

    @property
    def segments(self):
        return cells_per_segment_3d(self.nx, self.ny, self.nz)

    @property
    def breaks(self):
        return (X3_BREAKS, Y3_BREAKS, Z3_BREAKS)

    @property
    def n_nodes(self):
        return (2 * self.nx + 1) * (2 * self.ny + 1) * (2 * self.nz + 1)

    @property
    def n_dofs(self):
        return 7 * self.n_nodes

    @property
    def k_fine(self):
        return self.T / self.n_slices / self.m_fine

    @property
    def k_coarse(self):
        return self.T / self.n_slices / self.m_coarse


# 3D channel, 8 x 4 x 4 Q2 hexahedra (9,639 dofs): a small case of the 3D path.
SMALL3D_8x4x4 = Workload3D("fsi3d_q2_8x4x4_T1_8x4", nx=8, ny=4, nz=4, T=1.0, n_slices=8, m_fine=4)
# 3D channel at scale: 32 x 8 x 8 Q2 hexahedra (131,495 dofs), T = 1, 32 slices x 16 fine steps.
CHANNEL3D_32x8x8 = Workload3D("fsi3d_q2_32x8x8_T1_32x16", nx=32, ny=8, nz=8, T=1.0, n_slices=32, m_fine=16)


def node_axis(breaks, counts):
    """Node coordinates of the Q2 mesh along one axis: 2 n + 1 uniform nodes per
    segment of n cells, shared at the break points."""
    out = [breaks[0]]
    for (a, b), n in zip(zip(breaks[:-1], breaks[1:]), counts):
        out.extend(a + (b - a) * (np.arange(1, 2 * n + 1) / (2 * n)))
    return np.array(out)


def tip_node(w):
    """Index of the node at the top centre of the solid box (node (i, j) has id j * (2 nx + 1) + i)."""
    xn, yn = node_axis(X_BREAKS, w.nx_seg), node_axis(Y_BREAKS, w.ny_seg)
    (x0, x1), (_, y1) = SOLID_BOX
    i, j = int(np.argmin(abs(xn - 0.5 * (x0 + x1)))), int(np.argmin(abs(yn - y1)))
    if abs(xn[i] - 0.5 * (x0 + x1)) > 1e-12 or abs(yn[j] - y1) > 1e-12:
        raise ValueError("no node at the bar tip")
    return j * len(xn) + i


def uneven_batch(n=48, seed=1907, ny_range=(16, 48), slice_range=(16, 32), T=1.0, m_fine=16):
    """n independent instances of the channel problem with uneven meshes and
    materials, seeded: ny uniform on ny_range with nx = 4 ny; mu_s log-uniform
    on [2e5, 2e6] with lambda_s = 4 mu_s (Poisson ratio 0.4, as in the base
    material); mean inflow uniform on [0.5, 1.5]; slices uniform on
    slice_range; interval T with m_fine fine steps and one coarse step per slice."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        mu = float(np.exp(rng.uniform(math.log(2e5), math.log(2e6))))
        vbar = float(rng.uniform(0.5, 1.5))
        slices = int(rng.integers(slice_range[0], slice_range[1] + 1))
        out.append(Workload("uneven%02d_%dx%d" % (i, 4 * ny, ny), nx=4 * ny, ny=ny, T=T, n_slices=slices,
                            m_fine=m_fine, material=Material(mu_s=mu, lambda_s=4.0 * mu, vbar=vbar)))
    return out


def random_state(n_nodes, seed, v_scale=1.0, u_scale=2e-3, p_scale=100.0):
    """Seeded random nodal state [n_nodes, 5] = (v_x, v_y, u_x, u_y, p).

    The displacement amplitude is kept small so that the ALE map stays
    invertible (J > 0) on the meshes used in the tests.
    """
    rng = np.random.default_rng(seed)
    U = np.empty((n_nodes, 5))
    U[:, 0:2] = v_scale * rng.uniform(-1.0, 1.0, (n_nodes, 2))
    U[:, 2:4] = u_scale * rng.uniform(-1.0, 1.0, (n_nodes, 2))
    U[:, 4] = p_scale * rng.uniform(-1.0, 1.0, n_nodes)
    return U


def developed_state(w, t, seed, bend=2e-3):
    """Seeded smooth nodal state [n_nodes, 5] resembling a developed flow at time t:
    the ramped parabolic inflow profile carried through the channel and slowed
    near the bar, a bending displacement of the bar (u_x growing with height,
    fading into the fluid), a linear pressure drop, plus low-frequency seeded
    perturbations of every field. Inputs only: no discrete equation is solved."""
    rng = np.random.default_rng(seed)
    xn, yn = node_axis(X_BREAKS, w.nx_seg), node_axis(Y_BREAKS, w.ny_seg)
    X, Y = np.meshgrid(xn, yn)          # node (i, j) at [j, i]: id j * len(xn) + i
    H = Y_BREAKS[-1]
    m = w.material
    s = 0.5 * (1.0 - math.cos(math.pi * t / m.ramp_t)) if t < m.ramp_t else 1.0
    (x0, x1), (y0, y1) = SOLID_BOX
    xc = 0.5 * (x0 + x1)
    # distance-like weight to the bar (0 inside), used to fade the fields
    dx = np.maximum(np.maximum(x0 - X, X - x1), 0.0)
    dy = np.maximum(Y - y1, 0.0)
    dist = np.hypot(dx, dy)
    near = np.exp(-dist / 0.05)
    inside = (X >= x0 - 1e-12) & (X <= x1 + 1e-12) & (Y <= y1 + 1e-12)

    def mode(scale):
        a = rng.uniform(-1.0, 1.0, (3, 3))
        f = np.zeros_like(X)
        for p in range(3):
            for q in range(3):
                f += a[p, q] * np.sin((p + 1) * math.pi * X / 2.0) * np.sin((q + 1) * math.pi * Y / H)
        return scale * f

    U = np.zeros(X.shape + (5,))
    prof = 1.5 * m.vbar * s * 4.0 * Y * (H - Y) / H ** 2
    U[..., 0] = prof * (1.0 - near) + mode(0.05 * s)
    U[..., 1] = -0.3 * prof * near * np.sign(X - xc) + mode(0.02 * s)
    U[..., 2] = bend * (np.minimum(Y, y1) / y1) ** 2 * np.where(inside, 1.0, near) + mode(bend * 0.05)
    U[..., 3] = mode(bend * 0.05)
    U[..., 4] = 50.0 * s * (2.0 - X) + mode(5.0 * s)
    wall = (np.abs(Y) < 1e-12) | (np.abs(Y - H) < 1e-12) | (np.abs(X) < 1e-12) | (np.abs(X - X_BREAKS[-1]) < 1e-12)
    U[..., 2][wall] = 0.0
    U[..., 3][wall] = 0.0
    U[..., 0:2][inside] *= 1e-2
    return U.reshape(-1, 5)
