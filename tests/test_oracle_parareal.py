"""Pins of the oracle's Parareal driver and speedup model (CPU only)."""
import os

import numpy as np
import pytest

from oracle import parareal as pr

HERE = os.path.dirname(__file__)


def test_speedup_model_matches_printed_value():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "speedup_model.txt")) if l.strip() and not l.startswith("#")]
    for r, K, N, S, tol in rows:
        assert abs(pr.speedup_model(float(r), int(K), int(N)) - float(S)) <= float(tol)


@pytest.mark.parametrize("lam,N,m", [(-1.0, 8, 10), (-5.0, 6, 4), (0.3, 5, 7)])
def test_parareal_dahlquist_closed_form(lam, N, m):
    dt = 1.0 / N
    a = (1 + lam * dt / (2 * m)) ** m / (1 - lam * dt / (2 * m)) ** m   # m trapezoidal steps
    b = 1.0 / (1 - lam * dt)                                             # one implicit Euler step
    fine = lambda u, n: a * u
    coarse = lambda u, n: b * u
    hist = pr.parareal(np.array(1.0), N, coarse, fine, N)
    for i, it in enumerate(hist):
        for n in range(N + 1):
            ref = pr.dahlquist_parareal_closed_form(a, b, n, i)
            assert abs(float(it[n]) - ref) <= 1e-13 * max(1.0, abs(ref))
    # k = N iterations reproduce the serial fine solution
    ser = pr.serial(np.array(1.0), N, fine)
    assert all(abs(float(hist[N][n]) - float(ser[n])) <= 1e-14 for n in range(N + 1))


def test_parareal_frozen_slices_are_bitwise_serial():
    """After iteration i the first i boundary values equal the serial run exactly."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((4, 4)) * 0.3
    fine = lambda u, n: np.tanh(M @ u) + 0.1 * n
    coarse = lambda u, n: 0.9 * np.tanh(M @ u) + 0.1 * n
    N = 6
    hist = pr.parareal(rng.standard_normal(4), N, coarse, fine, N)
    ser = pr.serial(hist[0][0], N, fine)
    for i in range(N + 1):
        for n in range(i + 1):
            assert np.array_equal(hist[i][n], ser[n])


def test_parareal_fsi_reaches_serial_fine_solution():
    """Parareal on the ALE-FSI step (tiny mesh): after iteration i the first i
    slice boundaries are bit-for-bit the serial fine solution, and iteration N
    reproduces it everywhere (Sec. 4.1)."""
    from oracle import fsi as of
    from paper_1907_01252_gb300 import workloads as wl
    mesh = of.make_mesh(wl.X_BREAKS, wl.Y_BREAKS, wl.cells_per_segment(wl.X_BREAKS, 8),
                        wl.cells_per_segment(wl.Y_BREAKS, 2), wl.SOLID_BOX)
    model = of.FSIModel(mesh, wl.Material())
    N, m, T = 3, 2, 0.06
    dt = T / N
    fine = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, m)
    coarse = lambda U, n: model.propagate(U, n * dt, (n + 1) * dt, 1, theta=1.0)
    U0 = np.zeros((mesh.n_nodes, 5))
    hist = pr.parareal(U0, N, coarse, fine, N)
    ser = pr.serial(U0, N, fine)
    for i in range(N + 1):
        for n in range(i + 1):
            assert np.array_equal(hist[i][n], ser[n])
    assert not np.array_equal(hist[0][N], ser[N])      # the coarse predictor differs
