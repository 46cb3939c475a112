"""FP64 CPU oracle: Parareal iteration and speedup model (test infrastructure only).

Sec. 3 of Margenberg & Richter. The interval I = [0, T] is cut into N slices
of length T/N; C and F advance a state over one slice with a coarse and a fine
step size. The recursion Eq. (parareal:iteration) is

    U_0^i = U(0),   U_{n+1}^0 = C(U_n^0)                      (predictor sweep)
    U_{n+1}^{i+1} = C(U_n^{i+1}) + F(U_n^i) - C(U_n^i)

evaluated here as F(U_n^i) + (C(U_n^{i+1}) - C(U_n^i)): for a slice whose
input did not change the bracket is exactly zero, so the first i+1 boundary
values after iteration i+1 are bit-for-bit the serial fine solution (the
property noted in Sec. 4.1: after the i-th iteration the solution on the i-th
interval does not improve any more).
"""
from __future__ import annotations

import numpy as np


def parareal(U0, n_slices, coarse, fine, n_iter):
    """Run n_iter Parareal iterations.

    coarse(U, n), fine(U, n): propagate state U over slice n (t_n -> t_{n+1}).
    Returns the list of iterates; iterate i is a list of N+1 boundary states.
    """
    U = [np.array(U0, dtype=float, copy=True)]
    C_old = []
    for n in range(n_slices):                       # predictor sweep (i = 0)
        C_old.append(coarse(U[n], n))
        U.append(C_old[n])
    history = [list(U)]
    for i in range(n_iter):
        F_val = [fine(U[n], n) for n in range(n_slices)]   # parallel part
        U_new = [U[0]]
        C_new = []
        for n in range(n_slices):                   # sequential corrected sweep
            C_new.append(coarse(U_new[n], n))
            U_new.append(F_val[n] + (C_new[n] - C_old[n]))
        U, C_old = U_new, C_new
        history.append(list(U))
    return history


def serial(U0, n_slices, fine):
    """The serial fine solution at the slice boundaries."""
    U = [np.array(U0, dtype=float, copy=True)]
    for n in range(n_slices):
        U.append(fine(U[n], n))
    return U


def dahlquist_parareal_closed_form(lam_f, lam_c, n, i, u0=1.0):
    """Closed form of iterate i at boundary n for linear scalar propagators.

    With F u = a u and C u = b u the recursion is linear and
    U_n^i = sum_{j=0}^{i} binom(n, j) (a - b)^j b^(n-j) u0
    (Gander and Vandewalle 2007, used here only as an independent check).
    """
    from math import comb
    a, b = lam_f, lam_c
    return sum(comb(n, j) * (a - b) ** j * b ** (n - j) for j in range(0, min(i, n) + 1)) * u0


def speedup_model(r, n_iter, n_slices):
    """Eq. (eq:speedup): S = 1 / (r + (K/N)(1 + r)), r = h_F / h_C, K iterations, N slices."""
    return 1.0 / (r + (n_iter / n_slices) * (1.0 + r))
