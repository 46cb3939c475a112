"""The float-float dot product of csrc/fsi_ff.h (FP64-class accuracy on the FP32 pipe),
compiled for the host, against exact rational sums: block-row dot products of the
lengths and magnitude spreads of the FSI Jacobians (5 x 25 entries in 2D, 7 x 189 in
3D; entries from 1e-8 to 1e7)."""
import ctypes as C
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("ff") / "libff.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, os.path.join(HERE, "native", "ff_host.cpp")],
                   check=True)
    lib = C.CDLL(out)
    P = C.POINTER(C.c_double)
    for f in (lib.ff_dot_host, lib.f64_dot_host):
        f.argtypes, f.restype = [P, P, C.c_int], C.c_double
    return lib


def ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def exact(a, x):
    return float(sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x)))


@pytest.mark.parametrize("n", [125, 1323])
def test_float_float_dot_is_fp64_class(lib, n):
    """Error relative to sum |a_i x_i|: below 2^-45 on every row (FP64 summation of the
    same rows is shown beside it), with mixed signs and a spread of 15 decades."""
    rng = np.random.default_rng(n)
    worst_ff = worst_64 = 0.0
    for trial in range(40):
        a = rng.choice([-1, 1], n) * 10.0 ** rng.uniform(-8, 7, n)
        x = rng.choice([-1, 1], n) * 10.0 ** rng.uniform(-6, 2, n)
        ref = exact(a, x)
        mag = float(np.sum(np.abs(a * x)))
        worst_ff = max(worst_ff, abs(lib.ff_dot_host(ptr(a), ptr(x), n) - ref) / mag)
        worst_64 = max(worst_64, abs(lib.f64_dot_host(ptr(a), ptr(x), n) - ref) / mag)
    assert worst_ff <= 2.0 ** -45, (worst_ff, worst_64)


def test_float_float_split_and_cancellation(lib):
    """Exact cancellation cases: a row whose products cancel to a tiny remainder keeps the
    remainder to 2^-45 of sum |a x|; values beyond float precision survive the split."""
    a = np.array([1.0 + 2.0 ** -30, -1.0, 3.0e5, -3.0e5, 1e-7])
    x = np.array([1.0, 1.0, 1.0 + 2.0 ** -40, 1.0, 1.0])
    ref = exact(a, x)
    got = lib.ff_dot_host(ptr(a), ptr(x), len(a))
    mag = float(np.sum(np.abs(a * x)))
    assert abs(got - ref) <= 2.0 ** -45 * mag, (got, ref)
    one = np.array([np.pi]), np.array([1.0])
    assert abs(lib.ff_dot_host(ptr(one[0]), ptr(one[1]), 1) - np.pi) <= 2.0 ** -47 * np.pi
