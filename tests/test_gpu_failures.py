"""Failure detection through the C ABI, made on the host side (no GPU fault):
a non-finite input, exhausted iteration limits and bad sizes return their
status codes, every loop ends, and healthy slices of the same batch keep the
result they have when run alone."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"
W = wl.Workload("fail", nx=16, ny=4, T=0.5, n_slices=4, m_fine=2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def ctx_for(S=2, **kw):
    from paper_1907_01252_gb300 import fsi
    return fsi.Context(W, max_batch=S, **kw)


def test_nan_slice_reports_enan_and_spares_the_other_slice():
    from paper_1907_01252_gb300 import fsi
    ctx = ctx_for()
    U = torch.zeros((2, ctx.n_dofs), dtype=torch.float64, device=DEV)
    U[1, 7] = math.nan
    k = W.k_fine
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi_theta_step(U, [0.0, 0.0], k, 0.5 + k, U_new=(out := torch.empty_like(U)))
    assert e.value.code == fsi.FSI_ENAN
    assert e.value.slice_status == [fsi.FSI_OK, fsi.FSI_ENAN]
    alone, st = ctx.fsi_theta_step(U[:1].contiguous(), [0.0], k, 0.5 + k)
    assert st["slice_status"] == [fsi.FSI_OK]
    assert torch.equal(out[0], alone[0])
    # the fine propagator on a context of one slice runs the two slices as two batches:
    # the second batch's statuses land at its offset
    with pytest.raises(fsi.FsiError) as e:
        ctx_for(S=1).fsi_fine(U, [0.0, 0.0])
    assert e.value.slice_status == [fsi.FSI_OK, fsi.FSI_ENAN]


def test_newton_iteration_limit_reports_enewton():
    from paper_1907_01252_gb300 import fsi
    ctx = ctx_for(S=1, newton_maxit=1)
    U = torch.zeros((1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi_theta_step(U, [0.0], W.k_coarse, 1.0)       # a large step needs more than one iteration
    assert e.value.code == fsi.FSI_ENEWTON
    assert e.value.slice_status == [fsi.FSI_ENEWTON]


def test_gmres_iteration_limit_reports_egmres():
    """Linear solves stopped at their iteration limit still correct the Newton
    iterate; when Newton then fails, the slice reports FSI_EGMRES (the cause)."""
    from paper_1907_01252_gb300 import fsi
    ctx = ctx_for(S=1, gmres_maxit=2, newton_maxit=3)
    U = torch.zeros((1, ctx.n_dofs), dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi_theta_step(U, [0.0], W.k_coarse, 1.0)
    assert e.value.code == fsi.FSI_EGMRES
    assert e.value.slice_status == [fsi.FSI_EGMRES]


def test_bad_sizes_are_rejected():
    from paper_1907_01252_gb300 import fsi
    ctx = ctx_for(S=2)
    U = torch.zeros((3, ctx.n_dofs), dtype=torch.float64, device=DEV)
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi_theta_step(U, [0.0] * 3, W.k_fine, 0.5)      # more slices than max_batch
    assert e.value.code == fsi.FSI_EINVAL
    with pytest.raises(fsi.FsiError) as e:
        ctx.fsi_residual(U, U, [0.0] * 3, W.k_fine, 0.5)
    assert e.value.code == fsi.FSI_EINVAL
    with pytest.raises(fsi.FsiError):
        fsi.Context(W, max_batch=0)
    with pytest.raises(fsi.FsiError):
        fsi.Context(W, max_batch=1, gmres_restart=100)
    with pytest.raises(fsi.FsiError):
        fsi.Context(W, max_batch=1, newton_eta=1.5)
