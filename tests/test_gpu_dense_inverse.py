"""The coarsest-level dense solver through the C ABI: the cluster kernel and
the one-CTA kernel give the same inverse (same pivots, same arithmetic), both
agree with numpy's inverse, pivoting is exercised, singular input is reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def batch(S, n, seed, zero_diag=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((S, n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    if zero_diag:      # every step must pivot
        A = A[:, ::-1, :].copy()
    return A


@pytest.mark.parametrize("n,S", [(1, 1), (7, 3), (135, 2), (325, 2), (400, 1), (600, 1)])
def test_cluster_and_single_cta_inverses_agree_with_numpy(n, S):
    from paper_1907_01252_gb300 import fsi
    for zero_diag in (False, True):
        A = batch(S, n, 7 + n, zero_diag)
        At = torch.tensor(A, device=DEV)
        inv0 = fsi.dense_invert(At, method=0).cpu().numpy()
        inv1 = fsi.dense_invert(At, method=1).cpu().numpy()
        assert np.array_equal(inv0, inv1), (n, zero_diag)
        assert np.array_equal(At.cpu().numpy(), A)          # input untouched
        for s in range(S):
            ref = np.linalg.inv(A[s])
            cond = np.linalg.cond(A[s])
            # Gauss-Jordan with partial pivoting: error O(n eps cond) relative to the inverse
            tol = 50 * n * np.finfo(float).eps * cond * np.abs(ref).max()
            assert np.abs(inv0[s] - ref).max() <= tol, (n, s, zero_diag)


def test_singular_matrix_is_reported():
    from paper_1907_01252_gb300 import fsi
    A = batch(2, 40, 3)
    A[1, 5, :] = 0.0
    with pytest.raises(fsi.FsiError) as e:
        fsi.dense_invert(torch.tensor(A, device=DEV), method=0)
    assert e.value.code == fsi.FSI_EJAC
