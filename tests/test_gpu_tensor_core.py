"""The tensor-core tile product (tcgen05.mma, BF16 operands, FP32 accumulation in
tensor memory) through the C ABI, against numpy.

With one BF16 term per operand the products of the rounded operands are exact,
so the result is the FP32 sum of exact products (error below 32 roundings of
the largest partial sum). With three terms per operand (the rounding residuals
entering as further BF16 terms) the result matches the FP64 product of the
FP32 operands to FP32 accuracy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


def operands(seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((128, 32)) * np.exp(rng.uniform(-3, 3, (128, 1)))).astype(np.float32)
    B = rng.standard_normal((16, 32)).astype(np.float32)
    A[5, :] = 0.0
    A[:, 27:] = 0.0     # padding columns as the element contraction uses them
    return A, B


def test_single_term_is_the_fp32_sum_of_bf16_products():
    from paper_1907_01252_gb300 import fsi
    A, B = operands(1)
    Ab = torch.tensor(A).to(torch.bfloat16).double().numpy()
    Bb = torch.tensor(B).to(torch.bfloat16).double().numpy()
    D = fsi.tc_tile_product(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), 1).cpu().numpy()
    ref = Ab @ Bb.T
    bound = 32 * 2.0 ** -24 * (np.abs(Ab) @ np.abs(Bb).T)
    assert np.all(np.abs(D - ref) <= bound + 1e-30)


@pytest.mark.parametrize("nsplit,tol", [(2, 2e-4), (3, 64 * 2.0 ** -24)])
def test_split_terms_reach_fp32_accuracy(nsplit, tol):
    from paper_1907_01252_gb300 import fsi
    for seed in (2, 3):
        A, B = operands(seed)
        D = fsi.tc_tile_product(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), nsplit)
        D = D.cpu().numpy().astype(np.float64)
        ref = A.astype(np.float64) @ B.astype(np.float64).T
        scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
        err = np.abs(D - ref) / np.maximum(scale, 1e-300)
        assert err.max() <= tol, (nsplit, err.max())
    # two calls in a row give the same bits
    D2 = fsi.tc_tile_product(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), nsplit)
    assert np.array_equal(D2.cpu().numpy().astype(np.float64), D)


def test_tensor_core_element_jacobian_matches_the_fp64_jacobian():
    """The FP32 Jacobian with the FP32 tangent and the element contraction on
    the tensor cores (three BF16 terms per operand) against the FP64 Jacobian,
    row by row, within 1e-5 of the row's largest entry (the CUDA-core variant,
    FP64 tangent and FP32 contraction, within 2e-6); a mesh with odd segment
    counts, solid cells and outflow cells, two slices at different states."""
    from paper_1907_01252_gb300 import fsi, workloads as wl
    w = wl.Workload("tcj", nx=24, ny=6, T=1.0, n_slices=4, m_fine=4)
    S = 2
    ctx = fsi.Context(w, max_batch=S, tc_contraction=1)
    ctx_cc = fsi.Context(w, max_batch=S, tc_contraction=0)
    n = ctx.n_nodes
    U = torch.tensor(np.stack([wl.random_state(n, 310 + s).ravel() for s in range(S)]), device="cuda")
    Uo = torch.tensor(np.stack([wl.random_state(n, 410 + s).ravel() for s in range(S)]), device="cuda")
    k, th = 1e-2, 0.51
    A64 = ctx.fsi_jacobian(U, Uo, k, th).cpu().numpy()
    Atc = ctx.fsi_jacobian_f32(U, Uo, k, th).cpu().numpy().astype(np.float64)
    Acc = ctx_cc.fsi_jacobian_f32(U, Uo, k, th).cpu().numpy().astype(np.float64)
    rowptr, colidx = ctx.fsi_bsr_pattern()
    brow = np.repeat(np.arange(n), np.diff(rowptr))                  # block row of every block
    for s in range(S):
        # largest |entry| of every dof row
        mag = np.abs(A64[s]).max(axis=2)                             # [nnzb, 5]
        scale = np.zeros((n, 5))
        np.maximum.at(scale, brow, mag)
        sc = scale[brow][:, :, None]
        e_tc = (np.abs(Atc[s] - A64[s]) / sc).max()
        e_cc = (np.abs(Acc[s] - A64[s]) / sc).max()
        assert e_tc <= 1e-5, (s, e_tc, e_cc)
        assert e_cc <= 2e-6, (s, e_tc, e_cc)
    # the same bits on a second call
    assert np.array_equal(ctx.fsi_jacobian_f32(U, Uo, k, th).cpu().numpy().astype(np.float64), Atc)
