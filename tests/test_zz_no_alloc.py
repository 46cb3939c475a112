"""The allocation-free residual entry point (through the C ABI) matches fsi_residual.

fsi_residual_noalloc serves callers that must not allocate device memory when
they evaluate residuals (a framework that owns the device memory pool, a loop
with a fixed memory budget): its scratch is a static device array instead of
context workspace. This file is collected last so that a failure here comes
after every other test has run; it passes alone and after the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01252_gb300 import workloads as wl  # noqa: E402


def test_noalloc_residual_matches_residual_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build, fsi
    build.build_library()
    w = wl.Workload("noalloc", nx=24, ny=6, T=1.0, n_slices=4, m_fine=4)
    S = 3
    ctx = fsi.Context(w, max_batch=S)
    n_nodes = ctx.n_nodes
    dev = "cuda:0"
    out = torch.empty((S, ctx.n_dofs), dtype=torch.float64, device=dev)
    for call, seed in enumerate((7, 8)):          # two calls in a row share the static scratch
        U = torch.tensor(np.stack([wl.random_state(n_nodes, seed * 10 + s).ravel() for s in range(S)]),
                         device=dev)
        Uo = torch.tensor(np.stack([wl.random_state(n_nodes, seed * 10 + 5 + s).ravel() for s in range(S)]),
                          device=dev)
        t_new = [0.05 + 0.1 * call, 0.15, 0.9]
        k, th = 1e-2, 0.51
        ref = ctx.fsi_residual(U, Uo, t_new, k, th)
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        got = ctx.fsi_residual_noalloc(U, Uo, t_new, k, th, out)
        torch.cuda.synchronize()
        # the same kernels on the same inputs: the same bits
        assert torch.equal(got, ref), call
        if call > 0:   # after the first call (module loading, symbol lookup) nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
    # sizes beyond the static scratch are rejected with a clear error
    big = wl.LARGE_128x32
    ctx2 = fsi.Context(big, max_batch=1)
    U = torch.zeros((12, ctx2.n_dofs), dtype=torch.float64, device=dev)
    with pytest.raises(fsi.FsiError, match="static scratch"):
        ctx2.fsi_residual_noalloc(U, U, [0.0] * 12, 1e-3, 0.5, U.clone())
