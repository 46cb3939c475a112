"""The launch profiler (CUDA events around the library's own launches) with
and without CUDA graphs: timing never changes a result, every timed kernel
reports time, launches and algorithmic flops, and graph replays are timed too."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01252_gb300 import workloads as wl  # noqa: E402

DEV = "cuda:0"
W = wl.Workload("prof", nx=16, ny=4, T=0.5, n_slices=4, m_fine=2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1907_01252_gb300 import build
    build.build_library()


@pytest.mark.parametrize("graph_max_batch", [0, 4])
def test_profiled_step_is_bitwise_unprofiled_and_timed(graph_max_batch):
    from paper_1907_01252_gb300 import fsi
    ctx = fsi.Context(W, max_batch=2, graph_max_batch=graph_max_batch)
    U = torch.zeros((2, ctx.n_dofs), dtype=torch.float64, device=DEV)
    t = [0.0, W.T / W.n_slices]
    ref, _ = ctx.fsi_coarse(U, t)
    names = fsi.kernel_names()
    try:
        fsi.profile_enable(names)
        got, _ = ctx.fsi_coarse(U, t)
        torch.cuda.synchronize()
        for name in ("k_bsr_spmv", "k_vanka_cell", "k_cell_jacobian", "k_dots_partial"):
            ms, launches, flops = fsi.profile_read(name)
            assert launches > 0 and ms > 0.0 and flops > 0.0, name
        # a second profiled call (graphs already captured under this epoch) adds to the totals
        before = fsi.profile_read("k_bsr_spmv")[1]
        again, _ = ctx.fsi_coarse(U, t)
        torch.cuda.synchronize()
        assert fsi.profile_read("k_bsr_spmv")[1] > before
    finally:
        fsi.profile_enable([])
    assert torch.equal(got, ref)
    assert torch.equal(again, ref)
