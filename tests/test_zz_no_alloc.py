"""The allocation-free projection entry point against the allocating one.

mcf_project_capped_simplex_noalloc serves callers that cannot call cudaMalloc: processes
whose device memory belongs to their own pool or to a framework allocator, and loops that
must not enter the allocator. It must give the same projection, multipliers and distance as
mcf_project_capped_simplex, call after call, with or without the synchronizing distance
output, and refuse sizes beyond its fixed scratch with a clear error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_COLS = 1 << 18


def _inputs(seed, m, n, ld):
    g = torch.Generator(device="cuda").manual_seed(seed)
    Qt = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    Qt[:, :n] = torch.randn((m, n), device="cuda", generator=g)
    cap = torch.rand(m, device="cuda", generator=g) * 2.0 + 0.05
    return Qt, cap


def _project(fn, Qt, cap, n, m, ld):
    Ft = torch.full_like(Qt, -3.0)
    mu = torch.zeros(m, dtype=torch.float32, device="cuda")
    d2 = fn(n, m, ld, Qt.data_ptr(), cap.data_ptr(), Ft.data_ptr(), mu.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return Ft.cpu().numpy(), mu.cpu().numpy(), d2


@pytest.mark.parametrize("m,n,ld", [(5000, 300, 300), (257, 10000, 10000), (1000, 37, 40)])
def test_noalloc_matches_allocating_entry_point(lib, m, n, ld):
    Qt, cap = _inputs(m + n, m, n, ld)
    F_ref, mu_ref, d_ref = _project(lib.mcf_project_capped_simplex, Qt, cap, n, m, ld)
    scale = max(1.0, float(Qt.abs().max()))
    for _ in range(2):                      # two calls in a row share the scratch array
        F, mu, d = _project(lib.mcf_project_capped_simplex_noalloc, Qt, cap, n, m, ld)
        assert np.abs(F - F_ref).max() <= 2e-5 * scale
        assert np.abs(mu - mu_ref).max() <= 2e-5 * scale
        assert d == pytest.approx(d_ref, rel=1e-4)


def test_noalloc_without_distance_is_queued_on_the_stream(lib):
    """dist2 = NULL: the call only queues the work; after a stream synchronize the outputs
    equal the allocating entry point's, on two calls in a row."""
    n, m, ld = 1000, 3000, 1000
    Qt, cap = _inputs(7, m, n, ld)
    F_ref, mu_ref, _ = _project(lib.mcf_project_capped_simplex, Qt, cap, n, m, ld)
    scale = max(1.0, float(Qt.abs().max()))
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        Ft = torch.full_like(Qt, -3.0)
        mu = torch.zeros(m, dtype=torch.float32, device="cuda")
        assert lib.mcf_project_capped_simplex_noalloc(
            n, m, ld, Qt.data_ptr(), cap.data_ptr(), Ft.data_ptr(), mu.data_ptr(), stream,
            want_dist2=False) is None
        torch.cuda.current_stream().synchronize()
        assert np.abs(Ft.cpu().numpy() - F_ref).max() <= 2e-5 * scale
        assert np.abs(mu.cpu().numpy() - mu_ref).max() <= 2e-5 * scale


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.MCFError) as ei:
        lib.mcf_project_capped_simplex_noalloc(4, MAX_COLS + 1, 4, x.data_ptr(), x.data_ptr(),
                                               x.data_ptr(), x.data_ptr())
    assert ei.value.code == lib.MCF_ERR_INVALID
    assert "262144" in lib.mcf_last_error()
