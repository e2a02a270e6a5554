"""tdb_split_gemm_noalloc: the split-precision GEMM for callers that cannot
allocate device memory, checked against tdb_split_gemm (which allocates its
own buffers) on two calls in a row.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.  It must also pass on its own in a
fresh process: the first call there performs the one-time scratch lookup.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_03174_gb300 import binding
    return binding


def _run_noalloc(B, A, Bm, fmt, torch):
    # the test allocates the caller-owned device buffers; the entry point itself does not
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(Bm).cuda()
    dC = torch.full((A.shape[0], Bm.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    B.tdb_split_gemm_noalloc(A.shape[0], Bm.shape[1], A.shape[1], dA.data_ptr(), dB.data_ptr(), fmt,
                             dC.data_ptr(), s.cuda_stream)
    s.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_noalloc_matches_the_allocating_entry_point_on_two_calls(B, fmt):
    import torch
    rng = np.random.default_rng(100 + fmt)
    shapes = [(200, 136, 300), (128, 256, 64)]     # the second call reuses the scratch
    for M, N, K in shapes:
        A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-4, 0, size=(M, K)))
        Bm = rng.normal(size=(K, N)) * np.exp(rng.uniform(-4, 0, size=(K, N)))
        ref, _ = B.tdb_split_gemm(A, Bm, fmt=fmt)
        got = _run_noalloc(B, A, Bm, fmt, torch)
        scale = np.abs(A) @ np.abs(Bm)
        assert np.all(np.isfinite(got))
        tol = 2.0 ** -20 + 16 * 2.0 ** -24 * np.sqrt(K) if fmt != 1 else 1e-4
        assert np.max(np.abs(got - ref) / scale) < tol
        assert np.max(np.abs(got - A @ Bm) / scale) < tol


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_noalloc_reports_a_device_failure_as_nan_and_recovers(B, fmt):
    """The call returns before its GPU work runs, so a device-side failure (here an
    operand piece that overflows because A holds an Inf) shows up as C filled with NaN;
    the next call starts from a cleared flag and is exact again."""
    import torch
    rng = np.random.default_rng(200 + fmt)
    M, N, K = 96, 80, 120
    A = rng.normal(size=(M, K))
    Bm = rng.normal(size=(K, N))
    bad = A.copy()
    bad[3, 7] = np.inf
    got = _run_noalloc(B, bad, Bm, fmt, torch)
    assert np.all(np.isnan(got))
    got = _run_noalloc(B, A, Bm, fmt, torch)
    scale = np.abs(A) @ np.abs(Bm)
    tol = 2.0 ** -20 + 16 * 2.0 ** -24 * np.sqrt(K) if fmt != 1 else 1e-4
    assert np.all(np.isfinite(got)) and np.max(np.abs(got - A @ Bm) / scale) < tol


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    import torch
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.TdbError) as e:
        B.tdb_split_gemm_noalloc(1024, 1024, 1024, d.data_ptr(), d.data_ptr(), 0, d.data_ptr(), None)
    assert e.value.status == 9 and "8 MiB" in str(e.value)
    with pytest.raises(B.TdbError) as e:
        B.tdb_split_gemm_noalloc(8, 8, 2 ** 31 - 1, d.data_ptr(), d.data_ptr(), 0, d.data_ptr(), None)
    assert e.value.status == 1
