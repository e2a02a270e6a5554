"""The tcgen05 split-precision GEMM against a numpy FP64 product.

Error model: each operand is carried as hi + lo 16-bit pieces; the dropped
lo*lo product and the piece rounding leave ~2^-22 (FP16 pieces, scaled) or
~2^-16 (BF16 pieces) relative error per product, plus FP32 accumulation
(~2^-24 sqrt(K)).  Errors are measured against |A| @ |B| elementwise.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_1912_03174_gb300 import binding
    return binding


SHAPES = [(128, 128, 64), (40, 40, 40), (130, 200, 300), (256, 384, 1024), (1024, 1024, 1024)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_fp16_pieces_match_fp64(B, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-6, 0, size=(M, K)))
    Bm = rng.normal(size=(K, N)) * np.exp(rng.uniform(-6, 0, size=(K, N)))
    C, ms = B.tdb_split_gemm(A, Bm, fmt=0)
    ref = A @ Bm
    scale = np.abs(A) @ np.abs(Bm)
    rel = np.max(np.abs(C - ref) / scale)
    # pieces (2^-20 with margin) + FP32 accumulation (2^-24 sqrt(K), x16 for the max over elements)
    assert rel < 2.0 ** -20 + 16 * 2.0 ** -24 * np.sqrt(K), rel
    assert ms > 0


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (130, 200, 300)])
def test_bf16_pieces_match_fp64_to_16_bits(B, M, N, K):
    rng = np.random.default_rng(5)
    A = rng.normal(size=(M, K))
    Bm = rng.normal(size=(K, N))
    C, _ = B.tdb_split_gemm(A, Bm, fmt=1)
    C16, _ = B.tdb_split_gemm(A, Bm, fmt=0)
    ref = A @ Bm
    scale = np.abs(A) @ np.abs(Bm)
    e_bf = np.max(np.abs(C - ref) / scale)
    e_fp = np.max(np.abs(C16 - ref) / scale)
    assert e_bf < 1e-4, e_bf
    # FP32 accumulation (~2^-24 sqrt(K)) bounds the FP16-piece error here, so the
    # gap to the 16-bit BF16 pieces is a few x, not 2^6
    assert e_fp < e_bf / 2, (e_fp, e_bf)


def test_exact_small_integers(B):
    # small integers are exact in every piece format: the result must be exact
    rng = np.random.default_rng(1)
    A = rng.integers(-8, 9, size=(192, 320)).astype(float)
    Bm = rng.integers(-8, 9, size=(320, 136)).astype(float)
    for fmt in (0, 1):
        C, _ = B.tdb_split_gemm(A, Bm, fmt=fmt)
        assert np.array_equal(C, A @ Bm)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (130, 200, 300), (256, 384, 1024),
                                   (200, 136, 2048), (128, 256, 3000)])
def test_head_scheme_matches_fp64(B, M, N, K):
    # K > 1024: one exact head accumulator per 1024-deep slice of K
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-6, 0, size=(M, K)))
    Bm = rng.normal(size=(K, N)) * np.exp(rng.uniform(-6, 0, size=(K, N)))
    C, _ = B.tdb_split_gemm(A, Bm, fmt=2)
    ref = A @ Bm
    scale = np.abs(A) @ np.abs(Bm)
    rel = np.max(np.abs(C - ref) / scale)
    assert rel < 2.0 ** -20 + 16 * 2.0 ** -24 * np.sqrt(K), rel


@pytest.mark.parametrize("K", [1024, 2048])
def test_head_scheme_removes_the_accumulation_bias(B, K):
    # all products positive: the FP32 tensor-core accumulation truncates, so the
    # hi/lo scheme comes out systematically low by ~K 2^-25; the integer heads sum
    # exactly, leaving only the tails' share (~2^-7 of it)
    rng = np.random.default_rng(11)
    A = rng.uniform(0, 1, (256, K))
    Bm = rng.uniform(0, 1, (K, 256))
    ref = A @ Bm
    bias = {}
    for fmt in (0, 2):
        C, _ = B.tdb_split_gemm(A, Bm, fmt=fmt)
        bias[fmt] = float(np.mean((C - ref) / ref))
    assert bias[0] < -1e-6, bias              # measured ~ -7e-6 on GB300
    assert abs(bias[2]) < abs(bias[0]) / 20, bias


def test_head_scheme_rejects_k_beyond_three_slices(B):
    A = np.ones((128, 3073))
    with pytest.raises(B.TdbError) as e:
        B.tdb_split_gemm(A, A.T.copy(), fmt=2)
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# integer-slice product (TDB_FP64_SLICED): six 7-bit slices, exact accumulation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (130, 200, 300), (256, 384, 1024),
                                   (200, 136, 2048), (64, 100, 4096)])
def test_slice_gemm_is_fp64_accurate(B, M, N, K):
    rng = np.random.default_rng(3 * M + 5 * N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-6, 0, size=(M, K)))
    Bm = rng.normal(size=(K, N)) * np.exp(rng.uniform(-6, 0, size=(K, N)))
    C, _ = B.tdb_slice_gemm(A, Bm)
    ref = A @ Bm
    # the slices keep 42 bits of each entry relative to its row (A) or column (B)
    # maximum; the kept pairs leave out terms below 7 2^-42 of those maxima
    bound = K * np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(Bm), axis=0)[None, :]
    assert np.all(np.abs(C - ref) <= 2.0 ** -38 * bound), np.max(np.abs(C - ref) / bound)
    rel = np.max(np.abs(C - ref) / (np.abs(A) @ np.abs(Bm)))
    assert rel < 1e-9, rel


def test_slice_gemm_is_exact_on_integers_and_powers_of_two(B):
    rng = np.random.default_rng(5)
    A = rng.integers(-64, 65, size=(150, 520)).astype(float)
    Bm = rng.integers(-64, 65, size=(520, 90)).astype(float) * 2.0 ** -20
    C, _ = B.tdb_slice_gemm(A, Bm)
    assert np.array_equal(C, A @ Bm)


def test_slice_gemm_has_no_accumulation_bias(B):
    # the all-positive product whose FP32 tensor-core accumulation comes out low
    rng = np.random.default_rng(11)
    A = rng.uniform(0, 1, (256, 2048))
    Bm = rng.uniform(0, 1, (2048, 256))
    C, _ = B.tdb_slice_gemm(A, Bm)
    ref = A @ Bm
    assert np.max(np.abs(C - ref) / ref) < 1e-11
    assert abs(float(np.mean((C - ref) / ref))) < 1e-13


def test_slice_gemm_rejects_k_beyond_4096(B):
    A = np.ones((64, 4097))
    with pytest.raises(B.TdbError) as e:
        B.tdb_slice_gemm(A, A.T.copy())
    assert e.value.status == 1
