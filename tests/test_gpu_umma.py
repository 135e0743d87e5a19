"""The tensor-core BF16x3 product of the shared-matrix batch (tcgen05, TMA),
through the C ABI, against the exact (FP64) product of the same FP32 operands.

With the split x = x_hi + x_lo, x_hi = bf16(x) (relative error <= 2^-9) and
x_lo = bf16(x - x_hi) (the same, of the remainder), every entry of
A_hi V_lo + A_lo V_hi + A_hi V_hi misses a v by at most 3 * 2^-18 |a| |v| (the
dropped A_lo V_lo term and the two remainders), and FP32 accumulation of 3K
products adds at most (3K + 2) 2^-24 times the sum of their magnitudes: the test
bound is (3 * 2^-18 + (3K + 2) 2^-24) sum_k |a_mk| |v_nk| per entry.  Sizes
cover partial tiles in M (128 rows per tile), N (up to 256 instances per tile)
and K (64 per stage), both operand orientations, and the shapes of the bench's
shared-matrix batch at reduced size."""
import numpy as np
import pytest

from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return lib()


def _bound(Aop, V):
    K = Aop.shape[1]
    mag = np.abs(V.astype(np.float64)) @ np.abs(Aop.astype(np.float64)).T  # N x M
    return (3 * 2.0 ** -18 + (3 * K + 2) * 2.0 ** -24) * mag


CASES = [  # (M, N, K, a_mn_major)
    (128, 32, 64, 0),
    (300, 40, 200, 0),
    (200, 70, 300, 1),
    (1000, 257, 777, 0),
    (1000, 257, 777, 1),
    (2048, 512, 4096, 0),
    (4096, 512, 2048, 1),
]


@pytest.mark.parametrize("tile_k", [32, 64])
@pytest.mark.parametrize("M,N,K,mn", CASES)
def test_bf16x3_product_within_its_error_bound(C, M, N, K, mn, tile_k):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K + mn)
    A = rng.standard_normal((K, M) if mn else (M, K)).astype(np.float32) / np.sqrt(K)
    V = rng.standard_normal((N, K)).astype(np.float32)
    D = C.mpax_dense_bf16x3(torch.from_numpy(A).cuda(), torch.from_numpy(V).cuda(),
                            a_mn_major=bool(mn), tile_k=tile_k).cpu().numpy()
    Aop = A.T if mn else A
    exact = V.astype(np.float64) @ Aop.astype(np.float64).T  # N x M
    err = np.abs(D.astype(np.float64) - exact)
    bound = _bound(Aop, V)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    # far below one BF16 product's error (~2^-9 relative): the split keeps ~16 bits
    assert np.max(err) < 1e-3 * np.max(np.abs(exact)) + 1e-30
    if tile_k == 64:  # both pipeline shapes form the same sums in the same order
        D32 = C.mpax_dense_bf16x3(torch.from_numpy(A).cuda(), torch.from_numpy(V).cuda(),
                                  a_mn_major=bool(mn), tile_k=32).cpu().numpy()
        assert np.array_equal(D, D32)


def test_bf16x3_host_pointers_and_bad_sizes(C):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((96, 80)).astype(np.float32)
    V = rng.standard_normal((5, 80)).astype(np.float32)
    D = C.mpax_dense_bf16x3(A, V)
    exact = V.astype(np.float64) @ A.astype(np.float64).T
    assert np.all(np.abs(D - exact) <= _bound(A, V))
    with pytest.raises(C.MpaxError) as ei:
        C.mpax_dense_bf16x3(np.zeros((0, 8), np.float32), V[:, :8])
    assert ei.value.status == 1
