"""FP32 products on the tensor cores (hps_sgemm_tc: every FP32 value split
exactly into three BF16 terms, six BF16 products per K step, per-block FP32
accumulators summed in registers) against the product in extended precision.

Bound per entry: the FP32 GEMM bound (K + 2) 2^-24 (|alpha| |A| |B| + |beta| |C|)
with room for the dropped terms a2 b3, a3 b2, a3 b3 (2^-24 of |a b| each).
The error measured against it also checks the accumulation: with one tensor
memory accumulator over a long K the error grew with every MMA (the reason
for the per-block accumulators); here it must stay near a plain FP32 chain's."""
import numpy as np
import pytest

from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def run_tc32(A, B, C, alpha, beta, lda=None, ldb=None, ldc=None):
    torch = pytest.importorskip("torch")
    M, K = A.shape
    N = B.shape[1]
    lda, ldb, ldc = lda or M, ldb or K, ldc or M

    def colmajor(X, ld):
        buf = np.zeros((X.shape[1], ld), np.float32)  # column j at buf[j, :rows]
        buf[:, :X.shape[0]] = X.T
        return torch.from_numpy(buf).cuda()

    dA, dB, dC = colmajor(A, lda), colmajor(B, ldb), colmajor(C, ldc)
    st = hps.lib().hps_sgemm_tc(M, N, K, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb, beta,
                                dC.data_ptr(), ldc)
    assert st == hps.HPS_OK, hps.lib().hps_last_error()
    out = dC.cpu().numpy()
    return out[:, :M].T.copy(), out


def check(M, N, K, alpha, beta, seed, spread=0.0, **ld):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, K)) * np.exp(spread * rng.standard_normal((M, K)))).astype(np.float32)
    B = (rng.standard_normal((K, N)) * np.exp(spread * rng.standard_normal((K, N)))).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    got, raw = run_tc32(A, B, C, np.float32(alpha), np.float32(beta), **ld)
    Al, Bl, Cl = (x.astype(np.longdouble) for x in (A, B, C))
    want = np.longdouble(alpha) * (Al @ Bl) + np.longdouble(beta) * Cl
    scale = abs(alpha) * (np.abs(Al) @ np.abs(Bl)) + abs(beta) * np.abs(Cl)
    err = np.abs(got.astype(np.longdouble) - want)
    bound = (K + 2) * 2.0 ** -24 * scale
    assert np.all(err <= bound), float(np.max(err / bound))
    return float(np.max(err / scale)), raw


@pytest.mark.parametrize("M,N,K", [(96, 16, 32), (128, 64, 64), (196, 64, 196), (196, 56, 196),
                                   (300, 200, 450), (257, 129, 1000), (130, 65, 33)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (0.5, -2.0)])
def test_tc32_vs_extended_precision(M, N, K, alpha, beta):
    rel, _ = check(M, N, K, alpha, beta, seed=M + N + K)
    # far inside the FP32 bound: the accumulation does not grow with K
    assert rel < 64 * 2.0 ** -24, rel


def test_tc32_wide_dynamic_range_and_leading_dimensions():
    check(200, 70, 300, 1.0, 1.0, seed=5, spread=3.0, lda=203, ldb=301, ldc=256)


def test_tc32_small_products_take_the_tile_kernels():
    # below M = 96 or K = 32 the tile kernels run the product, same contract
    check(40, 30, 200, 1.0, 1.0, seed=7)
    check(200, 30, 16, 1.0, 0.0, seed=8)


def test_tc32_is_deterministic_and_leaves_padding_alone():
    _, raw1 = check(196, 64, 196, -1.0, 1.0, seed=9, ldc=200)
    _, raw2 = check(196, 64, 196, -1.0, 1.0, seed=9, ldc=200)
    assert np.array_equal(raw1, raw2)
    assert np.all(raw1[:, 196:] == 0.0)  # rows M .. ldc-1 of C untouched
