"""FP64 GEMM on the tensor cores (hps_dgemm_tc: exact BF16 splitting, tcgen05
MMAs with exact FP32 accumulation, 64-bit fixed-point combination) against
products in extended precision.  Bound per entry: the splitting truncates each
row of A and column of B below 2^-56 of its largest entry and drops slice
pairs below 2^-70, so |C - C_exact| <= K 2^-53 max|A_i.| max|B_.j| (generous)
plus the final FP64 rounding of C."""
import numpy as np
import pytest

from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def run_tc(A, B, C, alpha, beta):
    torch = pytest.importorskip("torch")
    # column-major device buffers: the contiguous storage of the transposes
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()
    M, K = A.shape
    N = B.shape[1]
    st = hps.lib().hps_dgemm_tc(M, N, K, alpha, dA.data_ptr(), M, dB.data_ptr(), K, beta,
                                dC.data_ptr(), M)
    assert st == hps.HPS_OK, hps.lib().hps_last_error()
    return dC.cpu().numpy().T.copy()


def exact(A, B, C, alpha, beta):
    Al, Bl, Cl = (x.astype(np.longdouble) for x in (A, B, C))
    return np.longdouble(alpha) * (Al @ Bl) + np.longdouble(beta) * Cl


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 200, 450), (257, 129, 1000),
                                   (130, 70, 17), (256, 128, 896)])
def test_tc_gemm_matches_extended_precision(M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-14, 14, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-14, 14, (1, N)))
    A[3, :] = 0.0  # a zero row
    B[:, 5] *= 1e-300  # tiny column
    B[:, 7] = 0.0  # a zero column
    C = rng.standard_normal((M, N))
    for alpha, beta in ((1.0, 0.0), (1.0, 1.0), (-0.5, 2.0)):
        got = run_tc(A, B, C, alpha, beta)
        ref = exact(A, B, C, alpha, beta)
        bound = (K * 2.0 ** -53 * abs(alpha) * np.max(np.abs(A), axis=1)[:, None]
                 * np.max(np.abs(B), axis=0)[None, :] + 2.0 ** -52 * np.abs(ref.astype(np.float64))
                 + 2.0 ** -52 * abs(beta) * np.abs(C))
        err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
        assert np.all(err <= bound), (alpha, beta, np.max(err / np.maximum(bound, 1e-300)))


def test_tc_gemm_is_deterministic():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((384, 448))
    B = rng.standard_normal((448, 192))
    C = rng.standard_normal((384, 192))
    a = run_tc(A, B, C, 1.0, 1.0)
    b = run_tc(A, B, C, 1.0, 1.0)
    assert np.array_equal(a, b)
