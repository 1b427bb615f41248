"""The mixed mode's leaf inverse (Gauss-Jordan with partial pivoting, the
whole 196 x 196 matrix in registers, through hps_sinv_gj) against the
definition of the inverse, on the oracle's own leaf operators A_ii (Section
3.1: interior rows and columns of A on a p = 16 leaf) and on random and
structured matrices.

Bounds: the residual of a backward-stable FP32 inversion, componentwise
|A X - I| <= n u (|A| |X|) with u = 2^-24 (measured on these matrices by an
FP32 emulation of the same elimination: 0.04 .. 0.21 of it), and the forward
error against the FP64 inverse of the FP32 matrix within the inversion bound
n u cond(A) (measured: up to 0.31 of it, at cond(A) = 1).  A wrong pivot row,
multiplier or un-permutation is off by O(1)."""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300.build import build

pytestmark = pytest.mark.gpu
N = 196
U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def gpu_inverse(mats, expect=None):
    torch = pytest.importorskip("torch")
    A = np.ascontiguousarray(np.stack([m.T for m in mats]).astype(np.float32))  # column-major
    dA = torch.from_numpy(A).cuda()
    dX = torch.full_like(dA, -7.0)
    st = hps.lib().hps_sinv_gj(N, len(mats), dA.data_ptr(), dX.data_ptr())
    assert st == (hps.HPS_OK if expect is None else expect), hps.lib().hps_last_error()
    assert np.array_equal(dA.cpu().numpy(), A, equal_nan=True)  # A is only read
    return [x.T.copy() for x in dX.cpu().numpy()]


def leaf_operator(seed, convection=False, h=1.0 / 256):
    """A_ii of one p = 16 leaf of the variable-speed Helmholtz problem
    (-Lap u - 80^2 (1 - 0.5 exp(-|x-c|^2/0.02)) u), optionally with a strong
    convection term, at a random position in the unit square."""
    p, q = 16, 14
    ops = O.LeafOps(p, q, h, h)
    t = np.cos(np.pi * np.arange(p) / (p - 1))[::-1]
    X, Y = np.meshgrid(t, t)
    x0, y0 = np.random.default_rng(seed).uniform(0.0, 1.0 - h, 2)
    xx, yy = x0 + h * (X + 1) / 2, y0 + h * (Y + 1) / 2
    co = {"c11": np.ones(p * p), "c22": np.ones(p * p),
          "c": (-6400.0 * (1 - 0.5 * np.exp(-((xx - 0.5) ** 2 + (yy - 0.5) ** 2) / 0.02))).ravel()}
    if convection:
        co["c1"] = (-1e3 * np.cos(4 * yy)).ravel()
        co["c2"] = (1e3 * np.sin(4 * xx)).ravel()
    A = ops.operator(co)
    return A[np.ix_(ops.Ji, ops.Ji)]


def check_inverse(A, X):
    A64 = A.astype(np.float32).astype(np.float64)
    X64 = X.astype(np.float64)
    R = A64 @ X64 - np.eye(N)
    S = np.abs(A64) @ np.abs(X64)
    assert np.all(np.abs(R) <= N * U * S), float(np.max(np.abs(R) / (N * U * S)))
    Xr = np.linalg.inv(A64)
    fwd = np.max(np.abs(X64 - Xr)) / np.max(np.abs(Xr))
    assert fwd <= N * U * np.linalg.cond(A64), fwd


def test_leaf_operators():
    mats = [leaf_operator(1), leaf_operator(2, convection=True), leaf_operator(3, h=1.0 / 64),
            leaf_operator(4, convection=True, h=1.0 / 16)]
    for A, X in zip(mats, gpu_inverse(mats)):
        check_inverse(A, X)


@pytest.mark.parametrize("cond", [1.0, 1e2, 1e4])
def test_random_matrices_of_given_condition(cond):
    rng = np.random.default_rng(int(np.log10(cond)) + 11)
    mats = []
    for _ in range(3):
        Q1, _ = np.linalg.qr(rng.standard_normal((N, N)))
        Q2, _ = np.linalg.qr(rng.standard_normal((N, N)))
        mats.append((Q1 * np.logspace(0, -np.log10(cond), N)) @ Q2.T)
    for A, X in zip(mats, gpu_inverse(mats)):
        check_inverse(A, X)


def test_pivoting_is_exact_on_permutations_and_zero_diagonals():
    """A permutation matrix (pivots of 1: every operation exact) inverts to its
    transpose bit for bit; so does a signed permutation with a zero diagonal,
    which the elimination can only take through row pivoting."""
    rng = np.random.default_rng(5)
    P = np.eye(N)[rng.permutation(N)]
    Z = np.zeros((N, N))
    for i in range(N):
        Z[i, (i + 1) % N] = (-1.0) ** i * 2.0
    X = gpu_inverse([P, Z])
    assert np.array_equal(X[0], P.T.astype(np.float32))
    assert np.array_equal(X[1], np.linalg.inv(Z).astype(np.float32))


def test_batch_equals_solo():
    mats = [leaf_operator(s, convection=bool(s % 2)) for s in range(6)]
    batch = gpu_inverse(mats)
    solo = gpu_inverse([mats[3]])[0]
    assert np.array_equal(batch[3], solo)


def test_singular_and_non_finite_matrices_are_reported():
    good = leaf_operator(7)
    zero_col = good.copy()
    zero_col[:, 40] = 0.0  # column 40 stays zero through the elimination
    nan = good.copy()
    nan[3, 9] = np.nan
    gpu_inverse([good, zero_col], expect=hps.HPS_ESINGULAR)
    assert "matrix 1" in hps.lib().hps_last_error().decode()
    gpu_inverse([nan, good], expect=hps.HPS_ESINGULAR)
    assert "matrix 0" in hps.lib().hps_last_error().decode()


def test_shape_limit():
    torch = pytest.importorskip("torch")
    a = torch.zeros(100 * 100, dtype=torch.float32, device="cuda")
    x = torch.zeros_like(a)
    assert hps.lib().hps_sinv_gj(100, 1, a.data_ptr(), x.data_ptr()) == hps.HPS_EINVAL
    assert b"n = 196" in hps.lib().hps_last_error()
    b = torch.zeros(2 * N * N + 4, dtype=torch.float32, device="cuda")
    assert hps.lib().hps_sinv_gj(N, 2, b.data_ptr(), b.data_ptr() + 4 * N * N) == hps.HPS_EINVAL
    assert b"overlap" in hps.lib().hps_last_error()
    y = torch.zeros(N * N, dtype=torch.float32, device="cuda")  # sized for one inverse
    assert hps.lib().hps_sinv_gj(N, 1, b.data_ptr() + 4, y.data_ptr()) == hps.HPS_EINVAL
    assert b"aligned" in hps.lib().hps_last_error()
