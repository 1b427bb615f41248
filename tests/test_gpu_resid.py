"""The mixed mode's FP64 residual kernels on raw leaves (hps_leaf_residual)
against the oracle's leaf operator A (Section 3.1) and flux map L4 L3
(Section 3.2, Steps 3-4), both evaluated in extended precision: r = -(A w) at
the interior Chebyshev nodes and the side fluxes at the Gauss points, for the
tensor-core kernel (exact BF16 digit products) and the FP64-pipe kernel (even
and odd parts).

Bounds per output, against the sum of the absolute terms |A||w| (or |F||w|):
the oracle builds D its own way (V' V^-1), so kernel and oracle may differ by
the rounding of the tables, 1e-13 of that sum; the two kernels apply the same
tables, so they agree to 2^-46 of it (64 roundings).  A wrong digit, table
row, sign or index is off by O(1) of the sum."""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def gpu_residual(p, q, hx, hy, co, w, tc):
    torch = pytest.importorskip("torch")
    nrhs, nl = w.shape[:2]
    ni = (p - 2) ** 2

    def dev(a):
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()

    dc = {k: dev(co.get(k)) for k in ("c11", "c22", "c")}
    dw = dev(w)
    r = torch.full((nl, nrhs, ni), -7.0, dtype=torch.float64, device="cuda")
    fl = torch.full((nrhs, nl, 4 * q), -7.0, dtype=torch.float64, device="cuda")
    ptr = {k: (None if v is None else v.data_ptr()) for k, v in dc.items()}
    st = hps.lib().hps_leaf_residual(p, q, nl, hx, hy, ptr["c11"], ptr["c22"], ptr["c"],
                                     dw.data_ptr(), nrhs, r.data_ptr(), fl.data_ptr(), tc)
    assert st == hps.HPS_OK, hps.lib().hps_last_error()
    return r.cpu().numpy(), fl.cpu().numpy()


def reference(p, q, hx, hy, co, w):
    """-(A w) at the interior nodes and L4 L3 w, with the sums of |terms|."""
    ops = O.LeafOps(p, q, hx, hy)
    nrhs, nl = w.shape[:2]
    ni = (p - 2) ** 2
    r, rs = np.zeros((nl, nrhs, ni)), np.zeros((nl, nrhs, ni))
    fl, fs = np.zeros((nrhs, nl, 4 * q)), np.zeros((nrhs, nl, 4 * q))
    FL = ops.F.astype(np.longdouble)
    for l in range(nl):
        A = ops.operator({k: (None if co.get(k) is None else co[k][l]) for k in O.COEFF_NAMES})
        AL = A[ops.Ji].astype(np.longdouble)
        WL = w[:, l].reshape(nrhs, p * p).T.astype(np.longdouble)
        r[l] = (-(AL @ WL)).T.astype(np.float64)
        rs[l] = (np.abs(AL) @ np.abs(WL)).T.astype(np.float64)
        fl[:, l] = (FL @ WL).T.astype(np.float64)
        fs[:, l] = (np.abs(FL) @ np.abs(WL)).T.astype(np.float64)
    return r, rs, fl, fs


def leaves(p, nl, nrhs, seed, hx=1 / 64, hy=1 / 48, terms=("c11", "c22", "c")):
    """Smooth positive diffusion, a signed zeroth-order field, and grids that
    mix smooth fields with noise over scales 1e-8 .. 1e8."""
    rng = np.random.default_rng(seed)
    t = np.cos(np.pi * np.arange(p) / (p - 1))[::-1]
    X, Y = np.meshgrid(t, t)
    co = {}
    for k in terms:
        f = np.stack([(1.5 + 0.5 * np.sin(3 * X + l) * np.cos(2 * Y - l)) if k != "c" else
                      -6400.0 * (1 - 0.5 * np.exp(-(X - 0.3 * l) ** 2 - Y ** 2)) for l in range(nl)])
        co[k] = f.reshape(nl, p * p)
    w = np.empty((nrhs, nl, p, p))
    for k in range(nrhs):
        for l in range(nl):
            smooth = np.sin(2.1 * X + 0.7 * k + l) * np.cosh(0.9 * Y) + 0.3 * X * Y
            scale = 10.0 ** rng.uniform(-8, 8)
            w[k, l] = scale * (smooth + 10.0 ** rng.uniform(-12, 0) * rng.standard_normal((p, p)))
    return co, w.reshape(nrhs, nl, p * p), hx, hy


@pytest.mark.parametrize("nrhs", [1, 8, 13, 40])
def test_residual_and_fluxes_vs_oracle(nrhs):
    p, q, nl = 16, 14, 5
    co, w, hx, hy = leaves(p, nl, nrhs, seed=nrhs)
    r0, rs, f0, fs = reference(p, q, hx, hy, co, w)
    out = {}
    for tc in (1, 0):
        r, fl = gpu_residual(p, q, hx, hy, co, w, tc)
        assert np.all(np.abs(r - r0) <= 1e-13 * rs), (tc, np.max(np.abs(r - r0) / rs))
        assert np.all(np.abs(fl - f0) <= 1e-13 * fs), (tc, np.max(np.abs(fl - f0) / fs))
        out[tc] = (r, fl)
    # the two kernels apply the same tables: they differ by their own
    # rounding (an FP64 chain of about 16 operations in the even/odd kernel)
    dr = np.max(np.abs(out[1][0] - out[0][0]) / rs)
    df = np.max(np.abs(out[1][1] - out[0][1]) / fs)
    assert dr <= 2.0 ** -46 and df <= 2.0 ** -46, (dr, df)


@pytest.mark.parametrize("terms,q", [(("c11", "c22"), 14), (("c",), 14), (("c11", "c22", "c"), 16),
                                     (("c11", "c22", "c"), 1), (("c11", "c22", "c"), 9)])
def test_partial_operators_and_gauss_counts(terms, q):
    p, nl, nrhs = 16, 3, 9
    co, w, hx, hy = leaves(p, nl, nrhs, seed=len(terms) + q, terms=terms)
    r0, rs, f0, fs = reference(p, q, hx, hy, co, w)
    r, fl = gpu_residual(p, q, hx, hy, co, w, 1)
    floor = 1e-300  # c alone: r = c w exactly where w is, zero sums elsewhere
    assert np.all(np.abs(r - r0) <= 1e-13 * rs + floor)
    assert np.all(np.abs(fl - f0) <= 1e-13 * fs + floor)


def test_zero_nan_and_extreme_grids():
    """A zero grid gives zeros; a grid holding a NaN gives NaN at all of its
    outputs and leaves the other grids alone; grids near 1e-250 and 1e+250
    keep their accuracy (the digits are relative to each grid's exponent)."""
    p, q, nl, nrhs = 16, 14, 2, 12
    co, w, hx, hy = leaves(p, nl, nrhs, seed=3)
    w = w.reshape(nrhs, nl, p * p)
    w[0, 0] = 0.0
    w[1, 1, 17] = np.nan
    w[2, 0] *= 1e-250 / np.max(np.abs(w[2, 0]))
    w[3, 1] *= 1e250 / np.max(np.abs(w[3, 1]))
    r, fl = gpu_residual(p, q, hx, hy, co, w, 1)
    assert np.all(r[0, 0] == 0.0) and np.all(fl[0, 0] == 0.0)
    assert np.all(np.isnan(r[1, 1])) and np.all(np.isnan(fl[1, 1]))
    good = np.ones((nrhs, nl), dtype=bool)
    good[1, 1] = False
    wg = np.where(good[..., None], w, 0.0)
    r0, rs, f0, fs = reference(p, q, hx, hy, co, wg)
    rg, fg = r.transpose(1, 0, 2)[good], fl[good]
    assert np.all(np.isfinite(rg)) and np.all(np.isfinite(fg))
    assert np.all(np.abs(rg - r0.transpose(1, 0, 2)[good]) <= 1e-13 * rs.transpose(1, 0, 2)[good])
    assert np.all(np.abs(fg - f0[good]) <= 1e-13 * fs[good])


def test_tensor_core_kernel_shape_limits():
    torch = pytest.importorskip("torch")
    p, q = 12, 10
    w = torch.zeros(p * p, dtype=torch.float64, device="cuda")
    r = torch.zeros((p - 2) ** 2, dtype=torch.float64, device="cuda")
    fl = torch.zeros(4 * q, dtype=torch.float64, device="cuda")
    st = hps.lib().hps_leaf_residual(p, q, 1, 0.1, 0.1, None, None, None, w.data_ptr(), 1,
                                     r.data_ptr(), fl.data_ptr(), 1)
    assert st == hps.HPS_EINVAL
    # the FP64-pipe kernel takes any order
    st = hps.lib().hps_leaf_residual(p, q, 1, 0.1, 0.1, None, None, None, w.data_ptr(), 1,
                                     r.data_ptr(), fl.data_ptr(), 0)
    assert st == hps.HPS_OK
