"""Post-processing through the C ABI: the root DtN map applied to Dirichlet
data (hps_apply_dtn, the T_apply of Section 9.1) and the solution evaluated at
arbitrary points (hps_interpolate, Section 5.3), against the oracle.

Tolerances: T^1 f is compared with the oracle's boundary fluxes of its own
sparse-LU solution at 1e-10 of max|g| (the FP64 bar of the solver); point
values at 1e-13 of max|u| (the two sides evaluate the same interpolant in
different but stable forms, barycentric and product)."""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

UNIT = (0.0, 1.0, 0.0, 1.0)
SKEW = (-0.3, 0.9, 0.1, 1.7)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def varcoef(x, y):
    return {"c11": 1 + 0.3 * np.sin(x + 2 * y), "c12": 0.2 * np.cos(3 * x - y),
            "c22": 1.2 + 0.1 * x * y, "c1": 5 * np.cos(x), "c2": -4 * np.sin(2 * y),
            "c": 7 * np.exp(x * y)}


def coeffs(dom, nx, ny, p, fn):
    xy = hps.hps_cheb_nodes(dom, nx, ny, p)
    co = fn(xy[..., 0], xy[..., 1])
    return {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
            for k, v in co.items()}


def fourier_data(dom, nx, ny, q, nrhs, seed0=0):
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    return np.ascontiguousarray(np.stack(
        [I.fourier_boundary(seed0 + s, bxy[:, 0], bxy[:, 1], dom) for s in range(nrhs)]))


@pytest.mark.parametrize("nrhs", [1, 3, 9, 20])
def test_apply_dtn_matches_oracle(nrhs):
    """Variable coefficients on a skewed domain, 3 x 2 leaves: 1 to 20
    right-hand sides (one to three passes of the few-right-hand-side kernel)."""
    dom, nx, ny, p, q = SKEW, 3, 2, 12, 10
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, varcoef), form_root_dtn=True)
    f = fourier_data(dom, nx, ny, q, nrhs)
    g = hps.hps_apply_dtn(h, f)
    h.close()
    want = O.dtn_apply(O.make_problem(dom, nx, ny, p, q, varcoef), f)
    err = np.max(np.abs(g - want)) / np.max(np.abs(want))
    assert err < 1e-10, err


def test_apply_dtn_many_rhs_on_the_tensor_cores():
    """8 x 8 leaves (nbnd = 448) and 130 right-hand sides: the product is large
    enough for the tensor-core FP64 GEMM."""
    dom, nx, ny, p, q = UNIT, 8, 8, 16, 14
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, I.convection_diffusion),
                      form_root_dtn=True)
    f = fourier_data(dom, nx, ny, q, 130, seed0=40)
    g = hps.hps_apply_dtn(h, f)
    g1 = hps.hps_apply_dtn(h, np.ascontiguousarray(f[:7]))
    h.close()
    want = O.dtn_apply(O.make_problem(dom, nx, ny, p, q, I.convection_diffusion), f)
    err = np.max(np.abs(g - want)) / np.max(np.abs(want))
    assert err < 1e-10, err
    assert np.max(np.abs(g[:7] - g1)) / np.max(np.abs(g1)) < 1e-13


def test_apply_dtn_linear_solution_is_exact():
    """u = 2x - 3y + 1 (Laplace): the fluxes are 2 on vertical sides and -3 on
    horizontal ones, up to rounding."""
    dom, nx, ny, p, q = SKEW, 4, 3, 10, 8
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, I.laplace), form_root_dtn=True)
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    f = np.ascontiguousarray((2 * bxy[:, 0] - 3 * bxy[:, 1] + 1)[None, :])
    g = hps.hps_apply_dtn(h, f)[0]
    h.close()
    side = np.concatenate([np.full(nx * q, 0), np.full(ny * q, 1), np.full(nx * q, 2),
                           np.full(ny * q, 3)])
    want = np.where((side == 0) | (side == 2), -3.0, 2.0)
    assert np.max(np.abs(g - want)) < 1e-10


def test_apply_dtn_device_pointers_and_single_leaf():
    torch = pytest.importorskip("torch")
    dom, p, q = UNIT, 14, 12
    h = hps.hps_build(dom, 1, 1, p, q, coeffs(dom, 1, 1, p, varcoef), form_root_dtn=True)
    f = fourier_data(dom, 1, 1, q, 2)
    g = hps.hps_apply_dtn(h, f)
    fd = torch.from_numpy(f).cuda()
    gd = torch.empty_like(fd)
    hps.hps_apply_dtn(h, fd, gd, device_ptrs=True)
    h.close()
    assert np.array_equal(gd.cpu().numpy(), g)
    want = O.dtn_apply(O.make_problem(dom, 1, 1, p, q, varcoef), f)
    assert np.max(np.abs(g - want)) / np.max(np.abs(want)) < 1e-10


def test_apply_dtn_mixed_mode_uses_the_formed_map():
    """Mixed mode keeps T^1 as formed from the FP32 lower levels (no refinement):
    it agrees with the FP64 map to FP32 accuracy."""
    dom, nx, ny, p, q = UNIT, 4, 4, 12, 10
    co = coeffs(dom, nx, ny, p, varcoef)
    f = fourier_data(dom, nx, ny, q, 2)
    h = hps.hps_build(dom, nx, ny, p, q, co, form_root_dtn=True)
    g64 = hps.hps_apply_dtn(h, f)
    h.close()
    h = hps.hps_build(dom, nx, ny, p, q, co, form_root_dtn=True, precision=hps.HPS_MIXED)
    gmx = hps.hps_apply_dtn(h, f)
    h.close()
    err = np.max(np.abs(gmx - g64)) / np.max(np.abs(g64))
    assert 0 < err < 1e-3, err


def test_apply_dtn_needs_the_root_map_and_one_problem():
    dom, nx, ny, p, q = UNIT, 2, 2, 8, 6
    co = coeffs(dom, nx, ny, p, I.laplace)
    f = fourier_data(dom, nx, ny, q, 1)
    h = hps.hps_build(dom, nx, ny, p, q, co)
    _, st = hps.hps_apply_dtn(h, f, check=False)
    h.close()
    assert st == hps.HPS_EINVAL
    pr = {"domain": dom, "nx": nx, "ny": ny, "p": p, "q": q, "coeffs": co}
    bh = hps.hps_build_batch([pr, pr], form_root_dtn=True)
    _, st = hps.hps_apply_dtn(bh, f, check=False)
    bh.close()
    assert st == hps.HPS_EINVAL


def _points(dom, nx, ny, n, seed):
    x0, x1, y0, y1 = dom
    rng = np.random.default_rng(seed)
    pts = np.column_stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)])
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    edges = [[x0, y0], [x1, y1], [x0, y1], [x1, y0], [x0 + hx, y0 + hy],
             [x0 + hx, 0.37 * y0 + 0.63 * y1], [0.71 * x0 + 0.29 * x1, y0 + hy], [x1, 0.5 * (y0 + y1)]]
    return np.ascontiguousarray(np.vstack([pts, edges]))


def test_interpolate_matches_oracle():
    """Three solutions of a variable-coefficient problem at random points, leaf
    edges, leaf corners and the domain's corners."""
    dom, nx, ny, p, q = SKEW, 3, 2, 12, 10
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, varcoef))
    u = hps.hps_solve(h, fourier_data(dom, nx, ny, q, 3))
    pts = _points(dom, nx, ny, 300, 8)
    out = hps.hps_interpolate(h, u, pts)
    h.close()
    want = O.evaluate_points(O.make_problem(dom, nx, ny, p, q, varcoef), u, pts)
    assert np.max(np.abs(out - want)) < 1e-13 * np.max(np.abs(want))


def test_interpolate_recovers_the_exact_solution():
    """exp(x) sin(y) solves Laplace's equation: the solution evaluated anywhere
    matches it to spectral accuracy."""
    dom, nx, ny, p, q = UNIT, 4, 4, 16, 14
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, I.laplace))
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    u = hps.hps_solve(h, np.ascontiguousarray(I.exp_sin(bxy[:, 0], bxy[:, 1])[None, :]))
    pts = _points(dom, nx, ny, 500, 9)
    out = hps.hps_interpolate(h, u, pts)[0]
    h.close()
    want = I.exp_sin(pts[:, 0], pts[:, 1])
    assert np.max(np.abs(out - want)) / np.max(np.abs(want)) < 1e-11


def test_interpolate_edge_cases():
    torch = pytest.importorskip("torch")
    dom, nx, ny, p, q = UNIT, 2, 2, 8, 6
    h = hps.hps_build(dom, nx, ny, p, q, coeffs(dom, nx, ny, p, I.laplace))
    u = hps.hps_solve(h, fourier_data(dom, nx, ny, q, 1))
    # no points
    out = hps.hps_interpolate(h, u, np.zeros((0, 2)))
    assert out.shape == (1, 0)
    # a point outside: rejected before device work with host arrays
    bad = np.array([[0.5, 0.5], [1.0 + 1e-12, 0.5]])
    _, st = hps.hps_interpolate(h, u, bad, check=False)
    assert st == hps.HPS_EINVAL
    # with device arrays: NaN there, the other point evaluated, HPS_EINVAL
    ud = torch.from_numpy(u).cuda()
    xd = torch.from_numpy(bad).cuda()
    od = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    _, st = hps.hps_interpolate(h, ud, xd, od, device_ptrs=True, check=False)
    ref = hps.hps_interpolate(h, u, np.ascontiguousarray(bad[:1]))
    h.close()
    o = od.cpu().numpy()
    assert st == hps.HPS_EINVAL and np.isnan(o[0, 1]) and o[0, 0] == ref[0, 0]
