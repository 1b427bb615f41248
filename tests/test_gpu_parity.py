"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative max error <= 1e-10 over all output nodes (the FP64 bar);
the Laplace ladder is also held to 1e-11, since the merges are exact in exact
arithmetic (Remark 5.1) and only rounding, amplified by the
conditioning of the DtN maps for oscillatory boundary data, separates the two
eliminations.
"""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

UNIT = (0.0, 1.0, 0.0, 1.0)
SKEW = (-0.3, 0.9, 0.1, 1.7)
TOL = 1e-10

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def varcoef(x, y):
    return {"c11": 1 + 0.3 * np.sin(x + 2 * y), "c12": 0.2 * np.cos(3 * x - y),
            "c22": 1.2 + 0.1 * x * y, "c1": 5 * np.cos(x), "c2": -4 * np.sin(2 * y),
            "c": 7 * np.exp(x * y)}


def gpu_coeffs(dom, nx, ny, p, fn):
    xy = hps.hps_cheb_nodes(dom, nx, ny, p)
    co = fn(xy[..., 0], xy[..., 1])
    return {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
            for k, v in co.items()}


def boundary_data(dom, nx, ny, q, seeds=(0, 1), with_exp=True):
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    rows = [I.exp_sin(bxy[:, 0], bxy[:, 1])] if with_exp else []
    rows += [I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], dom) for s in seeds]
    return np.ascontiguousarray(np.stack(rows))


def compare(dom, nx, ny, p, q, fn, f, solver="global"):
    h = hps.hps_build(dom, nx, ny, p, q, gpu_coeffs(dom, nx, ny, p, fn))
    u = hps.hps_solve(h, f)
    h.close()
    prob = O.make_problem(dom, nx, ny, p, q, fn)
    if solver == "global":
        sol, _, _ = O.solve_global(prob, f.T)
    else:
        sol = O.solve_condensed(prob, f.T)
    err = np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w))
    return err, u, sol


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (1, 2), (2, 2), (4, 4), (8, 8)])
def test_laplace_ladder(nx, ny):
    """One leaf (leaf kernels only), one and two merge levels, up to 8 x 8."""
    f = boundary_data(UNIT, nx, ny, 14)
    err, _, _ = compare(UNIT, nx, ny, 16, 14, I.laplace, f)
    assert err < 1e-11, err


@pytest.mark.parametrize("nx,ny,p,q", [(3, 5, 12, 10), (5, 3, 12, 10), (7, 1, 10, 8),
                                       (1, 6, 10, 8), (5, 3, 9, 8), (2, 3, 6, 3), (7, 1, 8, 8),
                                       (1, 5, 9, 9)])
def test_variable_coefficients_uneven_trees(nx, ny, p, q):
    """All six coefficients of eq. defA on a skewed domain, trees from
    non-power-of-two grids (splits at floor(n/2)), q < p, and q = p on strips
    (no interior vertex, so the system stays nonsingular)."""
    f = boundary_data(SKEW, nx, ny, q)
    err, _, _ = compare(SKEW, nx, ny, p, q, varcoef, f)
    assert err < TOL, err


def test_large_leaf_unstaged_panels():
    """p = 24: the 484 x 484 leaf matrices exceed the shared-memory panel
    budget, so the panel factorisation runs on global memory."""
    f = boundary_data(UNIT, 2, 2, 22)
    err, _, _ = compare(UNIT, 2, 2, 24, 22, varcoef, f)
    assert err < TOL, err


def test_config_8x8_laplace_exact_solution():
    """8 x 8 leaves, p = 16, q = 14, Laplace, f = exp(x) sin(y), 1 RHS: parity
    with the oracle and agreement with the exact solution."""
    bxy = hps.hps_boundary_nodes_grid(UNIT, 8, 8, 14)
    f = np.ascontiguousarray(I.exp_sin(bxy[:, 0], bxy[:, 1])[None, :])
    err, u, _ = compare(UNIT, 8, 8, 16, 14, I.laplace, f)
    assert err < 1e-12, err
    xy = hps.hps_cheb_nodes(UNIT, 8, 8, 16)
    ex = I.exp_sin(xy[..., 0], xy[..., 1])
    assert np.max(np.abs(u[0] - ex)) / np.max(np.abs(ex)) < 1e-12


def test_config_64x64_convection_diffusion_16rhs():
    """The benchmarked workload at full size: 64 x 64 leaves, p = 16, q = 14,
    c1 = -100 cos(4 pi y), c2 = 100 sin(4 pi x), 16 Fourier right-hand sides
    (seeds 0..15), against the oracle's condensed solve of the same system."""
    f = boundary_data(UNIT, 64, 64, 14, seeds=range(16), with_exp=False)
    err, _, _ = compare(UNIT, 64, 64, 16, 14, I.convection_diffusion, f, solver="condensed")
    assert err < TOL, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_level_lu_ragged_blocks(precision):
    """40 x 40 leaves with q = 13: the top merge's interface system has
    m = 520 = 2 * 256 + 8 unknowns, so the two-level LU runs two full outer
    blocks (the first trailing update on the tensor cores) and a ragged one of
    8 rows whose updates fall back to FP64 FMAs; the levels below keep the
    one-level LU."""
    n, p, q = 40, 15, 13
    f = boundary_data(UNIT, n, n, q, seeds=(3, 4), with_exp=True)
    prec = hps.HPS_MIXED if precision == "mixed" else hps.HPS_FP64
    h = hps.hps_build(UNIT, n, n, p, q, gpu_coeffs(UNIT, n, n, p, varcoef), precision=prec)
    u = hps.hps_solve(h, f)
    h.close()
    sol = O.solve_condensed(O.make_problem(UNIT, n, n, p, q, varcoef), f.T)
    err = np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w))
    assert err < TOL, err


def test_device_pointers_match_host_pointers():
    torch = pytest.importorskip("torch")
    dom, nx, ny, p, q = SKEW, 3, 4, 12, 10
    co = gpu_coeffs(dom, nx, ny, p, varcoef)
    f = boundary_data(dom, nx, ny, q)
    h = hps.hps_build(dom, nx, ny, p, q, co)
    u_host = hps.hps_solve(h, f)
    h.close()
    dco = {k: (None if v is None else torch.from_numpy(v).cuda()) for k, v in co.items()}
    hd = hps.hps_build(dom, nx, ny, p, q, dco, device_ptrs=True)
    fd = torch.from_numpy(f).cuda()
    ud = torch.empty((f.shape[0], nx * ny, p, p), dtype=torch.float64, device="cuda")
    hps.hps_solve(hd, fd, ud)
    torch.cuda.synchronize()
    hd.close()
    assert np.array_equal(ud.cpu().numpy(), u_host)


def test_multi_rhs_equals_single_solves():
    dom, nx, ny, p, q = UNIT, 4, 3, 12, 10
    h = hps.hps_build(dom, nx, ny, p, q, gpu_coeffs(dom, nx, ny, p, varcoef))
    f = boundary_data(dom, nx, ny, q, seeds=(0, 1, 2, 3))
    u = hps.hps_solve(h, f)
    for r in range(f.shape[0]):
        ur = hps.hps_solve(h, np.ascontiguousarray(f[r:r + 1]))
        assert np.array_equal(ur[0], u[r])
    again = hps.hps_solve(h, f)
    assert np.array_equal(again, u)
    h.close()


def test_root_dtn_option_does_not_change_solution():
    dom, nx, ny, p, q = UNIT, 4, 2, 10, 8
    co = gpu_coeffs(dom, nx, ny, p, varcoef)
    f = boundary_data(dom, nx, ny, q)
    a = hps.hps_build(dom, nx, ny, p, q, co)
    b = hps.hps_build(dom, nx, ny, p, q, co, form_root_dtn=True)
    assert np.array_equal(hps.hps_solve(a, f), hps.hps_solve(b, f))
    a.close()
    b.close()


def test_singular_leaf_reported():
    """A zero operator makes every leaf's A_ii singular: the build reports
    HPS_ESINGULAR instead of returning numbers."""
    zero = {"c11": np.zeros(4 * 64), "c22": np.zeros(4 * 64)}
    st = hps.hps_build(UNIT, 2, 2, 8, 6, zero, check=False)
    assert st == hps.HPS_ESINGULAR
    # the context is still usable afterwards
    f = boundary_data(UNIT, 2, 2, 6)
    err, _, _ = compare(UNIT, 2, 2, 8, 6, I.laplace, f)
    assert err < 1e-11
