"""Mixed precision with iterative refinement (FP32 leaves and lower merges,
FP64 top merges, FP64 residual of the global collocation system) against the
FP64 oracle.  Tolerance: relative max error <= 1e-10 after refinement."""
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


def setup(dom, nx, ny, p, q, fn, seeds=(0, 1)):
    xy = hps.hps_cheb_nodes(dom, nx, ny, p)
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
          for k, v in fn(xy[..., 0], xy[..., 1]).items()}
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    f = np.ascontiguousarray(np.stack([I.exp_sin(bxy[:, 0], bxy[:, 1])] +
                                      [I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], dom) for s in seeds]))
    return co, f


def run(dom, nx, ny, p, q, co, f, **kw):
    h = hps.hps_build(dom, nx, ny, p, q, co, precision=hps.HPS_MIXED, **kw)
    info = hps.SolveInfo()
    u = hps.hps_solve(h, f, info=info, check=False)
    h.close()
    return u, info


@pytest.mark.parametrize("dom,nx,ny,p,q,fn", [
    (UNIT, 1, 1, 16, 14, I.laplace), (UNIT, 8, 8, 16, 14, I.laplace),
    (SKEW, 5, 3, 9, 8, varcoef), (SKEW, 3, 5, 12, 10, varcoef), (UNIT, 1, 7, 10, 8, varcoef),
    (UNIT, 16, 16, 16, 14, I.convection_diffusion), (UNIT, 2, 2, 24, 22, varcoef)])
def test_mixed_matches_oracle(dom, nx, ny, p, q, fn):
    co, f = setup(dom, nx, ny, p, q, fn)
    u, info = run(dom, nx, ny, p, q, co, f)
    assert info.status == hps.HPS_OK and 1 <= info.iterations <= 10
    # the last correction applied: at most refine_tol, or small enough that the
    # contraction of the last two predicts the next one below refine_tol
    assert info.last_update <= 1e-6
    sol = O.solve_condensed(O.make_problem(dom, nx, ny, p, q, fn), f.T)
    err = np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w))
    assert err < TOL, err


def test_all_float_merges_still_converge():
    """fp64_top_levels = 0: every merge in FP32; refinement still reaches the
    FP64 solution on a benign problem."""
    co, f = setup(UNIT, 8, 8, 12, 10, I.convection_diffusion)
    u, info = run(UNIT, 8, 8, 12, 10, co, f, fp64_top_levels=0)
    assert info.status == hps.HPS_OK
    h = hps.hps_build(UNIT, 8, 8, 12, 10, co)
    u64 = hps.hps_solve(h, f)
    h.close()
    assert np.max(np.abs(u - u64)) / np.max(np.abs(u64)) < TOL


def test_oscillatory_helmholtz_with_stated_tolerance():
    """-Lap u - 40^2 (1 - 0.5 bump) u = 0 on 16 x 16 leaves: the FP64 residual
    resolves about 1e-10 here, so the stated refinement tolerance is 1e-9."""
    fn = lambda x, y: I.gaussian_bump_helmholtz(x, y, 40.0)
    co, f = setup(UNIT, 16, 16, 16, 14, fn)
    u, info = run(UNIT, 16, 16, 16, 14, co, f, refine_tol=1e-9)
    assert info.status == hps.HPS_OK
    sol = O.solve_condensed(O.make_problem(UNIT, 16, 16, 16, 14, fn), f.T)
    assert np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w)) < 1e-9


def test_not_converged_is_reported():
    co, f = setup(UNIT, 4, 4, 12, 10, varcoef)
    u, info = run(UNIT, 4, 4, 12, 10, co, f, max_refine=1, refine_tol=1e-15)
    assert info.status == hps.HPS_ENOTCONVERGED and info.iterations == 1
    assert np.all(np.isfinite(u))


@pytest.mark.parametrize("depth", [0, 1, 3, 8])
def test_refinement_depths_match_oracle(depth):
    """Plain refinement (depth 0) and Anderson histories of 1, 3 and 8 all reach
    the FP64 solution."""
    co, f = setup(SKEW, 6, 4, 12, 10, varcoef)
    u, info = run(SKEW, 6, 4, 12, 10, co, f, refine_depth=depth)
    assert info.status == hps.HPS_OK, (info.iterations, info.last_update)
    sol = O.solve_condensed(O.make_problem(SKEW, 6, 4, 12, 10, varcoef), f.T)
    assert np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w)) < TOL


def test_acceleration_needs_fewer_corrections():
    """kappa = 80 on 32 x 32 leaves, leaf operators left uncorrected: the FP32
    factors leave a slowly decaying error mode; after the same number of
    corrections the accelerated iteration has removed more of it than plain
    refinement (a smaller last correction), and both reach the oracle."""
    co, f = setup(UNIT, 32, 32, 16, 14, I.gaussian_bump_helmholtz, seeds=(3,))
    _, j0 = run(UNIT, 32, 32, 16, 14, co, f, refine_depth=0, max_refine=3, leaf_refine=0,
                refine_tol=1e-30)
    _, j3 = run(UNIT, 32, 32, 16, 14, co, f, refine_depth=3, max_refine=3, leaf_refine=0,
                refine_tol=1e-30)
    assert j0.iterations == 3 and j3.iterations == 3
    assert j3.last_update < j0.last_update, (j3.last_update, j0.last_update)
    u0, i0 = run(UNIT, 32, 32, 16, 14, co, f, refine_depth=0, max_refine=30, leaf_refine=0)
    u3, i3 = run(UNIT, 32, 32, 16, 14, co, f, refine_depth=3, max_refine=30, leaf_refine=0)
    assert i0.status == hps.HPS_OK and i3.status == hps.HPS_OK
    sol = O.solve_condensed(O.make_problem(UNIT, 32, 32, 16, 14, I.gaussian_bump_helmholtz), f.T)
    for u in (u0, u3):
        assert np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w)) < TOL


@pytest.mark.parametrize("precision", [hps.HPS_FP64, hps.HPS_MIXED])
def test_each_rhs_is_independent_of_the_others(precision):
    """Every right-hand side is eliminated and refined on its own, so solving
    it alone or among others gives the same bits."""
    co, f = setup(SKEW, 5, 4, 12, 10, varcoef, seeds=(0, 1, 2))
    h = hps.hps_build(SKEW, 5, 4, 12, 10, co, precision=precision)
    together = hps.hps_solve(h, f)
    for r in range(f.shape[0]):
        alone = hps.hps_solve(h, np.ascontiguousarray(f[r:r + 1]))
        assert np.array_equal(alone[0], together[r]), r
    h.close()


def test_leaf_dtn_formed_from_the_corrected_operator():
    """One leaf of the 256 x 256 Helmholtz grid (h = 1/256, kappa = 80), its
    DtN map formed in mixed mode and applied to Fourier data.  Formed from the
    FP32 LU's Y, T carries cond(A_ii) units of FP32 rounding, amplified by the
    side derivatives; formed from Y + dY (one correction against the FP64
    residual of A_ii Y = -A_ie L1, Section 3.2, eq. leaf_solve) it carries
    little more than the FP32 rounding of T itself."""
    h0 = 1.0 / 256
    dom = (0.5, 0.5 + h0, 0.25, 0.25 + h0)
    p, q = 16, 14
    co, _ = setup(dom, 1, 1, p, q, I.gaussian_bump_helmholtz)
    bxy = hps.hps_boundary_nodes_grid(dom, 1, 1, q)
    f = np.ascontiguousarray(np.stack([I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], dom)
                                       for s in range(4)]))
    want = O.dtn_apply(O.make_problem(dom, 1, 1, p, q, I.gaussian_bump_helmholtz), f)
    err = {}
    for lr in (0, 1):
        h = hps.hps_build(dom, 1, 1, p, q, co, precision=hps.HPS_MIXED, form_root_dtn=True,
                          leaf_refine=lr)
        g = hps.hps_apply_dtn(h, f)
        h.close()
        err[lr] = np.max(np.abs(g - want)) / np.max(np.abs(want))
    assert err[1] < 3e-7, err
    assert err[1] < 0.35 * err[0], err


def test_leaf_correction_shrinks_the_first_correction():
    """kappa = 80 on 32 x 32 leaves.  With every merge in FP64, what is left of
    the low-precision solve's error (the first refinement correction) comes
    from the FP32 leaves; correcting each leaf's Y once before its DtN map is
    formed shrinks it more than tenfold.  With the default FP32 lower merges,
    no more corrections reach the tolerance and the result matches the
    oracle."""
    co, f = setup(UNIT, 32, 32, 16, 14, I.gaussian_bump_helmholtz, seeds=(3,))
    first, iters, us = {}, {}, {}
    for lr in (0, 1):
        _, i1 = run(UNIT, 32, 32, 16, 14, co, f, leaf_refine=lr, max_refine=1,
                    refine_tol=1e-30, fp64_top_levels=64)
        first[lr] = i1.last_update
        us[lr], info = run(UNIT, 32, 32, 16, 14, co, f, leaf_refine=lr, max_refine=30)
        assert info.status == hps.HPS_OK
        iters[lr] = info.iterations
    assert first[1] < 0.1 * first[0], first
    assert iters[1] <= iters[0], iters
    sol = O.solve_condensed(O.make_problem(UNIT, 32, 32, 16, 14, I.gaussian_bump_helmholtz), f.T)
    assert np.max(np.abs(us[1] - sol.w)) / np.max(np.abs(sol.w)) < TOL
