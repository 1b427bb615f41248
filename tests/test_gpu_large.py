"""Full-size checks of the variable-speed Helmholtz workload (kappa = 80,
256 x 256 leaves, p = 16, q = 14: 16.8 M collocation nodes), where the oracle
cannot solve the whole system:

  * the same coefficient field on 32 x 32 and 64 x 64 leaves against the
    oracle's solve, in both precisions (element by element, 1e-10 relative);
  * at full size, both precisions against the oracle's leaf-local FP64
    residual of (E1, E2), the continuity of shared sides and the Dirichlet
    data, on sampled leaves, and mixed precision against FP64.

This problem is close to resonance (the solution is about 30 times larger
than its data) and its conditioning grows about 4.5 times per doubling of the
leaf count.  Rounding-level changes of the differentiation matrices alone
(correctly rounded D and D^2 against other exact-in-exact-arithmetic
constructions) move the oracle's own solution by 1e-11 relative at 32 x 32
leaves, so two FP64 solves of the 256 x 256 system, both with residuals at
rounding level, differ by a few 1e-10: mixed against FP64 is held to 5e-10
there, and the residual check carries the full-size evidence.
"""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

UNIT = (0.0, 1.0, 0.0, 1.0)
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def coeffs(dom, n, p, fn):
    xy = hps.hps_cheb_nodes(dom, n, n, p)
    co = fn(xy[..., 0], xy[..., 1])
    return {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
            for k, v in co.items()}


def fourier(dom, n, q, nrhs, seed0=0):
    bxy = hps.hps_boundary_nodes_grid(dom, n, n, q)
    return np.ascontiguousarray(np.stack([I.fourier_boundary(seed0 + s, bxy[:, 0], bxy[:, 1], dom)
                                          for s in range(nrhs)]))


@pytest.mark.parametrize("n", [32, 64])
def test_helmholtz_field_vs_oracle(n):
    p, q = 16, 14
    f = fourier(UNIT, n, q, 3)
    co = coeffs(UNIT, n, p, I.gaussian_bump_helmholtz)
    sol = O.solve_condensed(O.make_problem(UNIT, n, n, p, q, I.gaussian_bump_helmholtz), f.T)
    for prec in (hps.HPS_FP64, hps.HPS_MIXED):
        h = hps.hps_build(UNIT, n, n, p, q, co, precision=prec, max_refine=30)
        info = hps.SolveInfo()
        u = hps.hps_solve(h, f, info=info)
        h.close()
        err = np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w))
        assert err < 1e-10, (prec, err, info.iterations, info.last_update)


def test_helmholtz_256_full_size():
    n, p, q, nrhs = 256, 16, 14, 4
    co = coeffs(UNIT, n, p, I.gaussian_bump_helmholtz)
    f = fourier(UNIT, n, q, nrhs, seed0=7)
    h = hps.hps_build(UNIT, n, n, p, q, co)
    u64 = hps.hps_solve(h, f)
    h.close()
    h = hps.hps_build(UNIT, n, n, p, q, co, precision=hps.HPS_MIXED, max_refine=30)
    info = hps.SolveInfo()
    umx = hps.hps_solve(h, f, info=info, check=False)
    h.close()
    del co
    assert info.status == hps.HPS_OK
    rel = np.max(np.abs(umx - u64)) / np.max(np.abs(u64))
    prob = O.make_problem(UNIT, n, n, p, q, I.gaussian_bump_helmholtz)
    rng = np.random.default_rng(11)
    leaves = sorted(set(rng.choice(n * n, 40, replace=False).tolist()) |
                    {0, n - 1, n * (n - 1), n * n - 1, n * (n // 2) + n // 2 - 1})
    res = {name: O.sampled_residual(prob, u, f, leaves) for name, u in (("fp64", u64), ("mixed", umx))}
    msg = (rel, info.iterations, info.last_update, res)
    assert rel < 5e-10, msg
    for r in res.values():
        assert r["e1"] < 1e-14 and r["e2"] < 1e-14, msg
        assert r["cont"] < 1e-13 and r["gamma"] < 1e-13, msg
