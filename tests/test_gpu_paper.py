"""The paper's own problems with known solutions (Section 9.1) at its order
p = 21 through the C ABI, in both precisions.

q = 19 (q = p leaves the composite system singular once the grid has interior
vertices).  Each solution is compared with the oracle's element by element
(1e-10 relative) and with the exact solution: E_pot, the largest error at the
Chebyshev nodes, and E_grad, the largest error of the boundary flux T^1 f
(hps_apply_dtn: d/dx on the vertical sides, d/dy on the horizontal ones), must
not exceed what Table 2 prints for the paper's own runs at its tightest
tolerance (tests/golden/table2_errors_eps1e-12.txt).
"""
from pathlib import Path

import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

UNIT = (0.0, 1.0, 0.0, 1.0)
GOLDEN = Path(__file__).resolve().parent / "golden"
P, Q = 21, 19

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def table2():
    out = {}
    for ln in (GOLDEN / "table2_errors_eps1e-12.txt").read_text().splitlines():
        if ln.strip() and not ln.startswith("#"):
            name, epot, egrad = ln.split()
            out[name] = (float(epot), float(egrad))
    return out


def known(problem):
    """(coefficient function, u, du/dx, du/dy) of Section 9.1's problem: the
    field of a source at (-2, 0), log r for Laplace, Y0(80 r) for Helmholtz I."""
    import scipy.special
    r = lambda x, y: np.hypot(x + 2.0, y)
    if problem == "laplace":
        return (I.laplace, lambda x, y: np.log(r(x, y)),
                lambda x, y: (x + 2.0) / r(x, y) ** 2, lambda x, y: y / r(x, y) ** 2)
    k = 80.0
    return (lambda x, y: I.constant_helmholtz(x, y, k),
            lambda x, y: scipy.special.y0(k * r(x, y)),
            lambda x, y: -k * scipy.special.y1(k * r(x, y)) * (x + 2.0) / r(x, y),
            lambda x, y: -k * scipy.special.y1(k * r(x, y)) * y / r(x, y))


def exact_flux(bxy, n, ux, uy):
    side = np.concatenate([np.full(n * Q, 0), np.full(n * Q, 1), np.full(n * Q, 2),
                           np.full(n * Q, 3)])
    return np.where((side == 0) | (side == 2), uy(bxy[:, 0], bxy[:, 1]),
                    ux(bxy[:, 0], bxy[:, 1]))


@pytest.mark.parametrize("problem,n", [("laplace", 4), ("helmholtz_I", 16)])
@pytest.mark.parametrize("precision", [hps.HPS_FP64, hps.HPS_MIXED])
def test_known_solution_at_p21(problem, n, precision):
    coef, u, ux, uy = known(problem)
    xy = hps.hps_cheb_nodes(UNIT, n, n, P)
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
          for k, v in coef(xy[..., 0], xy[..., 1]).items()}
    bxy = hps.hps_boundary_nodes_grid(UNIT, n, n, Q)
    f = np.ascontiguousarray(u(bxy[:, 0], bxy[:, 1])[None, :])
    h = hps.hps_build(UNIT, n, n, P, Q, co, precision=precision, form_root_dtn=True,
                      max_refine=30)
    info = hps.SolveInfo()
    w = hps.hps_solve(h, f, info=info)
    g = hps.hps_apply_dtn(h, f)
    h.close()
    assert info.status == hps.HPS_OK
    sol = O.solve_condensed(O.make_problem(UNIT, n, n, P, Q, coef), f.T)
    assert np.max(np.abs(w - sol.w)) / np.max(np.abs(sol.w)) < 1e-10
    epot_paper, egrad_paper = table2()[problem]
    e_pot = np.max(np.abs(w[0] - u(xy[..., 0], xy[..., 1])))
    assert e_pot <= epot_paper, (e_pot, epot_paper)
    if precision == hps.HPS_FP64:  # mixed mode applies its FP32-formed lower maps
        e_grad = np.max(np.abs(g[0] - exact_flux(bxy, n, ux, uy)))
        assert e_grad <= egrad_paper, (e_grad, egrad_paper)


def test_helmholtz_I_p21_on_64x64_leaves():
    """Helmholtz I on 64 x 64 leaves at p = 21 (1.8 M Chebyshev nodes, about
    51 wavelengths across the domain), beyond the oracle's reach here: both
    precisions meet Table 2's E_pot against the exact solution and agree to
    1e-10."""
    n = 64
    coef, u, _, _ = known("helmholtz_I")
    xy = hps.hps_cheb_nodes(UNIT, n, n, P)
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
          for k, v in coef(xy[..., 0], xy[..., 1]).items()}
    bxy = hps.hps_boundary_nodes_grid(UNIT, n, n, Q)
    f = np.ascontiguousarray(u(bxy[:, 0], bxy[:, 1])[None, :])
    sols = {}
    for prec in (hps.HPS_FP64, hps.HPS_MIXED):
        h = hps.hps_build(UNIT, n, n, P, Q, co, precision=prec, max_refine=30)
        info = hps.SolveInfo()
        sols[prec] = hps.hps_solve(h, f, info=info)
        h.close()
        assert info.status == hps.HPS_OK
    exact = u(xy[..., 0], xy[..., 1])
    epot_paper, _ = table2()["helmholtz_I"]
    for w in sols.values():
        assert np.max(np.abs(w[0] - exact)) <= epot_paper
    a, b = sols[hps.HPS_MIXED], sols[hps.HPS_FP64]
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-10
