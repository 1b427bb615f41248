"""Batched build and solve of independent problems of uneven size and order p
(hps_build_batch / hps_solve_batch): each problem's result equals its solo run
bit for bit (the same arithmetic: per-leaf and per-merge work does not depend
on the other problems of a launch, and refinement runs per right-hand side),
and the batch matches the FP64 oracle in both modes."""
import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def uneven_batch(n_prob=6, seed=3, nmax=12):
    """Problems in the style of the uneven-batch workload: n log-uniform, p in
    {12, 16, 20}, q = p - 2, random smooth coefficient fields (small sizes so
    the oracle can check every problem)."""
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(n_prob):
        nx = int(round(np.exp(rng.uniform(np.log(2), np.log(nmax)))))
        ny = int(round(np.exp(rng.uniform(np.log(2), np.log(nmax)))))
        p = int(rng.choice([12, 16, 20]))
        dom = (0.0, 1.0, 0.0, 1.0)
        fn = lambda x, y, k=k: I.random_smooth_operator(seed * 100 + k, x, y)
        xy = hps.hps_cheb_nodes(dom, nx, ny, p)
        co = {n: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
              for n, v in fn(xy[..., 0], xy[..., 1]).items()}
        bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, p - 2)
        f = np.ascontiguousarray(np.stack([I.fourier_boundary(10 * k + s, bxy[:, 0], bxy[:, 1], dom)
                                           for s in range(3)]))
        probs.append(dict(domain=dom, nx=nx, ny=ny, p=p, q=p - 2, coeffs=co, fn=fn, f=f))
    return probs


@pytest.mark.parametrize("precision", [hps.HPS_FP64, hps.HPS_MIXED])
def test_batch_equals_solo_and_oracle(precision):
    probs = uneven_batch()
    bh = hps.hps_build_batch(probs, precision=precision)
    assert hps.lib().hps_batch_size(bh.ptr) == len(probs)
    us = [np.empty((3, pr["nx"] * pr["ny"], pr["p"], pr["p"])) for pr in probs]
    info = hps.SolveInfo()
    hps.hps_solve_batch(bh, [pr["f"] for pr in probs], us, info=info)
    assert info.status == hps.HPS_OK
    bh.close()
    for pr, u in zip(probs, us):
        h = hps.hps_build(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"], pr["coeffs"],
                          precision=precision)
        solo = hps.hps_solve(h, pr["f"])
        h.close()
        assert np.array_equal(u, solo), (pr["nx"], pr["ny"], pr["p"])
        sol = O.solve_condensed(O.make_problem(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"],
                                               pr["fn"]), pr["f"].T)
        err = np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w))
        assert err < 1e-10, (pr["nx"], pr["ny"], pr["p"], err)


def test_single_problem_batch_equals_build():
    pr = uneven_batch(n_prob=1, seed=5)[0]
    bh = hps.hps_build_batch([pr])
    u = np.empty((3, pr["nx"] * pr["ny"], pr["p"], pr["p"]))
    hps.hps_solve_batch(bh, [pr["f"]], [u])
    h = hps.hps_build(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"], pr["coeffs"])
    assert np.array_equal(hps.hps_solve(h, pr["f"]), u)
    h.close()
    bh.close()


def test_batch_rejects_single_solve_entry():
    probs = uneven_batch(n_prob=2, seed=7, nmax=4)
    bh = hps.hps_build_batch(probs)
    u = np.empty((3, probs[0]["nx"] * probs[0]["ny"], probs[0]["p"], probs[0]["p"]))
    st = hps.lib().hps_solve_ex(bh.ptr, probs[0]["f"].ctypes.data, 3, u.ctypes.data, 0, None)
    assert st == hps.HPS_EINVAL
    bh.close()


def test_tall_panels_agree_alone_and_batched():
    """A 40 x 40 problem with q = 13 has a 520-unknown top merge: solved alone,
    its tall panels are factored by a thread-block cluster; in a batch of 33
    copies (too many matrices for the cluster path) by one CTA each.  Same
    pivots and FMAs: the solutions agree bit for bit."""
    dom, n, p, q = (0.0, 1.0, 0.0, 1.0), 40, 15, 13
    xy = hps.hps_cheb_nodes(dom, n, n, p)
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
          for k, v in I.random_smooth_operator(3, xy[..., 0], xy[..., 1]).items()}
    bxy = hps.hps_boundary_nodes_grid(dom, n, n, q)
    f = np.ascontiguousarray(np.stack([I.fourier_boundary(s, bxy[:, 0], bxy[:, 1], dom)
                                       for s in range(2)]))
    h = hps.hps_build(dom, n, n, p, q, co)
    u1 = hps.hps_solve(h, f)
    h.close()
    pr = {"domain": dom, "nx": n, "ny": n, "p": p, "q": q, "coeffs": co}
    bh = hps.hps_build_batch([pr] * 33)
    us = [np.empty((2, n * n, p, p)) for _ in range(33)]
    hps.hps_solve_batch(bh, [f] * 33, us)
    bh.close()
    assert np.array_equal(u1, us[0]) and np.array_equal(u1, us[32])
