"""The serving loop (include/hps_serve.h): builds and coalesced solves from
concurrent requests give the same bits as each request served alone, memory
admission evicts idle operators, and a served solve matches the oracle."""
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


def problem(n, p, fn):
    xy = hps.hps_cheb_nodes(UNIT, n, n, p)
    co = {k: (None if v is None else np.ascontiguousarray(v, dtype=np.float64))
          for k, v in fn(xy[..., 0], xy[..., 1]).items()}
    return dict(domain=UNIT, nx=n, ny=n, p=p, q=p - 2, coeffs=co)


def data(pr, nrhs, seed):
    bxy = hps.hps_boundary_nodes_grid(UNIT, pr["nx"], pr["ny"], pr["q"])
    return np.ascontiguousarray(np.stack([I.fourier_boundary(seed + s, bxy[:, 0], bxy[:, 1], UNIT)
                                          for s in range(nrhs)]))


def test_mix_equals_alone_and_direct_handle():
    helm = lambda x, y: I.constant_helmholtz(x, y, 30.0)
    specs = [(problem(8, 16, I.laplace), hps.HPS_FP64), (problem(12, 12, helm), hps.HPS_MIXED),
             (problem(16, 16, I.convection_diffusion), hps.HPS_MIXED),
             (problem(6, 20, helm), hps.HPS_FP64)]
    srv = hps.Server(workers=3, max_rhs_per_solve=16)
    ops = [srv.submit_build(pr, precision=prec) for pr, prec in specs]
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(24):
        i = int(rng.integers(len(ops)))
        f = data(specs[i][0], int(rng.integers(1, 7)), 100 * k)
        reqs.append((srv.submit_solve(ops[i], f), i, f))
    for op in ops:
        assert srv.wait(op).status == hps.HPS_OK
    mixed_results = {}
    coalesced = 0
    for rid, i, f in reqs:
        info = srv.wait(rid)
        assert info.status == hps.HPS_OK
        coalesced += info.batch_rhs > info.nrhs
        mixed_results[rid] = srv.result(rid, ops[i], f.shape[0])
        srv.release(rid)
    assert coalesced > 0
    # the same requests one at a time
    for rid, i, f in reqs:
        r2 = srv.submit_solve(ops[i], f)
        info = srv.wait(r2)
        assert info.status == hps.HPS_OK and info.batch_rhs == f.shape[0]
        assert np.array_equal(srv.result(r2, ops[i], f.shape[0]), mixed_results[rid])
        srv.release(r2)
    st = srv.stats()
    assert st["completed"] == st["submitted"] == len(ops) + 2 * len(reqs) and st["failed"] == 0
    srv.close()
    # and through a handle built directly
    for rid, i, f in reqs[:6]:
        pr, prec = specs[i]
        h = hps.hps_build(UNIT, pr["nx"], pr["ny"], pr["p"], pr["q"], pr["coeffs"], precision=prec)
        assert np.array_equal(hps.hps_solve(h, f), mixed_results[rid])
        h.close()


def test_served_solve_matches_oracle():
    pr = problem(6, 12, I.convection_diffusion)
    f = data(pr, 3, 7)
    srv = hps.Server(workers=2)
    op = srv.submit_build(pr, precision=hps.HPS_MIXED)
    rid = srv.submit_solve(op, f)
    assert srv.wait(rid).status == hps.HPS_OK
    u = srv.result(rid, op, 3)
    srv.close()
    sol = O.solve_condensed(O.make_problem(UNIT, 6, 6, 12, 10, I.convection_diffusion), f.T)
    assert np.max(np.abs(u - sol.w)) / np.max(np.abs(sol.w)) < 1e-10


def test_admission_evicts_idle_operators():
    """A budget that holds one operator's build at a time: each new build
    evicts the idle one before it; a solve queued on an evicted operator
    completes with HPS_ENOMEM, one queued before the eviction runs."""
    prs = [problem(16, 16, I.laplace) for _ in range(3)]
    peak, res, work = hps.hps_estimate_bytes([prs[0]], nrhs=2)
    srv = hps.Server(hbm_budget=int(peak + res // 2), workers=2)
    a = srv.submit_build(prs[0])
    fa = data(prs[0], 2, 1)
    sa = srv.submit_solve(a, fa)            # queued before the next build
    assert srv.wait(sa).status == hps.HPS_OK
    srv.release(sa)
    b = srv.submit_build(prs[1])
    assert srv.wait(b).status == hps.HPS_OK
    late = srv.submit_solve(a, fa)          # a was evicted to admit b
    assert srv.wait(late).status == hps.HPS_ENOMEM
    st = srv.stats()
    assert st["evicted_ops"] >= 1 and st["peak_bytes_in_use"] <= st["budget"]
    srv.close()


def test_work_that_can_never_fit_is_refused():
    """A build whose estimated peak exceeds the budget is refused when it is
    submitted, and a solve too large to sit beside its own resident operator
    completes with HPS_ENOMEM; neither waits for memory that can never come,
    and the server keeps serving what fits."""
    pr = problem(8, 12, I.laplace)
    peak, res, work = hps.hps_estimate_bytes([pr], nrhs=1)
    srv = hps.Server(hbm_budget=int(peak // 2), workers=1)
    try:
        with pytest.raises(hps.HpsError) as e:
            srv.submit_build(pr)
        assert e.value.status == hps.HPS_ENOMEM
    finally:
        srv.close()
    budget = int(peak + res)  # room for the build, then for the operator and small solves
    srv = hps.Server(hbm_budget=budget, workers=1)
    try:
        a = srv.submit_build(pr)
        assert srv.wait(a).status == hps.HPS_OK
        dof = pr["nx"] * pr["ny"] * pr["p"] ** 2
        nbig = budget // (8 * dof) + 2  # its result alone exceeds the budget
        big = srv.submit_solve(a, data(pr, nbig, 0))
        assert srv.wait(big, timeout=60.0).status == hps.HPS_ENOMEM
        ok = srv.submit_solve(a, data(pr, 2, 0))
        assert srv.wait(ok, timeout=60.0).status == hps.HPS_OK
    finally:
        srv.close()
