"""The allocation-free solve entry point against the ordinary one.

hps_solve_static serves callers that cannot allocate device memory when they
solve (a fixed memory budget reserved up front, or no allocator or device
synchronisation allowed while other work runs): its scratch is a static device
array.  Two calls in a row must each return what hps_solve_ex returns for the
same handle and data.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300 import inputs as I
from paper_1307_2665_gb300.build import build

TOL = 1e-12

pytestmark = pytest.mark.gpu


def test_static_solve_matches_solve_twice():
    torch = pytest.importorskip("torch")
    build()
    dom, nx, ny, p, q = (0.0, 1.0, 0.0, 1.0), 8, 8, 16, 14
    xy = hps.hps_cheb_nodes(dom, nx, ny, p)
    co = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda())
          for k, v in I.convection_diffusion(xy[..., 0], xy[..., 1]).items()}
    h = hps.hps_build(dom, nx, ny, p, q, co, device_ptrs=True)
    bxy = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    outs = []
    for seed0 in (0, 7):  # two calls in a row, different data
        f = torch.from_numpy(np.ascontiguousarray(np.stack(
            [I.fourier_boundary(seed0 + s, bxy[:, 0], bxy[:, 1], dom) for s in range(4)]))).cuda()
        ref = torch.empty((4, nx * ny, p, p), dtype=torch.float64, device="cuda")
        hps.hps_solve(h, f, ref)
        got = torch.full_like(ref, float("nan"))
        assert hps.hps_solve_static(h, f, got) == hps.HPS_OK
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err <= TOL, err
        outs.append(got.clone())
    assert not torch.equal(outs[0], outs[1])
    # too large for the static array: rejected with a clear message
    big = torch.zeros((4000, hps.hps_boundary_count(nx, ny, q)), dtype=torch.float64, device="cuda")
    ub = torch.empty((1,), dtype=torch.float64, device="cuda")
    assert hps.hps_solve_static(h, big, ub, check=False) == hps.HPS_EINVAL
    assert b"static array" in hps.lib().hps_last_error()
    # the largest nrhs that fits (a size above it is refused before any device
    # work) still matches the ordinary solve
    lo, hi = 4, 4000
    while hi - lo > 1:
        mid = (lo + hi) // 2
        fm = torch.zeros((mid, hps.hps_boundary_count(nx, ny, q)), dtype=torch.float64,
                         device="cuda")
        um = torch.empty((mid, nx * ny, p, p), dtype=torch.float64, device="cuda")
        if hps.hps_solve_static(h, fm, um, check=False) == hps.HPS_OK:
            lo = mid
        else:
            assert b"static array" in hps.lib().hps_last_error()
            hi = mid
        del fm, um
    f = torch.from_numpy(np.ascontiguousarray(np.stack(
        [I.fourier_boundary(s % 20, bxy[:, 0], bxy[:, 1], dom) for s in range(lo)]))).cuda()
    ref = torch.empty((lo, nx * ny, p, p), dtype=torch.float64, device="cuda")
    hps.hps_solve(h, f, ref)
    got = torch.full_like(ref, float("nan"))
    assert hps.hps_solve_static(h, f, got) == hps.HPS_OK
    torch.cuda.synchronize()
    assert float((got - ref).abs().max() / ref.abs().max()) <= TOL
    h.close()
    # a mixed-precision handle is refused with a message
    hm = hps.hps_build(dom, nx, ny, p, q, co, device_ptrs=True, precision=hps.HPS_MIXED)
    assert hps.hps_solve_static(hm, f[:1].contiguous(), got[:1].contiguous(),
                                check=False) == hps.HPS_EINVAL
    assert b"only FP64 handles" in hps.lib().hps_last_error()
    hm.close()
