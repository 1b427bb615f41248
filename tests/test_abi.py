"""The C-ABI library: it builds, loads, exports every symbol the headers in
include/ declare, and its host-only entry points (node coordinates, options, status
text, argument validation) behave as documented.  No GPU needed."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from oracle import hps_oracle as O
from paper_1307_2665_gb300 import hps
from paper_1307_2665_gb300.build import build

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _declared():
    names = set()
    for hdr in sorted((ROOT / "include").glob("*.h")):
        txt = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(hps_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 10
    L = ctypes.CDLL(str(ROOT / "paper_1307_2665_gb300" / "_lib" / "libhps.so"))
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hps.EXPORTS)


@pytest.mark.parametrize("dom,nx,ny,p,q", [((0, 1, 0, 1), 3, 2, 16, 14),
                                           ((-0.3, 0.9, 0.1, 1.7), 4, 7, 9, 9),
                                           ((2.0, 2.5, -1.0, 3.0), 1, 1, 5, 2)])
def test_node_coordinates_match_oracle(dom, nx, ny, p, q):
    """hps_cheb_nodes / hps_boundary_nodes_grid give the nodes the oracle uses
    (Chebyshev extreme points per leaf, Gauss-Legendre points on Gamma in
    counter-clockwise order) to rounding."""
    a = hps.hps_cheb_nodes(dom, nx, ny, p)
    b = O.cheb_grid(dom, nx, ny, p)
    assert np.max(np.abs(a - b)) < 1e-14 * max(1.0, np.max(np.abs(b)))
    ga = hps.hps_boundary_nodes_grid(dom, nx, ny, q)
    gb = O.boundary_points(O.Problem(dom, nx, ny, p, q, {}))
    assert ga.shape == gb.shape == (hps.hps_boundary_count(nx, ny, q), 2)
    assert np.max(np.abs(ga - gb)) < 1e-14 * max(1.0, np.max(np.abs(gb)))


def test_default_options_and_status_strings():
    o = hps.default_options()
    assert o.precision == hps.HPS_FP64 and o.device_ptrs == 0 and o.max_refine == 10
    assert abs(o.refine_tol - 1e-11) < 1e-20 and o.fp64_top_levels == 2
    L = hps.lib()
    for st in (0, -1, -2, -3, -4, -5):
        assert len(L.hps_status_string(st)) > 0
    assert L.hps_status_string(123) == b"unknown status"


@pytest.mark.parametrize("args", [
    dict(nx=0, ny=2, p=16, q=14), dict(nx=2, ny=2, p=2, q=1), dict(nx=2, ny=2, p=8, q=9),
    dict(nx=2, ny=2, p=8, q=0), dict(nx=2, ny=-1, p=8, q=4), dict(nx=2, ny=2, p=8, q=8)])
def test_build_rejects_bad_sizes_before_device_work(args):
    """Validation happens before any device work, so it runs without a GPU."""
    st = hps.hps_build((0, 1, 0, 1), args["nx"], args["ny"], args["p"], args["q"], {}, check=False)
    assert st == hps.HPS_EINVAL


def test_build_rejects_degenerate_domain():
    assert hps.hps_build((1, 1, 0, 1), 2, 2, 8, 6, {}, check=False) == hps.HPS_EINVAL
    assert hps.hps_build((0, 1, 0, float("nan")), 2, 2, 8, 6, {}, check=False) == hps.HPS_EINVAL


def test_null_pointer_arguments():
    L = hps.lib()
    assert L.hps_free(None) == hps.HPS_OK
    assert L.hps_solve(None, None, 1, None, None) == hps.HPS_EINVAL
    assert L.hps_cheb_nodes(hps.Domain(0, 1, 0, 1), 2, 2, 8, None) == hps.HPS_EINVAL
    assert L.hps_apply_dtn(None, None, 1, None, 0) == hps.HPS_EINVAL
    assert L.hps_interpolate(None, None, 1, None, 5, None, 0) == hps.HPS_EINVAL


def test_estimate_bytes_host_only():
    """hps_estimate_bytes works from the plan alone: the build peak covers the
    resident operator, the resident FP64 operator holds at least Y and S, and
    the solve workspace grows linearly with the number of right-hand sides."""
    pr = dict(domain=(0, 1, 0, 1), nx=16, ny=16, p=16, q=14, coeffs={})
    peak, res, w1 = hps.hps_estimate_bytes([pr], nrhs=1)
    _, _, w2 = hps.hps_estimate_bytes([pr], nrhs=2)
    _, _, w3 = hps.hps_estimate_bytes([pr], nrhs=3)
    y = 256 * 196 * 56 * 8
    assert res > y and peak >= res and w1 > 0
    assert w3 - w2 == w2 - w1
    peak_m, res_m, wm = hps.hps_estimate_bytes([pr], nrhs=1, precision=hps.HPS_MIXED)
    assert wm > w1  # refinement vectors
    with pytest.raises(hps.HpsError):
        hps.hps_estimate_bytes([dict(pr, q=17)])


def _s_entries(nx, ny, q):
    """Entries of S summed over the merges of an nx x ny leaf grid: the tree
    splits a box's longer side at floor(n/2) (ties: x), and a merge's S is
    m x n_e with m the shared edge's Gauss nodes and n_e the parent's exterior."""
    if nx == 1 and ny == 1:
        return 0
    if nx >= ny:
        m, kids = ny * q, [(nx // 2, ny), (nx - nx // 2, ny)]
    else:
        m, kids = nx * q, [(nx, ny // 2), (nx, ny - ny // 2)]
    return m * 2 * (nx + ny) * q + sum(_s_entries(x, y, q) for x, y in kids)


@pytest.mark.parametrize("nx,ny,p,q", [(64, 64, 16, 14), (7, 3, 12, 10), (1, 5, 8, 6)])
def test_resident_estimate_is_s_plus_y(nx, ny, p, q):
    """An FP64 handle keeps S of every merge (eq. U_parent) and Y of every leaf
    (eq. leaf_solve, (p-2)^2 x 4q), plus index maps of a few percent at most:
    the plan's estimate agrees with a count made here from the tree alone."""
    pr = dict(domain=(0, 1, 0, 1), nx=nx, ny=ny, p=p, q=q, coeffs={})
    _, res, _ = hps.hps_estimate_bytes([pr], nrhs=1)
    sy = 8 * (_s_entries(nx, ny, q) + nx * ny * (p - 2) ** 2 * 4 * q)
    assert sy <= res <= 1.02 * sy + 65536, (res, sy)


def test_server_without_device_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(hps.HpsError) as e:
        hps.Server()
    assert e.value.status == hps.HPS_EDEVICE


def _declarations():
    """(return type, name, parameter count) of every function the headers declare."""
    out = []
    for hdr in sorted((ROOT / "include").glob("*.h")):
        txt = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        for ret, name, params in re.findall(
                r"^\s*((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**)\s*(hps_[a-z_]+)\s*\(([^)]*)\)\s*;",
                txt, flags=re.M):
            params = " ".join(params.split())
            n = 0 if params in ("", "void") else params.count(",") + 1
            out.append((" ".join(ret.split()), name, n))
    return out


def test_binding_types_match_the_headers():
    """Every ctypes prototype of the binding has the header's return type
    (an int64_t result left at ctypes' default int would be truncated) and its
    number of parameters."""
    decls = _declarations()
    assert {d[1] for d in decls} == set(hps.EXPORTS)
    ret_map = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "void": None,
               "const char*": ctypes.c_char_p, "const char *": ctypes.c_char_p}
    L = hps.lib()
    for ret, name, n in decls:
        fn = getattr(L, name)
        assert fn.restype is ret_map[ret], (name, ret, fn.restype)
        assert fn.argtypes is not None and len(fn.argtypes) == n, (name, n, fn.argtypes)
