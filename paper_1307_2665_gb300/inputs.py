"""Seeded synthetic inputs for the composite spectral solver.

Every function here maps sample coordinates (x, y) to values: coefficient
fields of the operator of eq. defA and Dirichlet data f on the boundary.
The coordinates come from the caller (the solver's own node helpers, or the
test oracle's), so this module holds none of the discretisation: no nodes,
no differentiation, no interpolation.  Both sides of a parity test sample
the same functions here and nothing else is shared between them.

Sign convention: the operator is
    A u = -c11 u_xx - 2 c12 u_xy - c22 u_yy + c1 u_x + c2 u_y + c u
(eq. defA).  The numerical examples of Section 9 write their PDE as
-Lap u - c1 u_x - c2 u_y - c u = 0 (eq. example); the helpers for those
examples return coefficients already converted to the eq. defA signs.
"""
from __future__ import annotations

import numpy as np

COEFF_NAMES = ("c11", "c12", "c22", "c1", "c2", "c")


def _zeros_like(x):
    return np.zeros_like(np.asarray(x, dtype=np.float64))


def _ones_like(x):
    return np.ones_like(np.asarray(x, dtype=np.float64))


# ----------------------------------------------------------------- coefficients
def laplace(x, y):
    """-Lap u: c11 = c22 = 1, every other coefficient absent (None)."""
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": None, "c2": None, "c": None}


def convection_diffusion(x, y, amp=100.0):
    """c11 = c22 = 1, c1 = -amp cos(4 pi y), c2 = amp sin(4 pi x), c = 0 (eq. defA signs)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": -amp * np.cos(4 * np.pi * y), "c2": amp * np.sin(4 * np.pi * x),
            "c": None}


def gaussian_bump_helmholtz(x, y, kappa=80.0):
    """-Lap u - kappa^2 (1 - 0.5 exp(-((x-.5)^2 + (y-.5)^2)/0.02)) u = 0, as eq. defA coefficients."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    bump = 1.0 - 0.5 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.02)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": None, "c2": None, "c": -(kappa ** 2) * bump}


def constant_helmholtz(x, y, kappa):
    """-Lap u - kappa^2 u = 0 (Section 9.1, Helmholtz I/II), eq. defA signs."""
    x = np.asarray(x, np.float64)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": None, "c2": None, "c": -(kappa ** 2) * _ones_like(x)}


def paper_variable_helmholtz(x, y, kappa=640.0):
    """Section 9.2 'variable Helmholtz': eq. example c = kappa^2 (1 - (sin 4pi x sin 4pi y)^2)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    c81 = kappa ** 2 * (1.0 - (np.sin(4 * np.pi * x) * np.sin(4 * np.pi * y)) ** 2)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": None, "c2": None, "c": -c81}


def paper_diffusion_convection(x, y):
    """Section 9.2 'diffusion-convection': eq. example c1 = -1e4 cos(4pi y), c2 = -1e4 cos(4pi x)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    c1_81 = -1.0e4 * np.cos(4 * np.pi * y)
    c2_81 = -1.0e4 * np.cos(4 * np.pi * x)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": -c1_81, "c2": -c2_81, "c": None}


def paper_constant_convection(x, y):
    """Section 9.2 'constant convection': eq. example c2 = -1e5."""
    x = np.asarray(x, np.float64)
    return {"c11": _ones_like(x), "c12": None, "c22": _ones_like(x),
            "c1": None, "c2": 1.0e5 * _ones_like(x), "c": None}


def smooth_field(seed, x, y, nk=4):
    """A smooth random field on [0,1]^2: a sum over kx, ky < nk of
    a cos(pi kx x + phi) cos(pi ky y + psi) / (1 + kx^2 + ky^2), with a ~ N(0,1)
    and phases ~ U[0, 2pi) drawn from PCG64(seed).  Scaled so that its maximum
    modulus on a fixed 129 x 129 grid of [0,1]^2 is 1 (so the scale does not
    depend on where the field is sampled)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((nk, nk))
    phi = rng.uniform(0.0, 2 * np.pi, (nk, nk))
    psi = rng.uniform(0.0, 2 * np.pi, (nk, nk))

    def ev(xx, yy):
        out = np.zeros(np.broadcast(xx, yy).shape)
        for kx in range(nk):
            for ky in range(nk):
                out += (a[kx, ky] * np.cos(np.pi * kx * xx + phi[kx, ky])
                        * np.cos(np.pi * ky * yy + psi[kx, ky]) / (1.0 + kx * kx + ky * ky))
        return out

    g = np.linspace(0.0, 1.0, 129)
    gx, gy = np.meshgrid(g, g)
    scale = np.max(np.abs(ev(gx, gy)))
    return ev(np.asarray(x, np.float64), np.asarray(y, np.float64)) / scale


def random_smooth_operator(seed, x, y):
    """Uneven-batch operator: c11, c22 = 1 + 0.5 field, c12 = 0.2 field,
    c1, c2 = +-50 field (independent fields), c = 0."""
    f = [smooth_field(seed * 8 + k, x, y) for k in range(5)]
    return {"c11": 1.0 + 0.5 * f[0], "c12": 0.2 * f[1], "c22": 1.0 + 0.5 * f[2],
            "c1": 50.0 * f[3], "c2": -50.0 * f[4], "c": None}


# -------------------------------------------------------------- boundary data
def exp_sin(x, y):
    """u = exp(x) sin(y): harmonic, used as exact solution and as Dirichlet data."""
    return np.exp(np.asarray(x, np.float64)) * np.sin(np.asarray(y, np.float64))


def harmonic_poly(k, part, x, y):
    """Re or Im of (x + i y)^k (harmonic polynomial of degree k)."""
    z = (np.asarray(x, np.float64) + 1j * np.asarray(y, np.float64)) ** k
    return z.real if part == "re" else z.imag


def log_source(x, y, xs=-2.0, ys=0.0):
    """log |x_hat - x| with x_hat = (-2, 0) (Section 9.1, Laplace)."""
    return np.log(np.hypot(np.asarray(x, np.float64) - xs, np.asarray(y, np.float64) - ys))


def paper_table3_data(x, y):
    """f = cos(2 x1) (1 - 2 x2), the Dirichlet data of Section 9.2."""
    return np.cos(2 * np.asarray(x, np.float64)) * (1.0 - 2 * np.asarray(y, np.float64))


def boundary_arclength(x, y, domain):
    """Arclength s of boundary points counter-clockwise from (x0, y0):
    south side (s = x - x0), east, north, west.  Points must lie on the boundary."""
    x0, x1, y0, y1 = domain
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w, h = x1 - x0, y1 - y0
    tol = 1e-12 * max(w, h)
    s = np.empty_like(x)
    south = np.abs(y - y0) <= tol
    east = (np.abs(x - x1) <= tol) & ~south
    north = (np.abs(y - y1) <= tol) & ~south & ~east
    west = ~(south | east | north)
    s[south] = x[south] - x0
    s[east] = w + (y[east] - y0)
    s[north] = w + h + (x1 - x[north])
    s[west] = 2 * w + h + (y1 - y[west])
    return s


def fourier_boundary(seed, x, y, domain, nmodes=20):
    """Smooth random Dirichlet data: sum over k = 1..nmodes of
    a_k cos(2 pi k s / P) + b_k sin(2 pi k s / P), s the counter-clockwise
    arclength from (x0, y0), P the perimeter, a_k, b_k ~ N(0,1) from PCG64(seed).
    Periodic in s, hence continuous at the corners."""
    x0, x1, y0, y1 = domain
    per = 2 * ((x1 - x0) + (y1 - y0))
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(nmodes)
    b = rng.standard_normal(nmodes)
    s = boundary_arclength(x, y, domain)
    out = np.zeros_like(s)
    for k in range(1, nmodes + 1):
        out += a[k - 1] * np.cos(2 * np.pi * k * s / per) + b[k - 1] * np.sin(2 * np.pi * k * s / per)
    return out


def sample_coefficients(fn, xy):
    """Evaluate a coefficient function at node coordinates xy[..., 2]."""
    return fn(xy[..., 0], xy[..., 1])


def sample_on_leaf_grid(fn, xs, ys, nx, ny, p):
    """Coefficient samples of fn at every leaf's Chebyshev grid, evaluated on
    the tensor-product grid: xs (nx*p,) holds the x coordinates of the columns
    of leaves ix = 0..nx-1 in turn, ys (ny*p,) the y coordinates of the rows.
    Returns {name: (ny*nx, p, p) or None}, leaf l = iy*nx + ix, row index along
    y.  For large grids this evaluates each factor of a separable field once per
    grid line instead of once per node."""
    out = fn(np.asarray(xs, np.float64)[None, :], np.asarray(ys, np.float64)[:, None])
    res = {}
    for k in COEFF_NAMES:
        v = out.get(k)
        if v is None:
            res[k] = None
            continue
        g = np.broadcast_to(np.asarray(v, np.float64), (ny * p, nx * p))
        res[k] = np.ascontiguousarray(g.reshape(ny, p, nx, p).transpose(0, 2, 1, 3)
                                      .reshape(ny * nx, p, p))
    return res


def fourier_boundary_bank(seed, x, y, domain, nrhs, nmodes=20):
    """nrhs data sets of the form of fourier_boundary (a_k, b_k ~ N(0,1), drawn
    row by row from one PCG64(seed) stream), evaluated as one matrix product:
    returns (nrhs, len(x))."""
    x0, x1, y0, y1 = domain
    per = 2 * ((x1 - x0) + (y1 - y0))
    s = boundary_arclength(x, y, domain)
    k = np.arange(1, nmodes + 1)[:, None]
    basis = np.concatenate([np.cos(2 * np.pi * k * s / per), np.sin(2 * np.pi * k * s / per)])
    rng = np.random.Generator(np.random.PCG64(seed))
    ab = rng.standard_normal((nrhs, 2 * nmodes))
    return np.ascontiguousarray(ab @ basis)
