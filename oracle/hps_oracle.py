"""FP64 CPU oracle for the composite spectral collocation method of
Gillman & Martinsson (arXiv:1307.2665).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg (and its reference arm) may import or call anything here.  It
shares no code with the CUDA path: its constants, node orderings, assembly and
solvers are written independently, with NumPy/SciPy as plain library primitives.

What it computes.  The merges of Section 4 are exact in exact arithmetic (the
Remark 5.1): the hierarchical solver reaches, up to rounding, the
solution of ONE linear system, the global composite collocation system.  The
oracle writes that system out and solves it by sparse LU:

  unknowns  u at the Gauss nodes of every interior leaf edge (Section 2) and
            w at the (p-2)^2 interior Chebyshev nodes of every leaf (Section 3.1);
  (E1)      per leaf and per interior Chebyshev node, the collocation equation
            (A w_full)_i = F_i  (Section 3.1, eq. A_interior; F = 0 for eq. basic),
            where the boundary nodes of w_full carry L1 u_e: the per-side
            degree (q-1) Gauss interpolant evaluated at the side's Chebyshev
            points, corners averaged (Section 3.2, Step 1);
  (E2)      per Gauss node on an edge shared by leaves alpha (left / below) and
            beta (right / above): flux^alpha - flux^beta = G, flux being
            L4 L3 w_full: d/dx on vertical sides, d/dy on horizontal sides, in the
            global direction (Section 2, definition of v; Section 3.2, Steps 3-4).
            G = 0 for eq. basic: this is v_3^alpha = v_3^beta, the equation that
            eq. (U_parent) of Section 4 solves.

Non-zero F and G (a body load and a flux jump) are not in the paper; they are
the right-hand sides of the correction equation of iterative refinement.

Readings where the paper is silent or garbled:
  * Chebyshev nodes are the p extreme (Lobatto) points, so the boundary holds
    4(p-1) nodes and the interior (p-2)^2 (Section 3.1).
  * "Gaussian nodes" are Gauss-Legendre points.
  * p and q may differ (Section 3.2 assumes p = q): L1 extrapolates the degree
    (q-1) interpolant of a side to all p Chebyshev points of that side, corners
    included; L3 differentiates at all p side points; L4 evaluates the degree
    (p-1) interpolant of the side fluxes at the q Gauss points.
  * Corner conflicts of Step 1 are resolved by the arithmetic mean.

Solvers: `solve_global` assembles (E1, E2) and calls scipy.sparse.linalg.splu
(dense numpy.linalg.solve on request, for the brute-force check).
`solve_condensed` is the textbook static condensation of the same system
(eliminate each leaf's interior unknowns with a dense solve, then sparse LU of
the edge system); it is pinned to `solve_global` in the tests and is used where
the assembled system is too large.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, invariants, brute force, and the node counts N and N_tot that
Tables 1 and 3 print).  The point values of Table 3 are not reproduced by the
problems as Section 9.2 states them, so none of them serves as a pin.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import legendre as npleg

COEFF_NAMES = ("c11", "c12", "c22", "c1", "c2", "c")


# ============================================================ 1-D constants
def cheb_points(p):
    """Section 3.1: p Chebyshev extreme points on [-1, 1], in increasing order."""
    j = np.arange(p)
    return -np.cos(np.pi * j / (p - 1))


def cheb_diff(p):
    """Section 3.1: the spectral differentiation matrix on cheb_points(p).

    Written as its definition: D = V' V^{-1}, where V[j, k] = T_k(t_j) and
    V'[j, k] = T_k'(t_j), i.e. D maps the values of a polynomial of degree
    < p at the nodes to the values of its derivative at the nodes."""
    t = cheb_points(p)
    V = npcheb.chebvander(t, p - 1)
    Vd = np.empty((p, p))
    for k in range(p):
        c = np.zeros(p)
        c[k] = 1.0
        Vd[:, k] = npcheb.chebval(t, npcheb.chebder(c))
    return np.linalg.solve(V.T, Vd.T).T


def gauss_points(q):
    """Section 2: q Gauss-Legendre points and weights on [-1, 1], increasing."""
    x, w = npleg.leggauss(q)
    order = np.argsort(x)
    return x[order], w[order]


def interp_matrix(src, dst):
    """Lagrange interpolation: row i evaluates at dst[i] the polynomial of degree
    < len(src) through values at src (the re-tabulations of Section 3.2, Steps 1
    and 4, between a side's Gauss and Chebyshev nodes).  Written as
    V_dst V_src^{-1} in the Legendre basis."""
    n = len(src)
    Vs = npleg.legvander(np.asarray(src), n - 1)
    Vd = npleg.legvander(np.asarray(dst), n - 1)
    return np.linalg.solve(Vs.T, Vd.T).T


# ================================================================= geometry
@dataclass
class Problem:
    """A Dirichlet problem (eq. basic) on the rectangle domain = (x0, x1, y0, y1),
    split into nx-by-ny leaves, p Chebyshev points per leaf side, q Gauss points
    per leaf edge.  coeffs[name] is None (absent, i.e. zero) or an array of shape
    (ny*nx, p, p) sampled at cheb_grid(); leaf l = iy*nx + ix, local [a, b] with a
    the y index and b the x index."""
    domain: tuple
    nx: int
    ny: int
    p: int
    q: int
    coeffs: dict = field(default_factory=dict)

    @property
    def n_leaves(self):
        return self.nx * self.ny

    @property
    def hx(self):
        return (self.domain[1] - self.domain[0]) / self.nx

    @property
    def hy(self):
        return (self.domain[3] - self.domain[2]) / self.ny


def cheb_grid(domain, nx, ny, p):
    """Coordinates of every leaf's p x p Chebyshev grid (Section 3.1, the
    tensor grid of a leaf): shape (ny*nx, p, p, 2)."""
    x0, x1, y0, y1 = domain
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    t = (cheb_points(p) + 1.0) / 2.0
    out = np.empty((ny * nx, p, p, 2))
    for iy in range(ny):
        for ix in range(nx):
            l = iy * nx + ix
            xs = x0 + ix * hx + t * hx
            ys = y0 + iy * hy + t * hy
            out[l, :, :, 0] = xs[None, :]
            out[l, :, :, 1] = ys[:, None]
    return out


class EdgeNumbering:
    """Global numbering of the Gauss nodes (Section 2, the points x_k).

    Horizontal edge (row j in 0..ny, column i in 0..nx-1) node k:
        (j*nx + i)*q + k, at x = x0 + i hx + (g_k+1) hx/2, y = y0 + j hy.
    Vertical edge (column i in 0..nx, row j in 0..ny-1) node k:
        NH + (i*ny + j)*q + k, at x = x0 + i hx, y = y0 + j hy + (g_k+1) hy/2.
    """

    def __init__(self, prob: Problem):
        self.prob = prob
        nx, ny, q = prob.nx, prob.ny, prob.q
        self.NH = (ny + 1) * nx * q
        self.N = self.NH + (nx + 1) * ny * q
        g, _ = gauss_points(q)
        self.g = g

    def h(self, j, i):
        q = self.prob.q
        return (j * self.prob.nx + i) * q + np.arange(q)

    def v(self, i, j):
        q = self.prob.q
        return self.NH + (i * self.prob.ny + j) * q + np.arange(q)

    def coords(self):
        pr = self.prob
        x0, x1, y0, y1 = pr.domain
        hx, hy = pr.hx, pr.hy
        xy = np.empty((self.N, 2))
        t = (self.g + 1.0) / 2.0
        for j in range(pr.ny + 1):
            for i in range(pr.nx):
                idx = self.h(j, i)
                xy[idx, 0] = x0 + i * hx + t * hx
                xy[idx, 1] = y0 + j * hy
        for i in range(pr.nx + 1):
            for j in range(pr.ny):
                idx = self.v(i, j)
                xy[idx, 0] = x0 + i * hx
                xy[idx, 1] = y0 + j * hy + t * hy
        return xy

    def leaf_sides(self, ix, iy):
        """The leaf's 4q exterior Gauss nodes (its index set I_e, Section 2),
        sides S, E, N, W, each in increasing coordinate."""
        return np.concatenate([self.h(iy, ix), self.v(ix + 1, iy),
                               self.h(iy + 1, ix), self.v(ix, iy)])

    def is_boundary(self):
        pr = self.prob
        b = np.zeros(self.N, dtype=bool)
        for i in range(pr.nx):
            b[self.h(0, i)] = True
            b[self.h(pr.ny, i)] = True
        for j in range(pr.ny):
            b[self.v(0, j)] = True
            b[self.v(pr.nx, j)] = True
        return b

    def gamma_order(self):
        """Global ids of the Gauss nodes on Gamma (eq. basic), counter-clockwise from (x0, y0):
        south (increasing x), east (increasing y), north (decreasing x),
        west (decreasing y).  This is the order of the Dirichlet data f."""
        pr = self.prob
        parts = [self.h(0, i) for i in range(pr.nx)]
        parts += [self.v(pr.nx, j) for j in range(pr.ny)]
        parts += [self.h(pr.ny, i)[::-1] for i in reversed(range(pr.nx))]
        parts += [self.v(0, j)[::-1] for j in reversed(range(pr.ny))]
        return np.concatenate(parts)


def boundary_points(prob: Problem):
    """Coordinates of the Dirichlet nodes on Gamma (eq. basic) in the order of f."""
    en = EdgeNumbering(prob)
    return en.coords()[en.gamma_order()]


# ===================================================== per-leaf local operators
class LeafOps:
    """The leaf maps of Sections 3.1-3.2 for one leaf size (hx, hy)."""

    def __init__(self, p, q, hx, hy):
        self.p, self.q = p, q
        tc = cheb_points(p)
        tg, _ = gauss_points(q)
        D = cheb_diff(p)
        I = np.eye(p)
        # index (a, b) -> a*p + b, a along y, b along x
        self.Dx = np.kron(I, D) * (2.0 / hx)
        self.Dy = np.kron(D, I) * (2.0 / hy)
        self.Dxx = self.Dx @ self.Dx
        self.Dxy = self.Dx @ self.Dy
        self.Dyy = self.Dy @ self.Dy
        self.Pg2c = interp_matrix(tg, tc)  # p x q, Step 1
        self.Pc2g = interp_matrix(tc, tg)  # q x p, Step 4
        idx = np.arange(p * p).reshape(p, p)
        bnd = np.zeros((p, p), dtype=bool)
        bnd[0, :] = bnd[-1, :] = bnd[:, 0] = bnd[:, -1] = True
        self.Ji = idx[~bnd]            # interior, (p-2)^2, row-major
        self.Je = idx[bnd]
        # L1: p^2 x 4q, Step 1 (rows of interior nodes are zero)
        L1 = np.zeros((p * p, 4 * q))
        cnt = np.zeros(p * p)
        sides = {"S": (0, lambda b: (0, b)), "E": (1, lambda a: (a, p - 1)),
                 "N": (2, lambda b: (p - 1, b)), "W": (3, lambda a: (a, 0))}
        for name, (s, pos) in sides.items():
            for j in range(p):
                a, b = pos(j)
                r = a * p + b
                L1[r, s * q:(s + 1) * q] += self.Pg2c[j]
                cnt[r] += 1
        nz = cnt > 0
        L1[nz] /= cnt[nz][:, None]
        self.L1 = L1
        # flux map F = L4 L3: 4q x p^2, Steps 3-4
        F = np.zeros((4 * q, p * p))
        rowS = [0 * p + b for b in range(p)]
        rowN = [(p - 1) * p + b for b in range(p)]
        rowW = [a * p + 0 for a in range(p)]
        rowE = [a * p + (p - 1) for a in range(p)]
        F[0 * q:1 * q] = self.Pc2g @ self.Dy[rowS]
        F[1 * q:2 * q] = self.Pc2g @ self.Dx[rowE]
        F[2 * q:3 * q] = self.Pc2g @ self.Dy[rowN]
        F[3 * q:4 * q] = self.Pc2g @ self.Dx[rowW]
        self.F = F

    def operator(self, coef_leaf):
        """Section 3.1: A = -C11 Dx^2 - 2 C12 Dx Dy - C22 Dy^2 + C1 Dx + C2 Dy + C,
        the C's diagonal with the coefficient samples of this leaf."""
        p = self.p
        A = np.zeros((p * p, p * p))

        def c(name):
            v = coef_leaf.get(name)
            return None if v is None else np.asarray(v, np.float64).reshape(p * p)

        terms = (("c11", -1.0, self.Dxx), ("c12", -2.0, self.Dxy),
                 ("c22", -1.0, self.Dyy), ("c1", 1.0, self.Dx),
                 ("c2", 1.0, self.Dy))
        for name, s, M in terms:
            v = c(name)
            if v is not None:
                A += s * v[:, None] * M
        v = c("c")
        if v is not None:
            A += np.diag(v)
        return A


def _leaf_coef(prob, l):
    return {k: (None if prob.coeffs.get(k) is None else prob.coeffs[k][l]) for k in COEFF_NAMES}


# ================================================================ solvers
def _boundary_values(prob, en, f):
    """Scatter Dirichlet data f (order of EdgeNumbering.gamma_order, shape
    (nbnd,) or (nbnd, nrhs)) into a global Gauss-node array."""
    f = np.asarray(f, np.float64)
    if f.ndim == 1:
        f = f[:, None]
    U = np.zeros((en.N, f.shape[1]))
    U[en.gamma_order()] = f
    return U


def _as2d(a, rows):
    if a is None:
        return None
    a = np.asarray(a, np.float64)
    return a.reshape(rows, -1)


@dataclass
class Solution:
    """w_full on every leaf (the Chebyshev values of Section 3.1):
    (nrhs, n_leaves, p, p); u at all Gauss nodes (Section 2): (N, nrhs)."""
    w: np.ndarray
    u_gauss: np.ndarray


def solve_global(prob: Problem, f, F=None, G=None, dense=False):
    """Assemble (E1, E2) and solve: E1 is the collocation condition of Section
    3.1 (eq. A_interior) at every leaf's interior nodes, E2 the flux continuity
    v3^alpha = v3^beta of Section 4 that eq. U_parent solves, at every interior
    Gauss node.  f: Dirichlet data in gamma order, (nbnd,) or
    (nbnd, nrhs).  F: body load at interior Chebyshev nodes, (n_leaves, (p-2)^2,
    nrhs) or None.  G: flux jumps at the interior Gauss nodes, indexed by global
    Gauss id, (N, nrhs) or None (boundary entries ignored)."""
    p, q, nl = prob.p, prob.q, prob.n_leaves
    ni = (p - 2) ** 2
    en = EdgeNumbering(prob)
    ops = LeafOps(p, q, prob.hx, prob.hy)
    isb = en.is_boundary()
    U = _boundary_values(prob, en, f)
    nrhs = U.shape[1]
    # unknown numbering
    uid = -np.ones(en.N, dtype=np.int64)
    interior_nodes = np.nonzero(~isb)[0]
    uid[interior_nodes] = np.arange(len(interior_nodes))
    nu = len(interior_nodes)
    wbase = nu
    nunk = nu + nl * ni
    rows, cols, vals = [], [], []
    rhs = np.zeros((nunk, nrhs))
    Fb = None if F is None else np.asarray(F, np.float64).reshape(nl, ni, -1)
    # E1 rows: numbered like the w unknowns
    leaf_ext = []
    for iy in range(prob.ny):
        for ix in range(prob.nx):
            l = iy * prob.nx + ix
            ext = en.leaf_sides(ix, iy)
            leaf_ext.append(ext)
            A = ops.operator(_leaf_coef(prob, l))
            Ai = A[ops.Ji]
            Aie = Ai @ ops.L1            # ni x 4q on u_e
            Aii = Ai[:, ops.Ji]          # ni x ni on w_i
            r0 = wbase + l * ni
            rr = r0 + np.arange(ni)
            # w part
            R, C = np.meshgrid(rr, r0 + np.arange(ni), indexing="ij")
            m = Aii != 0
            rows.append(R[m]); cols.append(C[m]); vals.append(Aii[m])
            # u part
            ue_id = uid[ext]
            known = ue_id < 0
            if np.any(~known):
                sub = Aie[:, ~known]
                R, C = np.meshgrid(rr, ue_id[~known], indexing="ij")
                m = sub != 0
                rows.append(R[m]); cols.append(C[m]); vals.append(sub[m])
            if np.any(known):
                rhs[rr] -= Aie[:, known] @ U[ext[known]]
            if Fb is not None:
                rhs[rr] += Fb[l]
    # E2 rows: numbered like the u unknowns
    Gb = None if G is None else _as2d(G, en.N)

    def flux_rows(l, side):
        """Rows of flux = F w_full on one side (Section 3.2, Steps 3-4), as
        (coeffs on u_e, coeffs on w_i)."""
        Fs = ops.F[side * q:(side + 1) * q]
        return Fs @ ops.L1, Fs[:, ops.Ji]

    def add_pair(la, sa, lb, sb, gids):
        rr = uid[gids]
        for l, s, sg in ((la, sa, 1.0), (lb, sb, -1.0)):
            Fu, Fw = flux_rows(l, s)
            Fu = sg * Fu
            Fw = sg * Fw
            ext = leaf_ext[l]
            ue_id = uid[ext]
            known = ue_id < 0
            sub = Fu[:, ~known]
            R, C = np.meshgrid(rr, ue_id[~known], indexing="ij")
            m = sub != 0
            rows.append(R[m]); cols.append(C[m]); vals.append(sub[m])
            if np.any(known):
                rhs[rr] -= Fu[:, known] @ U[ext[known]]
            R, C = np.meshgrid(rr, wbase + l * ni + np.arange(ni), indexing="ij")
            m = Fw != 0
            rows.append(R[m]); cols.append(C[m]); vals.append(Fw[m])
        if Gb is not None:
            rhs[rr] += Gb[gids]

    for j in range(1, prob.ny):        # interior horizontal edges
        for i in range(prob.nx):
            add_pair((j - 1) * prob.nx + i, 2, j * prob.nx + i, 0, en.h(j, i))
    for i in range(1, prob.nx):        # interior vertical edges
        for j in range(prob.ny):
            add_pair(j * prob.nx + (i - 1), 1, j * prob.nx + i, 3, en.v(i, j))

    Aglob = scipy.sparse.csc_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(nunk, nunk))
    if dense:
        x = np.linalg.solve(Aglob.toarray(), rhs)
    else:
        # The collocation rows scale like 1/h^2 and the flux rows like 1/h:
        # equilibrate the rows before the LU and polish with two steps of FP64
        # iterative refinement (both only reduce the rounding error of the
        # library solve; the system solved is unchanged).
        rs = 1.0 / np.maximum(abs(Aglob).max(axis=1).toarray().ravel(), 1e-300)
        As = scipy.sparse.diags(rs) @ Aglob
        lu = scipy.sparse.linalg.splu(As.tocsc())
        x = lu.solve(rhs * rs[:, None])
        for _ in range(2):
            x = x + lu.solve((rhs - Aglob @ x) * rs[:, None])
    Ug = U.copy()
    Ug[interior_nodes] = x[:nu]
    wi = x[nu:].reshape(nl, ni, nrhs)
    return _assemble_w(prob, ops, en, Ug, wi), Aglob, rhs


def _assemble_w(prob, ops, en, Ug, wi):
    p, nl = prob.p, prob.n_leaves
    nrhs = Ug.shape[1]
    w = np.zeros((nrhs, nl, p * p))
    for iy in range(prob.ny):
        for ix in range(prob.nx):
            l = iy * prob.nx + ix
            ext = en.leaf_sides(ix, iy)
            full = ops.L1 @ Ug[ext]          # boundary rows; interior rows 0
            full[ops.Ji] = wi[l]
            w[:, l, :] = full.T
    return Solution(w=w.reshape(nrhs, nl, p, p), u_gauss=Ug)


def solve_condensed(prob: Problem, f, F=None, G=None):
    """Static condensation of the same system: per leaf, w_i = X u_e + A_ii^{-1} F_i
    with X = -A_ii^{-1} A_ie L1 (eq. leaf_solve), so the leaf's side fluxes are
    Tl u_e + hl; the E2 rows then involve edge unknowns only and are solved by
    sparse LU; finally each leaf's interior is recovered."""
    p, q, nl = prob.p, prob.q, prob.n_leaves
    ni = (p - 2) ** 2
    en = EdgeNumbering(prob)
    ops = LeafOps(p, q, prob.hx, prob.hy)
    isb = en.is_boundary()
    U = _boundary_values(prob, en, f)
    nrhs = U.shape[1]
    uid = -np.ones(en.N, dtype=np.int64)
    interior_nodes = np.nonzero(~isb)[0]
    uid[interior_nodes] = np.arange(len(interior_nodes))
    nu = len(interior_nodes)
    Fb = None if F is None else np.asarray(F, np.float64).reshape(nl, ni, -1)
    Gb = None if G is None else _as2d(G, en.N)
    T, H, X, Z, ext_all = [], [], [], [], []
    for iy in range(prob.ny):
        for ix in range(prob.nx):
            l = iy * prob.nx + ix
            A = ops.operator(_leaf_coef(prob, l))
            Ai = A[ops.Ji]
            B = Ai @ ops.L1
            if Fb is not None:
                B = np.concatenate([B, -Fb[l]], axis=1)
            sol = -np.linalg.solve(Ai[:, ops.Ji], B)
            Xl = sol[:, :4 * q]
            Wl = ops.L1.copy()
            Wl[ops.Ji] += Xl
            T.append(ops.F @ Wl)
            if Fb is not None:
                zl = sol[:, 4 * q:]
                H.append(ops.F[:, ops.Ji] @ zl)
                Z.append(zl)
            X.append(Xl)
            ext_all.append(en.leaf_sides(ix, iy))
    rows, cols, vals = [], [], []
    rhs = np.zeros((nu, nrhs))

    def add_pair(la, sa, lb, sb, gids):
        rr = uid[gids]
        for l, s, sg in ((la, sa, 1.0), (lb, sb, -1.0)):
            Ts = sg * T[l][s * q:(s + 1) * q]
            ext = ext_all[l]
            ue_id = uid[ext]
            known = ue_id < 0
            R, C = np.meshgrid(rr, ue_id[~known], indexing="ij")
            rows.append(R.ravel()); cols.append(C.ravel()); vals.append(Ts[:, ~known].ravel())
            if np.any(known):
                rhs[rr] -= Ts[:, known] @ U[ext[known]]
            if Fb is not None:
                rhs[rr] -= sg * H[l][s * q:(s + 1) * q]
        if Gb is not None:
            rhs[rr] += Gb[gids]

    for j in range(1, prob.ny):
        for i in range(prob.nx):
            add_pair((j - 1) * prob.nx + i, 2, j * prob.nx + i, 0, en.h(j, i))
    for i in range(1, prob.nx):
        for j in range(prob.ny):
            add_pair(j * prob.nx + (i - 1), 1, j * prob.nx + i, 3, en.v(i, j))
    Ug = U.copy()
    if nu > 0:
        K = scipy.sparse.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                    shape=(nu, nu))
        lu = scipy.sparse.linalg.splu(K)
        x = lu.solve(rhs)
        x = x + lu.solve(rhs - K @ x)  # one step of FP64 refinement of the library solve
        Ug[interior_nodes] = x
    wi = np.empty((nl, ni, nrhs))
    for l in range(nl):
        wi[l] = X[l] @ Ug[ext_all[l]]
        if Fb is not None:
            wi[l] += Z[l]
    return _assemble_w(prob, ops, en, Ug, wi)


def leaf_dtn(prob: Problem, l=0):
    """The leaf map T = L4 L3 L2 L1 of Section 3.2 (4q x 4q, sides S, E, N, W,
    each in increasing coordinate, fluxes in the global direction), and the
    leaf solution operator Y = -A_ii^{-1} A_ie L1 ((p-2)^2 x 4q, Section 5.3)."""
    ops = LeafOps(prob.p, prob.q, prob.hx, prob.hy)
    A = ops.operator(_leaf_coef(prob, l))
    Ai = A[ops.Ji]
    Y = -np.linalg.solve(Ai[:, ops.Ji], Ai @ ops.L1)
    W = ops.L1.copy()
    W[ops.Ji] += Y
    return ops.F @ W, Y


def residual(prob: Problem, sol: Solution, f, F=None, G=None):
    """FP64 residual of (E1, E2) (Section 3.1 eq. A_interior; Section 4 flux
    continuity) for a candidate solution, matrix-free.

    Returns (r1, r2): r1[l, i, rhs] = F_i - (A w_full)_i at each leaf's interior
    Chebyshev nodes; r2[k, rhs] = G_k - (flux^alpha - flux^beta)_k at each
    interior Gauss node k (global id; boundary entries zero).  w_full is rebuilt
    from the Gauss values (L1 on the boundary rows) and the interior values of
    the candidate, so a candidate whose corner values disagree with L1 is
    judged by its Gauss and interior values only."""
    p, q, nl = prob.p, prob.q, prob.n_leaves
    ni = (p - 2) ** 2
    en = EdgeNumbering(prob)
    ops = LeafOps(p, q, prob.hx, prob.hy)
    Ug = sol.u_gauss
    nrhs = Ug.shape[1]
    r1 = np.zeros((nl, ni, nrhs))
    fl = np.zeros((nl, 4 * q, nrhs))
    Fb = None if F is None else np.asarray(F, np.float64).reshape(nl, ni, -1)
    for iy in range(prob.ny):
        for ix in range(prob.nx):
            l = iy * prob.nx + ix
            ext = en.leaf_sides(ix, iy)
            full = ops.L1 @ Ug[ext]
            full[ops.Ji] = sol.w[:, l].reshape(nrhs, p * p).T[ops.Ji]
            A = ops.operator(_leaf_coef(prob, l))
            r1[l] = -(A[ops.Ji] @ full)
            if Fb is not None:
                r1[l] += Fb[l]
            fl[l] = ops.F @ full
    r2 = np.zeros((en.N, nrhs))
    for j in range(1, prob.ny):
        for i in range(prob.nx):
            la, lb = (j - 1) * prob.nx + i, j * prob.nx + i
            r2[en.h(j, i)] = -(fl[la][2 * q:3 * q] - fl[lb][0:q])
    for i in range(1, prob.nx):
        for j in range(prob.ny):
            la, lb = j * prob.nx + (i - 1), j * prob.nx + i
            r2[en.v(i, j)] = -(fl[la][q:2 * q] - fl[lb][3 * q:4 * q])
    if G is not None:
        Gb = _as2d(G, en.N)
        r2[~en.is_boundary()] += Gb[~en.is_boundary()]
    return r1, r2


def sampled_residual(prob: Problem, w, f, leaves):
    """Leaf-local check of a candidate solution given only its per-leaf values
    w_full (nrhs, n_leaves, p, p), on a subset of leaves, for problems too
    large to solve here.  For each listed leaf it evaluates

      e1     (A w_full)_i at the interior Chebyshev nodes (E1, Section 3.1),
             scaled by ||A_ii-rows||_inf ||w||_inf;
      e2     flux mismatch L4 L3 w^alpha - L4 L3 w^beta on its east and north
             edges (E2), scaled by ||L4 L3||_inf ||w||_inf;
      cont   the two leaves' values at the non-corner Chebyshev points of a
             shared side, which both come from the same Gauss values through
             L1 (Section 3.2, Step 1) and must agree, scaled by ||w||_inf;
      gamma  on sides lying on Gamma, the non-corner Chebyshev values against
             L1 f of that side (Step 1 with the Dirichlet data), same scale.

    f: (nrhs, nbnd) in the order of boundary_points.  Returns the maxima."""
    p, q = prob.p, prob.q
    ops = LeafOps(p, q, prob.hx, prob.hy)
    en = EdgeNumbering(prob)
    gpos = -np.ones(en.N, dtype=np.int64)
    gpos[en.gamma_order()] = np.arange(len(en.gamma_order()))
    f = np.atleast_2d(np.asarray(f, np.float64))
    w = np.asarray(w, np.float64)
    nrhs = w.shape[0]
    inner = np.arange(1, p - 1)
    rows = {"S": inner, "N": (p - 1) * p + inner, "W": inner * p, "E": inner * p + p - 1}
    fscale = np.max(np.sum(np.abs(ops.F), axis=1))
    out = {"e1": 0.0, "e2": 0.0, "cont": 0.0, "gamma": 0.0}

    def full(l):
        return w[:, l].reshape(nrhs, p * p).T

    for l in leaves:
        iy, ix = divmod(int(l), prob.nx)
        W = full(l)
        wmax = max(np.max(np.abs(W)), 1e-300)
        A = ops.operator(_leaf_coef(prob, l))[ops.Ji]
        out["e1"] = max(out["e1"], np.max(np.abs(A @ W)) / (np.max(np.sum(np.abs(A), 1)) * wmax))
        Fl = ops.F @ W
        for dx, dy, mine, theirs, rm, rt in ((1, 0, slice(q, 2 * q), slice(3 * q, 4 * q), "E", "W"),
                                              (0, 1, slice(2 * q, 3 * q), slice(0, q), "N", "S")):
            jx, jy = ix + dx, iy + dy
            if jx >= prob.nx or jy >= prob.ny:
                continue
            Wn = full(jy * prob.nx + jx)
            sc = max(wmax, np.max(np.abs(Wn)))
            out["e2"] = max(out["e2"], np.max(np.abs(Fl[mine] - (ops.F @ Wn)[theirs])) / (fscale * sc))
            out["cont"] = max(out["cont"], np.max(np.abs(W[rows[rm]] - Wn[rows[rt]])) / sc)
        sides = []
        if iy == 0:
            sides.append(("S", en.h(0, ix)))
        if iy == prob.ny - 1:
            sides.append(("N", en.h(prob.ny, ix)))
        if ix == 0:
            sides.append(("W", en.v(0, iy)))
        if ix == prob.nx - 1:
            sides.append(("E", en.v(prob.nx, iy)))
        for side, gids in sides:
            want = ops.Pg2c[1:p - 1] @ f[:, gpos[gids]].T
            out["gamma"] = max(out["gamma"], np.max(np.abs(W[rows[side]] - want)) / wmax)
    return out


# ============================================================ post-processing
def boundary_flux(prob: Problem, w):
    """The DtN map of the whole domain applied to the Dirichlet data of the
    solutions w (nrhs, n_leaves, p, p): at every Gamma Gauss node, in the order
    of f, the flux of Section 2 (d/dx on vertical sides, d/dy on horizontal
    sides, global direction), computed from the boundary leaf as L4 L3 w_full
    (Section 3.2, Steps 3-4; the map F of LeafOps).  This is T^1 f for the data
    f of the solve (Algorithm 1's root map), without forming T^1.
    Returns (nrhs, nbnd)."""
    w = np.asarray(w, np.float64)
    if w.ndim == 3:
        w = w[None]
    en = EdgeNumbering(prob)
    ops = LeafOps(prob.p, prob.q, prob.hx, prob.hy)
    q, nx, ny = prob.q, prob.nx, prob.ny
    G = np.zeros((en.N, w.shape[0]))
    for iy in range(ny):
        for ix in range(nx):
            if 0 < ix < nx - 1 and 0 < iy < ny - 1:
                continue
            fl = ops.F @ w[:, iy * nx + ix].reshape(w.shape[0], -1).T  # (4q, nrhs): S, E, N, W
            if iy == 0:
                G[en.h(0, ix)] = fl[0:q]
            if ix == nx - 1:
                G[en.v(nx, iy)] = fl[q:2 * q]
            if iy == ny - 1:
                G[en.h(ny, ix)] = fl[2 * q:3 * q]
            if ix == 0:
                G[en.v(0, iy)] = fl[3 * q:4 * q]
    return G[en.gamma_order()].T


def dtn_apply(prob: Problem, f):
    """T^1 f for Dirichlet data f (nrhs, nbnd), T^1 the DtN map of the whole
    domain (the root map of Algorithm 1; Section 9.1 times it as T_apply): the
    boundary fluxes of the global system's solution (sparse LU, solve_global)."""
    f = np.atleast_2d(np.asarray(f, np.float64))
    sol, _, _ = solve_global(prob, f.T)
    return boundary_flux(prob, sol.w)


def lagrange_basis(nodes, t):
    """Values at t of the Lagrange polynomials of the nodes (the leaf
    interpolant of Section 5.3), in product form:
    l_j(t) = prod_{k != j} (t - t_k) / (t_j - t_k)."""
    nodes = np.asarray(nodes, np.float64)
    out = np.ones(len(nodes))
    for j in range(len(nodes)):
        for k in range(len(nodes)):
            if k != j:
                out[j] *= (t - nodes[k]) / (nodes[j] - nodes[k])
    return out


def evaluate_points(prob: Problem, w, xy):
    """Section 5.3: the solutions w (nrhs, n_leaves, p, p) at points xy (npts, 2)
    by the tensor-product interpolant of the containing leaf's Chebyshev values.
    A point on an edge shared by two leaves takes the leaf to its east (north);
    one on the domain's east (north) side the last leaf.  Returns (nrhs, npts)."""
    w = np.asarray(w, np.float64)
    if w.ndim == 3:
        w = w[None]
    x0, x1, y0, y1 = prob.domain
    t = cheb_points(prob.p)
    out = np.empty((w.shape[0], len(xy)))
    for i, (x, y) in enumerate(np.asarray(xy, np.float64)):
        if not (x0 <= x <= x1 and y0 <= y <= y1):
            raise ValueError("point outside the domain")
        sx = (x - x0) / (x1 - x0) * prob.nx
        sy = (y - y0) / (y1 - y0) * prob.ny
        ix = min(int(np.floor(sx)), prob.nx - 1)
        iy = min(int(np.floor(sy)), prob.ny - 1)
        bx = lagrange_basis(t, 2.0 * (sx - ix) - 1.0)
        by = lagrange_basis(t, 2.0 * (sy - iy) - 1.0)
        out[:, i] = np.einsum("a,rab,b->r", by, w[:, iy * prob.nx + ix], bx)
    return out


# ================================================================ counting
def gauss_count(n, q):
    """N = 2 n (n+1) q Gauss nodes on an n x n leaf grid (Section 5.2)."""
    return 2 * n * (n + 1) * q


def total_count(n, p, q):
    """N_tot = N + (n (p-1) + 1)^2: Gauss nodes plus distinct Chebyshev nodes
    (the convention of Tables 1 and 3)."""
    return gauss_count(n, q) + (n * (p - 1) + 1) ** 2


def make_problem(domain, nx, ny, p, q, coeff_fn):
    """Sample coeff_fn(x, y) -> dict of the coefficients of eq. defA at this
    oracle's own Chebyshev grid (the collocation nodes of Section 3.1)."""
    xy = cheb_grid(domain, nx, ny, p)
    coeffs = coeff_fn(xy[..., 0], xy[..., 1])
    return Problem(domain=tuple(domain), nx=nx, ny=ny, p=p, q=q,
                   coeffs={k: (None if coeffs.get(k) is None else np.asarray(coeffs[k], np.float64))
                           for k in COEFF_NAMES})
