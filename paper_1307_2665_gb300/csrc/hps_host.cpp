// Host-side constants and the tree plan of the composite spectral solver.
//
// Constants (Section 3.1, 3.2): Chebyshev extreme points with the barycentric
// differentiation matrix, Gauss-Legendre points by Newton's method on the
// three-term Legendre recurrence, and Lagrange interpolation matrices in the
// first ("modified Lagrange") barycentric form, which stays accurate when a side
// interpolant is evaluated at the side's end points (Step 1 extrapolates the
// Gauss interpolant to the Chebyshev corners).
//
// Plan (Section 2 and Section 5.1): the binary tree over the leaves, each box's
// exterior ordering, and, per merge geometry, the maps that split the children's
// exterior nodes into J1, J2, J3 (Algorithm 1, line 6; Figure 3).
#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <tuple>

#include "hps_internal.hpp"

namespace hps {

namespace {

const double kPi = 3.14159265358979323846;

// Lagrange basis of nodes x evaluated at t: row-major (nt x n).
std::vector<double> lagrange_matrix(const std::vector<double>& x, const std::vector<double>& t) {
  const int n = (int)x.size(), nt = (int)t.size();
  std::vector<double> w(n);
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    w[j] = 1.0 / prod;
  }
  std::vector<double> P((size_t)nt * n, 0.0);
  for (int i = 0; i < nt; ++i) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (t[i] == x[j]) hit = j;
    if (hit >= 0) {
      P[(size_t)i * n + hit] = 1.0;
      continue;
    }
    double ell = 1.0;  // node polynomial prod_k (t - x_k)
    for (int k = 0; k < n; ++k) ell *= (t[i] - x[k]);
    for (int j = 0; j < n; ++j) P[(size_t)i * n + j] = ell * w[j] / (t[i] - x[j]);
  }
  return P;
}

}  // namespace

Consts make_consts(int p, int q) {
  Consts c;
  c.p = p;
  c.q = q;
  // Chebyshev extreme points, increasing: t_j = -cos(pi j/(p-1)), written as a
  // sine so that the set is exactly antisymmetric about 0.
  c.t.resize(p);
  for (int j = 0; j < p; ++j) c.t[j] = std::sin(kPi * (2.0 * j - (p - 1)) / (2.0 * (p - 1)));
  // Barycentric weights of the extreme points: (-1)^j, halved at both ends.
  std::vector<double> bw(p);
  for (int j = 0; j < p; ++j) bw[j] = ((j % 2) ? -1.0 : 1.0) * ((j == 0 || j == p - 1) ? 0.5 : 1.0);
  // Differentiation matrix.  Off-diagonal entries (bw_j / bw_i) / (t_i - t_j)
  // with the node difference written as 2 sin(pi (i+j) / (2(p-1)))
  // sin(pi (i-j) / (2(p-1))), free of the cancellation of t_i - t_j between
  // the clustered end nodes; the diagonal by the negative sum of the row (rows
  // of D annihilate constants).  The points are symmetric about 0, so D is
  // anti-centrosymmetric, D[p-1-i][p-1-j] = -D[i][j]: the upper rows are
  // computed and mirrored, so the symmetry holds bit for bit and kernels that
  // split grid lines into even and odd parts apply the same D.
  const int hr = (p + 1) / 2;  // computed rows (the centre row included for odd p)
  c.D.assign((size_t)p * p, 0.0);
  for (int i = 0; i < hr; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      const double dt = 2.0 * std::sin(kPi * (i + j) / (2.0 * (p - 1))) *
                        std::sin(kPi * (i - j) / (2.0 * (p - 1)));
      const double v = (bw[j] / bw[i]) / dt;
      c.D[(size_t)i * p + j] = v;
      diag -= v;
    }
    c.D[(size_t)i * p + i] = diag;
  }
  if (p % 2) {  // the centre row: exactly antisymmetric, zero diagonal
    const int m = p / 2;
    for (int j = m + 1; j < p; ++j) c.D[(size_t)m * p + j] = -c.D[(size_t)m * p + (p - 1 - j)];
    c.D[(size_t)m * p + m] = 0.0;
  }
  for (int i = hr; i < p; ++i)
    for (int j = 0; j < p; ++j)
      c.D[(size_t)i * p + j] = -c.D[(size_t)(p - 1 - i) * p + (p - 1 - j)];
  // D^2 = D D.  Off-diagonal entries of the upper rows summed with explicit
  // FMAs (the same bits on every host), mirrored into the lower rows (and the
  // centre row's right half); the diagonal of every row by the negative sum
  // of that row's off-diagonal entries in increasing column order.  Among the
  // constructions compared, this one put the 32 x 32-leaf Helmholtz solution
  // closest to the one with correctly rounded D and D^2 (the diagonal sums are
  // where the rounding of D^2 enters the smooth part of the solution most).
  // The mirrored rows' diagonals can differ from their mirror images by a unit
  // in the last place; every kernel reads this one table (the even / odd ones
  // add that difference back), so all paths apply the same operator.
  c.D2.assign((size_t)p * p, 0.0);
  for (int i = 0; i < hr; ++i)
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      double s = 0.0;
      for (int k = 0; k < p; ++k) s = std::fma(c.D[(size_t)i * p + k], c.D[(size_t)k * p + j], s);
      c.D2[(size_t)i * p + j] = s;
    }
  if (p % 2)
    for (int j = p / 2 + 1; j < p; ++j)
      c.D2[(size_t)(p / 2) * p + j] = c.D2[(size_t)(p / 2) * p + (p - 1 - j)];
  for (int i = hr; i < p; ++i)
    for (int j = 0; j < p; ++j)
      if (j != i) c.D2[(size_t)i * p + j] = c.D2[(size_t)(p - 1 - i) * p + (p - 1 - j)];
  for (int i = 0; i < p; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p; ++j)
      if (j != i) diag -= c.D2[(size_t)i * p + j];
    c.D2[(size_t)i * p + i] = diag;
  }
  // Gauss-Legendre points: Newton iteration on P_q from Chebyshev-like guesses.
  c.g.resize(q);
  c.gw.resize(q);
  for (int k = 0; k < q; ++k) {
    double x = -std::cos(kPi * (k + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int n = 2; n <= q; ++n) {
        double pn = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = pn;
      }
      double pq = (q == 1) ? x : p1;
      double pqm1 = (q == 1) ? 1.0 : p0;
      dp = q * (x * pq - pqm1) / (x * x - 1.0);
      double dx = pq / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute the derivative at the converged point for the weight
    double p0 = 1.0, p1 = x;
    for (int n = 2; n <= q; ++n) {
      double pn = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
      p0 = p1;
      p1 = pn;
    }
    double pq = (q == 1) ? x : p1, pqm1 = (q == 1) ? 1.0 : p0;
    dp = q * (x * pq - pqm1) / (x * x - 1.0);
    c.g[k] = x;
    c.gw[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  std::sort(c.g.begin(), c.g.end());
  // weights follow the sorted order (the rule is symmetric, recompute to be safe)
  for (int k = 0; k < q; ++k) {
    double x = c.g[k], p0 = 1.0, p1 = x;
    for (int n = 2; n <= q; ++n) {
      double pn = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
      p0 = p1;
      p1 = pn;
    }
    double pq = (q == 1) ? x : p1, pqm1 = (q == 1) ? 1.0 : p0;
    double dp = q * (x * pq - pqm1) / (x * x - 1.0);
    c.gw[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  c.Pg2c = lagrange_matrix(c.g, c.t);  // Step 1 (per side)
  c.Pc2g = lagrange_matrix(c.t, c.g);  // Step 4 (per side)
  return c;
}

std::vector<float> interior_flux_map(const Consts& c, double sx, double sy) {
  const int p = c.p, q = c.q, pi = p - 2, nq = 4 * q;
  std::vector<float> F((size_t)nq * pi * pi, 0.0f);
  for (int a = 1; a < p - 1; ++a)
    for (int b = 1; b < p - 1; ++b) {
      const size_t col = (size_t)((a - 1) * pi + (b - 1)) * nq;
      for (int k = 0; k < q; ++k) {
        const double pb = c.Pc2g[(size_t)k * p + b], pa = c.Pc2g[(size_t)k * p + a];
        F[col + 0 * q + k] = (float)(sy * pb * c.D[a]);                        // S: row 0
        F[col + 1 * q + k] = (float)(sx * pa * c.D[(size_t)(p - 1) * p + b]);  // E: column p-1
        F[col + 2 * q + k] = (float)(sy * pb * c.D[(size_t)(p - 1) * p + a]);  // N: row p-1
        F[col + 3 * q + k] = (float)(sx * pa * c.D[b]);                        // W: column 0
      }
    }
  return F;
}

// ------------------------------------------------------------------ the plan
namespace {

// Side offsets of a box's exterior ordering: S, E, N, W.
struct Sides {
  int S, E, N, W, n;
  Sides(int bx, int by, int q) {
    S = 0;
    E = bx * q;
    N = (bx + by) * q;
    W = (2 * bx + by) * q;
    n = 2 * (bx + by) * q;
  }
};

MergeShape make_shape(int split, int abx, int aby, int bbx, int bby, int q) {
  MergeShape s;
  s.split = split;
  Sides A(abx, aby, q), B(bbx, bby, q);
  int pbx = split == 0 ? abx + bbx : abx;
  int pby = split == 0 ? aby : aby + bby;
  Sides P(pbx, pby, q);
  s.na = A.n;
  s.nb = B.n;
  s.ne = P.n;
  s.src.assign(P.n, 0);
  auto alpha = [](int i) { return i; };
  auto beta = [](int i) { return -(i + 1); };
  if (split == 0) {
    // west alpha, east beta; J3 = alpha's east side = beta's west side
    s.m = aby * q;
    s.j3a = A.E;
    s.j3b = B.W;
    for (int k = 0; k < pbx * q; ++k) {
      s.src[P.S + k] = k < abx * q ? alpha(A.S + k) : beta(B.S + k - abx * q);
      s.src[P.N + k] = k < abx * q ? alpha(A.N + k) : beta(B.N + k - abx * q);
    }
    for (int k = 0; k < pby * q; ++k) {
      s.src[P.E + k] = beta(B.E + k);
      s.src[P.W + k] = alpha(A.W + k);
    }
  } else {
    // south alpha, north beta; J3 = alpha's north side = beta's south side
    s.m = abx * q;
    s.j3a = A.N;
    s.j3b = B.S;
    for (int k = 0; k < pbx * q; ++k) {
      s.src[P.S + k] = alpha(A.S + k);
      s.src[P.N + k] = beta(B.N + k);
    }
    for (int k = 0; k < pby * q; ++k) {
      s.src[P.E + k] = k < aby * q ? alpha(A.E + k) : beta(B.E + k - aby * q);
      s.src[P.W + k] = k < aby * q ? alpha(A.W + k) : beta(B.W + k - aby * q);
    }
  }
  s.cmap_a.assign(s.na, 0);
  s.cmap_b.assign(s.nb, 0);
  for (int j = 0; j < s.m; ++j) {
    s.cmap_a[s.j3a + j] = -(j + 1);
    s.cmap_b[s.j3b + j] = -(j + 1);
  }
  for (int k = 0; k < s.ne; ++k) {
    int v = s.src[k];
    if (v >= 0)
      s.cmap_a[v] = k;
    else
      s.cmap_b[-v - 1] = k;
  }
  return s;
}

}  // namespace

Plan make_forest(const std::vector<ProblemSpec>& specs) {
  Plan pl;
  std::map<std::tuple<int, int, int, int, int, int>, int> shape_ids;
  int leaf0 = 0;
  int64_t rff = 0;
  for (size_t k = 0; k < specs.size(); ++k) {
    const ProblemSpec& sp = specs[k];
    ProbInfo pi;
    pi.s = sp;
    pi.leaf0 = leaf0;
    pi.nl = sp.nx * sp.ny;
    pi.nbnd = 2 * (sp.nx + sp.ny) * sp.q;
    pi.hx = (sp.x1 - sp.x0) / sp.nx;
    pi.hy = (sp.y1 - sp.y0) / sp.ny;
    pi.rff_off = rff;
    pi.root = (int)pl.boxes.size();
    leaf0 += pi.nl;
    rff += pi.nbnd;
    pl.leaf_box.resize(leaf0, -1);
    pl.leaf_prob.resize(leaf0, (int)k);
    // breadth-first construction keeps parent index < child index (Section 2)
    Box root;
    root.ix0 = 0;
    root.iy0 = 0;
    root.bx = sp.nx;
    root.by = sp.ny;
    root.prob = (int)k;
    pl.boxes.push_back(root);
    for (size_t b = pi.root; b < pl.boxes.size(); ++b) {
      Box cur = pl.boxes[b];
      if (cur.bx == 1 && cur.by == 1) {
        pl.boxes[b].leaf = pi.leaf0 + cur.iy0 * sp.nx + cur.ix0;
        pl.leaf_box[pl.boxes[b].leaf] = (int)b;
        continue;
      }
      Box a, c;
      int split = (cur.bx >= cur.by) ? 0 : 1;  // split the longer side; ties split x
      if (split == 0) {
        int h = cur.bx / 2;
        a = {cur.ix0, cur.iy0, h, cur.by};
        c = {cur.ix0 + h, cur.iy0, cur.bx - h, cur.by};
      } else {
        int h = cur.by / 2;
        a = {cur.ix0, cur.iy0, cur.bx, h};
        c = {cur.ix0, cur.iy0 + h, cur.bx, cur.by - h};
      }
      a.parent = c.parent = (int)b;
      a.prob = c.prob = (int)k;
      pl.boxes[b].split = split;
      pl.boxes[b].child[0] = (int)pl.boxes.size();
      pl.boxes.push_back(a);
      pl.boxes[b].child[1] = (int)pl.boxes.size();
      pl.boxes.push_back(c);
    }
    // heights bottom-up within this problem (children have larger indices)
    for (int b = (int)pl.boxes.size() - 1; b >= pi.root; --b) {
      Box& x = pl.boxes[b];
      x.ne = 2 * (x.bx + x.by) * sp.q;
      if (x.child[0] >= 0)
        x.height = 1 + std::max(pl.boxes[x.child[0]].height, pl.boxes[x.child[1]].height);
    }
    pi.height = pl.boxes[pi.root].height;
    pl.height = std::max(pl.height, pi.height);
    // root exterior (S, E, N, W increasing) from f (counter-clockwise from (x0,y0))
    std::vector<int> m(pi.nbnd);
    Sides R(sp.nx, sp.ny, sp.q);
    const int nx = sp.nx, ny = sp.ny, q = sp.q;
    for (int kk = 0; kk < nx * q; ++kk) {
      m[R.S + kk] = kk;
      m[R.N + kk] = (nx + ny) * q + (nx * q - 1 - kk);
    }
    for (int kk = 0; kk < ny * q; ++kk) {
      m[R.E + kk] = nx * q + kk;
      m[R.W + kk] = (2 * nx + ny) * q + (ny * q - 1 - kk);
    }
    pl.root_from_f.insert(pl.root_from_f.end(), m.begin(), m.end());
    pl.probs.push_back(pi);
  }
  pl.levels.assign(pl.height + 1, {});
  for (int b = 0; b < (int)pl.boxes.size(); ++b) {
    Box& x = pl.boxes[b];
    if (x.child[0] < 0) continue;
    const Box& A = pl.boxes[x.child[0]];
    const Box& B = pl.boxes[x.child[1]];
    const int q = specs[x.prob].q;
    auto key = std::make_tuple(x.split, A.bx, A.by, B.bx, B.by, q);
    auto it = shape_ids.find(key);
    if (it == shape_ids.end()) {
      pl.shapes.push_back(make_shape(x.split, A.bx, A.by, B.bx, B.by, q));
      it = shape_ids.emplace(key, (int)pl.shapes.size() - 1).first;
    }
    x.shape = it->second;
    pl.levels[x.height].push_back(b);
  }
  int64_t off = 0;
  for (auto& x : pl.boxes) {
    x.ext_off = off;
    off += x.ne;
  }
  pl.ext_total = off;
  return pl;
}

void cheb_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int p,
                      double* xy) {
  Consts c = make_consts(p, 1);
  const double hx = (x1 - x0) / nx, hy = (y1 - y0) / ny;
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix) {
      size_t l = (size_t)iy * nx + ix;
      for (int a = 0; a < p; ++a)
        for (int b = 0; b < p; ++b) {
          size_t n = (l * p + a) * p + b;
          xy[2 * n] = x0 + ix * hx + 0.5 * (c.t[b] + 1.0) * hx;
          xy[2 * n + 1] = y0 + iy * hy + 0.5 * (c.t[a] + 1.0) * hy;
        }
    }
}

void boundary_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int q,
                          double* xy) {
  Consts c = make_consts(std::max(q, 2), q);
  const double hx = (x1 - x0) / nx, hy = (y1 - y0) / ny;
  size_t n = 0;
  auto put = [&](double x, double y) {
    xy[2 * n] = x;
    xy[2 * n + 1] = y;
    ++n;
  };
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < q; ++k) put(x0 + i * hx + 0.5 * (c.g[k] + 1.0) * hx, y0);
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k < q; ++k) put(x1, y0 + j * hy + 0.5 * (c.g[k] + 1.0) * hy);
  for (int i = nx - 1; i >= 0; --i)
    for (int k = q - 1; k >= 0; --k) put(x0 + i * hx + 0.5 * (c.g[k] + 1.0) * hx, y1);
  for (int j = ny - 1; j >= 0; --j)
    for (int k = q - 1; k >= 0; --k) put(x0, y0 + j * hy + 0.5 * (c.g[k] + 1.0) * hy);
}

}  // namespace hps
