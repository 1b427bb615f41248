// Internal declarations shared by the translation units of libhps.
//
// Layout conventions (all device matrices are column-major, element (i, j) of
// an m-row matrix at i + j*ld):
//   * A box's exterior Gauss nodes (its I_e, Section 2) are ordered by side,
//     south, east, north, west, each side in increasing coordinate and made of
//     q nodes per leaf segment.  A leaf therefore has 4q exterior nodes.
//   * T of a box with ne exterior nodes is ne x ne: T(i, j) = d flux_i / d u_j,
//     the flux being d/dy on horizontal sides and d/dx on vertical sides, in the
//     global direction (Section 2, vector v).
//   * S of a merge is m x ne (m = |J3|, ne = parent's exterior size); its
//     columns follow the parent's exterior order.
//   * Y of a leaf is ni x 4q, ni = (p-2)^2 interior Chebyshev nodes in
//     row-major (y-major) order.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hps {

// ------------------------------------------------------------ 1-D constants
// Section 3.1 (Chebyshev grid, spectral differentiation) and Section 3.2
// (Steps 1 and 4: re-tabulation between Gauss and Chebyshev points on a side).
struct Consts {
  int p = 0, q = 0;
  std::vector<double> t;     // p Chebyshev extreme points on [-1,1], increasing
  std::vector<double> D;     // p x p differentiation matrix, row-major D[i*p+j]
  std::vector<double> D2;    // p x p, D*D, exactly centrosymmetric
  std::vector<double> g;     // q Gauss-Legendre points on [-1,1], increasing
  std::vector<double> gw;    // their weights
  std::vector<double> Pg2c;  // p x q row-major: value at t_i of the degree q-1 interpolant
  std::vector<double> Pc2g;  // q x p row-major: value at g_k of the degree p-1 interpolant
};
Consts make_consts(int p, int q);
// Side fluxes (Section 3.2, Steps 3-4: d/dy on S and N, d/dx on E and W, then
// the side interpolant at the q Gauss points) of values at the interior
// Chebyshev nodes only: the 4q x (p-2)^2 map L4 L3 restricted to the interior
// columns, for a leaf with scalings sx = 2/hx, sy = 2/hy; column-major (ld 4q),
// rows in the order S, E, N, W, columns (a-1)(p-2) + (b-1).
std::vector<float> interior_flux_map(const Consts& c, double sx, double sy);

// --------------------------------------------------------------------- plan
// One plan may hold several independent problems (a forest): every problem
// has its own tree, and the leaves / merges of all problems at the same height
// are processed by the same batched launches.
struct ProblemSpec {
  double x0, x1, y0, y1;
  int nx, ny, p, q;
};

struct ProbInfo {
  ProblemSpec s;
  int root = 0;           // box index of the problem's root
  int leaf0 = 0, nl = 0;  // global leaf range (leaf l = leaf0 + iy*nx + ix)
  int height = 0;
  int nbnd = 0;
  int64_t rff_off = 0;    // offset of this problem's map in root_from_f
  double hx = 0, hy = 0;
};

struct Box {
  int ix0, iy0, bx, by;  // leaf extent
  int parent = -1;
  int child[2] = {-1, -1};
  int split = -1;        // 0: children share a vertical edge (west alpha, east beta)
                         // 1: children share a horizontal edge (south alpha, north beta)
  int height = 0;        // 0 for a leaf
  int leaf = -1;         // global leaf index for a leaf box
  int prob = 0;          // problem this box belongs to
  int ne = 0;            // exterior size 2*(bx+by)*q
  int shape = -1;        // merge shape index (parents only)
  int64_t ext_off = 0;   // offset (in nodes) of this box in the exterior-value pool
};

// Geometry of one merge, shared by all merges with equal child extents and q.
struct MergeShape {
  int split, m, ne, na, nb;  // |J3|, parent / alpha / beta exterior sizes
  int j3a, j3b;              // first J3 position in alpha's / beta's exterior
  std::vector<int> src;      // ne: parent position -> alpha index (>= 0) or beta index -(v+1)
  std::vector<int> cmap_a;   // na: alpha position -> parent position (>= 0) or J3 index -(j+1)
  std::vector<int> cmap_b;   // nb: same for beta
};

struct Plan {
  std::vector<ProbInfo> probs;
  std::vector<Box> boxes;
  std::vector<int> leaf_box;        // global leaf -> box
  std::vector<int> leaf_prob;       // global leaf -> problem
  std::vector<MergeShape> shapes;
  std::vector<std::vector<int>> levels;  // levels[h] (h >= 1): parent boxes of height h, all problems
  int height = 0;                   // largest root height
  int64_t ext_total = 0;            // sum of ne over boxes
  std::vector<int> root_from_f;     // per problem: root exterior position -> index into its f
  int n_leaves() const { return (int)leaf_box.size(); }
};
Plan make_forest(const std::vector<ProblemSpec>& specs);

void cheb_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int p,
                      double* xy);
void boundary_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int q,
                          double* xy);

}  // namespace hps
