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
  std::vector<double> g;     // q Gauss-Legendre points on [-1,1], increasing
  std::vector<double> gw;    // their weights
  std::vector<double> Pg2c;  // p x q row-major: value at t_i of the degree q-1 interpolant
  std::vector<double> Pc2g;  // q x p row-major: value at g_k of the degree p-1 interpolant
};
Consts make_consts(int p, int q);

// --------------------------------------------------------------------- plan
struct Box {
  int ix0, iy0, bx, by;  // leaf extent
  int parent = -1;
  int child[2] = {-1, -1};
  int split = -1;        // 0: children share a vertical edge (west alpha, east beta)
                         // 1: children share a horizontal edge (south alpha, north beta)
  int height = 0;        // 0 for a leaf
  int leaf = -1;         // leaf index l = iy*nx + ix for a leaf box
  int ne = 0;            // exterior size 2*(bx+by)*q
  int shape = -1;        // merge shape index (parents only)
  int64_t ext_off = 0;   // offset (in nodes) of this box in the exterior-value pool
};

// Geometry of one merge, shared by all merges with equal child extents.
struct MergeShape {
  int split, m, ne, na, nb;  // |J3|, parent / alpha / beta exterior sizes
  int j3a, j3b;              // first J3 position in alpha's / beta's exterior
  std::vector<int> src;      // ne: parent position -> alpha index (>= 0) or beta index -(v+1)
  std::vector<int> cmap_a;   // na: alpha position -> parent position (>= 0) or J3 index -(j+1)
  std::vector<int> cmap_b;   // nb: same for beta
};

struct Plan {
  double x0, x1, y0, y1;
  int nx, ny, p, q;
  std::vector<Box> boxes;           // boxes[0] is the root
  std::vector<int> leaf_box;        // leaf l -> box
  std::vector<MergeShape> shapes;
  std::vector<std::vector<int>> levels;  // levels[h] (h >= 1): parent boxes of height h
  int height = 0;                   // root height
  int64_t ext_total = 0;            // sum of ne over boxes
  std::vector<int> root_from_f;     // root exterior position -> index into f
};
Plan make_plan(double x0, double x1, double y0, double y1, int nx, int ny, int p, int q);

void cheb_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int p,
                      double* xy);
void boundary_node_coords(double x0, double x1, double y0, double y1, int nx, int ny, int q,
                          double* xy);

}  // namespace hps
