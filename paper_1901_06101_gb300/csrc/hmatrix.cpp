// Host-side geometry for kernel matrices whose rows and columns are points:
// the KD-tree ordering the paper assumes before compressing an off-diagonal
// block (Sec. 5: rows and columns permuted by a KD-tree partitioning), and the
// admissible blocks of a hierarchical-matrix partition built on the same
// trees, each of which can be compressed by H-BACA (Sec. 1: H-BACA as the
// low-rank compression tool of hierarchical matrices).
//
// The cluster tree halves an index range [s0, s0 + s) into a first child of
// ceil(s / 2) and a second of floor(s / 2) indices -- the index tree of H-BACA
// (Alg. 3) -- after sorting the node's points along the widest side of their
// bounding box, so every H-BACA leaf of an ordered point set is a spatial cell.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "hbaca.h"
#include "run.h"

namespace {

struct Box {
  std::vector<double> lo, hi;
};

Box bounding_box(const double* pts, int dim, const int64_t* idx, int64_t count) {
  Box b{std::vector<double>(dim, INFINITY), std::vector<double>(dim, -INFINITY)};
  for (int64_t t = 0; t < count; ++t)
    for (int k = 0; k < dim; ++k) {
      const double v = pts[idx[t] * dim + k];
      b.lo[k] = std::min(b.lo[k], v);
      b.hi[k] = std::max(b.hi[k], v);
    }
  return b;
}

// Order idx[s0 .. s0+s) so that every node of the halving tree down to nodes
// of at most `leaf` points holds one side of a split along its widest side.
void kd_order(const double* pts, int dim, std::vector<int64_t>& idx, int64_t s0, int64_t s, int64_t leaf) {
  if (s <= leaf || s < 2) return;
  const Box b = bounding_box(pts, dim, idx.data() + s0, s);
  int k = 0;
  for (int j = 1; j < dim; ++j)
    if (b.hi[j] - b.lo[j] > b.hi[k] - b.lo[k]) k = j;
  const int64_t a = (s + 1) / 2;
  auto first = idx.begin() + s0;
  std::nth_element(first, first + a, first + s, [&](int64_t u, int64_t v) {
    const double pu = pts[u * dim + k], pv = pts[v * dim + k];
    return pu < pv || (pu == pv && u < v);
  });
  kd_order(pts, dim, idx, s0, a, leaf);
  kd_order(pts, dim, idx, s0 + a, s - a, leaf);
}

double box_diam(const Box& b) {
  double s = 0.0;
  for (size_t k = 0; k < b.lo.size(); ++k) s += (b.hi[k] - b.lo[k]) * (b.hi[k] - b.lo[k]);
  return std::sqrt(s);
}

double box_dist(const Box& a, const Box& b) {
  double s = 0.0;
  for (size_t k = 0; k < a.lo.size(); ++k) {
    const double g = std::max({0.0, b.lo[k] - a.hi[k], a.lo[k] - b.hi[k]});
    s += g * g;
  }
  return std::sqrt(s);
}

struct Blocks {
  const double* x;
  const double* y;
  int dim;
  int64_t leaf;
  double eta;
  std::vector<int64_t> ix, iy;  // identity index lists (points are already ordered)
  std::vector<int64_t> out;     // (r0, m, c0, n, admissible) per block
};

void partition(Blocks& B, int64_t r0, int64_t m, int64_t c0, int64_t n) {
  const Box bx = bounding_box(B.x, B.dim, B.ix.data() + r0, m);
  const Box by = bounding_box(B.y, B.dim, B.iy.data() + c0, n);
  const bool adm = std::min(box_diam(bx), box_diam(by)) <= B.eta * box_dist(bx, by);
  const bool leaf_x = m <= B.leaf || m < 2, leaf_y = n <= B.leaf || n < 2;
  if (adm || (leaf_x && leaf_y)) {
    B.out.insert(B.out.end(), {r0, m, c0, n, adm ? 1 : 0});
    return;
  }
  const int64_t am = (m + 1) / 2, an = (n + 1) / 2;
  if (leaf_y || (!leaf_x && m >= n)) {  // split the rows
    partition(B, r0, am, c0, n);
    partition(B, r0 + am, m - am, c0, n);
  } else {  // split the columns
    partition(B, r0, m, c0, an);
    partition(B, r0, m, c0 + an, n - an);
  }
}

}  // namespace

extern "C" {

hbaca_status hbaca_kdtree_order(const double* points, int64_t n, int32_t dim, int64_t leaf, int64_t* perm) {
  if (!points || !perm || n < 1 || dim < 1 || dim > 1024 || leaf < 1)
    return hbaca::record_error(HBACA_INVALID_ARG, "need points, perm, n >= 1, 1 <= dim <= 1024, leaf >= 1");
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  kd_order(points, dim, idx, 0, n, leaf);
  std::memcpy(perm, idx.data(), (size_t)n * sizeof(int64_t));
  hbaca::record_error(HBACA_OK, "");
  return HBACA_OK;
}

int64_t hbaca_hmatrix_blocks(const double* x, int64_t m, const double* y, int64_t n, int32_t dim, int64_t leaf,
                             double eta, int64_t* blocks, int64_t max_blocks) {
  if (!x || !y || m < 1 || n < 1 || dim < 1 || dim > 1024 || leaf < 1 || !(eta > 0.0)) {
    hbaca::record_error(HBACA_INVALID_ARG, "need x, y, m, n >= 1, 1 <= dim <= 1024, leaf >= 1, eta > 0");
    return -1;
  }
  Blocks B{x, y, dim, leaf, eta, std::vector<int64_t>(m), std::vector<int64_t>(n), {}};
  std::iota(B.ix.begin(), B.ix.end(), 0);
  std::iota(B.iy.begin(), B.iy.end(), 0);
  partition(B, 0, m, 0, n);
  const int64_t count = (int64_t)B.out.size() / 5;
  if (blocks) std::memcpy(blocks, B.out.data(), (size_t)std::min(count, std::max<int64_t>(max_blocks, 0)) * 5 * 8);
  hbaca::record_error(HBACA_OK, "");
  return count;
}

}  // extern "C"
