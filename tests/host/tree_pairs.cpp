// Host harness for tests/test_tree_host.py: the tree of tree_core.cuh (the header the
// tree neighbour-list kernels use) built over given fixed-point coordinates in a
// given order, queried for every particle; writes every pair i < j whose
// minimum-image distance (FP64 on the fixed-point difference) is below r.
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../paper_1308_5587_gb300/csrc/tree_core.cuh"

using namespace gbmd;

extern "C" long long tree_pairs(int n, const uint32_t* u, const int* order, const double* L,
                                double r, long long cap, int* pairs) {
  const int P = tree_leaves(n);
  std::vector<TreeBox> box(2 * (size_t)P);
  for (int b = 0; b < P; ++b) {
    TreeBox t = tree_empty_box();
    for (int k = 0; k < TREE_LEAF; ++k) {
      const int m = b * TREE_LEAF + k;
      if (m < n) {
        const int i = order[m];
        tree_box_add(t, u[3 * i], u[3 * i + 1], u[3 * i + 2]);
      }
    }
    box[P + b] = t;
  }
  for (int k = P - 1; k >= 1; --k) box[k] = tree_box_union(box[2 * k], box[2 * k + 1]);
  float fs[3];
  for (int a = 0; a < 3; ++a) fs[a] = (float)(L[a] / 4294967296.0);
  const float r2 = (float)(r * r * (1.0 + 1e-5));
  long long cnt = 0;
  for (int i = 0; i < n; ++i) {
    const int seen = tree_query(box.data(), P, u[3 * i], u[3 * i + 1], u[3 * i + 2], fs[0], fs[1],
                                fs[2], r2, 2 * P, [&](int b) {
      for (int k = 0; k < TREE_LEAF; ++k) {
        const int m = b * TREE_LEAF + k;
        if (m >= n) break;
        const int j = order[m];
        if (j <= i) continue;
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
          const double d = (double)(int32_t)(u[3 * i + a] - u[3 * j + a]) * (L[a] / 4294967296.0);
          d2 += d * d;
        }
        if (d2 < r * r) {
          if (cnt < cap) {
            pairs[2 * cnt] = i;
            pairs[2 * cnt + 1] = j;
          }
          ++cnt;
        }
      }
    });
    if (seen < 0) return -1;
  }
  return cnt;
}
