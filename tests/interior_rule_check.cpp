// Host-side check of the split polar interior-density rule
// (paper_1608_04607_gb300/csrc/interior_rule.cuh, shared with the CUDA
// kernel): reads n, the n-point Gauss-Legendre nodes and weights, then cases
// of one face (P0 P1 P2, inward normal, e1, e2) and a point r, and prints
// every node as "w R dx dy".
#include <cstdio>
#include <vector>

#include "interior_rule.cuh"

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1 || n < 1 || n > 64) return 1;
  std::vector<double> gx(n), gw(n);
  for (int i = 0; i < n; ++i)
    if (std::scanf("%lf", &gx[i]) != 1) return 1;
  for (int i = 0; i < n; ++i)
    if (std::scanf("%lf", &gw[i]) != 1) return 1;
  double P[3][3], nin[3], e1[3], e2[3], r[3];
  while (true) {
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i)
      for (int c = 0; c < 3 && ok; ++c) ok = std::scanf("%lf", &P[i][c]) == 1;
    for (double* a : {nin, e1, e2, r})
      for (int c = 0; c < 3 && ok; ++c) ok = std::scanf("%lf", &a[c]) == 1;
    if (!ok) break;
    for (int k = 0; k < 6 * n * n; ++k) {
      const dfm::rule::PolarNode q = dfm::rule::polar_node(P, nin, e1, e2, r, n, k, gx.data(), gw.data());
      std::printf("%.17g %.17g %.17g %.17g\n", q.w, q.R, q.dx, q.dy);
    }
  }
  return 0;
}
