// Host-side check of the Zernike evaluation of the kernels for bases above
// N_p = 8 (paper_1608_04607_gb300/csrc/zernike_wide.h, shared with the CUDA
// code): reads Np and points "px py", prints per point one line of the N_b
// values in basis order evaluated in FP64, one in FP32, and a line with the
// number of times each basis index was emitted.
#include <cstdio>
#include <vector>

#include "zernike_wide.h"

int main() {
  int Np = 0;
  if (std::scanf("%d", &Np) != 1 || Np < 0 || Np > dfm::zw::kNpW) return 1;
  const int nb = (Np + 1) * (Np + 2) / 2;
  double px = 0, py = 0;
  while (std::scanf("%lf %lf", &px, &py) == 2) {
    std::vector<double> zd(nb, 0.0);
    std::vector<float> zf(nb, 0.f);
    std::vector<int> cnt(nb, 0);
    bool bad = false;
    dfm::zw::zernike_wide<double>(Np, px, py, [&](int idx, int n, int m, double z) {
      if (idx < 0 || idx >= nb || idx != (n * (n + 2) + m) / 2) {
        bad = true;
        return;
      }
      zd[idx] = z;
      ++cnt[idx];
    });
    dfm::zw::zernike_wide<float>(Np, (float)px, (float)py, [&](int idx, int, int, float z) {
      if (idx >= 0 && idx < nb) zf[idx] = z;
    });
    if (bad) return 2;
    for (int i = 0; i < nb; ++i) std::printf("%.17g%c", zd[i], i + 1 < nb ? ' ' : '\n');
    for (int i = 0; i < nb; ++i) std::printf("%.9g%c", (double)zf[i], i + 1 < nb ? ' ' : '\n');
    for (int i = 0; i < nb; ++i) std::printf("%d%c", cnt[i], i + 1 < nb ? ' ' : '\n');
  }
  return 0;
}
