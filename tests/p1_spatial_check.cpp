// Host-side check of the closed-form spatial matrix of the linear spatial
// basis (paper_1608_04607_gb300/csrc/p1_basis.h, shared with the CUDA
// assembly): reads lines "sA sB sC dz area_obc x pA pB pC rB rC rD" and prints
// the nine entries M[b][a] (row-major) per line.
#include <cstdio>

#include "p1_basis.h"

int main() {
  float sA, sB, sC, dz, area, x;
  int pos[6];
  while (std::scanf("%f %f %f %f %f %f %d %d %d %d %d %d", &sA, &sB, &sC, &dz, &area, &x, &pos[0], &pos[1], &pos[2],
                    &pos[3], &pos[4], &pos[5]) == 12) {
    float M[3][3];
    dfm::p1::p1_spatial(sA, sB, sC, dz, area, x, pos, M);
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) std::printf("%.9g%c", (double)M[b][a], (b == 2 && a == 2) ? '\n' : ' ');
  }
  return 0;
}
