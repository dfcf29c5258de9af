// Zernike polynomials of orders up to 20 for the kernels of bases above
// N_p = 8 (wide.cu).  Plain arithmetic with no CUDA intrinsics, so the same
// function serves the device kernels and a host-side check against the
// oracle's closed form.
#pragma once

#include "launch_geometry.h"

#ifdef __CUDACC__
#define DFM_ZW_HD __host__ __device__
#else
#define DFM_ZW_HD
#endif

namespace dfm {
namespace zw {

constexpr int kNpW = geom::kWideMaxNp;

// Z_n^m(px, py) for n = 0..Np (Np <= 20), m-major: for each m >= 0 the
// angular factors rho^m cos(m phi), rho^m sin(m phi) as Re, Im of
// (px + i py)^m, and the radial factor Q_n^m = R_n^m / rho^m by Kintner's
// three-term recurrence in n at fixed m (E. C. Kintner, Optica Acta 23, 1976):
//   Q_m^m = 1,  Q_{m+2}^m = (m + 2) rho^2 - (m + 1),
//   K1 Q_n^m = (K2 rho^2 + K3) Q_{n-2}^m + K4 Q_{n-4}^m,
//   K1 = (n + m)(n - m)(n - 2)/2, K2 = 2n(n - 1)(n - 2),
//   K3 = -m^2 (n - 1) - n(n - 1)(n - 2), K4 = -n(n + m - 2)(n - m - 2)/2.
// It defines the same polynomials as the recursion of Sec. 3.1 (zernike<NP>
// in node.cuh) but holds two radial values instead of two whole orders, which
// keeps these kernels' registers for their accumulators.  emit(idx, n, m, z)
// receives Z_n^m at basis index idx = (n (n + 2) + m) / 2 (m < 0: the sine
// function).
template <typename T, typename Emit>
DFM_ZW_HD inline void zernike_wide(int Np, T px, T py, Emit&& emit) {
  const T r2 = px * px + py * py;
  T cr = T(1), ci = T(0);
#pragma unroll
  for (int m = 0; m <= kNpW; ++m) {
    if (m > Np) break;
    if (m > 0) {
      const T t = cr * px - ci * py;
      ci = cr * py + ci * px;
      cr = t;
    }
    T qa = T(0), qb = T(0);  // Q_{n-4}^m, Q_{n-2}^m
#pragma unroll
    for (int n = m; n <= kNpW; n += 2) {
      if (n > Np) break;
      T qn;
      if (n == m) {
        qn = T(1);
      } else if (n == m + 2) {
        qn = T(m + 2) * r2 - T(m + 1);
      } else {
        const T k1 = T((n + m) * (n - m) * (n - 2) / 2);
        const T k2 = T(2 * n * (n - 1) * (n - 2));
        const T k3 = T(-m * m * (n - 1) - n * (n - 1) * (n - 2));
        const T k4 = T(-n * (n + m - 2) * (n - m - 2) / 2);
        qn = ((k2 / k1) * r2 + k3 / k1) * qb + (k4 / k1) * qa;
      }
      qa = qb;
      qb = qn;
      if (m == 0) {
        emit((n * (n + 2)) / 2, n, 0, qn);
      } else {
        emit((n * (n + 2) + m) / 2, n, m, qn * cr);
        emit((n * (n + 2) - m) / 2, n, -m, qn * ci);
      }
    }
  }
}

}  // namespace zw
}  // namespace dfm
