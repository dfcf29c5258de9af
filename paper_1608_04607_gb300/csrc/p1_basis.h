// The linear spatial basis on each face (DFM_BASIS(Np, 1)), for the
// assembly and interior-density kernels of wide.cu.  Plain arithmetic with no
// CUDA intrinsics, so the same functions serve the device kernels and a
// host-side check against the oracle's clipping route.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define DFM_P1_HD __host__ __device__
#else
#define DFM_P1_HD
#endif

namespace dfm {
namespace p1 {

// sqrt|T| phi_a at the face's vertex k (frame order): the orthonormal affine
// functions from Gram-Schmidt of (1, l_1, l_2), l_k the barycentric coordinate
// of vertex k: 1; sqrt(18) (l_1 - 1/3); sqrt(24) (l_2 - 1/3 + (l_1 - 1/3) / 2).
DFM_P1_HD inline float value(int a, int k) {
  if (a == 0) return 1.f;
  if (a == 1) return 4.24264068712f * ((k == 1 ? 1.f : 0.f) - 1.f / 3.f);
  return 4.89897948557f * ((k == 2 ? 1.f : 0.f) - 1.f / 3.f + 0.5f * ((k == 1 ? 1.f : 0.f) - 1.f / 3.f));
}
DFM_P1_HD inline double value_d(int a, int k) {
  if (a == 0) return 1.0;
  if (a == 1) return 4.2426406871192851 * ((k == 1 ? 1.0 : 0.0) - 1.0 / 3.0);
  return 4.8989794855663561 * ((k == 2 ? 1.0 : 0.0) - 1.0 / 3.0 + 0.5 * ((k == 1 ? 1.0 : 0.0) - 1.0 / 3.0));
}

// F(j, k)(x) = Int_0^1 t^j (1 - t)^k e^{-x t} dt for (j, k) = (2, 1), (1, 2),
// (0, 3): the moments of the damping over the visible triangle OBC (L = L_O
// l_O, x = mu L_O).  Below x = 2 the Taylor series sum_m (-x)^m / m!
// (j + m)! k! / (j + m + k + 1)! (22 terms: the first omitted one is below
// 2^22 / 22! < 4e-15);
// above, the exact I_n = Int_0^1 t^n e^{-x t} dt = n! / x^(n+1) (1 - e^{-x}
// sum_{i<=n} x^i / i!) combined, whose cancellation is mild there.
DFM_P1_HD inline void p1_moments(float x, float& f21, float& f12, float& f03) {
  if (x < 2.f) {
    float t21 = 1.f / 12.f, t12 = 1.f / 12.f, t03 = 1.f / 4.f;
    f21 = t21;
    f12 = t12;
    f03 = t03;
#pragma unroll
    for (int m = 0; m < 22; ++m) {
      // T_{m+1} / T_m = -x / (m + 1) * (j + m + 1) / (j + m + k + 2), j + k = 3
      const float c = -x / (float)(m + 1) / (float)(m + 5);
      t21 *= c * (float)(m + 3);
      t12 *= c * (float)(m + 2);
      t03 *= c * (float)(m + 1);
      f21 += t21;
      f12 += t12;
      f03 += t03;
    }
    return;
  }
  const float e = expf(-x), ix = 1.f / x;
  const float i0 = ix * (1.f - e);
  const float i1 = ix * ix * (1.f - e * (1.f + x));
  const float i2 = 2.f * ix * ix * ix * (1.f - e * (1.f + x + 0.5f * x * x));
  const float i3 = 6.f * ix * ix * ix * ix * (1.f - e * (1.f + x + 0.5f * x * x + x * x * x / 6.f));
  f21 = i2 - i3;
  f12 = i1 - 2.f * i2 + i3;
  f03 = i0 - 3.f * i1 + 3.f * i2 - i3;
}

// Spatial matrix M[b][a] = Int_{OBC} (sqrt|T_l| phi_a)(s) (sqrt|T_l'| psi_b)(y(s)) e^{-mu L(s)} ds
// of one direction (Sec. 3.3 with the linear basis): the visible triangle
// OBC has O with barycentrics (s_A, s_B+, s_C+) / den on the source face, L
// affine with L(O) = L_O and zero on BC, and the exit point y(s) is the
// affine image with y(O) = Y_O of barycentrics (d_z, s_B-, s_C-) / den on the
// destination face BCD (x+ = max(x, 0), x- = max(-x, 0)).  Both integrand
// factors are barycentric interpolations of their values at (O, B, C) and
// (Y_O, B, C), so M = 2 |OBC| sum_ij phi_a(V_i) psi_b(W_j) k_ij with
// k_OO = F21, k_OB = k_OC = F12 / 2, k_BB = k_CC = F03 / 3, k_BC = F03 / 6.
// pos: source-face positions of A, B, C, receiving-face positions of B, C, D.
DFM_P1_HD inline void p1_spatial(float sA, float sB, float sC, float dz, float area_obc, float x,
                                           const int* pos, float M[3][3]) {
  const float den = sA + fmaxf(sB, 0.f) + fmaxf(sC, 0.f);
  const float inv = 1.f / den;
  const float oa = sA * inv, ob = fmaxf(sB, 0.f) * inv, oc = fmaxf(sC, 0.f) * inv;
  const float yd = dz * inv, yb = fmaxf(-sB, 0.f) * inv, yc = fmaxf(-sC, 0.f) * inv;
  float f21, f12, f03;
  p1_moments(x, f21, f12, f03);
  const float kOO = f21, kOB = 0.5f * f12, kBB = f03 / 3.f, kBC = f03 / 6.f;
  float phO[3], phB[3], phC[3], psY[3], psB[3], psC[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    phB[a] = value(a, pos[1]);
    phC[a] = value(a, pos[2]);
    phO[a] = oa * value(a, pos[0]) + ob * phB[a] + oc * phC[a];
    psB[a] = value(a, pos[3]);
    psC[a] = value(a, pos[4]);
    psY[a] = yd * value(a, pos[5]) + yb * psB[a] + yc * psC[a];
  }
  const float s2 = 2.f * area_obc;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float gO = psY[b] * kOO + (psB[b] + psC[b]) * kOB;  // sum_j psi_b(W_j) k_Oj
    const float gB = psY[b] * kOB + psB[b] * kBB + psC[b] * kBC;
    const float gC = psY[b] * kOB + psB[b] * kBC + psC[b] * kBB;
#pragma unroll
    for (int a = 0; a < 3; ++a) M[b][a] = s2 * (phO[a] * gO + phB[a] * gB + phC[a] * gC);
  }
}

}  // namespace p1
}  // namespace dfm
