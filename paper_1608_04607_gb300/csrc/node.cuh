// Node arithmetic shared by the assembly and adjoint kernels (Sec. 3.1-3.4):
// per-pair constants, direction patches, the closed-form spatial integral
// and the Zernike recursion.  Included by assemble.cu, adjoint.cu and source.cu; every
// symbol is TU-local (anonymous namespace).
#pragma once

#include <math.h>

#include "dfm_internal.cuh"

namespace dfm {
namespace {

// ---------------------------------------------------------------------------
// Per-pair constants (FP32, in the source face frame: x = e1, y = e2, z = n)
// ---------------------------------------------------------------------------
struct PairConst {
  float mA[3], mB[3], mC[3];  // s_X(d) = m_X . d
  float R1[3], R2[3];         // receiving face axes e1', e2' in the source frame
  float A[3], B[3], C[3], D[3];  // tet vertices in the source frame
  float area_src;             // |ABC|
  float mu;                   // damping of the tet
  float scale;                // lambda / sqrt(|T_l| |T_l'|)
  int out_row, slot;          // destination of the block
  // heterogeneous media (Sec. 3.3 transmission law) at the exit face l':
  // kind 0 = no interface (lambda in scale), 1 = the part transmitted into the
  // neighbour (weight lambda_t(d), receiving momentum scaled by qscale =
  // c_i / c_j), 2 = the part reflected back into the tet (weight
  // 1 - lambda_t(d), received by face l' itself), -1 = no block
  float ndst[3];              // inward normal of face l' in the source frame
  float c_ratio;              // c_i / c_j (Snell: sin theta_t = c_ratio sin theta_r)
  float z_src, z_dst;         // impedances rho_f c of the tet and of the neighbour
  float qscale;               // factor on the receiving tangential momentum
  int kind;
};
static_assert(sizeof(PairConst) == 160, "PairConst layout");

// Acoustic transmission probability across an interface (Sec. 3.3):
//   lambda_t = 4 z_dst z_src cos_r cos_t / (z_dst cos_r + z_src cos_t)^2,
// cos_t from Snell's law, zero beyond the critical angle.  cos_t^2 =
// 1 - c^2 (1 - cos_r^2) is formed as (1 - c^2) + c^2 cos_r^2: the direct form
// cancels for grazing rays in FP32 (cos_r = 1e-3 lost 3% of cos_t, and every
// cos_r below 2.4e-4 gave total reflection at equal speeds).
template <typename T>
__host__ __device__ inline T transmission_prob(T cos_r, T c_ratio, T z_src, T z_dst) {
  const T c2 = c_ratio * c_ratio;
  const T ct2 = (T(1) - c2) + c2 * cos_r * cos_r;
  if (ct2 <= T(0)) return T(0);
  const T cos_t = sqrt(ct2);
  const T den = z_dst * cos_r + z_src * cos_t;
  return T(4) * z_dst * z_src * cos_r * cos_t / (den * den);
}

// The reflected share 1 - lambda_t, formed as ((a - b) / (a + b))^2 with
// a = z_dst cos_r, b = z_src cos_t (the same quantity: (a + b)^2 - (a - b)^2
// = 4ab) so that nearly matched impedances do not cancel in FP32; 1 beyond
// the critical angle.
template <typename T>
__host__ __device__ inline T reflection_prob(T cos_r, T c_ratio, T z_src, T z_dst) {
  const T c2 = c_ratio * c_ratio;
  const T ct2 = (T(1) - c2) + c2 * cos_r * cos_r;
  if (ct2 <= T(0)) return T(1);
  const T a = z_dst * cos_r, b = z_src * sqrt(ct2);
  const T r = (a - b) / (a + b);
  return r * r;
}

// Weight of a ray d (source frame) in the pair's part of the operator.
template <typename T>
__device__ __forceinline__ T media_weight(const PairConst& pc, T d0, T d1, T d2) {
  if (pc.kind <= 0) return T(1);
  const T cos_r = -(d0 * (T)pc.ndst[0] + d1 * (T)pc.ndst[1] + d2 * (T)pc.ndst[2]);
  return pc.kind == 1 ? transmission_prob<T>(cos_r, (T)pc.c_ratio, (T)pc.z_src, (T)pc.z_dst)
                      : reflection_prob<T>(cos_r, (T)pc.c_ratio, (T)pc.z_src, (T)pc.z_dst);
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One thread per face pair p = 12 t + 3 f + k (k-th destination face l' != f).
// c_tet, rhof_tet: per-tet speed and fluid density (NULL: 1).  part 0: the
// blocks received across l' (transmitted, or reflected at the boundary);
// part 1: the blocks reflected at an interface between different media, kind
// -1 where there is none.
__global__ void pair_setup_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets,
                                  const int32_t* __restrict__ recv, const double* __restrict__ refl,
                                  const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet,
                                  double mu_uniform, int64_t npairs, PairConst* __restrict__ out,
                                  const double* __restrict__ c_tet = nullptr,
                                  const double* __restrict__ rhof_tet = nullptr, int part = 0) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int64_t t = p / 12;
  const int f = (int)((p % 12) / 3);
  const int k = (int)(p % 3);
  const int fp = k + (k >= f ? 1 : 0);
  const FaceGeom g = geom[4 * t + f];
  const int32_t* tv = tets + 4 * t;
  // local coordinates of the tet's vertices
  double loc[4][3];
  for (int v = 0; v < 4; ++v) {
    double r[3];
    for (int c = 0; c < 3; ++c) r[c] = V[3 * (int64_t)tv[v] + c] - g.o[c];
    loc[v][0] = dot3(r, g.e1);
    loc[v][1] = dot3(r, g.e2);
    loc[v][2] = dot3(r, g.n);
  }
  // A = vertex fp (on the source face), B, C the other two face vertices in face order, D = vertex f
  int bc[2], nb = 0;
  for (int j = 1; j <= 3; ++j) {
    const int v = (f + j) & 3;
    if (v != fp) bc[nb++] = v;
  }
  const double* A = loc[fp];
  const double* B = loc[bc[0]];
  const double* C = loc[bc[1]];
  const double* D = loc[f];
  const double D3 = D[2];
  // m_X = (-D3 grad beta_X, beta_X(D')) for the in-plane barycentric coordinate beta_X
  auto mvec = [&](const double* X, const double* Y, const double* Z, float* m) {
    const double zy0 = Z[0] - Y[0], zy1 = Z[1] - Y[1];
    const double den = zy0 * (X[1] - Y[1]) - zy1 * (X[0] - Y[0]);
    const double gx = -zy1 / den, gy = zy0 / den;
    const double betaD = (zy0 * (D[1] - Y[1]) - zy1 * (D[0] - Y[0])) / den;
    m[0] = (float)(-D3 * gx);
    m[1] = (float)(-D3 * gy);
    m[2] = (float)betaD;
  };
  PairConst pc;
  mvec(A, B, C, pc.mA);
  mvec(B, C, A, pc.mB);
  mvec(C, A, B, pc.mC);
  const int32_t R0 = recv[4 * t + fp];
  const bool boundary = (R0 == 4 * t + fp);
  // media of the tet and of the neighbour across l'
  const int64_t ti = R0 / 4;
  const double cj = c_tet ? c_tet[t] : 1.0, ci = c_tet ? c_tet[ti] : 1.0;
  const double zj = cj * (rhof_tet ? rhof_tet[t] : 1.0), zi = ci * (rhof_tet ? rhof_tet[ti] : 1.0);
  const bool interface = !boundary && (ci != cj || zi != zj);
  // part 1 blocks are received by face l' of the tet itself
  const int32_t R = part == 1 ? (int32_t)(4 * t + fp) : R0;
  const FaceGeom gr = geom[R];
  pc.R1[0] = (float)dot3(gr.e1, g.e1);
  pc.R1[1] = (float)dot3(gr.e1, g.e2);
  pc.R1[2] = (float)dot3(gr.e1, g.n);
  pc.R2[0] = (float)dot3(gr.e2, g.e1);
  pc.R2[1] = (float)dot3(gr.e2, g.e2);
  pc.R2[2] = (float)dot3(gr.e2, g.n);
  for (int c = 0; c < 3; ++c) {
    pc.A[c] = (float)A[c];
    pc.B[c] = (float)B[c];
    pc.C[c] = (float)C[c];
    pc.D[c] = (float)D[c];
  }
  pc.area_src = (float)g.area;
  pc.mu = (float)(mu_tet ? mu_tet[t] : mu_uniform);
  const double lam = boundary ? refl[R] : 1.0;
  pc.scale = (float)(lam / sqrt(g.area * geom[4 * t + fp].area));
  pc.out_row = R;
  pc.slot = f - (f > fp ? 1 : 0);
  const FaceGeom gd = geom[4 * t + fp];
  pc.ndst[0] = (float)dot3(gd.n, g.e1);
  pc.ndst[1] = (float)dot3(gd.n, g.e2);
  pc.ndst[2] = (float)dot3(gd.n, g.n);
  pc.c_ratio = (float)(ci / cj);
  pc.z_src = (float)zj;
  pc.z_dst = (float)zi;
  pc.qscale = (part == 0 && interface) ? (float)(ci / cj) : 1.f;
  pc.kind = part == 0 ? (interface ? 1 : 0) : (interface ? 2 : -1);
  out[p] = pc;
}

// ---------------------------------------------------------------------------
// Node arithmetic
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <typename T> __device__ __forceinline__ T exp_t(T x);
template <> __device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// phi2(x) = (x - 1 + e^{-x}) / x^2 = sum_k (-x)^k / (k+2)!; the series below
// x = 1/2 avoids the cancellation of the closed form (Sec. 3.3; mu = 0 gives 1/2).
template <typename T>
__device__ __forceinline__ T phi2(T x) {
  if (x < T(0.5)) {
    // Horner on 14 terms: |x| < 1/2 gives truncation < 0.5^14/16! ~ 3e-18
    const T c[13] = {T(1.0 / 2), T(1.0 / 6), T(1.0 / 24), T(1.0 / 120), T(1.0 / 720), T(1.0 / 5040),
                     T(1.0 / 40320), T(1.0 / 362880), T(1.0 / 3628800), T(1.0 / 39916800),
                     T(1.0 / 479001600), T(1.0 / 6227020800.0), T(1.0 / 87178291200.0)};
    T s = c[12];
#pragma unroll
    for (int i = 11; i >= 0; --i) s = c[i] - x * s;
    return s;
  }
  return (x - T(1) + exp_t<T>(-x)) / (x * x);
}

// Zernike polynomials Z_n^m(p), p = (px, py) in the unit disc (Sec. 3.1),
// by the paper's radial recursion written for Q_n^m = R_n^m / rho^m:
//   Q_n^n = 1,  Q_n^0 = 2 rho^2 Q_{n-1}^1 - Q_{n-2}^0,
//   Q_n^m = Q_{n-1}^{m-1} + rho^2 Q_{n-1}^{m+1} - Q_{n-2}^m  (0 < m < n),
// and cos(m phi) rho^m, sin(m phi) rho^m = Re, Im of (px + i py)^m.  This is a
// polynomial in (px, py): no angle, no division, no special case at rho = 0.
template <int NP, typename T>
__device__ __forceinline__ void zernike(T px, T py, T* Z) {
  const T r2 = px * px + py * py;
  T Q[NP + 1][NP + 1];
  T cr[NP + 1], ci[NP + 1];
  cr[0] = T(1);
  ci[0] = T(0);
#pragma unroll
  for (int m = 1; m <= NP; ++m) {
    cr[m] = cr[m - 1] * px - ci[m - 1] * py;
    ci[m] = cr[m - 1] * py + ci[m - 1] * px;
  }
#pragma unroll
  for (int n = 0; n <= NP; ++n) {
#pragma unroll
    for (int m = n & 1; m <= n; m += 2) {
      if (m == n) Q[n][m] = T(1);
      else if (m == 0) Q[n][m] = T(2) * r2 * Q[n - 1][1] - Q[n - 2][0];
      else Q[n][m] = Q[n - 1][m - 1] + r2 * Q[n - 1][m + 1] - Q[n - 2][m];
    }
  }
#pragma unroll
  for (int n = 0; n <= NP; ++n) {
#pragma unroll
    for (int m = -n; m <= n; m += 2) {
      const int idx = (n * (n + 2) + m) / 2;
      const int am = m < 0 ? -m : m;
      Z[idx] = m == 0 ? Q[n][0] : (m > 0 ? Q[n][am] * cr[am] : Q[n][am] * ci[am]);
    }
  }
}

template <int NP>
struct Tile {
  static constexpr int NB = (NP + 1) * (NP + 2) / 2;
  static constexpr int NBP = ((NB + 7) / 8) * 8;  // padded block side
  static constexpr int TR = NBP / 8;              // rows per lane (8 row groups)
  static constexpr int TC = NBP / 4;              // columns per lane (4 column groups)
  // staging row stride: NBP + 4 keeps rows 16-byte aligned and shifts each
  // row by 16 bytes modulo 128, so eight lanes storing 16-byte vectors of
  // eight consecutive rows hit eight distinct bank groups
  static constexpr int LD = NBP + 4;
};

constexpr int kWarps = 4;        // warps (face pairs) per block
constexpr int kMaxQ = 32;        // largest per-patch Gauss order
constexpr int kStack = 16;       // subdivision stack entries per warp
constexpr int kPatchBuf = 32;    // patches processed per chunk
constexpr int kMaxDepth = 4;     // deepest subdivision level

struct Poly {
  float v[4][3];  // unit generators (v[3] = v[0] for a triangle)
  int nv, depth;
};

__device__ __forceinline__ void nrm3(float* a) {
  const float s = rsqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  a[0] *= s;
  a[1] *= s;
  a[2] *= s;
}

__device__ __forceinline__ void mid3(const float* a, const float* b, float* out) {
  out[0] = a[0] + b[0];
  out[1] = a[1] + b[1];
  out[2] = a[2] + b[2];
  nrm3(out);
}

__device__ __forceinline__ float dotf(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Region r of the destination face (0 interior, 1 wedge at A, 2 strip on AB,
// 3 strip on AC) as unit generators (Sec. 3.3: the regions of P).
__device__ inline void region_poly(const PairConst& pc, int r, Poly& P) {
  const float* A = pc.A;
  const float* B = pc.B;
  const float* C = pc.C;
  const float* D = pc.D;
  float g[4][3];
  auto sub = [](const float* x, const float* y, float* o) {
    o[0] = x[0] - y[0];
    o[1] = x[1] - y[1];
    o[2] = x[2] - y[2];
  };
  switch (r) {
    case 0: sub(D, A, g[0]); sub(D, B, g[1]); sub(D, C, g[2]); P.nv = 3; break;
    case 1: sub(D, A, g[0]); sub(B, A, g[1]); sub(C, A, g[2]); P.nv = 3; break;
    case 2: sub(D, A, g[0]); sub(D, B, g[1]); sub(C, B, g[2]); sub(C, A, g[3]); P.nv = 4; break;
    default: sub(D, A, g[0]); sub(D, C, g[1]); sub(B, C, g[2]); sub(B, A, g[3]); P.nv = 4; break;
  }
  for (int k = 0; k < P.nv; ++k) {
    nrm3(g[k]);
    P.v[k][0] = g[k][0];
    P.v[k][1] = g[k][1];
    P.v[k][2] = g[k][2];
  }
  if (P.nv == 3) {
    P.v[3][0] = P.v[0][0];
    P.v[3][1] = P.v[0][1];
    P.v[3][2] = P.v[0][2];
  }
  P.depth = 0;
}

// bilinear coefficients a, b, c, d of Eq. (Parametr) from v1..v4
__device__ __forceinline__ void bilinear_coeffs(const Poly& P, float* out12) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float v1 = P.v[0][c], v2 = P.v[1][c], v3 = P.v[2][c], v4 = P.v[3][c];
    out12[c] = 0.25f * (v1 + v2 + v3 + v4);
    out12[3 + c] = 0.25f * (v2 - v1 + v3 - v4);
    out12[6 + c] = 0.25f * (v3 + v4 - v1 - v2);
    out12[9 + c] = 0.25f * (v3 - v4 + v1 - v2);
  }
}

// Per-warp direction-patch state: the subdivision stack and a buffer of
// patches (bilinear coefficients a, b, c, d) ready for quadrature.
struct PatchSmem {
  Poly stack[kStack];
  float patch[kPatchBuf][12];
  int sp;      // stack size
  int npatch;  // patches in the buffer
};

// Lane 0: pop polygons, split those with an edge longer than the threshold,
// emit the rest into the patch buffer until it is full or the stack is empty.
__device__ inline void fill_patches(PatchSmem& S, float cos_max) {
  S.npatch = 0;
  while (S.sp > 0 && S.npatch < kPatchBuf) {
    Poly P = S.stack[--S.sp];
    float minc = 1.f;
    for (int e = 0; e < P.nv; ++e) minc = fminf(minc, dotf(P.v[e], P.v[(e + 1) % P.nv]));
    const bool split = (minc < cos_max) && (P.depth < kMaxDepth) && (S.sp + 4 <= kStack);
    if (!split) {
      bilinear_coeffs(P, S.patch[S.npatch++]);
      continue;
    }
    Poly c[4];
    for (int i = 0; i < 4; ++i) {
      c[i].depth = P.depth + 1;
      c[i].nv = P.nv;
    }
    if (P.nv == 3) {
      float ab[3], bc[3], ca[3];
      mid3(P.v[0], P.v[1], ab);
      mid3(P.v[1], P.v[2], bc);
      mid3(P.v[2], P.v[0], ca);
      const float* tri[4][3] = {{P.v[0], ab, ca}, {ab, P.v[1], bc}, {ca, bc, P.v[2]}, {ab, bc, ca}};
      for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k)
          for (int x = 0; x < 3; ++x) c[i].v[k][x] = tri[i][k < 3 ? k : 0][x];
    } else {
      float ab[3], bc[3], cd[3], da[3], m[3];
      mid3(P.v[0], P.v[1], ab);
      mid3(P.v[1], P.v[2], bc);
      mid3(P.v[2], P.v[3], cd);
      mid3(P.v[3], P.v[0], da);
      m[0] = P.v[0][0] + P.v[1][0] + P.v[2][0] + P.v[3][0];
      m[1] = P.v[0][1] + P.v[1][1] + P.v[2][1] + P.v[3][1];
      m[2] = P.v[0][2] + P.v[1][2] + P.v[2][2] + P.v[3][2];
      nrm3(m);
      const float* q[4][4] = {{P.v[0], ab, m, da}, {ab, P.v[1], bc, m}, {m, bc, P.v[2], cd}, {da, m, cd, P.v[3]}};
      for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k)
          for (int x = 0; x < 3; ++x) c[i].v[k][x] = q[i][k][x];
    }
    for (int i = 0; i < 4; ++i) S.stack[S.sp++] = c[i];
  }
}


// d/dx phi2(x) = (2 - x - (x + 2) e^{-x}) / x^3 = sum_j (-1)^(j+1) (j+1) x^j / (j+3)!;
// the series below x = 1 avoids the cancellation of the closed form.
template <typename T>
__device__ __forceinline__ T phi2_prime(T x) {
  if (x < T(1)) {
    // coefficients (-1)^(j+1) (j+1)/(j+3)!, j = 0..14
    const T c[15] = {T(-1.0 / 6), T(2.0 / 24), T(-3.0 / 120), T(4.0 / 720), T(-5.0 / 5040), T(6.0 / 40320),
                     T(-7.0 / 362880), T(8.0 / 3628800), T(-9.0 / 39916800), T(10.0 / 479001600),
                     T(-11.0 / 6227020800.0), T(12.0 / 87178291200.0), T(-13.0 / 1307674368000.0),
                     T(14.0 / 20922789888000.0), T(-15.0 / 355687428096000.0)};
    T s = c[14];
#pragma unroll
    for (int i = 13; i >= 0; --i) s = c[i] + x * s;
    return s;
  }
  return (T(2) - x - (x + T(2)) * exp_t<T>(-x)) / (x * x * x);
}

// k-th derivative of phi2 (k <= 3): phi2^(k)(x) = (-1)^k Int_0^1 (1-u) u^k e^{-x u} du.
// Below x = 1 the Taylor series sum_m (-1)^(m+k) (m+k)!/(m! (m+k+2)!) x^m
// (20 terms); above, a 16-point Gauss rule on the integral (the integrand is
// smooth), so no cancellation occurs at any x >= 0.
template <typename T>
__device__ __forceinline__ T phi2_deriv(int k, T x) {
  if (k == 0 && x < T(0.5)) return phi2<T>(x);
  if (x < T(1)) {
    T fk = T(1);  // k!
    for (int i = 2; i <= k; ++i) fk *= T(i);
    T term = ((k & 1) ? T(-1) : T(1)) * fk / (fk * T(k + 1) * T(k + 2));  // (-1)^k k!/(k+2)!
    T sum = term;
#pragma unroll 4
    for (int m = 0; m < 19; ++m) {
      term *= -x * T(m + k + 1) / (T(m + 1) * T(m + k + 3));
      sum += term;
    }
    return sum;
  }
  const T gx[8] = {T(0.0950125098376374), T(0.2816035507792589), T(0.4580167776572274), T(0.6178762444026438),
                   T(0.7554044083550030), T(0.8656312023878318), T(0.9445750230732326), T(0.9894009349916499)};
  const T gw[8] = {T(0.1894506104550685), T(0.1826034150449236), T(0.1691565193950025), T(0.1495959888165767),
                   T(0.1246289712555339), T(0.0951585116824928), T(0.0622535239386479), T(0.0271524594117541)};
  T sum = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const T u = T(0.5) * (T(1) + T(sgn) * gx[i]);
      T uk = T(1);
      for (int j = 0; j < k; ++j) uk *= u;
      sum += T(0.5) * gw[i] * (T(1) - u) * uk * exp_t<T>(-x * u);
    }
  return (k & 1) ? -sum : sum;
}

// Geometry of one quadrature node of a patch: direction d (unit, source
// frame), Jacobian of Sec. 3.4 (includes cos theta), and the closed-form
// quantities |OBC| and L_O of Sec. 3.3 (valid = s_A > 0).
template <typename T>
struct NodeGeom {
  T d0, d1, d2, jac, Anab, LO;
  bool valid;
};

template <typename T>
__device__ __forceinline__ NodeGeom<T> node_geom(const float* cf, T xi, T eta, const PairConst& pc) {
  NodeGeom<T> g;
  T f[3], fx[3], fe[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T a = cf[c], b = cf[3 + c], cc = cf[6 + c], d = cf[9 + c];
    f[c] = a + b * xi + cc * eta + d * xi * eta;
    fx[c] = b + d * eta;
    fe[c] = cc + d * xi;
  }
  const T r2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
  const T rinv = rsqrt_t<T>(r2);
  const T det = f[0] * (fx[1] * fe[2] - fx[2] * fe[1]) + f[1] * (fx[2] * fe[0] - fx[0] * fe[2]) +
                f[2] * (fx[0] * fe[1] - fx[1] * fe[0]);
  const T ri2 = rinv * rinv;
  g.jac = fabs(f[2] * det) * ri2 * ri2;
  g.d0 = f[0] * rinv;
  g.d1 = f[1] * rinv;
  g.d2 = f[2] * rinv;
  const T sA = (T)pc.mA[0] * g.d0 + (T)pc.mA[1] * g.d1 + (T)pc.mA[2] * g.d2;
  const T sB = (T)pc.mB[0] * g.d0 + (T)pc.mB[1] * g.d1 + (T)pc.mB[2] * g.d2;
  const T sC = (T)pc.mC[0] * g.d0 + (T)pc.mC[1] * g.d1 + (T)pc.mC[2] * g.d2;
  g.valid = sA > T(0);
  const T den = sA + fmax(sB, T(0)) + fmax(sC, T(0));
  const T inv = g.valid ? T(1) / den : T(0);
  g.LO = (T)pc.D[2] * inv;
  g.Anab = (T)pc.area_src * sA * inv;
  return g;
}

// inverse Zernike norm (2n+2)/(eps_m pi) of basis index i (Sec. 3.1-3.2)
__device__ __forceinline__ float zernike_invnorm(int i) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= i) ++n;
  const int m = 2 * i - n * (n + 2);
  return (float)((2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI));
}

}  // namespace
}  // namespace dfm
