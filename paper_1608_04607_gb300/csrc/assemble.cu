// Assembly of the discretised transfer operator B (Sec. 3.2-3.4).
//
// For a tet with source face l = ABC' (A the face vertex not on the
// destination face l', B, C the shared vertices, D the apex) and an inward
// direction d, the set of source points whose ray leaves through l' is the
// triangle OBC of Sec. 3.3; the damping length is affine on it, zero on BC,
// so its damped area is
//   S(d) = 2 |OBC| phi2(mu L_O),  phi2(x) = (x - 1 + e^{-x}) / x^2,
// the closed form of Sec. 3.3 (|OBC| = h|BC|/2, L_O = L_max).  We evaluate
// |OBC| and L_O without locating O explicitly: with s_X(d) = d_z beta_X(P(d))
// (beta the barycentric coordinates of the point P where the ray through D
// meets the source plane), s_X is LINEAR in d, s_X(d) = m_X . d, and in each
// of the four non-empty direction regions (P inside ABC, beyond vertex A,
// beyond edge AB, beyond edge AC)
//   den = s_A + max(s_B, 0) + max(s_C, 0),  L_O = D3 / den,  |OBC| = |ABC| s_A / den,
// with D3 the apex height.  No division by cos(theta) appears, so grazing
// directions and directions near the shared edges stay well conditioned.
//
// The direction integral runs over the four non-empty sub-regions of the
// paper's seven (Sec. 3.4), each a spherical polygon mapped from [-1,1]^2 by
// the bilinear map of Eq. (Parametr) projected onto the hemisphere, with the
// Jacobian f_3 det[f, f_xi, f_eta] / |f|^4 (which includes cos theta).  Where
// the paper refines with adaptive Clenshaw-Curtis, we split a region into
// patches (midpoint subdivision on the sphere) until every patch edge
// subtends at most max_patch_deg, then apply a fixed tensor Gauss-Legendre
// rule of order q on every patch.
//
// Work decomposition: a one-thread-per-pair FP64 set-up kernel writes the
// per-pair constants (local frame, the linear forms m_X, the receiving frame)
// in FP32; the assembly kernel runs one warp per face pair.  Lanes evaluate
// one quadrature node each (geometry, closed-form S, two Zernike vectors by
// the recursion of Sec. 3.1 in Cartesian form), stage w Z(p') and Z(p) in
// shared memory, then the warp accumulates the rank-32 update of the N_b x N_b
// block with every lane owning a TR x TC register tile.
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
  float pad[4];
};
static_assert(sizeof(PairConst) == 144, "PairConst layout");

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One thread per face pair p = 12 t + 3 f + k (k-th destination face l' != f).
__global__ void pair_setup_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets,
                                  const int32_t* __restrict__ recv, const double* __restrict__ refl,
                                  const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet,
                                  double mu_uniform, int64_t npairs, PairConst* __restrict__ out) {
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
  const int32_t R = recv[4 * t + fp];
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
  const double lam = (R == 4 * t + fp) ? refl[R] : 1.0;
  pc.scale = (float)(lam / sqrt(g.area * geom[4 * t + fp].area));
  pc.out_row = R;
  pc.slot = f - (f > fp ? 1 : 0);
  pc.pad[0] = pc.pad[1] = pc.pad[2] = pc.pad[3] = 0.f;
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
  static constexpr int LD = NBP + 1;              // staging row stride (odd: conflict-free stores)
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
__device__ void region_poly(const PairConst& pc, int r, Poly& P) {
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

// Shared memory of one warp.
template <int NP, typename T>
struct WarpSmem {
  Poly stack[kStack];
  float patch[kPatchBuf][12];
  T zq[32 * Tile<NP>::LD];  // w * Z(p') per node
  T zp[32 * Tile<NP>::LD];  // Z(p) per node
  int sp;                   // stack size
  int npatch;               // patches in the buffer
};

// Lane 0: pop polygons, split those with an edge longer than the threshold,
// emit the rest into the patch buffer until it is full or the stack is empty.
template <int NP, typename T>
__device__ void fill_patches(WarpSmem<NP, T>& S, float cos_max) {
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

template <int NP, typename T>
__global__ void __launch_bounds__(kWarps * 32)
assemble_kernel(const PairConst* __restrict__ pairs, int64_t npairs, const double* __restrict__ gl_x,
                const double* __restrict__ gl_w, int q, float cos_max, T* __restrict__ vals, int64_t row_stride,
                unsigned long long* __restrict__ node_count) {
  using TL = Tile<NP>;
  constexpr int NB = TL::NB, TR = TL::TR, TC = TL::TC, LD = TL::LD;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  WarpSmem<NP, T>* smem = reinterpret_cast<WarpSmem<NP, T>*>(dyn_smem);
  T* s_x = reinterpret_cast<T*>(smem + kWarps);
  T* s_w = s_x + kMaxQ;
  float* s_ninv = reinterpret_cast<float*>(s_w + kMaxQ);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  WarpSmem<NP, T>& S = smem[wid];
  if (threadIdx.x < q) {
    s_x[threadIdx.x] = (T)gl_x[threadIdx.x];
    s_w[threadIdx.x] = (T)gl_w[threadIdx.x];
  }
  if (threadIdx.x < NB) {
    // inverse Zernike norm (2n+2)/(eps_m pi) of basis index i (Sec. 3.1-3.2)
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= (int)threadIdx.x) ++n;
    const int m = 2 * (int)threadIdx.x - n * (n + 2);
    s_ninv[threadIdx.x] = (float)((2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI));
  }
  // zero the staging buffers once (padding columns stay zero)
  for (int i = lane; i < 32 * LD; i += 32) {
    S.zq[i] = T(0);
    S.zp[i] = T(0);
  }
  __syncthreads();
  const int qq = q * q;
  const int a0 = (lane >> 2) * TR;
  const int b0 = (lane & 3) * TC;

  {
    const int64_t p = (int64_t)blockIdx.x * kWarps + wid;
    if (p >= npairs) return;  // no block-wide barrier follows
    const PairConst pc = pairs[p];
    T acc[TR][TC];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int c = 0; c < TC; ++c) acc[r][c] = T(0);
    if (lane == 0) {
      S.sp = 0;
      for (int r = 3; r >= 0; --r) region_poly(pc, r, S.stack[S.sp++]);
    }
    __syncwarp();
    const T mA0 = pc.mA[0], mA1 = pc.mA[1], mA2 = pc.mA[2];
    const T mB0 = pc.mB[0], mB1 = pc.mB[1], mB2 = pc.mB[2];
    const T mC0 = pc.mC[0], mC1 = pc.mC[1], mC2 = pc.mC[2];
    const T D3 = pc.D[2], Af = pc.area_src, mu = pc.mu;
    unsigned long long pair_nodes = 0;
    while (true) {
      if (lane == 0) fill_patches<NP, T>(S, cos_max);
      __syncwarp();
      const int npatch = S.npatch;
      if (npatch == 0) break;
      const int nodes = npatch * qq;
      pair_nodes += nodes;
      for (int base = 0; base < nodes; base += 32) {
        const int k = base + lane;
        T Zp[NB], Zq[NB];
        T wnode = T(0);
        if (k < nodes) {
          const int pi = k / qq;
          const int rem = k - pi * qq;
          const int i = rem / q;
          const int j = rem - i * q;
          const float* cf = S.patch[pi];
          const T xi = s_x[i], eta = s_x[j];
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
          const T jac = fabs(f[2] * det) * ri2 * ri2;
          const T d0 = f[0] * rinv, d1 = f[1] * rinv, d2 = f[2] * rinv;
          const T sA = mA0 * d0 + mA1 * d1 + mA2 * d2;
          const T sB = mB0 * d0 + mB1 * d1 + mB2 * d2;
          const T sC = mC0 * d0 + mC1 * d1 + mC2 * d2;
          if (sA > T(0)) {
            const T den = sA + fmax(sB, T(0)) + fmax(sC, T(0));
            const T inv = T(1) / den;
            const T LO = D3 * inv;
            const T Anab = Af * sA * inv;
            wnode = s_w[i] * s_w[j] * jac * T(2) * Anab * phi2<T>(mu * LO);
          }
          zernike<NP, T>(d0, d1, Zp);
          const T qx = d0 * (T)pc.R1[0] + d1 * (T)pc.R1[1] + d2 * (T)pc.R1[2];
          const T qy = d0 * (T)pc.R2[0] + d1 * (T)pc.R2[1] + d2 * (T)pc.R2[2];
          zernike<NP, T>(qx, qy, Zq);
        } else {
#pragma unroll
          for (int c = 0; c < NB; ++c) Zp[c] = Zq[c] = T(0);
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          S.zq[lane * LD + c] = wnode * Zq[c];
          S.zp[lane * LD + c] = Zp[c];
        }
        __syncwarp();
        const int kmax = min(32, nodes - base);
        for (int kk = 0; kk < kmax; ++kk) {
          T av[TR], bv[TC];
#pragma unroll
          for (int r = 0; r < TR; ++r) av[r] = S.zq[kk * LD + a0 + r];
#pragma unroll
          for (int c = 0; c < TC; ++c) bv[c] = S.zp[kk * LD + b0 + c];
#pragma unroll
          for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
        __syncwarp();
      }
    }
    if (lane == 0) atomicAdd(node_count, pair_nodes);
    // epilogue: scale row a by lambda N_a / sqrt(|T_l||T_l'|) and store
    T* out = vals + (int64_t)pc.out_row * row_stride + (int64_t)pc.slot * NB * NB;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      const int a = a0 + r;
      if (a >= NB) continue;
      const T s = (T)pc.scale * (T)s_ninv[a];
#pragma unroll
      for (int c = 0; c < TC; ++c) {
        const int b = b0 + c;
        if (b < NB) out[a * NB + b] = acc[r][c] * s;
      }
    }
    __syncwarp();
  }
}

template <int NP, typename T>
constexpr size_t assemble_smem_bytes() {
  return sizeof(WarpSmem<NP, T>) * kWarps + 2 * kMaxQ * sizeof(T) + 64 * sizeof(float);
}

template <int NP, typename T>
int launch_assemble(const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                    float cos_max, T* vals, int64_t row_stride, unsigned long long* nodes, cudaStream_t st) {
  constexpr size_t smem = assemble_smem_bytes<NP, T>();
  static_assert(smem <= 220 * 1024, "assembly shared memory");
  DFM_CUDA_CHECK(cudaFuncSetAttribute(assemble_kernel<NP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (npairs + kWarps - 1) / kWarps;
  if (blocks > 0x7fffffff) return set_error(DFM_ERR_ARG, "dfm_assemble: too many face pairs");
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_ASSEMBLE, st);
    assemble_kernel<NP, T><<<(unsigned)blocks, kWarps * 32, smem, st>>>(pairs, npairs, glx, glw, q, cos_max, vals,
                                                                        row_stride, nodes);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

template <typename T>
int dispatch_np(int Np, const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                float cos_max, T* vals, int64_t row_stride, unsigned long long* nodes, cudaStream_t st) {
  switch (Np) {
    case 0: return launch_assemble<0, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 1: return launch_assemble<1, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 2: return launch_assemble<2, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 3: return launch_assemble<3, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 4: return launch_assemble<4, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 5: return launch_assemble<5, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 6: return launch_assemble<6, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 7: return launch_assemble<7, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    case 8: return launch_assemble<8, T>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, st);
    default: return set_error(DFM_ERR_ARG, "dfm_assemble: Np must be in 0..8");
  }
}

int check_params(const dfm_mesh* mesh, const dfm_params* p) {
  if (!mesh || !p) return set_error(DFM_ERR_ARG, "dfm_assemble: NULL mesh or params");
  if (p->Np < 0 || p->Np > 8) return set_error(DFM_ERR_ARG, "dfm_assemble: Np must be in 0..8");
  if (p->precision != DFM_F32 && p->precision != DFM_F64)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: precision must be DFM_F32 or DFM_F64");
  if (!p->mu && !(p->mu_uniform >= 0.0)) return set_error(DFM_ERR_ARG, "dfm_assemble: mu_uniform must be >= 0");
  const int q = p->quad_order ? p->quad_order : p->Np + 6;
  if (q < 1 || q > kMaxQ) return set_error(DFM_ERR_ARG, "dfm_assemble: quad_order must be in 1..32");
  const double deg = p->max_patch_deg > 0 ? p->max_patch_deg : 60.0;
  if (!(deg >= 10.0 && deg <= 180.0)) return set_error(DFM_ERR_ARG, "dfm_assemble: max_patch_deg must be in [10, 180]");
  return DFM_OK;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_assemble_into(const dfm_mesh* mesh, const dfm_params* p, dfm_op* op, void* stream) {
  int rc = check_params(mesh, p);
  if (rc) return rc;
  if (!op || op->mesh != mesh || op->Np != p->Np || op->precision != p->precision)
    return set_error(DFM_ERR_ARG, "dfm_assemble_into: operator does not match mesh/Np/precision");
  cudaStream_t st = as_stream(stream);
  const int q = p->quad_order ? p->quad_order : p->Np + 6;
  const double deg = p->max_patch_deg > 0 ? p->max_patch_deg : 60.0;
  const float cos_max = (float)cos(deg * M_PI / 180.0);
  const int64_t npairs = 12 * mesh->nt;
  // scratch: per-pair constants and the Gauss table, kept with the operator
  const int64_t need = npairs * (int64_t)sizeof(PairConst) + 2 * 64 * (int64_t)sizeof(double) + 256;
  if (op->work_bytes < need) {
    cudaFree(op->work);
    op->work = nullptr;
    op->work_bytes = 0;
    DFM_CUDA_CHECK(cudaMalloc(&op->work, need));
    op->work_bytes = need;
  }
  PairConst* pairs = reinterpret_cast<PairConst*>(op->work);
  double* glx = reinterpret_cast<double*>(reinterpret_cast<char*>(op->work) + npairs * sizeof(PairConst));
  double* glw = glx + 64;
  unsigned long long* nodes = reinterpret_cast<unsigned long long*>(glw + 64);
  DFM_CUDA_CHECK(cudaMemsetAsync(nodes, 0, sizeof(unsigned long long), st));
  rc = gauss_legendre_device(q, glx, glw, st);
  if (rc) return rc;
  const int bs = 128;
  pair_setup_kernel<<<(unsigned)((npairs + bs - 1) / bs), bs, 0, st>>>(mesh->verts, mesh->tets, mesh->recv,
                                                                       mesh->refl, mesh->geom, p->mu,
                                                                       p->mu_uniform, npairs, pairs);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  if (op->precision == DFM_F32)
    return dispatch_np<float>(p->Np, pairs, npairs, glx, glw, q, cos_max, (float*)op->vals, op->row_stride, nodes,
                              st);
  return dispatch_np<double>(p->Np, pairs, npairs, glx, glw, q, cos_max, (double*)op->vals, op->row_stride, nodes,
                             st);
}

extern "C" int dfm_assemble(const dfm_mesh* mesh, const dfm_params* p, void* stream, dfm_op** out) {
  if (!out) return set_error(DFM_ERR_ARG, "dfm_assemble: out is NULL");
  *out = nullptr;
  int rc = check_params(mesh, p);
  if (rc) return rc;
  dfm_op* op = new dfm_op();
  op->mesh = mesh;
  op->Np = p->Np;
  op->nb = nbasis(p->Np);
  op->precision = p->precision;
  op->nrows = mesh->nrows;
  op->row_stride = op_row_stride(op->nb);
  op->bytes = op->nrows * op->row_stride * elem_size(op->precision);
  cudaError_t e = cudaMalloc(&op->vals, op->bytes);
  if (e != cudaSuccess) {
    delete op;
    return cuda_error(e, "dfm_assemble: cudaMalloc(vals)");
  }
  // padding between rows stays zero
  e = cudaMemsetAsync(op->vals, 0, op->bytes, as_stream(stream));
  if (e != cudaSuccess) {
    dfm_op_destroy(op);
    return cuda_error(e, "dfm_assemble: cudaMemsetAsync");
  }
  rc = dfm_assemble_into(mesh, p, op, stream);
  if (rc) {
    dfm_op_destroy(op);
    return rc;
  }
  *out = op;
  return DFM_OK;
}

extern "C" void dfm_op_destroy(dfm_op* op) {
  if (!op) return;
  cudaFree(op->vals);
  cudaFree(op->work);
  cudaFree(op->swork);
  delete op;
}

extern "C" int dfm_op_info(const dfm_op* op, dfm_op_info_t* info) {
  if (!op || !info) return set_error(DFM_ERR_ARG, "dfm_op_info: NULL argument");
  info->Np = op->Np;
  info->nb = op->nb;
  info->precision = op->precision;
  info->n_rows = op->nrows;
  info->row_stride = op->row_stride;
  info->vals = op->vals;
  info->bytes = op->bytes;
  return DFM_OK;
}

extern "C" int dfm_op_copy_vals(const dfm_op* op, void* dst, int64_t bytes, void* stream) {
  if (!op || !dst) return set_error(DFM_ERR_ARG, "dfm_op_copy_vals: NULL argument");
  if (bytes != op->bytes) return set_error(DFM_ERR_ARG, "dfm_op_copy_vals: bytes must equal the operator size");
  DFM_CUDA_CHECK(cudaMemcpyAsync(dst, op->vals, bytes, cudaMemcpyDefault, as_stream(stream)));
  return DFM_OK;
}

extern "C" int dfm_op_nodes(const dfm_op* op, int64_t* nodes) {
  if (!op || !nodes || !op->work) return set_error(DFM_ERR_ARG, "dfm_op_nodes: NULL argument or no assembly yet");
  const int64_t npairs = 12 * op->mesh->nt;
  const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(
      reinterpret_cast<const char*>(op->work) + npairs * sizeof(PairConst) + 128 * sizeof(double));
  unsigned long long h = 0;
  DFM_CUDA_CHECK(cudaMemcpy(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost));
  *nodes = (int64_t)h;
  return DFM_OK;
}
