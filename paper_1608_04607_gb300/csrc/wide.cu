// Bases above N_p = 8 (N_b = 55 .. 231): the cuboid verification of Sec. 4.1
// runs the method up to N_p = 20, where one block holds 231 x 231 entries and
// neither a warp's register tile (the assembly of assemble.cu) nor a staged
// operator row (the pipelined applications of spmv.cu) fits.  This file holds
// the kernels of that range:
//
//  * the Zernike polynomials by a radial recurrence at fixed m that holds two
//    values instead of whole orders (zernike_wide.h), each Z_n^m handed to
//    the caller as it is formed;
//  * the assembly of B (Eq. B4DInt with the closed form of Sec. 3.3 and the
//    patch rule of Sec. 3.4), one block per (face pair, tile of test rows):
//    the block's threads each own an 8 x 8 register tile, and each pass
//    stages Z(p) and w Z(p') of up to 64 quadrature nodes in shared memory;
//  * the forward application y = x0 + alpha B x (FP32 blocks, FP32 or FP64
//    vectors), one block per operator row, a warp per test index streaming
//    the row's three block rows with coalesced loads;
//  * the directed boundary source (Eq. RhoNeumann) and the interior density
//    functional (Eq. IntDens) at these orders.
//
// The arithmetic per node and per entry is that of the narrow kernels; only
// the work decomposition differs.
#include <math.h>

#include <algorithm>

#include "dfm_internal.cuh"
#include "interior_rule.cuh"
#include "node.cuh"
#include "p1_basis.h"
#include "zernike_wide.h"

namespace dfm {
namespace {

// order n of basis index i (n (n + 1) / 2 <= i < (n + 1)(n + 2) / 2)
__device__ __forceinline__ int order_of(int i) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= i) ++n;
  return n;
}

// Per face pair p = 12 t + 3 f + k of the linear basis: positions of A (the
// source face's vertex not on the destination face), B, C in the source
// face's frame order, and of B, C, D (D the vertex opposite the source face)
// in the frame order of the receiving row's face, packed as bytes.
__global__ void p1_setup_kernel(const int32_t* __restrict__ tets, const int32_t* __restrict__ recv, int64_t npairs,
                                int2* __restrict__ pos) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int64_t t = p / 12;
  const int f = (int)((p % 12) / 3);
  const int k = (int)(p % 3);
  const int fp = k + (k >= f ? 1 : 0);
  int bcv[2], bcp[2], nb = 0;
  for (int j = 1; j <= 3; ++j) {
    const int v = (f + j) & 3;
    if (v != fp) {
      bcv[nb] = v;
      bcp[nb++] = j - 1;
    }
  }
  const int pA = ((fp - f) & 3) - 1;
  const int32_t R = recv[4 * t + fp];
  const int64_t tr = R / 4;
  const int fr = R % 4;
  const int32_t gB = tets[4 * t + bcv[0]], gC = tets[4 * t + bcv[1]], gD = tets[4 * t + f];
  int rB = 0, rC = 0, rD = 0;
  for (int j = 0; j < 3; ++j) {
    const int32_t g = tets[4 * tr + ((fr + 1 + j) & 3)];
    if (g == gB) rB = j;
    if (g == gC) rC = j;
    if (g == gD) rD = j;
  }
  pos[p] = make_int2(pA | (bcp[0] << 8) | (bcp[1] << 16), rB | (rC << 8) | (rD << 16));
}

// ---------------------------------------------------------------------------
// Assembly: block (pair p, tile y).  Threads [0, nc) evaluate Z(p) of the
// pass's nodes, threads [nc, 2 nc) w Z(p') restricted to the tile's rows
// (with NS = 1 stopping at the order of the tile's last row); then thread
// (rg, cg) adds the nodes' terms to its rows 8 rg .. 8 rg + 7 of the tile and
// its columns 4 cg .. 4 cg + 3 and NS NBP/2 + 4 cg .. NS NBP/2 + 4 cg + 3 (eight
// consecutive lanes then read 128 consecutive bytes of a staged row).  NS = 3
// (linear spatial basis): row (b, i) = b NB + i, column (a, j) = a NB + j, the
// term of a node w M[b][a] Z_i(p') Z_j(p) with M the spatial matrix of
// p1_spatial; the staged row vector of source function a holds w M[b][a] Z_i(p')
// and columns are padded to NBP per spatial function, so a 4-column group
// never spans two of them.
// ---------------------------------------------------------------------------
template <int NS, typename TO>
__global__ void __launch_bounds__(256, 2)
assemble_wide_kernel(const PairConst* __restrict__ pairs, const int2* __restrict__ p1pos,
                     const double* __restrict__ gl_x, const double* __restrict__ gl_w, int q, float cos_max,
                     TO* __restrict__ vals, int64_t row_stride, unsigned long long* __restrict__ node_count,
                     int moment, int Np, geom::WideAsm G) {
  __shared__ PatchSmem P;
  __shared__ PairConst pc;  // read by every thread from shared memory (keeps registers for acc)
  __shared__ int s_pos[6];
  extern __shared__ __align__(16) float wsm[];
  float* zq = wsm;                          // [NS][nc][ldq]  w (M) Z(p') of the tile's rows
  float* zp = zq + NS * G.nc * G.ldq;       // [nc][ldp]      Z(p)
  float* s_ninv = zp + G.nc * G.ldp;        // [trw]
  float* s_x = s_ninv + G.trw;              // [32]
  float* s_w = s_x + 32;                    // [32]
  const int tid = threadIdx.x;
  const int NB = G.nb;        // Zernike functions
  const int NR = G.nrow;      // block side NS NB
  const int row0 = blockIdx.y * G.trw;
  if (pairs[blockIdx.x].kind < 0) return;  // the whole block: no block for this pair in this part
  if (tid < (int)(sizeof(PairConst) / 4))
    reinterpret_cast<int*>(&pc)[tid] = reinterpret_cast<const int*>(pairs + blockIdx.x)[tid];
  if constexpr (NS > 1) {
    if (tid < 6) {
      const int2 w = p1pos[blockIdx.x];
      s_pos[tid] = ((tid < 3 ? w.x : w.y) >> (8 * (tid % 3))) & 0xff;
    }
  }
  if (tid < q) {
    s_x[tid] = (float)gl_x[tid];
    s_w[tid] = (float)gl_w[tid];
  }
  for (int a = tid; a < G.trw; a += blockDim.x)
    s_ninv[a] = row0 + a < NR ? zernike_invnorm((row0 + a) % NB) : 0.f;
  __syncthreads();  // pc, s_pos
  // w Z(p') needs orders 0..q_last
  const int q_last = NS == 1 ? order_of(min(row0 + G.trw, NB) - 1) : Np;
  const bool acc_thread = tid < G.cg * G.rg;
  const int cgi = tid % G.cg, rgi = tid / G.cg;
  const int half = NS * G.nbp / 2;
  // the thread's two column groups: spatial function a0/a1, Zernike column j0/j1
  // (one spatial function: a0 = a1 = 0, j0 = 4 cg, j1 = NBP/2 + 4 cg)
  const int c0 = 4 * cgi, c1 = half + 4 * cgi;
  const int a0 = NS == 1 ? 0 : c0 / G.nbp, j0 = c0 - a0 * G.nbp;
  const int a1 = NS == 1 ? 0 : c1 / G.nbp, j1 = c1 - a1 * G.nbp;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  if (tid == 0) {
    P.sp = 0;
    for (int r = 3; r >= 0; --r) region_poly(pc, r, P.stack[P.sp++]);
  }
  __syncthreads();
  const float mu = pc.mu;
  const int qq = q * q;
  unsigned long long pair_nodes = 0;
  while (true) {
    if (tid == 0) fill_patches(P, cos_max);
    __syncthreads();
    const int npatch = P.npatch;
    if (npatch == 0) break;
    const int nodes = npatch * qq;
    pair_nodes += nodes;
    for (int base = 0; base < nodes; base += G.nc) {
      if (tid < 2 * G.nc) {
        const bool is_q = tid >= G.nc;
        const int kl = is_q ? tid - G.nc : tid;
        const int k = base + kl;
        if (k < nodes) {
          const int pi = k / qq;
          const int rem = k - pi * qq;
          const int i = rem / q;
          const int j = rem - i * q;
          const NodeGeom<float> g = node_geom<float>(P.patch[pi], s_x[i], s_x[j], pc);
          if (!is_q) {
            float* row = zp + kl * G.ldp;
            zw::zernike_wide<float>(Np, g.d0, g.d1, [&](int idx, int, int, float z) { row[idx] = z; });
          } else {
            const float qx = pc.qscale * (g.d0 * pc.R1[0] + g.d1 * pc.R1[1] + g.d2 * pc.R1[2]);
            const float qy = pc.qscale * (g.d0 * pc.R2[0] + g.d1 * pc.R2[1] + g.d2 * pc.R2[2]);
            const int trw = G.trw;
            if constexpr (NS == 1) {
              float wnode = 0.f;
              if (g.valid) {
                // S = 2 |OBC| phi2(mu L_O) (Sec. 3.3); moment k: 2 |OBC| L_O^k phi2^(k)(mu L_O)
                float sk;
                if (moment == 0) {
                  sk = phi2<float>(mu * g.LO);
                } else {
                  sk = phi2_deriv<float>(moment, mu * g.LO);
                  for (int e = 0; e < moment; ++e) sk *= g.LO;
                }
                wnode = s_w[i] * s_w[j] * g.jac * 2.f * g.Anab * sk * media_weight<float>(pc, g.d0, g.d1, g.d2);
              }
              float* row = zq + kl * G.ldq;
              zw::zernike_wide<float>(q_last, qx, qy, [&](int idx, int, int, float z) {
                const int a = idx - row0;
                if (a >= 0 && a < trw) row[a] = wnode * z;
              });
            } else {
              float M[3][3];
              float wdir = 0.f;
              if (g.valid) {
                const float sA = pc.mA[0] * g.d0 + pc.mA[1] * g.d1 + pc.mA[2] * g.d2;
                const float sB = pc.mB[0] * g.d0 + pc.mB[1] * g.d1 + pc.mB[2] * g.d2;
                const float sC = pc.mC[0] * g.d0 + pc.mC[1] * g.d1 + pc.mC[2] * g.d2;
                p1::p1_spatial(sA, sB, sC, g.d2, g.Anab, mu * g.LO, s_pos, M);
                wdir = s_w[i] * s_w[j] * g.jac;
              } else {
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                  for (int a = 0; a < 3; ++a) M[b][a] = 0.f;
              }
              float* row = zq + kl * G.ldq;
              const int plane = G.nc * G.ldq;
              zw::zernike_wide<float>(Np, qx, qy, [&](int idx, int, int, float z) {
                const float wz = wdir * z;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                  const int r = b * NB + idx - row0;
                  if (r >= 0 && r < trw) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) row[a * plane + r] = wz * M[b][a];
                  }
                }
              });
            }
          }
        }
      }
      __syncthreads();
      if (acc_thread) {
        const int kmax = min(G.nc, nodes - base);
        const float* pa0 = zq + a0 * G.nc * G.ldq + 8 * rgi;
        const float* pa1 = NS == 1 ? pa0 : zq + a1 * G.nc * G.ldq + 8 * rgi;
        const float* pb0 = zp + j0;
        const float* pb1 = zp + j1;
#pragma unroll 2
        for (int kk = 0; kk < kmax; ++kk) {
          float av[8], aw[8];
          {
            const float4 u0 = *reinterpret_cast<const float4*>(pa0 + kk * G.ldq);
            const float4 u1 = *reinterpret_cast<const float4*>(pa0 + kk * G.ldq + 4);
            av[0] = u0.x; av[1] = u0.y; av[2] = u0.z; av[3] = u0.w;
            av[4] = u1.x; av[5] = u1.y; av[6] = u1.z; av[7] = u1.w;
          }
          if constexpr (NS == 1) {
#pragma unroll
            for (int r = 0; r < 8; ++r) aw[r] = av[r];
          } else {
            const float4 u0 = *reinterpret_cast<const float4*>(pa1 + kk * G.ldq);
            const float4 u1 = *reinterpret_cast<const float4*>(pa1 + kk * G.ldq + 4);
            aw[0] = u0.x; aw[1] = u0.y; aw[2] = u0.z; aw[3] = u0.w;
            aw[4] = u1.x; aw[5] = u1.y; aw[6] = u1.z; aw[7] = u1.w;
          }
          const float4 b0 = *reinterpret_cast<const float4*>(pb0 + kk * G.ldp);
          const float4 b1 = *reinterpret_cast<const float4*>(pb1 + kk * G.ldp);
          const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                make_float2(b1.z, b1.w)};
#pragma unroll
          for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float ar = c < 2 ? av[r] : aw[r];
              const float2 s2 = __ffma2_rn(make_float2(ar, ar), bv[c], make_float2(acc[r][2 * c], acc[r][2 * c + 1]));
              acc[r][2 * c] = s2.x;
              acc[r][2 * c + 1] = s2.y;
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0 && blockIdx.y == 0) atomicAdd(node_count, pair_nodes);
  if (!acc_thread) return;
  // epilogue: scale row (b, i) by lambda N_i / sqrt(|T_l||T_l'|) and store
  TO* out = vals + (int64_t)pc.out_row * row_stride + (int64_t)pc.slot * NR * NR;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int ar = row0 + 8 * rgi + r;
    if (ar >= NR) continue;
    const float s = pc.scale * s_ninv[8 * rgi + r];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int jj = c < 4 ? j0 + c : j1 + (c - 4);
      const int sa = c < 4 ? a0 : a1;
      if (jj < NB) out[(int64_t)ar * NR + sa * NB + jj] = (TO)(acc[r][c] * s);
    }
  }
}

// ---------------------------------------------------------------------------
// Forward application y = x0 + alpha B x: block per operator row R (strided),
// the row's source coefficients (tet t = recv[R] / 4, its faces other than
// the exit face recv[R] % 4, in slot order) staged in shared memory, warp per
// test index a reading B[R][k][a][.] with coalesced loads, a shuffle
// reduction per (a, right-hand side).
// ---------------------------------------------------------------------------
template <typename TX, typename TA>
__global__ void __launch_bounds__(256)
spmv_wide_kernel(const float* __restrict__ vals, int64_t row_stride, const int32_t* __restrict__ recv, int64_t nrows,
                 int nb, const TX* __restrict__ x, const TX* x0, TX* y, int R, TA alpha) {
  extern __shared__ __align__(16) unsigned char spmv_wsm[];
  TA* xs = reinterpret_cast<TA*>(spmv_wsm);  // [3][nb]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t total = nrows * nb;
  const int64_t nb2 = (int64_t)nb * nb;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int32_t src = recv[row];
    const int64_t t = src >> 2;
    const int e = src & 3;
    const float* brow = vals + row * row_stride;
    for (int r = 0; r < R; ++r) {
      __syncthreads();  // the previous right-hand side's readers are done
      for (int i = threadIdx.x; i < 3 * nb; i += blockDim.x) {
        const int k = i / nb, j = i - k * nb;
        const int f = k + (k >= e ? 1 : 0);
        xs[i] = (TA)x[r * total + (4 * t + f) * nb + j];
      }
      __syncthreads();
      for (int a = warp; a < nb; a += nw) {
        TA acc = TA(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float* bp = brow + k * nb2 + (int64_t)a * nb;
          const TA* xk = xs + k * nb;
#pragma unroll
          for (int u = 0; u < 8; ++u) {  // nb <= 256
            const int j = lane + 32 * u;
            if (j < nb) acc = fma((TA)__ldg(bp + j), xk[j], acc);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          const int64_t o = r * total + row * nb + a;
          const TA base = x0 ? (TA)x0[o] : TA(0);
          y[o] = (TX)(base + alpha * acc);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Directed boundary source (Eq. RhoNeumann), one thread per source: the
// coefficients N_nm Z_n^m(p_d) sqrt|T| of the unit-mass delta at p_d.
// ---------------------------------------------------------------------------
__global__ void directed_source_wide_kernel(int Np, const FaceGeom* __restrict__ geom, const int64_t* __restrict__ rows,
                                            const double* __restrict__ dirs, int n_src, int64_t nrows, int combine,
                                            double* __restrict__ rho0, int* __restrict__ bad, int stride) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int64_t r = rows[s];
  const FaceGeom F = geom[r];
  double px = 0.0, py = 0.0;  // the inward normal: p = 0
  if (dirs) {
    double d[3] = {dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2]};
    const double inv = 1.0 / sqrt(dot3(d, d));
    for (int c = 0; c < 3; ++c) d[c] *= inv;
    if (!(dot3(d, F.n) > 0.0)) {
      atomicOr(bad, 1);
      return;
    }
    px = dot3(d, F.e1);
    py = dot3(d, F.e2);
  }
  const double sa = sqrt(F.area);
  double* out = rho0 + ((combine ? 0 : (int64_t)s * nrows) + r) * stride;
  zw::zernike_wide<double>(Np, px, py, [&](int idx, int n, int m, double z) {
    out[idx] = (2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI) * z * sa;
  });
}

// ---------------------------------------------------------------------------
// Interior density coefficients at the centroid of a listed tet (Eq. IntDens),
// FP64: block per (listed tet, face), passes of 32 nodes whose kernel weight
// and Zernike vector warp 0 evaluates into shared memory, thread a summing
// basis functions a and a + 128 over the pass.  POLAR: the split polar rule of
// interior_rule.cuh (6 nq^2 nodes); otherwise the collapsed Gauss rule.
// ---------------------------------------------------------------------------
constexpr int kDensPass = 32;

template <bool POLAR, int NS>
__global__ void __launch_bounds__(128)
interior_density_wide_kernel(int Np, const double* __restrict__ V, const int32_t* __restrict__ tets,
                             const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet, double mu_uniform,
                             const int64_t* __restrict__ list, const double* __restrict__ weights,
                             const double* __restrict__ gl_x, const double* __restrict__ gl_w, int nq,
                             double* __restrict__ gvec, double* __restrict__ dgvec) {
  extern __shared__ __align__(16) double dens_wsm[];
  const int NB = (Np + 1) * (Np + 2) / 2;  // Zernike functions
  const int NR = NS * NB;                   // unknowns per row
  double* zs = dens_wsm;                    // [32][NB]
  double* kw = zs + kDensPass * NB;         // [NS][32] kernel weights (times each face function)
  double* kd = kw + NS * kDensPass;         // [NS][32] their mu-derivatives
  const int tid = threadIdx.x;
  const int i = (int)(blockIdx.x >> 2);
  const int l = (int)(blockIdx.x & 3);
  const int64_t e = list[i];
  const double wt = weights ? weights[i] : 1.0;
  const int32_t* tv = tets + 4 * e;
  double r[3] = {0, 0, 0};
  for (int v = 0; v < 4; ++v)
    for (int c = 0; c < 3; ++c) r[c] += 0.25 * V[3 * (int64_t)tv[v] + c];
  const FaceGeom F = geom[4 * e + l];
  double p[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) p[k][c] = V[3 * (int64_t)tv[(l + 1 + k) & 3] + c];
  // face vertices in plane coordinates (for barycentrics of the nodes' points)
  double fx1 = 0, fy1 = 0, fx2 = 0, fy2 = 0;
  for (int c = 0; c < 3; ++c) {
    fx1 += (p[1][c] - p[0][c]) * F.e1[c];
    fy1 += (p[1][c] - p[0][c]) * F.e2[c];
    fx2 += (p[2][c] - p[0][c]) * F.e1[c];
    fy2 += (p[2][c] - p[0][c]) * F.e2[c];
  }
  const double fdet = fx1 * fy2 - fx2 * fy1;
  const double mu = mu_tet ? mu_tet[e] : mu_uniform;
  double g0 = 0.0, g1 = 0.0, d0 = 0.0, d1 = 0.0;
  const int nodes = POLAR ? 6 * nq * nq : nq * nq;
  for (int base = 0; base < nodes; base += kDensPass) {
    if (tid < kDensPass) {
      const int k = base + tid;
      double ker = 0.0, dist = 0.0, dx = 0.0, dy = 0.0;
      double lb[3] = {1.0, 0.0, 0.0};  // barycentrics of the node's face point
      if (k < nodes) {
        if constexpr (POLAR) {
          const rule::PolarNode qn = rule::polar_node(p, F.n, F.e1, F.e2, r, nq, k, gl_x, gl_w);
          if (qn.w != 0.0) {
            ker = qn.w * exp(-mu * qn.R);
            dist = qn.R;
            dx = qn.dx;
            dy = qn.dy;
            if constexpr (NS > 1) {
              // the face point s = r - R unit(r - s), unit(r - s) = dx e1 + dy e2 + dz n
              const double dz = sqrt(fmax(0.0, 1.0 - dx * dx - dy * dy));
              double x = 0, y = 0;
              for (int c = 0; c < 3; ++c) {
                const double sc = r[c] - qn.R * (dx * F.e1[c] + dy * F.e2[c] + dz * F.n[c]) - p[0][c];
                x += sc * F.e1[c];
                y += sc * F.e2[c];
              }
              lb[1] = (fy2 * x - fx2 * y) / fdet;
              lb[2] = (-fy1 * x + fx1 * y) / fdet;
              lb[0] = 1.0 - lb[1] - lb[2];
            }
          }
        } else {
          const int ii = k / nq, jj = k - ii * nq;
          const double u = 0.5 * (1.0 + gl_x[ii]);
          const double v = (1.0 - u) * 0.5 * (1.0 + gl_x[jj]);
          const double w = gl_w[ii] * gl_w[jj] * 0.25 * (1.0 - u) * 2.0 * F.area;
          double rs[3];
          for (int c = 0; c < 3; ++c) rs[c] = r[c] - (p[0][c] + u * (p[1][c] - p[0][c]) + v * (p[2][c] - p[0][c]));
          dist = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
          const double id = 1.0 / dist;
          const double e0 = rs[0] * id, e1 = rs[1] * id, e2 = rs[2] * id;
          const double cosv = e0 * F.n[0] + e1 * F.n[1] + e2 * F.n[2];
          ker = w * cosv * exp(-mu * dist) * id * id;
          dx = e0 * F.e1[0] + e1 * F.e1[1] + e2 * F.e1[2];
          dy = e0 * F.e2[0] + e1 * F.e2[1] + e2 * F.e2[2];
          lb[0] = 1.0 - u - v;
          lb[1] = u;
          lb[2] = v;
        }
      }
#pragma unroll
      for (int sp = 0; sp < NS; ++sp) {
        const double ph = NS == 1 ? 1.0 : p1::value_d(sp, 0) * lb[0] + p1::value_d(sp, 1) * lb[1] +
                                              p1::value_d(sp, 2) * lb[2];
        kw[sp * kDensPass + tid] = ker * ph;
        kd[sp * kDensPass + tid] = -dist * ker * ph;
      }
      double* row = zs + tid * NB;
      zw::zernike_wide<double>(Np, dx, dy, [&](int idx, int, int, double z) { row[idx] = z; });
    }
    __syncthreads();
    const int kmax = min(kDensPass, nodes - base);
    const int s0 = tid / NB, i0 = tid - s0 * NB;              // unknown tid = s0 NB + i0
    const int s1 = (tid + 128) / NB, i1 = tid + 128 - s1 * NB;  // unknown tid + 128
    for (int kk = 0; kk < kmax; ++kk) {
      if (tid < NR) {
        const double z = zs[kk * NB + i0];
        g0 = fma(kw[s0 * kDensPass + kk], z, g0);
        d0 = fma(kd[s0 * kDensPass + kk], z, d0);
      }
      if (tid + 128 < NR) {
        const double z = zs[kk * NB + i1];
        g1 = fma(kw[s1 * kDensPass + kk], z, g1);
        d1 = fma(kd[s1 * kDensPass + kk], z, d1);
      }
    }
    __syncthreads();
  }
  const double s = wt / sqrt(F.area);
  double* gr = gvec + (4 * e + l) * NR;
  double* dr = dgvec ? dgvec + (4 * e + l) * NR : nullptr;
  if (tid < NR) {
    atomicAdd(&gr[tid], s * g0);
    if (dr) atomicAdd(&dr[tid], s * d0);
  }
  if (tid + 128 < NR) {
    atomicAdd(&gr[tid + 128], s * g1);
    if (dr) atomicAdd(&dr[tid + 128], s * d1);
  }
}

int device_sms() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return std::max(nsm, 1);
}

}  // namespace

int launch_assemble_wide(int Np, const void* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                         float cos_max, float* vals, int64_t row_stride, unsigned long long* nodes, int moment,
                         cudaStream_t st) {
  if (Np <= 8 || Np > geom::kWideMaxNp) return set_error(DFM_ERR_ARG, "dfm_assemble: the wide assembly takes Np in 9..20");
  if (q < 1 || q > kMaxQ) return set_error(DFM_ERR_ARG, "dfm_assemble: quad_order must be in 1..32");
  if (npairs > 0x7fffffff) return set_error(DFM_ERR_ARG, "dfm_assemble: too many face pairs");
  if (npairs == 0) return DFM_OK;
  const geom::WideAsm G = geom::wide_asm_geometry(nbasis(Np));
  if (G.smem > 200 * 1024 || G.threads > 256)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: wide assembly tile does not fit a block");
  DFM_CUDA_CHECK(cudaFuncSetAttribute(assemble_wide_kernel<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)G.smem));
  const dim3 grid((unsigned)npairs, (unsigned)G.ntile);
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_ASSEMBLE, st);
    assemble_wide_kernel<1, float><<<grid, G.threads, G.smem, st>>>(reinterpret_cast<const PairConst*>(pairs),
                                                                    nullptr, glx, glw, q, cos_max, vals, row_stride,
                                                                    nodes, moment, Np, G);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

int launch_assemble_p1(const dfm_mesh* mesh, int Np, const void* pairs, void* pos_scratch, int64_t npairs,
                       const double* glx, const double* glw, int q, float cos_max, float* vals, int64_t row_stride,
                       unsigned long long* nodes, cudaStream_t st) {
  if (Np < 0 || Np > 8) return set_error(DFM_ERR_ARG, "dfm_assemble: the linear spatial basis takes Np in 0..8");
  if (q < 1 || q > kMaxQ) return set_error(DFM_ERR_ARG, "dfm_assemble: quad_order must be in 1..32");
  if (npairs > 0x7fffffff) return set_error(DFM_ERR_ARG, "dfm_assemble: too many face pairs");
  if (npairs == 0) return DFM_OK;
  if (reinterpret_cast<uintptr_t>(pos_scratch) & 7) return set_error(DFM_ERR_ARG, "dfm_assemble: scratch alignment");
  int2* pos = reinterpret_cast<int2*>(pos_scratch);
  p1_setup_kernel<<<(unsigned)((npairs + 127) / 128), 128, 0, st>>>(mesh->tets, mesh->recv, npairs, pos);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  const geom::WideAsm G = geom::wide_asm_geometry(nbasis(Np), 3);
  if (G.smem > 200 * 1024 || G.threads > 256)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: linear-basis assembly tile does not fit a block");
  DFM_CUDA_CHECK(cudaFuncSetAttribute(assemble_wide_kernel<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)G.smem));
  const dim3 grid((unsigned)npairs, (unsigned)G.ntile);
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_ASSEMBLE, st);
    assemble_wide_kernel<3, float><<<grid, G.threads, G.smem, st>>>(reinterpret_cast<const PairConst*>(pairs), pos,
                                                                    glx, glw, q, cos_max, vals, row_stride, nodes, 0,
                                                                    Np, G);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

template <typename TX>
int apply_wide_t(const dfm_op* op, const TX* x, const TX* x0, TX* y, int R, double alpha, cudaStream_t st) {
  if (op->precision != DFM_F32) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: bases above Np = 8 need FP32 blocks");
  if (op->nb > 256) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: basis too large");
  const int32_t* recv = op->recv ? op->recv : op->mesh->recv;
  const size_t smem = 3 * (size_t)op->nb * sizeof(TX);
  const int64_t grid = std::min<int64_t>(op->nrows, (int64_t)device_sms() * 8);
  if (grid < 1) return DFM_OK;
  {
    ::dfm::KernelTimer timer_(sizeof(TX) == 8 ? DFM_KERNEL_SPMV64 : DFM_KERNEL_SPMV, st);
    spmv_wide_kernel<TX, TX><<<(unsigned)grid, 256, smem, st>>>(reinterpret_cast<const float*>(op->vals),
                                                                op->row_stride, recv, op->nrows, op->nb, x, x0, y, R,
                                                                (TX)alpha);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

int apply_wide(const dfm_op* op, const float* x, const float* x0, float* y, int R, double alpha, cudaStream_t st) {
  return apply_wide_t<float>(op, x, x0, y, R, alpha, st);
}

int apply_wide(const dfm_op* op, const double* x, const double* x0, double* y, int R, double alpha,
               cudaStream_t st) {
  return apply_wide_t<double>(op, x, x0, y, R, alpha, st);
}

int launch_directed_source_wide(int Np, const FaceGeom* geom, const int64_t* rows, const double* dirs, int n_src,
                                int64_t nrows, int combine, double* rho0, int* bad, int stride, cudaStream_t st) {
  directed_source_wide_kernel<<<(unsigned)((n_src + 127) / 128), 128, 0, st>>>(Np, geom, rows, dirs, n_src, nrows,
                                                                               combine, rho0, bad, stride);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

int launch_interior_density_wide(int Np, int ns, bool polar, const dfm_mesh* mesh, const double* mu,
                                 double mu_uniform, const int64_t* list, const double* weights, int n,
                                 const double* glx, const double* glw, int nq, double* gvec, double* dgvec,
                                 cudaStream_t st) {
  if (ns * nbasis(Np) > 256) return set_error(DFM_ERR_UNSUPPORTED, "dfm_interior_density: basis too large");
  const size_t smem = ((size_t)kDensPass * nbasis(Np) + 2 * ns * kDensPass) * sizeof(double);
  const unsigned blocks = (unsigned)(4 * (int64_t)n);
  auto go = [&](auto kernel) -> int {
    DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kernel<<<blocks, 128, smem, st>>>(Np, mesh->verts, mesh->tets, mesh->geom, mu, mu_uniform, list, weights, glx,
                                      glw, nq, gvec, dgvec);
    return DFM_OK;
  };
  int rc;
  if (ns == 1)
    rc = polar ? go(interior_density_wide_kernel<true, 1>) : go(interior_density_wide_kernel<false, 1>);
  else
    rc = polar ? go(interior_density_wide_kernel<true, 3>) : go(interior_density_wide_kernel<false, 3>);
  if (rc) return rc;
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

}  // namespace dfm
