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

#include <cuda_bf16.h>

#include "dfm_internal.cuh"
#include "node.cuh"

#include <algorithm>
#include <cstddef>
#include <type_traits>

namespace dfm {
namespace {

// Store one staged row: scale * v[0..NB) followed by zeros up to NBP, as
// 16-byte vectors for FP32 (rows are 16-byte aligned, see Tile::LD).
template <int NBP, int NB, typename T>
__device__ __forceinline__ void stage_row(T* row, const T* v, T scale) {
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int u = 0; u < NBP / 4; ++u) {
      float4 q;
      q.x = (4 * u + 0 < NB) ? scale * v[4 * u + 0 < NB ? 4 * u + 0 : 0] : 0.f;
      q.y = (4 * u + 1 < NB) ? scale * v[4 * u + 1 < NB ? 4 * u + 1 : 0] : 0.f;
      q.z = (4 * u + 2 < NB) ? scale * v[4 * u + 2 < NB ? 4 * u + 2 : 0] : 0.f;
      q.w = (4 * u + 3 < NB) ? scale * v[4 * u + 3 < NB ? 4 * u + 3 : 0] : 0.f;
      *reinterpret_cast<float4*>(row + 4 * u) = q;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NBP; ++c) row[c] = c < NB ? scale * v[c < NB ? c : 0] : T(0);
  }
}

// Load N consecutive staged values with the widest aligned vector loads.
template <int N, typename T>
__device__ __forceinline__ void load_run(const T* p, T* out) {
  if constexpr (std::is_same<T, float>::value && N % 4 == 0) {
#pragma unroll
    for (int u = 0; u < N / 4; ++u) {
      const float4 q = *reinterpret_cast<const float4*>(p + 4 * u);
      out[4 * u] = q.x;
      out[4 * u + 1] = q.y;
      out[4 * u + 2] = q.z;
      out[4 * u + 3] = q.w;
    }
  } else if constexpr (std::is_same<T, float>::value && N % 2 == 0) {
#pragma unroll
    for (int u = 0; u < N / 2; ++u) {
      const float2 q = *reinterpret_cast<const float2*>(p + 2 * u);
      out[2 * u] = q.x;
      out[2 * u + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < N; ++u) out[u] = p[u];
  }
}

// Shared memory of one warp: patch state plus the staged node vectors.
template <int NP, typename T>
struct WarpSmem {
  PatchSmem P;
  alignas(16) T zq[32 * Tile<NP>::LD];  // w * Z(p') per node (16-byte aligned rows)
  alignas(16) T zp[32 * Tile<NP>::LD];  // Z(p) per node
};

// QC > 0 fixes the per-patch Gauss order at compile time (the default
// N_p + 6), which turns the node-index divisions into multiplies.
// TO: storage type of the blocks (T, or BF16 rounded from FP32 sums).
template <int NP, typename T, int QC, typename TO>
__global__ void __launch_bounds__(kWarps * 32)
assemble_kernel(const PairConst* __restrict__ pairs, int64_t npairs, const double* __restrict__ gl_x,
                const double* __restrict__ gl_w, int q_rt, float cos_max, TO* __restrict__ vals, int64_t row_stride,
                unsigned long long* __restrict__ node_count, int moment) {
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
  const int q = QC > 0 ? QC : q_rt;
  if (threadIdx.x < q) {
    s_x[threadIdx.x] = (T)gl_x[threadIdx.x];
    s_w[threadIdx.x] = (T)gl_w[threadIdx.x];
  }
  if (threadIdx.x < NB) s_ninv[threadIdx.x] = zernike_invnorm(threadIdx.x);
  __syncthreads();
  const int qq = q * q;
  const int a0 = (lane >> 2) * TR;
  const int b0 = (lane & 3) * TC;

  {
    const int64_t p = (int64_t)blockIdx.x * kWarps + wid;
    if (p >= npairs) return;  // no block-wide barrier follows
    const PairConst pc = pairs[p];
    if (pc.kind < 0) return;  // no block for this pair in this part
    T acc[TR][TC];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int c = 0; c < TC; ++c) acc[r][c] = T(0);
    if (lane == 0) {
      S.P.sp = 0;
      for (int r = 3; r >= 0; --r) region_poly(pc, r, S.P.stack[S.P.sp++]);
    }
    __syncwarp();
    const T mu = pc.mu;
    unsigned long long pair_nodes = 0;
    while (true) {
      if (lane == 0) fill_patches(S.P, cos_max);
      __syncwarp();
      const int npatch = S.P.npatch;
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
          const NodeGeom<T> g = node_geom<T>(S.P.patch[pi], s_x[i], s_x[j], pc);
          if (g.valid) {
            // S = 2 |OBC| phi2(mu L_O) (Sec. 3.3); moment k: d^k S / d mu^k = 2 |OBC| L_O^k phi2^(k)(mu L_O)
            T sk;
            if (moment == 0) {
              sk = phi2<T>(mu * g.LO);
            } else {
              sk = phi2_deriv<T>(moment, mu * g.LO);
              for (int e = 0; e < moment; ++e) sk *= g.LO;
            }
            wnode = s_w[i] * s_w[j] * g.jac * T(2) * g.Anab * sk * media_weight<T>(pc, g.d0, g.d1, g.d2);
          }
          const T d0 = g.d0, d1 = g.d1, d2 = g.d2;
          zernike<NP, T>(d0, d1, Zp);
          // receiving momentum (scaled by c_i / c_j after a refraction)
          const T qx = (T)pc.qscale * (d0 * (T)pc.R1[0] + d1 * (T)pc.R1[1] + d2 * (T)pc.R1[2]);
          const T qy = (T)pc.qscale * (d0 * (T)pc.R2[0] + d1 * (T)pc.R2[1] + d2 * (T)pc.R2[2]);
          zernike<NP, T>(qx, qy, Zq);
        } else {
#pragma unroll
          for (int c = 0; c < NB; ++c) Zp[c] = Zq[c] = T(0);
        }
        stage_row<TL::NBP, NB>(&S.zq[lane * LD], Zq, wnode);
        stage_row<TL::NBP, NB>(&S.zp[lane * LD], Zp, T(1));
        __syncwarp();
        const int kmax = min(32, nodes - base);
#pragma unroll 2
        for (int kk = 0; kk < kmax; ++kk) {
          T av[TR], bv[TC];
          load_run<TR>(&S.zq[kk * LD + a0], av);
          load_run<TC>(&S.zp[kk * LD + b0], bv);
          if constexpr (std::is_same<T, float>::value) {
            // packed FP32 FMAs (two independent roundings, the same results
            // as scalar FMAs) halve the instructions of the rank-1 update
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              const float2 a2 = make_float2(av[r], av[r]);
#pragma unroll
              for (int c = 0; c < TC; c += 2) {
                const float2 p2 = __ffma2_rn(a2, make_float2(bv[c], bv[c + 1]), make_float2(acc[r][c], acc[r][c + 1]));
                acc[r][c] = p2.x;
                acc[r][c + 1] = p2.y;
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
              for (int c = 0; c < TC; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
          }
        }
        __syncwarp();
      }
    }
    if (lane == 0) atomicAdd(node_count, pair_nodes);
    // epilogue: scale row a by lambda N_a / sqrt(|T_l||T_l'|) and store
    TO* out = vals + (int64_t)pc.out_row * row_stride + (int64_t)pc.slot * NB * NB;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      const int a = a0 + r;
      if (a >= NB) continue;
      const T s = (T)pc.scale * (T)s_ninv[a];
#pragma unroll
      for (int c = 0; c < TC; ++c) {
        const int b = b0 + c;
        if (b < NB) {
          if constexpr (std::is_same<TO, __nv_bfloat16>::value)
            out[a * NB + b] = __float2bfloat16_rn(acc[r][c] * s);
          else
            out[a * NB + b] = acc[r][c] * s;
        }
      }
    }
    __syncwarp();
  }
}

using WarpSmem4f = WarpSmem<4, float>;
using WarpSmem8f = WarpSmem<8, float>;
static_assert(offsetof(WarpSmem4f, zq) % 16 == 0 && sizeof(WarpSmem4f) % 16 == 0, "16-byte aligned staging rows");
static_assert(offsetof(WarpSmem8f, zq) % 16 == 0 && sizeof(WarpSmem8f) % 16 == 0, "16-byte aligned staging rows");

template <int NP, typename T>
constexpr size_t assemble_smem_bytes() {
  return sizeof(WarpSmem<NP, T>) * kWarps + 2 * kMaxQ * sizeof(T) + 64 * sizeof(float);
}

template <int NP, typename T, int QC, typename TO>
int launch_assemble_q(const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                      float cos_max, TO* vals, int64_t row_stride, unsigned long long* nodes, int moment,
                      cudaStream_t st) {
  constexpr size_t smem = assemble_smem_bytes<NP, T>();
  static_assert(smem <= 220 * 1024, "assembly shared memory");
  DFM_CUDA_CHECK(
      cudaFuncSetAttribute(assemble_kernel<NP, T, QC, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (npairs + kWarps - 1) / kWarps;
  if (blocks > 0x7fffffff) return set_error(DFM_ERR_ARG, "dfm_assemble: too many face pairs");
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_ASSEMBLE, st);
    assemble_kernel<NP, T, QC, TO><<<(unsigned)blocks, kWarps * 32, smem, st>>>(pairs, npairs, glx, glw, q, cos_max,
                                                                                vals, row_stride, nodes, moment);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

template <int NP, typename T, typename TO>
int launch_assemble(const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                    float cos_max, TO* vals, int64_t row_stride, unsigned long long* nodes, int moment,
                    cudaStream_t st) {
  if (std::is_same<T, float>::value && q == NP + 6)
    return launch_assemble_q<NP, T, NP + 6, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment,
                                                st);
  return launch_assemble_q<NP, T, 0, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
}

template <typename T, typename TO = T>
int dispatch_np(int Np, const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                float cos_max, TO* vals, int64_t row_stride, unsigned long long* nodes, int moment, cudaStream_t st) {
  switch (Np) {
    case 0: return launch_assemble<0, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 1: return launch_assemble<1, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 2: return launch_assemble<2, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 3: return launch_assemble<3, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 4: return launch_assemble<4, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 5: return launch_assemble<5, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 6: return launch_assemble<6, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 7: return launch_assemble<7, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    case 8: return launch_assemble<8, T, TO>(pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
    default:
      // N_p = 9..20: one block per (face pair, tile of test rows), FP32 blocks
      if constexpr (std::is_same<T, float>::value && std::is_same<TO, float>::value)
        return launch_assemble_wide(Np, pairs, npairs, glx, glw, q, cos_max, vals, row_stride, nodes, moment, st);
      return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: Np above 8 is built for FP32 blocks only");
  }
}

int check_params(const dfm_mesh* mesh, const dfm_params* p) {
  if (!mesh || !p) return set_error(DFM_ERR_ARG, "dfm_assemble: NULL mesh or params");
  if (!basis_ok(p->Np, geom::kWideMaxNp))
    return set_error(DFM_ERR_ARG, "dfm_assemble: Np must be in 0..20 (0..8 with the linear spatial basis)");
  const int np = basis_np(p->Np);
  if (p->precision != DFM_F32 && p->precision != DFM_F64 && p->precision != DFM_BF16)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: precision must be DFM_F32, DFM_F64 or DFM_BF16");
  if (np > 8 && p->precision != DFM_F32)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: Np above 8 is built for DFM_F32 only");
  if (basis_ns(p->Np) > 1 && (p->precision != DFM_F32 || p->moment != 0 || p->c || p->rho_f))
    return set_error(DFM_ERR_UNSUPPORTED,
                     "dfm_assemble: the linear spatial basis is built for DFM_F32, moment 0 and uniform media");
  if (!p->mu && !(p->mu_uniform >= 0.0)) return set_error(DFM_ERR_ARG, "dfm_assemble: mu_uniform must be >= 0");
  const int q = p->quad_order ? p->quad_order : np + 6;
  if (q < 1 || q > kMaxQ) return set_error(DFM_ERR_ARG, "dfm_assemble: quad_order must be in 1..32");
  const double deg = p->max_patch_deg > 0 ? p->max_patch_deg : 60.0;
  if (!(deg >= 10.0 && deg <= 180.0)) return set_error(DFM_ERR_ARG, "dfm_assemble: max_patch_deg must be in [10, 180]");
  if (p->moment < 0 || p->moment > 3) return set_error(DFM_ERR_ARG, "dfm_assemble: moment must be in 0..3");
  if ((p->c || p->rho_f) && p->moment != 0)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_assemble: damping moments are built for uniform media only");
  return DFM_OK;
}

// identity row map of a reflection operator: row R receives from R's own tet
__global__ void iota_kernel(int32_t* __restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = (int32_t)i;
}

// the reflected part of op (heterogeneous media), created on first use; its
// time-out flag is op's
int ensure_reflection(dfm_op* op, cudaStream_t st) {
  if (op->rop) return DFM_OK;
  dfm_op* r = new dfm_op();
  r->mesh = op->mesh;
  r->Np = op->Np;
  r->ns = op->ns;
  r->nb = op->nb;
  r->precision = op->precision;
  r->nrows = op->nrows;
  r->row_stride = op->row_stride;
  r->bytes = op->bytes;
  r->dev_err = op->dev_err;
  cudaError_t e = cudaMalloc(&r->vals, r->bytes);
  if (e == cudaSuccess) e = cudaMalloc(&r->own_recv, sizeof(int32_t) * r->nrows);
  if (e != cudaSuccess) {
    cudaFree(r->vals);
    cudaFree(r->own_recv);
    delete r;
    return cuda_error(e, "dfm_assemble: reflected part");
  }
  iota_kernel<<<(unsigned)std::min<int64_t>((r->nrows + 255) / 256, 4096), 256, 0, st>>>(r->own_recv, r->nrows);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  r->recv = r->own_recv;
  op->rop = r;
  return DFM_OK;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_assemble_into(const dfm_mesh* mesh, const dfm_params* p, dfm_op* op, void* stream) {
  int rc = check_params(mesh, p);
  if (rc) return rc;
  if (!op || op->mesh != mesh || op->Np != basis_np(p->Np) || op->ns != basis_ns(p->Np) ||
      op->precision != p->precision)
    return set_error(DFM_ERR_ARG, "dfm_assemble_into: operator does not match mesh/Np/precision");
  const int np = op->Np;
  cudaStream_t st = as_stream(stream);
  op->lp_valid = false;  // the low-precision preconditioner copies follow the blocks
  op->lpT_valid = false;
  op->mu_uniform = p->mu ? -1.0 : p->mu_uniform;
  op->moment = p->moment;
  const int q = p->quad_order ? p->quad_order : np + 6;
  const double deg = p->max_patch_deg > 0 ? p->max_patch_deg : 60.0;
  const float cos_max = (float)cos(deg * M_PI / 180.0);
  const int64_t npairs = 12 * mesh->nt;
  // scratch: per-pair constants and the Gauss table, kept with the operator
  // (the linear spatial basis adds two words of vertex positions per pair)
  const int64_t base_need = npairs * (int64_t)sizeof(PairConst) + 2 * 64 * (int64_t)sizeof(double) + 256;
  const int64_t need = base_need + (op->ns > 1 ? 8 * npairs : 0);
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
  const bool media = p->c || p->rho_f;
  if (media) {
    rc = ensure_reflection(op, st);
    if (rc) return rc;
    op->rop->mu_uniform = op->mu_uniform;
    op->rop->moment = 0;
  } else if (op->rop) {  // uniform media now: no reflected part
    op->rop->dev_err = nullptr;
    dfm_op_destroy(op->rop);
    op->rop = nullptr;
  }
  const int bs = 128;
  // part 0: the blocks received across each exit face; part 1 (media): the
  // blocks reflected at interfaces, into the reflection operator
  for (int part = 0; part < (media ? 2 : 1); ++part) {
    dfm_op* dst = part == 0 ? op : op->rop;
    if (part == 1) DFM_CUDA_CHECK(cudaMemsetAsync(dst->vals, 0, dst->bytes, st));  // non-interface blocks stay 0
    pair_setup_kernel<<<(unsigned)((npairs + bs - 1) / bs), bs, 0, st>>>(mesh->verts, mesh->tets, mesh->recv,
                                                                         mesh->refl, mesh->geom, p->mu,
                                                                         p->mu_uniform, npairs, pairs, p->c,
                                                                         p->rho_f, part);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    if (op->ns > 1)
      rc = launch_assemble_p1(mesh, np, pairs, reinterpret_cast<char*>(op->work) + base_need, npairs, glx, glw, q,
                              cos_max, (float*)dst->vals, op->row_stride, nodes, st);
    else if (op->precision == DFM_F32)
      rc = dispatch_np<float>(np, pairs, npairs, glx, glw, q, cos_max, (float*)dst->vals, op->row_stride, nodes,
                              p->moment, st);
    else if (op->precision == DFM_BF16)
      rc = dispatch_np<float, __nv_bfloat16>(np, pairs, npairs, glx, glw, q, cos_max,
                                             (__nv_bfloat16*)dst->vals, op->row_stride, nodes, p->moment, st);
    else
      rc = dispatch_np<double>(np, pairs, npairs, glx, glw, q, cos_max, (double*)dst->vals, op->row_stride,
                               nodes, p->moment, st);
    if (rc) return rc;
  }
  return DFM_OK;
}

extern "C" int dfm_assemble(const dfm_mesh* mesh, const dfm_params* p, void* stream, dfm_op** out) {
  if (!out) return set_error(DFM_ERR_ARG, "dfm_assemble: out is NULL");
  *out = nullptr;
  int rc = check_params(mesh, p);
  if (rc) return rc;
  dfm_op* op = new dfm_op();
  op->mesh = mesh;
  op->Np = basis_np(p->Np);
  op->ns = basis_ns(p->Np);
  op->nb = basis_size(p->Np);
  op->precision = p->precision;
  op->nrows = mesh->nrows;
  op->row_stride = op_row_stride(op->nb);
  op->bytes = op->nrows * op->row_stride * elem_size(op->precision);
  cudaError_t e = cudaMalloc(&op->vals, op->bytes);
  if (e != cudaSuccess) {
    delete op;
    return cuda_error(e, "dfm_assemble: cudaMalloc(vals)");
  }
  e = cudaMalloc(&op->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(op->dev_err, 0, sizeof(int), as_stream(stream));
  if (e != cudaSuccess) {
    dfm_op_destroy(op);
    return cuda_error(e, "dfm_assemble: error flag");
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
  if (op->rop) {
    op->rop->dev_err = nullptr;  // shared with op
    dfm_op_destroy(op->rop);
  }
  cudaFree(op->own_recv);
  destroy_hop_graphs(op);
  forget_sweep(op->vals);
  forget_sweep(op->lp_vals);
  forget_sweep(op->lpT_vals);
  cudaFree(op->vals);
  cudaFree(op->work);
  cudaFree(op->swork);
  cudaFree(op->dev_err);
  cudaFree(op->lp_vals);
  cudaFree(op->lpT_vals);
  delete op;
}

extern "C" int dfm_op_info(const dfm_op* op, dfm_op_info_t* info) {
  if (!op || !info) return set_error(DFM_ERR_ARG, "dfm_op_info: NULL argument");
  info->Np = op->ns > 1 ? DFM_BASIS(op->Np, 1) : op->Np;
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

extern "C" int dfm_op_copy_reflected(const dfm_op* op, void* dst, int64_t bytes, void* stream) {
  if (!op || !dst) return set_error(DFM_ERR_ARG, "dfm_op_copy_reflected: NULL argument");
  if (!op->rop) return set_error(DFM_ERR_ARG, "dfm_op_copy_reflected: the operator has no reflected part");
  if (bytes != op->rop->bytes)
    return set_error(DFM_ERR_ARG, "dfm_op_copy_reflected: bytes must equal the operator size");
  DFM_CUDA_CHECK(cudaMemcpyAsync(dst, op->rop->vals, bytes, cudaMemcpyDefault, as_stream(stream)));
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
