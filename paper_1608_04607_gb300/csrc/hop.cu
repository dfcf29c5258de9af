// Polynomial-preconditioner hops on a low-precision copy of the blocks.
//
// The flexible inner solver evaluates z = p(B~) v = sum_{k<d} B~^k v by
// Horner's rule, z <- v + B~ z, with B~ the FP16 or BF16 rounding of the
// FP32 blocks, or their e4m3 rounding with one FP32 scale per operator row.
// A hop reads a half (a quarter) of the operator bytes of an FP32 application;
// the result only preconditions (the Arnoldi relation uses the FP32 operator),
// so the rounding costs accuracy of the preconditioner, not of the solution.
//
// Layouts, chosen so that a consumer thread reads whole vectors only:
//  - the copy: per operator row, per block k (3), per column chunk c
//    (NBP / 8 chunks, NBP = NB rounded up to 8), per test index a (NB): the 8
//    trial values b = 8c .. 8c+7 of B_k[a][.] (zero for b >= NB), 16 bytes
//    in FP16/BF16, 8 bytes in e4m3.  The threads forming outputs
//    a = 0..NB-1 of a row read consecutive chunks (no shared-memory bank
//    conflicts).  An e4m3 row ends (after padding to 16 bytes) with a 16-byte
//    field holding its FP32 scale s_R: the row's values are s_R q.
//  - hop vectors (v and the intermediate z): FP16 holding v times a power of
//    two (FP16 and e4m3 copies) or FP32 (BF16 copy), each face's NB
//    coefficients padded with zeros to NBP, so that a face starts on a
//    16-byte boundary and a tet's 4 faces form one 16-byte-aligned run.
// The last hop of a Horner chain writes the unpadded FP32 layout of the
// solver's vectors.
//
// The pipeline follows the FP32 application: a producer warp streams tiles of
// consecutive rows into shared memory - the operator rows and the x0 slice by
// bulk copies (TMA), each row's source-tet coefficients (a scattered 16-byte
// aligned run of 4 NBP values) by 16-byte cp.async copies issued by the
// producer lanes, all completing on the stage's mbarrier - and eight consumer
// warps form the outputs (one thread per row and padded test index).  Waits
// are bounded and a time-out sets the operator's error flag.  Measured at
// N_b = 15 (e4m3 copy): cp.async gathers and 16-row tiles took a hop from
// 41.5 to 36.8 us against bulk copies and 8-row tiles.
//
// The kernel and its launcher live in hop_kernel.cuh; hop_launch_*.cu
// instantiate them per copy format (parallel compilation).
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hop_frag.cuh"
#include "hop_kernel.cuh"
#include "tune.h"

namespace dfm {
namespace {

using namespace hopk;
using geom::kFragGroupMin;

// FP16 and e4m3 copies of bases padded to a multiple of 16 are stored
// fragment-ordered and hopped on tensor cores (hop_frag.cuh), except for one
// to three right-hand sides on the smallest such bases (padded width 16),
// whose rows are too short for the tensor-core consumer's per-row cost: there
// the CUDA-core hop on the chunk-ordered copy runs faster (29.5 against
// 39 us per e4m3 hop at N_b = 15 on 192,000 rows)
bool frag_copy(int nb, int precision, int R) {
  if (!geom::frag_basis(nb) || (precision != DFM_F16 && precision != DFM_FP8E4M3)) return false;
  return R >= kFragGroupMin || hop_nbp(nb) > 16;
}

// FP16/BF16 copy: element i of the copy <- its block entry (0 in pads); the
// blocks are FP32, or BF16 for a BF16 operator
// Entry e of row J of the copy.  Forward (recvT == NULL): row J's own blocks.
// Transposed: row J = 4t + l holds, for k = 0..2 and l' = the k-th face of t
// other than l, the block that face l of t sends to row R = recvT[4t + l'],
// transposed: entry (a, b) = B_{R, s}[b][a], s = l - (l > l') the slot of
// face l among the faces of t other than l'.
template <typename S>
__device__ __forceinline__ float copy_entry_at(const S* src, int64_t row_stride, const int32_t* recvT, int64_t J,
                                               int64_t e, int nb, int nbp) {
  if (!recvT) return copy_entry(src + J * row_stride, e, nb, nbp);
  const int k = (int)(e / ((int64_t)nb * nbp));
  int64_t rem = e - (int64_t)k * nb * nbp;
  const int c = (int)(rem / (nb * 8));
  rem -= (int64_t)c * nb * 8;
  const int a = (int)(rem / 8);
  const int b = c * 8 + (int)(rem - a * 8);
  if (b >= nb) return 0.f;
  const int l = (int)(J & 3);
  const int lq = k + (k >= l ? 1 : 0);
  const int64_t Rr = recvT[(J & ~int64_t(3)) + lq];
  const int slot = l - (l > lq ? 1 : 0);
  return (float)src[Rr * row_stride + (int64_t)slot * nb * nb + (int64_t)b * nb + a];
}

template <typename E, typename S>
__global__ void to_hop16_kernel(const S* __restrict__ src, int64_t row_stride, E* __restrict__ dst, int64_t nrows,
                                int nb, int nbp, const int32_t* __restrict__ recvT) {
  const int64_t row_elems = 3 * (int64_t)nb * nbp;
  const int64_t total = nrows * row_elems;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / row_elems;
    const int64_t e = i - row * row_elems;
    const float v = copy_entry_at(src, row_stride, recvT, row, e, nb, nbp);
    if constexpr (std::is_same<E, __half>::value)
      dst[i] = __float2half_rn(v);
    else
      dst[i] = __float2bfloat16_rn(v);
  }
}

// e4m3 copy: one warp per operator row; s_R = max |entry| / 448, q = e4m3(v / s_R)
template <typename S>
__global__ void to_hop8_kernel(const S* __restrict__ src, int64_t row_stride, unsigned char* __restrict__ dst,
                               int64_t nrows, int nb, int nbp, int64_t body_bytes, int64_t row_bytes,
                               const int32_t* __restrict__ recvT) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_entries = 3 * (int64_t)nb * nb;
  const int64_t n_vals = 3 * (int64_t)nb * nbp;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < nrows; row += warps) {
    float mx = 0.f;
    if (!recvT) {
      const S* sr = src + row * row_stride;
      for (int64_t e = lane; e < n_entries; e += 32) mx = fmaxf(mx, fabsf((float)sr[e]));
    } else {
      for (int64_t e = lane; e < n_vals; e += 32) mx = fmaxf(mx, fabsf(copy_entry_at(src, row_stride, recvT, row, e, nb, nbp)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = mx > 0.f ? mx / 448.f : 1.f;
    unsigned char* dr = dst + row * row_bytes;
    for (int64_t e = lane; e < body_bytes; e += 32) {
      const float v = e < n_vals ? copy_entry_at(src, row_stride, recvT, row, e, nb, nbp) : 0.f;
      dr[e] = (unsigned char)__nv_cvt_float_to_fp8(v / s, __NV_SATFINITE, __NV_E4M3);
    }
    if (lane < 4) reinterpret_cast<float*>(dr + body_bytes)[lane] = lane == 0 ? s : 0.f;
  }
}

// Fragment-ordered copy (hop_frag.cuh): one warp per row; FP16 values, or
// e4m3 values with s_R = max |entry| / 448 as in to_hop8_kernel.  Entry (a, b)
// of block k is B_k[a][b] (forward) or, transposed, the entry (b, a) of the
// block that face l of t sends to its k-th receiving row (as copy_entry_at).
template <typename E, typename S>
__global__ void to_frag_kernel(const S* __restrict__ src, int64_t row_stride, unsigned char* __restrict__ dst,
                               int64_t nrows, int nb, int nbp, int64_t row_bytes, const int32_t* __restrict__ recvT) {
  constexpr bool kFp8 = std::is_same<E, __nv_fp8_e4m3>::value;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_vals = 3 * (int64_t)nb * nbp;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < nrows; row += warps) {
    auto entry = [&](int64_t e) -> float {
      const fragk::FragPos p = fragk::frag_pos(e, nb, nbp);
      if (p.b >= nb) return 0.f;
      if (!recvT) return (float)src[row * row_stride + (int64_t)p.k * nb * nb + (int64_t)p.a * nb + p.b];
      const int l = (int)(row & 3);
      const int lq = p.k + (p.k >= l ? 1 : 0);
      const int64_t Rr = recvT[(row & ~int64_t(3)) + lq];
      const int slot = l - (l > lq ? 1 : 0);
      return (float)src[Rr * row_stride + (int64_t)slot * nb * nb + (int64_t)p.b * nb + p.a];
    };
    unsigned char* dr = dst + row * row_bytes;
    if constexpr (kFp8) {
      float mx = 0.f;
      for (int64_t e = lane; e < n_vals; e += 32) mx = fmaxf(mx, fabsf(entry(e)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float s = mx > 0.f ? mx / 448.f : 1.f;
      for (int64_t e = lane; e < n_vals; e += 32)
        dr[e] = (unsigned char)__nv_cvt_float_to_fp8(entry(e) / s, __NV_SATFINITE, __NV_E4M3);
      if (lane < 4) reinterpret_cast<float*>(dr + n_vals)[lane] = lane == 0 ? s : 0.f;
    } else {
      for (int64_t e = lane; e < n_vals; e += 32) reinterpret_cast<__half*>(dr)[e] = __float2half_rn(entry(e));
    }
  }
}

// v (FP32 [R][rows][nb]) times scale into the grouped hop layout
// [G][rows][NBP][8] (right-hand side q = 8 g + j; zero past R and nb): one
// thread per (g, row, a), 8 reads coalesced over a, one 16-byte store
__global__ void frag_pack_kernel(const float* __restrict__ v, __half* __restrict__ vp, int64_t rows, int nb, int nbp,
                                 int R, int G, float scale) {
  const int64_t total = (int64_t)G * rows * nbp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(i % nbp);
    const int64_t gr = i / nbp;
    const int64_t row = gr % rows;
    const int g = (int)(gr / rows);
    __half h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int q = 8 * g + j;
      h[j] = __float2half_rn(q < R && a < nb ? v[((int64_t)q * rows + row) * nb + a] * scale : 0.f);
    }
    uint4 u;
    memcpy(&u, h, 16);
    reinterpret_cast<uint4*>(vp)[i] = u;
  }
}

template <typename V>
__global__ void hop_pack_kernel(const float* __restrict__ v, V* __restrict__ vp, int64_t rows, int nb, int nbp,
                                float scale) {
  const int64_t total = rows * nbp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / nbp;
    const int a = (int)(i - row * nbp);
    vp[i] = (V)(a < nb ? v[row * nb + a] * scale : 0.f);
  }
}

// largest |x_i| (non-negative floats order like their bit patterns)
__global__ void amax_kernel(const float* __restrict__ x, int64_t n, unsigned* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

int grid_for_elems(int64_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)std::max(nsm, 1) * 8));
}

}  // namespace

int prepare_lowp(const dfm_op* cop, int precision, cudaStream_t st, int trans, int R) {
  dfm_op* op = const_cast<dfm_op*>(cop);
  if ((op->precision != DFM_F32 && op->precision != DFM_BF16) ||
      (precision != DFM_F16 && precision != DFM_BF16 && precision != DFM_FP8E4M3))
    return set_error(DFM_ERR_UNSUPPORTED,
                     "preconditioner copy: needs an FP32 or BF16 operator and DFM_F16, DFM_BF16 or DFM_FP8E4M3");
  if (!narrow_nb(op->nb))
    return set_error(DFM_ERR_UNSUPPORTED, "preconditioner copy: built for the bases of the per-warp kernels "
                                          "(Np <= 8; with the linear spatial basis Np = 0 or 4)");
  void*& vals = trans ? op->lpT_vals : op->lp_vals;
  int64_t& have = trans ? op->lpT_bytes : op->lp_bytes;
  int& prec = trans ? op->lpT_precision : op->lp_precision;
  bool& valid = trans ? op->lpT_valid : op->lp_valid;
  bool& frag = trans ? op->lpT_frag : op->lp_frag;
  const bool want_frag = frag_copy(op->nb, precision, R);
  const int32_t* recvT = trans ? op->mesh->recv : nullptr;
  const int nb = op->nb, nbp = hop_nbp(nb);
  const int64_t row_bytes = precision == DFM_FP8E4M3 ? copy_row_bytes<__nv_fp8_e4m3>(nb, nbp)
                                                     : copy_row_bytes<__half>(nb, nbp);
  const int64_t bytes = op->nrows * row_bytes;
  if (vals && have < bytes) {
    forget_sweep(vals);
    DFM_CUDA_CHECK(cudaFree(vals));
    vals = nullptr;
    valid = false;
  }
  if (!vals) {
    DFM_CUDA_CHECK(cudaMalloc(&vals, bytes));
    have = bytes;
  }
  if (!valid || prec != precision || frag != want_frag) {
    auto convert = [&](auto src) {
      using S = std::remove_const_t<std::remove_pointer_t<decltype(src)>>;
      if (want_frag) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((op->nrows * 32 + 255) / 256, 4096));
        if (precision == DFM_FP8E4M3)
          to_frag_kernel<__nv_fp8_e4m3, S><<<grid, 256, 0, st>>>(src, op->row_stride, (unsigned char*)vals, op->nrows,
                                                                 nb, nbp, row_bytes, recvT);
        else
          to_frag_kernel<__half, S><<<grid, 256, 0, st>>>(src, op->row_stride, (unsigned char*)vals, op->nrows, nb,
                                                          nbp, row_bytes, recvT);
      } else if (precision == DFM_FP8E4M3) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((op->nrows * 32 + 255) / 256, 4096));
        to_hop8_kernel<S><<<grid, 256, 0, st>>>(src, op->row_stride, (unsigned char*)vals, op->nrows, nb, nbp,
                                                copy_body_bytes<__nv_fp8_e4m3>(nb, nbp), row_bytes, recvT);
      } else {
        const int grid = grid_for_elems(op->nrows * 3 * (int64_t)nb * nbp);
        if (precision == DFM_F16)
          to_hop16_kernel<__half, S><<<grid, 256, 0, st>>>(src, op->row_stride, (__half*)vals, op->nrows, nb, nbp,
                                                            recvT);
        else
          to_hop16_kernel<__nv_bfloat16, S><<<grid, 256, 0, st>>>(src, op->row_stride, (__nv_bfloat16*)vals,
                                                                   op->nrows, nb, nbp, recvT);
      }
    };
    if (op->precision == DFM_F32)
      convert((const float*)op->vals);
    else
      convert((const __nv_bfloat16*)op->vals);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    prec = precision;
    frag = want_frag;
    valid = true;
  }
  return DFM_OK;
}

namespace {

// one hop over all R right-hand sides (kHopMaxRhs per launch)
template <typename V>
int hop_apply_t(const dfm_op* op, const V* xp, const V* x0p, void* y, int R, bool out_padded, float out_scale,
                int trans, cudaStream_t st) {
  const LowpView cp = lowp_of(op, trans);
  const int64_t stride_p = op->nrows * (int64_t)hop_nbp(op->nb);
  const int64_t stride_y = out_padded ? stride_p : op->nrows * (int64_t)op->nb;
  const int64_t ybytes = out_padded ? (int64_t)sizeof(V) : 4;
  // right-hand sides per launch: at most kHopMaxRhs, and few enough that two
  // stages fit in shared memory (large bases with many right-hand sides)
  const bool fp8 = cp.precision == DFM_FP8E4M3;
  const int rchunk = geom::hop_rhs_chunk(op->nb, fp8 ? 1 : 2, fp8, (int)sizeof(V));
  if (rchunk < 1) return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: a tile does not fit shared memory");
  for (int r0 = 0; r0 < R; r0 += rchunk) {
    const int Rp = std::min(rchunk, R - r0);
    const V* x = xp + r0 * stride_p;
    const V* x0 = x0p + r0 * stride_p;
    void* yy = static_cast<char*>(y) + r0 * stride_y * ybytes;
    int rc;
    if constexpr (std::is_same<V, __half>::value) {
      if (cp.precision == DFM_F16)
        rc = hop_launch_f16(op, x, x0, yy, Rp, out_scale, out_padded, trans, st);
      else
        rc = hop_launch_fp8(op, x, x0, yy, Rp, out_scale, out_padded, trans, st);
    } else {
      rc = hop_launch_bf16(op, x, x0, yy, Rp, out_scale, out_padded, trans, st);
    }
    if (rc) return rc;
  }
  return DFM_OK;
}

// Candidate geometries of the tensor-core hop for the autotuner: tile rows
// in multiples of the rows that give each warp of a consumer group one item,
// 2, 4, 6 or 8 stages, every stage at most 100 KB and all within the budget.
std::vector<tune::Geometry> frag_candidates(int nb, bool fp8, int w, int rgl) {
  const int64_t row = geom::frag_row_stage_bytes(nb, fp8 ? 1 : 2, fp8, w, rgl);
  const int unit = rgl >= geom::kFragGroupWarps ? 1 : geom::kFragGroupWarps / rgl;
  std::vector<tune::Geometry> out;
  for (int m : {1, 2, 3, 4, 6, 8}) {
    const int rpt = unit * m;
    if (rpt > 32 || rpt * row > 100 * 1024) continue;
    for (int st : {2, 4, 6, 8})  // multiples of the consumer groups (see geom::frag_geometry)
      if (st * rpt * row <= geom::kStageBudget) out.push_back(tune::Geometry{rpt, st, 0.f});
  }
  return out;
}

tune::Geometry frag_default(int nb, bool fp8, int w, int rgl) {
  const geom::Frag g = geom::frag_geometry(nb, fp8 ? 1 : 2, fp8, w, rgl);
  return tune::Geometry{g.rpt, g.stages, 0.f};
}

// One hop on the fragment-ordered copy over all R right-hand sides: R <= 3
// in the [R][rows][NBP] layout, one launch per right-hand side; R >= 4 in
// groups of 8 ([G][rows][NBP][8]), two groups per launch.
int hop_apply_frag(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int R, bool out_padded,
                   float out_scale, int trans, cudaStream_t st) {
  const LowpView cp = lowp_of(op, trans);
  const int nb = op->nb, nbp = hop_nbp(nb);
  const int64_t rows = op->nrows;
  const bool fp8 = cp.precision == DFM_FP8E4M3;
  int dev = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  // each launch shape takes the tile rows and stages the autotuner picked for it
  auto launch = [&](const __half* x, const __half* x0, void* yy, int w, int rgl, int rhs_here) -> int {
    auto go = [&](int rpt, int stages) -> int {
      return fp8 ? hop_frag_launch_fp8(op, x, x0, yy, w, rgl, rhs_here, out_padded, out_scale, trans, rpt, stages, st)
                 : hop_frag_launch_f16(op, x, x0, yy, w, rgl, rhs_here, out_padded, out_scale, trans, rpt, stages, st);
    };
    const tune::Key key{0, nb, cp.precision, w, rgl, trans, rows, dev};
    tune::Geometry g;
    const int rc = tune::choose(key, st, frag_candidates(nb, fp8, w, rgl), frag_default(nb, fp8, w, rgl), go, &g);
    if (rc) return rc;
    return go(g.rpt, g.stages);
  };
  if (R < kFragGroupMin) {
    for (int r = 0; r < R; ++r) {
      void* yy = out_padded ? static_cast<void*>(static_cast<__half*>(y) + r * rows * nbp)
                            : static_cast<void*>(static_cast<float*>(y) + r * rows * nb);
      const int rc = launch(xp + r * rows * nbp, x0p + r * rows * nbp, yy, 1, 1, 1);
      if (rc) return rc;
    }
    return DFM_OK;
  }
  const int G = (R + 7) / 8;
  const int64_t plane = rows * nbp * 8;
  for (int g0 = 0; g0 < G; g0 += 2) {
    const int rgl = std::min(2, G - g0);
    void* yy = out_padded ? static_cast<void*>(static_cast<__half*>(y) + g0 * plane)
                          : static_cast<void*>(static_cast<float*>(y) + (int64_t)g0 * 8 * rows * nb);
    const int rc = launch(xp + g0 * plane, x0p + g0 * plane, yy, 8, rgl, std::min(16, R - 8 * g0));
    if (rc) return rc;
  }
  return DFM_OK;
}

// CUDA graphs of the hop chains.  A Horner chain is a pack of v, d - 1 hops
// and nothing else; the hops between the first and the last read and write
// only the chain's fixed scratch (vp, ha, hb), so for a given operator copy,
// right-hand-side count, degree and scratch they are the same launches every
// time.  The first chain of a shape runs eagerly (the autotuner picks its
// geometries then), the second is captured into a graph, later ones replay
// it: one launch instead of d - 3.  The pack (reading v) and the last hop
// (writing z) stay outside the graph.
struct HopGraph {
  const void* copy;
  int prec;
  bool frag;
  int trans, R, d;
  const void *vp, *ha, *hb;
  float vscale;
  int state;  // 0: seen once, 1: captured, 2: capture failed (eager)
  cudaGraphExec_t exec;
  long long nodes;
};
struct HopGraphs {
  std::vector<HopGraph> g;
  cudaStream_t cap = nullptr;  // private stream the chains are captured on
};
constexpr size_t kMaxHopGraphs = 16;
std::atomic<int> g_hop_graphs{1};
std::atomic<long long> g_hop_graph_replays{0};

int chain(const dfm_op* op, int R, int d, const float* v, float* z, void* vp, void* ha, void* hb, float vscale,
          int trans, cudaStream_t st) {
  const LowpView cp = lowp_of(op, trans);
  const bool bf16 = cp.precision == DFM_BF16;  // FP32 hop vectors, unscaled
  const float vs = bf16 ? 1.0f : vscale;
  const int nb = op->nb, nbp = hop_nbp(nb);
  const int64_t rows = (int64_t)R * op->nrows;
  if (bf16) {
    hop_pack_kernel<float><<<grid_for_elems(rows * nbp), 256, 0, st>>>(v, static_cast<float*>(vp), rows, nb, nbp, 1.0f);
  } else if (cp.frag && R >= kFragGroupMin) {
    const int G = (R + 7) / 8;
    frag_pack_kernel<<<grid_for_elems((int64_t)G * op->nrows * nbp), 256, 0, st>>>(v, static_cast<__half*>(vp),
                                                                                  op->nrows, nb, nbp, R, G, vs);
  } else {
    hop_pack_kernel<__half><<<grid_for_elems(rows * nbp), 256, 0, st>>>(v, static_cast<__half*>(vp), rows, nb, nbp,
                                                                       vs);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  // one hop: dst = vp + B~ src (the last one unpadded FP32 into z)
  auto hop = [&](const void* src, void* dst, bool last, cudaStream_t s) -> int {
    if (bf16)
      return hop_apply_t<float>(op, static_cast<const float*>(src), static_cast<const float*>(vp), dst, R, !last,
                                1.0f, trans, s);
    if (cp.frag)
      return hop_apply_frag(op, static_cast<const __half*>(src), static_cast<const __half*>(vp), dst, R, !last,
                            1.0f / vs, trans, s);
    return hop_apply_t<__half>(op, static_cast<const __half*>(src), static_cast<const __half*>(vp), dst, R, !last,
                               1.0f / vs, trans, s);
  };
  void* h[2] = {ha, hb};
  // hops 1 .. d - 2 into the scratch
  auto middle = [&](cudaStream_t s) -> int {
    const void* src = vp;
    for (int k = 1; k <= d - 2; ++k) {
      const int rc = hop(src, h[k & 1], false, s);
      if (rc) return rc;
      src = h[k & 1];
    }
    return DFM_OK;
  };
  int rc = DFM_OK;
  bool issued = false;  // the middle hops are on the stream
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DFM_CUDA_CHECK(cudaStreamIsCapturing(st, &cap));
  if (d - 2 >= 2 && g_hop_graphs.load() && cap == cudaStreamCaptureStatusNone) {
    dfm_op* mop = const_cast<dfm_op*>(op);
    if (!mop->hop_graphs) mop->hop_graphs = new HopGraphs();
    std::vector<HopGraph>& list = static_cast<HopGraphs*>(mop->hop_graphs)->g;
    HopGraph* ent = nullptr;
    for (HopGraph& e : list)
      if (e.copy == cp.vals && e.prec == cp.precision && e.frag == cp.frag && e.trans == trans && e.R == R &&
          e.d == d && e.vp == vp && e.ha == ha && e.hb == hb && e.vscale == vs) {
        ent = &e;
        break;
      }
    if (!ent) {  // first use: eager (the autotuner decides here)
      if (list.size() >= kMaxHopGraphs) {
        if (list.front().exec) cudaGraphExecDestroy(list.front().exec);
        list.erase(list.begin());
      }
      list.push_back(HopGraph{cp.vals, cp.precision, cp.frag, trans, R, d, vp, ha, hb, vs, 0, nullptr, 0});
      rc = middle(st);
      issued = true;
    } else if (ent->state == 0) {
      // second use: capture on the operator's private stream (nothing runs
      // there; the legacy default stream cannot be captured), replay below
      // on the caller's stream
      ent->state = 2;
      HopGraphs* gs = static_cast<HopGraphs*>(mop->hop_graphs);
      if (!gs->cap && cudaStreamCreateWithFlags(&gs->cap, cudaStreamNonBlocking) != cudaSuccess) gs->cap = nullptr;
      if (gs->cap && cudaStreamBeginCapture(gs->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        set_capturing(true);
        const int crc = middle(gs->cap);
        set_capturing(false);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(gs->cap, &graph);
        size_t n = 0;
        if (crc == DFM_OK && ee == cudaSuccess && graph && cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess &&
            n > 0 && cudaGraphInstantiate(&ent->exec, graph, 0) == cudaSuccess) {
          ent->state = 1;
          ent->nodes = (long long)n;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      (void)cudaGetLastError();  // a failed capture leaves this chain to eager launches
    }
    if (!issued && ent && ent->state == 1) {
      {
        ::dfm::KernelTimer timer_(trans ? DFM_KERNEL_SPMV16_T : DFM_KERNEL_SPMV16, st, (int)ent->nodes);
        DFM_CUDA_CHECK(cudaGraphLaunch(ent->exec, st));
      }
      count_launches(ent->nodes);
      g_hop_graph_replays.fetch_add(1);
      issued = true;
    }
  }
  if (!issued) rc = middle(st);
  if (rc) return rc;
  return hop(d >= 3 ? h[(d - 2) & 1] : vp, z, true, st);
}
}  // namespace

int hop_horner(const dfm_op* op, int R, int d, const float* v, float* z, void* vp, void* ha, void* hb, float vscale,
               cudaStream_t st, int trans) {
  if (!op || !lowp_of(op, trans).valid || !v || !z || R < 1 || d < 1)
    return set_error(DFM_ERR_ARG, "preconditioner: no low-precision copy, NULL vector or bad degree");
  if ((reinterpret_cast<uintptr_t>(vp) | reinterpret_cast<uintptr_t>(ha) | reinterpret_cast<uintptr_t>(hb) |
       reinterpret_cast<uintptr_t>(lowp_of(op, trans).vals)) & 15)
    return set_error(DFM_ERR_ARG, "preconditioner: hop vectors and copy must be 16-byte aligned");
  if (d == 1) {
    DFM_CUDA_CHECK(cudaMemcpyAsync(z, v, sizeof(float) * (int64_t)R * op->nrows * op->nb, cudaMemcpyDeviceToDevice, st));
    return DFM_OK;
  }
  // FP16 and e4m3 copies run the hops on FP16 vectors (v scaled by vscale);
  // the BF16 copy on FP32 vectors
  return chain(op, R, d, v, z, vp, ha, hb, vscale, trans, st);
}

void destroy_hop_graphs(dfm_op* op) {
  if (!op || !op->hop_graphs) return;
  auto* gs = static_cast<HopGraphs*>(op->hop_graphs);
  for (HopGraph& e : gs->g)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (gs->cap) cudaStreamDestroy(gs->cap);
  delete gs;
  op->hop_graphs = nullptr;
}

}  // namespace dfm

extern "C" int dfm_hop_graphs(int mode) {
  using namespace dfm;
  if (mode < -1 || mode > 1) return set_error(DFM_ERR_ARG, "dfm_hop_graphs: mode must be -1, 0 or 1");
  if (mode >= 0) g_hop_graphs.store(mode);
  return g_hop_graphs.load();
}

extern "C" long long dfm_hop_graph_replays(void) { return dfm::g_hop_graph_replays.load(); }

extern "C" int dfm_precond_apply(const dfm_op* op, int precision, int degree, int transpose, const float* x, float* z,
                                 int R, void* stream) {
  using namespace dfm;
  if (!op || !x || !z || R < 1) return set_error(DFM_ERR_ARG, "dfm_precond_apply: NULL operator/vector or R < 1");
  if (x == z) return set_error(DFM_ERR_ARG, "dfm_precond_apply: z must not alias x");
  if (degree < 1 || degree > 64) return set_error(DFM_ERR_ARG, "dfm_precond_apply: degree must be in 1..64");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(z)) & 15)
    return set_error(DFM_ERR_ARG, "dfm_precond_apply: x and z must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  int rc = prepare_lowp(op, precision, st, transpose ? 1 : 0, R);
  if (rc) return rc;
  const int64_t rows = (int64_t)R * op->nrows;
  const int64_t elems = rows * hop_nbp(op->nb);
  char* scratch = nullptr;
  const int64_t vec_bytes = (elems * 4 + 255) / 256 * 256;
  DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&scratch), 3 * vec_bytes + 256, st));
  // FP16 hop vectors hold x * 2^-(e + 8) with 2^e >= max |x|, as in the solver
  // (whose vectors have unit norm): products and sums stay far from the FP16
  // overflow threshold
  unsigned* amax_d = reinterpret_cast<unsigned*>(scratch + 3 * vec_bytes);
  unsigned amax_bits = 0;
  cudaError_t e = cudaMemsetAsync(amax_d, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    amax_kernel<<<grid_for_elems(rows * op->nb), 256, 0, st>>>(x, rows * op->nb, amax_d);
    DFM_LAUNCHED();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&amax_bits, amax_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    float amax;
    memcpy(&amax, &amax_bits, 4);
    int ex = 0;
    if (amax > 0.f && std::isfinite(amax)) frexpf(amax, &ex);  // amax < 2^ex
    const float vscale = ldexpf(1.0f, -(ex + 8));
    rc = hop_horner(op, R, degree, x, z, scratch, scratch + vec_bytes, scratch + 2 * vec_bytes, vscale, st,
                    transpose ? 1 : 0);
  }
  const cudaError_t ef = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_error(e, "dfm_precond_apply");
  if (rc) return rc;
  if (ef != cudaSuccess) return cuda_error(ef, "dfm_precond_apply: cudaFreeAsync");
  return DFM_OK;
}
