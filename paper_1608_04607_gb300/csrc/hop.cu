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
//  - hop vectors (v and the intermediate z): FP32, each face's NB
//    coefficients padded with zeros to NBP, so that a face starts on a
//    32-byte boundary and a tet's 4 faces form one 16-byte-aligned run.
// The last hop of a Horner chain writes the unpadded FP32 layout of the
// solver's vectors.
//
// The pipeline is the one of the FP32 application: a producer warp streams
// tiles of consecutive rows (operator rows, each row's source-tet
// coefficients and the x0 slice) into shared memory with bulk copies, four
// consumer warps form the outputs; waits are bounded and a time-out sets the
// operator's error flag.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "dfm_internal.cuh"
#include "tma_pipe.cuh"

namespace dfm {
namespace {

using namespace pipe;

constexpr int kHopStages = 4;
constexpr int kHopConsumerWarps = 4;
constexpr int kHopMaxRhs = 16;  // right-hand sides staged per pass
// operator bytes per hop kept in L2 for the next one (which sweeps the other way)
constexpr int64_t kHopL2KeepBytes = 64ll << 20;

// Entry e of one row of the copy (value index in copy order) from the row's
// FP32 blocks: e -> (block k, chunk c, test index a, slot j), trial b = 8c + j.
template <typename S>
__device__ __forceinline__ float copy_entry(const S* row, int64_t e, int nb, int nbp) {
  const int k = (int)(e / ((int64_t)nb * nbp));
  int64_t rem = e - (int64_t)k * nb * nbp;
  const int c = (int)(rem / (nb * 8));
  rem -= (int64_t)c * nb * 8;
  const int a = (int)(rem / 8);
  const int b = c * 8 + (int)(rem - a * 8);
  return b < nb ? (float)row[(int64_t)k * nb * nb + (int64_t)a * nb + b] : 0.f;
}

// Storage formats of the copy: bytes per value, whether rows carry a scale,
// and the decoding of one 8-value chunk into 4 pairs of floats.
template <typename E>
struct Codec;

template <>
struct Codec<__half> {
  static constexpr int kEB = 2;
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ void decode8(const unsigned char* p, float2 f[4]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h;
      memcpy(&h, &w[i], 4);
      f[i] = __half22float2(h);
    }
  }
};

template <>
struct Codec<__nv_bfloat16> {
  static constexpr int kEB = 2;
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ void decode8(const unsigned char* p, float2 f[4]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 h;
      memcpy(&h, &w[i], 4);
      f[i] = __bfloat1622float2(h);
    }
  }
};

// the same chunks as 4 half2 (FP16 vector path; FP16 and e4m3 copies)
template <typename E>
__device__ __forceinline__ void decode8h(const unsigned char* p, __half2 h[4]);

template <>
__device__ __forceinline__ void decode8h<__half>(const unsigned char* p, __half2 h[4]) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  memcpy(h, &v, 16);
}

template <>
__device__ __forceinline__ void decode8h<__nv_fp8_e4m3>(const unsigned char* p, __half2 h[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const uint32_t w[2] = {v.x, v.y};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
    const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
    memcpy(&h[i], &hr, 4);
  }
}

template <>
struct Codec<__nv_fp8_e4m3> {
  static constexpr int kEB = 1;
  static constexpr bool kScaled = true;
  static __device__ __forceinline__ void decode8(const unsigned char* p, float2 f[4]) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const uint32_t w[2] = {v.x, v.y};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
      __half2 h;
      memcpy(&h, &hr, 4);
      f[i] = __half22float2(h);
    }
  }
};

// bytes of one operator row of the copy: the values (padded to 16 bytes) and,
// for scaled formats, a 16-byte field whose first 4 bytes hold s_R
template <typename E>
__host__ __device__ constexpr int64_t copy_body_bytes(int nb, int nbp) {
  return (3 * (int64_t)nb * nbp * Codec<E>::kEB + 15) / 16 * 16;
}
template <typename E>
__host__ __device__ constexpr int64_t copy_row_bytes(int nb, int nbp) {
  return copy_body_bytes<E>(nb, nbp) + (Codec<E>::kScaled ? 16 : 0);
}

// y = x0 + alpha B~ x for R right-hand sides; x, x0 of type V (float, or
// __half holding a scaled copy of the vector) padded to NBP per face row; y
// padded of type V (OUTP), or FP32 unpadded (NB per face row) times out_scale.
// With V = __half each block's 8-value chunks are multiplied and summed in
// packed FP16 (one rounding per fused multiply-add; 2 x NBP/8 products per
// lane) and the three block sums are added in FP32.
template <int NB, typename E, typename V, bool OUTP>
__global__ void __launch_bounds__(32 * (kHopConsumerWarps + 1))
hop_kernel(const unsigned char* __restrict__ vals, const int32_t* __restrict__ recv, int64_t nrows,
           const V* __restrict__ xp, const V* __restrict__ x0p, void* __restrict__ yv, int R, float alpha,
           float out_scale, int stages, int reverse, int64_t keep_from, int* __restrict__ err) {
  constexpr int NBP = (NB + 7) / 8 * 8;
  constexpr int NC = NBP / 8;
  constexpr int RPT = (32 * kHopConsumerWarps) / NBP;  // rows per tile
  constexpr int EB = Codec<E>::kEB;
  constexpr unsigned ROW_BYTES = (unsigned)copy_row_bytes<E>(NB, NBP);
  constexpr unsigned BODY_BYTES = (unsigned)copy_body_bytes<E>(NB, NBP);
  constexpr unsigned XBLK = 4 * NBP * (unsigned)sizeof(V);
  constexpr unsigned X0ROW = NBP * (unsigned)sizeof(V);
  constexpr bool VH = std::is_same<V, __half>::value;
  static_assert(RPT >= 1 && RPT <= 32, "rows per tile");
  static_assert(ROW_BYTES % 16 == 0 && X0ROW % 16 == 0, "rows must keep 16-byte alignment");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kHopStages;
  int32_t* s_recv = reinterpret_cast<int32_t*>(smem_raw + 128);
  const int64_t stage_bytes = (int64_t)RPT * ROW_BYTES + (int64_t)R * RPT * (XBLK + X0ROW);
  unsigned char* stage0 = smem_raw + 128 + ((kHopStages * RPT * 4 + 127) / 128) * 128;
  const int64_t ntiles = (nrows + RPT - 1) / RPT;
  const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kHopConsumerWarps);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto tile_first_row = [&](int64_t i) {
    const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
    return (reverse ? ntiles - 1 - tile : tile) * RPT;
  };
  if (warp == 0) {
    // ---------------- producer ----------------
    const uint64_t pol_last = l2_policy_evict_last();
    const uint64_t pol_first = l2_policy_evict_first();
    int64_t issued = 0;
    bool ok = true;
    int32_t next_src = 0;
    if (mine > 0) {
      const int64_t R0 = tile_first_row(0);
      if (lane < RPT && R0 + lane < nrows) next_src = recv[R0 + lane];
    }
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      const int64_t R0 = tile_first_row(i);
      const int nr = (int)std::min<int64_t>(RPT, nrows - R0);
      const int32_t src = next_src;
      if (i + 1 < mine) {
        const int64_t R1 = tile_first_row(i + 1);
        if (lane < RPT && R1 + lane < nrows) next_src = recv[R1 + lane];
      }
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      int32_t* rs = s_recv + s * RPT;
      if (lane < nr) rs[lane] = src;
      __syncwarp();  // the row map is written before lane 0's arrive publishes the stage
      fence_proxy_async_smem();
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], (unsigned)nr * ROW_BYTES + (unsigned)(R * nr) * (XBLK + X0ROW));
        const uint64_t pol = (blockIdx.x + i * (int64_t)gridDim.x) >= keep_from ? pol_last : pol_first;
        bulk_copy_g2s_hint(st, vals + R0 * (int64_t)ROW_BYTES, (unsigned)nr * ROW_BYTES, &full[s], pol);
        for (int rhs = 0; rhs < R; ++rhs)
          bulk_copy_g2s(st + (int64_t)RPT * ROW_BYTES + (int64_t)R * RPT * XBLK + (int64_t)rhs * RPT * X0ROW,
                        x0p + ((int64_t)rhs * nrows + R0) * NBP, (unsigned)nr * X0ROW, &full[s]);
      }
      if (lane < nr)
        for (int rhs = 0; rhs < R; ++rhs)
          bulk_copy_g2s(st + (int64_t)RPT * ROW_BYTES + ((int64_t)rhs * RPT + lane) * XBLK,
                        xp + ((int64_t)rhs * nrows + 4 * (int64_t)(src >> 2)) * NBP, XBLK, &full[s]);
      issued = i + 1;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    // drain: every issued stage must have landed before the block's shared memory goes away
    if (lane == 0)
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j)
        mbar_wait_bounded(&full[j % stages], (unsigned)((j / stages) & 1));
    return;
  }
  // ---------------- consumers: thread (r, a), a < NBP ----------------
  const int ctid = threadIdx.x - 32;
  const int r = ctid / NBP;
  const int a = ctid - r * NBP;
  for (int64_t i = 0; i < mine; ++i) {
    const int s = (int)(i % stages);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((i / stages) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const unsigned char* st = stage0 + s * stage_bytes;
    const int64_t R0 = tile_first_row(i);
    const int nr = (int)std::min<int64_t>(RPT, nrows - R0);
    if (r < nr) {
      const int lp = s_recv[s * RPT + r] & 3;
      const unsigned char* brow = st + r * ROW_BYTES;
      float scale = 1.f;
      if constexpr (Codec<E>::kScaled) scale = *reinterpret_cast<const float*>(brow + BODY_BYTES);
      for (int rhs = 0; rhs < R; ++rhs) {
        const V* xs = reinterpret_cast<const V*>(st + (int64_t)RPT * ROW_BYTES + ((int64_t)rhs * RPT + r) * XBLK);
        const V* x0s =
            reinterpret_cast<const V*>(st + (int64_t)RPT * ROW_BYTES + (int64_t)R * RPT * XBLK + (int64_t)rhs * RPT * X0ROW);
        float out = 0.f;
        if (a < NB) {
          float sum = 0.f;
          if constexpr (VH) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const int l = k + (k >= lp ? 1 : 0);
              const __half* xl = reinterpret_cast<const __half*>(xs) + l * NBP;
              const unsigned char* bk = brow + k * NB * NBP * EB;
              __half2 acc0 = __float2half2_rn(0.f), acc1 = __float2half2_rn(0.f);
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                __half2 bh[4], xh[4];
                decode8h<E>(bk + (c * NB + a) * 8 * EB, bh);
                const uint4 xv = *reinterpret_cast<const uint4*>(xl + c * 8);
                memcpy(xh, &xv, 16);
                acc0 = __hfma2(bh[0], xh[0], acc0);
                acc1 = __hfma2(bh[1], xh[1], acc1);
                acc0 = __hfma2(bh[2], xh[2], acc0);
                acc1 = __hfma2(bh[3], xh[3], acc1);
              }
              const float2 f0 = __half22float2(acc0), f1 = __half22float2(acc1);
              sum += (f0.x + f0.y) + (f1.x + f1.y);
            }
          } else {
            float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                             make_float2(0.f, 0.f)};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const int l = k + (k >= lp ? 1 : 0);
              const float* xl = reinterpret_cast<const float*>(xs) + l * NBP;
              const unsigned char* bk = brow + k * NB * NBP * EB;
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                float2 bv[4];
                Codec<E>::decode8(bk + (c * NB + a) * 8 * EB, bv);
                const float4 xa = *reinterpret_cast<const float4*>(xl + c * 8);
                const float4 xb = *reinterpret_cast<const float4*>(xl + c * 8 + 4);
                acc[0] = __ffma2_rn(bv[0], make_float2(xa.x, xa.y), acc[0]);
                acc[1] = __ffma2_rn(bv[1], make_float2(xa.z, xa.w), acc[1]);
                acc[2] = __ffma2_rn(bv[2], make_float2(xb.x, xb.y), acc[2]);
                acc[3] = __ffma2_rn(bv[3], make_float2(xb.z, xb.w), acc[3]);
              }
            }
            sum = ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
          }
          out = (float)x0s[r * NBP + a] + alpha * (scale * sum);
        }
        const int64_t row = (int64_t)rhs * nrows + R0 + r;
        if constexpr (OUTP)
          reinterpret_cast<V*>(yv)[row * NBP + a] = (V)out;  // pads (a >= NB) written as 0
        else if (a < NB)
          reinterpret_cast<float*>(yv)[row * NB + a] = out * out_scale;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// FP16/BF16 copy: element i of the copy <- its block entry (0 in pads); the
// blocks are FP32, or BF16 for a BF16 operator
template <typename E, typename S>
__global__ void to_hop16_kernel(const S* __restrict__ src, int64_t row_stride, E* __restrict__ dst, int64_t nrows,
                                int nb, int nbp) {
  const int64_t row_elems = 3 * (int64_t)nb * nbp;
  const int64_t total = nrows * row_elems;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / row_elems;
    const int64_t e = i - row * row_elems;
    const float v = copy_entry(src + row * row_stride, e, nb, nbp);
    if constexpr (std::is_same<E, __half>::value)
      dst[i] = __float2half_rn(v);
    else
      dst[i] = __float2bfloat16_rn(v);
  }
}

// e4m3 copy: one warp per operator row; s_R = max |entry| / 448, q = e4m3(v / s_R)
template <typename S>
__global__ void to_hop8_kernel(const S* __restrict__ src, int64_t row_stride, unsigned char* __restrict__ dst,
                               int64_t nrows, int nb, int nbp, int64_t body_bytes, int64_t row_bytes) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_entries = 3 * (int64_t)nb * nb;
  const int64_t n_vals = 3 * (int64_t)nb * nbp;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; row < nrows; row += warps) {
    const S* sr = src + row * row_stride;
    float mx = 0.f;
    for (int64_t e = lane; e < n_entries; e += 32) mx = fmaxf(mx, fabsf((float)sr[e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float s = mx > 0.f ? mx / 448.f : 1.f;
    unsigned char* dr = dst + row * row_bytes;
    for (int64_t e = lane; e < body_bytes; e += 32) {
      const float v = e < n_vals ? copy_entry(sr, e, nb, nbp) : 0.f;
      dr[e] = (unsigned char)__nv_cvt_float_to_fp8(v / s, __NV_SATFINITE, __NV_E4M3);
    }
    if (lane < 4) reinterpret_cast<float*>(dr + body_bytes)[lane] = lane == 0 ? s : 0.f;
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

template <typename E, typename V, bool OUTP>
int launch_hop(const dfm_op* op, const V* xp, const V* x0p, void* y, int R, float out_scale, cudaStream_t st) {
  const int nb = op->nb;
  const int nbp = hop_nbp(nb);
  const int rpt = (32 * kHopConsumerWarps) / nbp;
  const int64_t row_bytes = copy_row_bytes<E>(nb, nbp);
  const int64_t vb = (int64_t)sizeof(V);
  const int64_t stage_bytes = rpt * row_bytes + (int64_t)R * rpt * (4 * nbp * vb + nbp * vb);
  const int64_t budget = 200 * 1024 - 1024;
  const int stages = (int)std::min<int64_t>(kHopStages, budget / stage_bytes);
  if (stages < 2) return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: a tile does not fit shared memory");
  const size_t smem = 128 + ((kHopStages * rpt * 4 + 127) / 128) * 128 + (size_t)stages * stage_bytes;
  int dev = 0, nsm = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto go = [&](auto kernel) -> int {
    DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * (kHopConsumerWarps + 1), smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (op->nrows + rpt - 1) / rpt;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    const int64_t keep_from = std::max<int64_t>(0, ntiles - kHopL2KeepBytes / (rpt * row_bytes));
    {
      ::dfm::KernelTimer timer_(DFM_KERNEL_SPMV16, st);
      kernel<<<(unsigned)grid, 32 * (kHopConsumerWarps + 1), smem, st>>>(
          reinterpret_cast<const unsigned char*>(op->lp_vals), op->mesh->recv, op->nrows, xp, x0p, y, R, 1.0f,
          out_scale, stages, next_sweep_direction(op->lp_vals), keep_from, op->dev_err);
    }
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    return DFM_OK;
  };
  switch (nb) {
    case 1: return go(hop_kernel<1, E, V, OUTP>);
    case 3: return go(hop_kernel<3, E, V, OUTP>);
    case 6: return go(hop_kernel<6, E, V, OUTP>);
    case 10: return go(hop_kernel<10, E, V, OUTP>);
    case 15: return go(hop_kernel<15, E, V, OUTP>);
    case 21: return go(hop_kernel<21, E, V, OUTP>);
    case 28: return go(hop_kernel<28, E, V, OUTP>);
    case 36: return go(hop_kernel<36, E, V, OUTP>);
    case 45: return go(hop_kernel<45, E, V, OUTP>);
    default: return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: unsupported basis size");
  }
}

}  // namespace

int prepare_lowp(const dfm_op* cop, int precision, cudaStream_t st) {
  dfm_op* op = const_cast<dfm_op*>(cop);
  if ((op->precision != DFM_F32 && op->precision != DFM_BF16) ||
      (precision != DFM_F16 && precision != DFM_BF16 && precision != DFM_FP8E4M3))
    return set_error(DFM_ERR_UNSUPPORTED,
                     "preconditioner copy: needs an FP32 or BF16 operator and DFM_F16, DFM_BF16 or DFM_FP8E4M3");
  const int nb = op->nb, nbp = hop_nbp(nb);
  const int64_t row_bytes = precision == DFM_FP8E4M3 ? copy_row_bytes<__nv_fp8_e4m3>(nb, nbp)
                                                     : copy_row_bytes<__half>(nb, nbp);
  const int64_t bytes = op->nrows * row_bytes;
  if (op->lp_vals && op->lp_bytes < bytes) {
    forget_sweep(op->lp_vals);
    DFM_CUDA_CHECK(cudaFree(op->lp_vals));
    op->lp_vals = nullptr;
    op->lp_valid = false;
  }
  if (!op->lp_vals) {
    DFM_CUDA_CHECK(cudaMalloc(&op->lp_vals, bytes));
    op->lp_bytes = bytes;
  }
  if (!op->lp_valid || op->lp_precision != precision) {
    auto convert = [&](auto src) {
      using S = std::remove_const_t<std::remove_pointer_t<decltype(src)>>;
      if (precision == DFM_FP8E4M3) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((op->nrows * 32 + 255) / 256, 4096));
        to_hop8_kernel<S><<<grid, 256, 0, st>>>(src, op->row_stride, (unsigned char*)op->lp_vals, op->nrows, nb, nbp,
                                                copy_body_bytes<__nv_fp8_e4m3>(nb, nbp), row_bytes);
      } else {
        const int grid = grid_for_elems(op->nrows * 3 * (int64_t)nb * nbp);
        if (precision == DFM_F16)
          to_hop16_kernel<__half, S><<<grid, 256, 0, st>>>(src, op->row_stride, (__half*)op->lp_vals, op->nrows, nb,
                                                            nbp);
        else
          to_hop16_kernel<__nv_bfloat16, S><<<grid, 256, 0, st>>>(src, op->row_stride, (__nv_bfloat16*)op->lp_vals,
                                                                   op->nrows, nb, nbp);
      }
    };
    if (op->precision == DFM_F32)
      convert((const float*)op->vals);
    else
      convert((const __nv_bfloat16*)op->vals);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    op->lp_precision = precision;
    op->lp_valid = true;
  }
  return DFM_OK;
}

namespace {

// one hop over all R right-hand sides (kHopMaxRhs per launch)
template <typename V>
int hop_apply_t(const dfm_op* op, const V* xp, const V* x0p, void* y, int R, bool out_padded, float out_scale,
                cudaStream_t st) {
  const int64_t stride_p = op->nrows * (int64_t)hop_nbp(op->nb);
  const int64_t stride_y = out_padded ? stride_p : op->nrows * (int64_t)op->nb;
  const int64_t ybytes = out_padded ? (int64_t)sizeof(V) : 4;
  for (int r0 = 0; r0 < R; r0 += kHopMaxRhs) {
    const int Rp = std::min(kHopMaxRhs, R - r0);
    const V* x = xp + r0 * stride_p;
    const V* x0 = x0p + r0 * stride_p;
    void* yy = static_cast<char*>(y) + r0 * stride_y * ybytes;
    int rc;
    if constexpr (std::is_same<V, __half>::value) {
      if (op->lp_precision == DFM_F16)
        rc = out_padded ? launch_hop<__half, V, true>(op, x, x0, yy, Rp, out_scale, st)
                        : launch_hop<__half, V, false>(op, x, x0, yy, Rp, out_scale, st);
      else
        rc = out_padded ? launch_hop<__nv_fp8_e4m3, V, true>(op, x, x0, yy, Rp, out_scale, st)
                        : launch_hop<__nv_fp8_e4m3, V, false>(op, x, x0, yy, Rp, out_scale, st);
    } else {
      rc = out_padded ? launch_hop<__nv_bfloat16, V, true>(op, x, x0, yy, Rp, out_scale, st)
                      : launch_hop<__nv_bfloat16, V, false>(op, x, x0, yy, Rp, out_scale, st);
    }
    if (rc) return rc;
  }
  return DFM_OK;
}

template <typename V>
int horner_t(const dfm_op* op, int R, int d, const float* v, float* z, void* vp_, void* ha_, void* hb_, float vscale,
             cudaStream_t st) {
  V* vp = static_cast<V*>(vp_);
  V* h[2] = {static_cast<V*>(ha_), static_cast<V*>(hb_)};
  const int64_t rows = (int64_t)R * op->nrows;
  hop_pack_kernel<V><<<grid_for_elems(rows * hop_nbp(op->nb)), 256, 0, st>>>(v, vp, rows, op->nb, hop_nbp(op->nb),
                                                                           vscale);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  const V* src = vp;
  for (int k = 1; k < d; ++k) {
    const bool last = (k == d - 1);
    void* dst = last ? static_cast<void*>(z) : static_cast<void*>(h[k & 1]);
    const int rc = hop_apply_t<V>(op, src, vp, dst, R, !last, 1.0f / vscale, st);
    if (rc) return rc;
    src = h[k & 1];
  }
  return DFM_OK;
}

}  // namespace

int hop_horner(const dfm_op* op, int R, int d, const float* v, float* z, void* vp, void* ha, void* hb, float vscale,
               cudaStream_t st) {
  if (!op || !op->lp_valid || !v || !z || R < 1 || d < 1)
    return set_error(DFM_ERR_ARG, "preconditioner: no low-precision copy, NULL vector or bad degree");
  if ((reinterpret_cast<uintptr_t>(vp) | reinterpret_cast<uintptr_t>(ha) | reinterpret_cast<uintptr_t>(hb) |
       reinterpret_cast<uintptr_t>(op->lp_vals)) & 15)
    return set_error(DFM_ERR_ARG, "preconditioner: hop vectors and copy must be 16-byte aligned");
  if (d == 1) {
    DFM_CUDA_CHECK(cudaMemcpyAsync(z, v, sizeof(float) * (int64_t)R * op->nrows * op->nb, cudaMemcpyDeviceToDevice, st));
    return DFM_OK;
  }
  // FP16 and e4m3 copies run the hops on FP16 vectors (v scaled by vscale);
  // the BF16 copy on FP32 vectors
  if (op->lp_precision == DFM_BF16) return horner_t<float>(op, R, d, v, z, vp, ha, hb, 1.0f, st);
  return horner_t<__half>(op, R, d, v, z, vp, ha, hb, vscale, st);
}

}  // namespace dfm

extern "C" int dfm_precond_apply(const dfm_op* op, int precision, int degree, const float* x, float* z, int R,
                                 void* stream) {
  using namespace dfm;
  if (!op || !x || !z || R < 1) return set_error(DFM_ERR_ARG, "dfm_precond_apply: NULL operator/vector or R < 1");
  if (x == z) return set_error(DFM_ERR_ARG, "dfm_precond_apply: z must not alias x");
  if (degree < 1 || degree > 64) return set_error(DFM_ERR_ARG, "dfm_precond_apply: degree must be in 1..64");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(z)) & 15)
    return set_error(DFM_ERR_ARG, "dfm_precond_apply: x and z must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  int rc = prepare_lowp(op, precision, st);
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
    rc = hop_horner(op, R, degree, x, z, scratch, scratch + vec_bytes, scratch + 2 * vec_bytes, vscale, st);
  }
  const cudaError_t ef = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_error(e, "dfm_precond_apply");
  if (rc) return rc;
  if (ef != cudaSuccess) return cuda_error(ef, "dfm_precond_apply: cudaFreeAsync");
  return DFM_OK;
}
