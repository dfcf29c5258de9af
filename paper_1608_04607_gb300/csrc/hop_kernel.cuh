// Kernel of the preconditioner hops (hop.cu describes the method and the
// layouts): storage formats of the low-precision copy, the warp-specialised
// hop kernel and its launcher.  Instantiated per copy format in
// hop_launch_*.cu so that the formats compile in parallel.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "dfm_internal.cuh"
#include "tma_pipe.cuh"

namespace dfm {
namespace hopk {

using namespace pipe;

constexpr int kHopStages = 2;  // with 32-row tiles: 29.5 us per e4m3 hop (3 stages: 30.8, 4: 30.9)
// tile and stage geometry: launch_geometry.h (shared with the host-side check)
using geom::kHopConsumerWarps;
using geom::kHopMaxRhs;
constexpr int kHopRhsInner = 4;  // right-hand sides sharing each decoded chunk (multi-RHS launches)
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
  return geom::hop_body_bytes(nb, Codec<E>::kEB);
}
template <typename E>
__host__ __device__ constexpr int64_t copy_row_bytes(int nb, int nbp) {
  return copy_body_bytes<E>(nb, nbp) + (Codec<E>::kScaled ? 16 : 0);
}

// rows per tile (one or two consumer passes), see geom::hop_tile_rows
template <typename E>
__host__ __device__ constexpr int hop_tile_rows(int nb) {
  return geom::hop_tile_rows(nb, Codec<E>::kEB, Codec<E>::kScaled);
}

// y = x0 + alpha B~ x for R right-hand sides; x, x0 of type V (float, or
// __half holding a scaled copy of the vector) padded to NBP per face row; y
// padded of type V (OUTP), or FP32 unpadded (NB per face row) times out_scale.
// With V = __half each block's 8-value chunks are multiplied and summed in
// packed FP16 (one rounding per fused multiply-add; 2 x NBP/8 products per
// lane) and the three block sums are added in FP32.  With FP16 vectors the
// right-hand sides are taken RC at a time, each decoded chunk of B~ serving
// all RC of them.
template <int NB, typename E, typename V, bool OUTP, int RC, bool TR>
__global__ void __launch_bounds__(32 * (kHopConsumerWarps + 1))
hop_kernel(const unsigned char* __restrict__ vals, const int32_t* __restrict__ recv, int64_t nrows,
           const V* __restrict__ xp, const V* __restrict__ x0p, void* __restrict__ yv, int R, float alpha,
           float out_scale, int stages, int reverse, int64_t keep_from, int* __restrict__ err) {
  constexpr int NBP = (NB + 7) / 8 * 8;
  constexpr int NC = NBP / 8;
  constexpr int RSTEP = (32 * kHopConsumerWarps) / NBP;  // rows of one consumer pass
  constexpr int RPT = hop_tile_rows<E>(NB);                   // rows per tile (one or two passes)
  constexpr int EB = Codec<E>::kEB;
  constexpr unsigned ROW_BYTES = (unsigned)copy_row_bytes<E>(NB, NBP);
  constexpr unsigned BODY_BYTES = (unsigned)copy_body_bytes<E>(NB, NBP);
  constexpr unsigned XBLK_D = 4 * NBP * (unsigned)sizeof(V);  // bytes of a source tet's coefficients
  constexpr unsigned XBLK = XBLK_D;                             // their stride in shared memory
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
      mbar_init(&full[s], 1 + 32);  // the producer's expect_tx arrival + one cp.async arrival per producer lane
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
    // per tile row: the rows whose coefficients it gathers.  Forward: the
    // source tet of row R (recv[R] / 4), whose 4 faces are consecutive rows.
    // Transposed: the receiving rows recv[4t + l'] of the row's own tet t,
    // one gathered face row each (read as one 16-byte vector of recv).
    auto row_sources = [&](int64_t row) -> int4 {
      if constexpr (TR) {
        return *reinterpret_cast<const int4*>(recv + (row & ~int64_t(3)));
      } else {
        const int32_t q = recv[row];
        return make_int4(q, q, q, q);
      }
    };
    int4 next_src = make_int4(0, 0, 0, 0);
    if (mine > 0) {
      const int64_t R0 = tile_first_row(0);
      if (lane < RPT && R0 + lane < nrows) next_src = row_sources(R0 + lane);
    }
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      const int64_t R0 = tile_first_row(i);
      const int nr = (int)std::min<int64_t>(RPT, nrows - R0);
      const int4 src = next_src;
      if (i + 1 < mine) {
        const int64_t R1 = tile_first_row(i + 1);
        if (lane < RPT && R1 + lane < nrows) next_src = row_sources(R1 + lane);
      }
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      int32_t* rs = s_recv + s * RPT;
      // the consumers skip face (entry & 3) of the gathered four: the source
      // tet's exit face (forward) or the row's own face (transposed)
      if (lane < nr) rs[lane] = TR ? (int32_t)(R0 + lane) : src.x;
      __syncwarp();  // the row map is written before lane 0's arrive publishes the stage
      fence_proxy_async_smem();
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], (unsigned)nr * ROW_BYTES + (unsigned)(R * nr) * X0ROW);
        const uint64_t pol = (blockIdx.x + i * (int64_t)gridDim.x) >= keep_from ? pol_last : pol_first;
        bulk_copy_g2s_hint(st, vals + R0 * (int64_t)ROW_BYTES, (unsigned)nr * ROW_BYTES, &full[s], pol);
        for (int rhs = 0; rhs < R; ++rhs)
          bulk_copy_g2s(st + (int64_t)RPT * ROW_BYTES + (int64_t)R * RPT * XBLK + (int64_t)rhs * RPT * X0ROW,
                        x0p + ((int64_t)rhs * nrows + R0) * NBP, (unsigned)nr * X0ROW, &full[s]);
      }
      if (lane < nr)
        for (int rhs = 0; rhs < R; ++rhs) {
          unsigned char* dst =
              st + (int64_t)RPT * ROW_BYTES + ((int64_t)rhs * RPT + lane) * XBLK;
          if constexpr (!TR) {
            const unsigned char* srcp =
                reinterpret_cast<const unsigned char*>(xp + ((int64_t)rhs * nrows + 4 * (int64_t)(src.x >> 2)) * NBP);
#pragma unroll
            for (unsigned off = 0; off < XBLK_D; off += 16) cp_async16(dst + off, srcp + off);
          } else {
            const int32_t fr[4] = {src.x, src.y, src.z, src.w};
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              const unsigned char* srcp =
                  reinterpret_cast<const unsigned char*>(xp + ((int64_t)rhs * nrows + fr[f]) * NBP);
#pragma unroll
              for (unsigned off = 0; off < XBLK_D / 4; off += 16)
                cp_async16(dst + f * (XBLK_D / 4) + off, srcp + off);
            }
          }
        }
      cp_async_arrive_noinc(&full[s]);
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
  const int r0c = ctid / NBP;
  const int a = ctid - r0c * NBP;
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
    for (int r = r0c; r0c < RSTEP && r < nr; r += RSTEP) {
      const int lp = s_recv[s * RPT + r] & 3;
      const unsigned char* brow = st + r * ROW_BYTES;
      float scale = 1.f;
      if constexpr (Codec<E>::kScaled) scale = *reinterpret_cast<const float*>(brow + BODY_BYTES);
      const unsigned char* xbase = st + (int64_t)RPT * ROW_BYTES;
      const V* x0base = reinterpret_cast<const V*>(xbase + (int64_t)R * RPT * XBLK);
      if constexpr (VH) {
       for (int q0 = 0; q0 < R; q0 += RC) {
        float sum[RC];
#pragma unroll
        for (int q = 0; q < RC; ++q) sum[q] = 0.f;
        if (a < NB) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int l = k + (k >= lp ? 1 : 0);
            const unsigned char* bk = brow + k * NB * NBP * EB;
            __half2 acc0[RC], acc1[RC];
#pragma unroll
            for (int q = 0; q < RC; ++q) acc0[q] = acc1[q] = __float2half2_rn(0.f);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              __half2 bh[4];
              decode8h<E>(bk + (c * NB + a) * 8 * EB, bh);
#pragma unroll
              for (int q = 0; q < RC; ++q) {
                if (q0 + q < R) {
                  const __half* xl =
                      reinterpret_cast<const __half*>(xbase + ((int64_t)(q0 + q) * RPT + r) * XBLK) + l * NBP + c * 8;
                  const uint4 xv = *reinterpret_cast<const uint4*>(xl);
                  __half2 xh[4];
                  memcpy(xh, &xv, 16);
                  acc0[q] = __hfma2(bh[0], xh[0], acc0[q]);
                  acc1[q] = __hfma2(bh[1], xh[1], acc1[q]);
                  acc0[q] = __hfma2(bh[2], xh[2], acc0[q]);
                  acc1[q] = __hfma2(bh[3], xh[3], acc1[q]);
                }
              }
            }
#pragma unroll
            for (int q = 0; q < RC; ++q) {
              const float2 f0 = __half22float2(acc0[q]), f1 = __half22float2(acc1[q]);
              sum[q] += (f0.x + f0.y) + (f1.x + f1.y);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          if (q0 + q < R) {
            const int qq = q0 + q;
            const float out = a < NB ? (float)x0base[((int64_t)qq * RPT + r) * NBP + a] + alpha * (scale * sum[q]) : 0.f;
            const int64_t row = (int64_t)qq * nrows + R0 + r;
            if constexpr (OUTP)
              reinterpret_cast<V*>(yv)[row * NBP + a] = (V)out;  // pads (a >= NB) written as 0
            else if (a < NB)
              reinterpret_cast<float*>(yv)[row * NB + a] = out * out_scale;
          }
        }
       }
      } else {
        for (int rhs = 0; rhs < R; ++rhs) {
          const float* xs = reinterpret_cast<const float*>(xbase + ((int64_t)rhs * RPT + r) * XBLK);
          float out = 0.f;
          if (a < NB) {
            float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                             make_float2(0.f, 0.f)};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const int l = k + (k >= lp ? 1 : 0);
              const float* xl = xs + l * NBP;
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
            const float sum =
                ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
            out = (float)x0base[((int64_t)rhs * RPT + r) * NBP + a] + alpha * (scale * sum);
          }
          const int64_t row = (int64_t)rhs * nrows + R0 + r;
          if constexpr (OUTP)
            reinterpret_cast<V*>(yv)[row * NBP + a] = (V)out;
          else if (a < NB)
            reinterpret_cast<float*>(yv)[row * NB + a] = out * out_scale;
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <typename E, typename V, bool OUTP, int RC>
int launch_hop(const dfm_op* op, const V* xp, const V* x0p, void* y, int R, float out_scale, int trans,
               cudaStream_t st) {
  const void* copy = lowp_of(op, trans).vals;
  const int nb = op->nb;
  const int nbp = hop_nbp(nb);
  const int rpt = hop_tile_rows<E>(nb);
  const int64_t row_bytes = copy_row_bytes<E>(nb, nbp);
  const int64_t stage_bytes = geom::hop_stage_bytes(nb, Codec<E>::kEB, Codec<E>::kScaled, (int)sizeof(V), R);
  const int stages = geom::hop_stages(stage_bytes, kHopStages);
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
      ::dfm::KernelTimer timer_(trans ? DFM_KERNEL_SPMV16_T : DFM_KERNEL_SPMV16, st);
      kernel<<<(unsigned)grid, 32 * (kHopConsumerWarps + 1), smem, st>>>(
          reinterpret_cast<const unsigned char*>(copy), op->mesh->recv, op->nrows, xp, x0p, y, R, 1.0f,
          out_scale, stages, next_sweep_direction(copy), keep_from, op->dev_err);
    }
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    return DFM_OK;
  };
  auto go_nb = [&](auto nbc) -> int {
    constexpr int NBC = decltype(nbc)::value;
    // FP16 hop vectors on a basis padded to a multiple of 16 wider than 16
    // always run on the fragment-ordered copy (hop.cu, frag_copy)
    if constexpr (std::is_same<V, __half>::value && geom::frag_basis(NBC) && NBC > 16)
      return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: this shape uses the tensor-core hop");
    else
      return trans ? go(hop_kernel<NBC, E, V, OUTP, RC, true>) : go(hop_kernel<NBC, E, V, OUTP, RC, false>);
  };
  switch (nb) {
    case 1: return go_nb(std::integral_constant<int, 1>{});
    case 3: return go_nb(std::integral_constant<int, 3>{});
    case 6: return go_nb(std::integral_constant<int, 6>{});
    case 10: return go_nb(std::integral_constant<int, 10>{});
    case 15: return go_nb(std::integral_constant<int, 15>{});
    case 21: return go_nb(std::integral_constant<int, 21>{});
    case 28: return go_nb(std::integral_constant<int, 28>{});
    case 36: return go_nb(std::integral_constant<int, 36>{});
    case 45: return go_nb(std::integral_constant<int, 45>{});
    default: return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: unsupported basis size");
  }
}


}  // namespace hopk

// y = x0 + B~ x on the copy of op (one copy format per entry point); x, x0
// padded vectors of type V; y padded (outp) or FP32 unpadded times out_scale.
int hop_launch_f16(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int R, float out_scale, bool outp,
                   int trans, cudaStream_t st);
int hop_launch_fp8(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int R, float out_scale, bool outp,
                   int trans, cudaStream_t st);
int hop_launch_bf16(const dfm_op* op, const float* xp, const float* x0p, void* y, int R, float out_scale, bool outp,
                    int trans, cudaStream_t st);

}  // namespace dfm
