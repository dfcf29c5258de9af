// Preconditioner hops on tensor cores for bases whose padded width NBP (NB
// rounded up to 8) is a multiple of 16: NB = 10, 15, 28, 45 (N_p = 3, 4, 6,
// 8), with the FP16 and e4m3 copies.  hop.cu describes the method; this file
// holds the fragment-ordered copy layout, the hop vector layouts, the kernel
// and its launcher.
//
// Per operator row a hop is Y (NB x R) = sum_k B~_k X_k over the row's three
// blocks, a dense contraction: it runs as mma.sync.m16n8k16 products (FP16
// operands, FP32 accumulators) with the blocks as the 16 x 16 A tiles and the
// source faces' coefficients as the 16 x 8 B tiles (8 right-hand sides, or
// one right-hand side in column 0).
//
// Fragment-ordered copy.  Each block (NB x NB, test x trial) is cut into
// 16 x 16 tiles (m-tile mt over test indices, k-tile kt over trial indices,
// trial indices >= NB zero), stored per block in the order (mt, kt).  A tile
// holds, for lane (g, t) = (lane / 4, lane % 4) of the consuming warp, first
// its four values of row g: columns 2t, 2t+1, 2t+8, 2t+9 (128 values for the
// warp), then the same four of row g + 8 for the lanes whose row g + 8 < NB
// (the last m-tile of a block holds vm = NB - 16 mt < 16 rows: 16 vm values).
// One 4-value load per row half gives a lane its A-fragment registers, and a
// block keeps NB x NBP values, as in the vector-friendly layout.  An e4m3 row
// ends with the 16-byte scale field.
//
// Hop vectors.  One right-hand side (W = 1): [rows][NBP] FP16, the face rows
// of a right-hand side one after the other (right-hand sides of a launch
// group are run one launch each).  Several (W = 8): groups of 8 right-hand
// sides, group plane [rows][NBP][8] (right-hand side innermost; sides past R
// zero): a tet's four faces are one contiguous 4 x NBP x 16-byte run, fetched
// by one bulk copy, and the 8 x 8 B sub-tiles come out of shared memory with
// ldmatrix.trans (16-byte rows, no bank conflicts).
//
// Pipeline.  A producer warp issues only bulk copies (TMA): per tile the
// copy rows and the x0 slice of each group, and per tile row the source tet's
// four face rows of each group (forward) or the three receiving rows
// (transposed), all completing on the stage's mbarrier.  Eight consumer warps
// form two groups that take alternate tiles (the stage count is even, so a
// stage is always reused by the group that consumed it last, which keeps the
// barriers' phase parities unambiguous); within a tile a warp owns whole
// (row, group) items: for each block and k-tile one ldmatrix gives the B
// fragment shared by the MT m-tiles.  Waits are bounded; a time-out sets the
// operator's error flag.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "dfm_internal.cuh"
#include "tma_pipe.cuh"

namespace dfm {
namespace fragk {

using namespace pipe;
using geom::kFragGroupWarps;
using geom::kFragGroups;

constexpr int64_t kFragL2KeepBytes = 64ll << 20;  // copy bytes per hop kept in L2 for the next (reversed) sweep

template <typename E>
struct FragFmt;
template <>
struct FragFmt<__half> {
  static constexpr int kEB = 2;
  static constexpr bool kScaled = false;
};
template <>
struct FragFmt<__nv_fp8_e4m3> {
  static constexpr int kEB = 1;
  static constexpr bool kScaled = true;
};

using geom::frag_pos;
using geom::FragPos;

__device__ __forceinline__ uint32_t e4m3x2_to_h2(uint32_t pair16) {
  const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(pair16 & 0xFFFFu), __NV_E4M3);
  uint32_t u;
  memcpy(&u, &hr, 4);
  return u;
}

__device__ __forceinline__ void mma_16816(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// B fragment of a 16 (k) x 8 (n) tile stored row-major with 16-byte rows
// (k rows of 8 halves): lanes 0..15 address rows 0..15
__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t& b0, uint32_t& b1, unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
               : "=r"(b0), "=r"(b1)
               : "r"(addr)
               : "memory");
}

// A fragment of tile (mt, kt) of one block: rows vm of the tile are stored
template <typename E, int NB, int NBP>
__device__ __forceinline__ void load_a(const unsigned char* bk, int mt, int kt, int lane, uint32_t& a0, uint32_t& a1,
                                       uint32_t& a2, uint32_t& a3) {
  const int vm = NB - 16 * mt < 16 ? NB - 16 * mt : 16;
  constexpr int EB = FragFmt<E>::kEB;
  const unsigned char* tile = bk + (16 * mt * NBP + kt * 16 * vm) * EB;
  const bool has_hi = lane < (vm - 8) * 4;
  if constexpr (EB == 1) {
    const uint32_t lo = *reinterpret_cast<const uint32_t*>(tile + lane * 4);
    const uint32_t hi = has_hi ? *reinterpret_cast<const uint32_t*>(tile + 128 + lane * 4) : 0u;
    a0 = e4m3x2_to_h2(lo);
    a2 = e4m3x2_to_h2(lo >> 16);
    a1 = e4m3x2_to_h2(hi);
    a3 = e4m3x2_to_h2(hi >> 16);
  } else {
    const uint2 lo = *reinterpret_cast<const uint2*>(tile + lane * 8);
    const uint2 hi = has_hi ? *reinterpret_cast<const uint2*>(tile + 256 + lane * 8) : make_uint2(0u, 0u);
    a0 = lo.x;
    a2 = lo.y;
    a1 = hi.x;
    a3 = hi.y;
  }
}

// y = x0 + alpha B~ x on the fragment-ordered copy.  W = 1: one right-hand
// side; W = 8: RGL (1 or 2) groups of 8 right-hand sides (planes of
// plane = nrows NBP 8 halves).  OUTP: y in the hop layout (FP16, pads written
// 0); else FP32 [q][nrows][NB] times out_scale for the right-hand sides
// q < rhs_here.  TR: the transposed copy (gathers from the receiving rows).
template <int NB, typename E, int W, bool OUTP, bool TR>
__global__ void __launch_bounds__(32 * (1 + kFragGroups * kFragGroupWarps), 1)
hop_frag_kernel(const unsigned char* __restrict__ vals, const int32_t* __restrict__ recv, int64_t nrows,
                const __half* __restrict__ xp, const __half* __restrict__ x0p, void* __restrict__ yv, int rgl,
                int rhs_here, float alpha, float out_scale, int rpt, int stages, int reverse, int64_t keep_from,
                int* __restrict__ err) {
  constexpr int NBP = (NB + 7) / 8 * 8;
  constexpr int MT = NBP / 16;
  constexpr int KT = NBP / 16;
  constexpr int EB = FragFmt<E>::kEB;
  constexpr unsigned BODY = (unsigned)((3 * NB * NBP * EB + 15) / 16 * 16);
  constexpr unsigned ROW = BODY + (FragFmt<E>::kScaled ? 16u : 0u);
  constexpr unsigned XR = NBP * W * 2;  // bytes of one face row of one group
  static_assert(NBP % 16 == 0, "tensor-core hop needs NBP % 16 == 0");
  static_assert(W == 1 || W == 8, "one or eight right-hand sides per group");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + geom::kFragMaxStages;
  int32_t* s_lp = reinterpret_cast<int32_t*>(smem_raw + 128);
  unsigned char* stage0 = smem_raw + 128 + ((geom::kFragMaxStages * 32 * 4 + 127) / 128) * 128;
  const int64_t plane = nrows * (int64_t)NBP * W;  // halves per group plane
  const int64_t x_off = (int64_t)rpt * ROW;
  const int64_t x0_off = x_off + (int64_t)rpt * rgl * 4 * XR;
  const int64_t stage_bytes = x0_off + (int64_t)rgl * rpt * XR;
  const int64_t ntiles = (nrows + rpt - 1) / rpt;
  const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // one right-hand side: a source face row is only 2 NBP bytes, too small for
  // a bulk copy each (the copy engine's per-request cost dominates), so the
  // producer lanes gather them with 16-byte cp.async copies that arrive on the
  // stage barrier once per lane; groups of 8 use one bulk copy per tile row
  constexpr bool kLsuGather = (W == 1);
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], kLsuGather ? 1 + 32 : 1);  // the producer's arrive.expect_tx (+ a cp.async arrival per lane)
      mbar_init(&empty[s], kFragGroupWarps);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto tile_first_row = [&](int64_t i) {
    const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
    return (reverse ? ntiles - 1 - tile : tile) * rpt;
  };
  if (warp == 0) {
    // ---------------- producer ----------------
    const uint64_t pol_last = l2_policy_evict_last();
    const uint64_t pol_first = l2_policy_evict_first();
    int64_t issued = 0;
    bool ok = true;
    // forward: the source tet of row R (recv[R] / 4), its 4 faces consecutive
    // rows; transposed: the receiving rows recv[4t + l'] of the row's own tet
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
      if (lane < rpt && R0 + lane < nrows) next_src = row_sources(R0 + lane);
    }
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      const int64_t R0 = tile_first_row(i);
      const int nr = (int)std::min<int64_t>(rpt, nrows - R0);
      const int4 src = next_src;
      if (i + 1 < mine) {
        const int64_t R1 = tile_first_row(i + 1);
        if (lane < rpt && R1 + lane < nrows) next_src = row_sources(R1 + lane);
      }
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      // the face each row skips: the source tet's exit face (forward) or the
      // row's own face (transposed)
      if (lane < nr) s_lp[s * 32 + lane] = TR ? (int32_t)((R0 + lane) & 3) : (src.x & 3);
      __syncwarp();  // the map is written before lane 0's arrive publishes the stage
      const unsigned gathered = TR ? 3u : 4u;
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], (unsigned)nr * ROW + (unsigned)(rgl * nr) * XR * (kLsuGather ? 1u : 1u + gathered));
        const uint64_t pol = (blockIdx.x + i * (int64_t)gridDim.x) >= keep_from ? pol_last : pol_first;
        bulk_copy_g2s_hint(st, vals + R0 * (int64_t)ROW, (unsigned)nr * ROW, &full[s], pol);
        for (int g = 0; g < rgl; ++g)
          bulk_copy_g2s(st + x0_off + (int64_t)g * rpt * XR, x0p + g * plane + R0 * (int64_t)NBP * W,
                        (unsigned)nr * XR, &full[s]);
      }
      if constexpr (kLsuGather) {
        // 16-byte chunks of the tile rows' source face rows over the lanes:
        // row r's gathered face f comes from the lane holding row r's sources
        constexpr int CH = XR / 16;  // chunks per face row
        const int total = nr * 4 * CH;
        for (int base = 0; base < total; base += 32) {  // uniform trip count: the shuffles see every lane
          const int item = base + lane;
          const int r = (item < total ? item : 0) / (4 * CH);
          const int f = ((item < total ? item : 0) / CH) & 3;
          const int c = (item < total ? item : 0) % CH;
          const int32_t sx = __shfl_sync(0xffffffffu, src.x, r);
          int32_t srow;
          bool skip = item >= total;
          if constexpr (!TR) {
            srow = 4 * (sx >> 2) + f;
          } else {
            const int32_t sy = __shfl_sync(0xffffffffu, src.y, r), sz = __shfl_sync(0xffffffffu, src.z, r);
            const int32_t sw = __shfl_sync(0xffffffffu, src.w, r);
            srow = f == 0 ? sx : (f == 1 ? sy : (f == 2 ? sz : sw));
            skip = skip || f == (int)((R0 + r) & 3);  // the row's own face is not needed
          }
          if (!skip)
            cp_async16(st + x_off + ((int64_t)r * 4 + f) * XR + c * 16,
                       reinterpret_cast<const unsigned char*>(xp + (int64_t)srow * NBP) + c * 16);
        }
        cp_async_arrive_noinc(&full[s]);
      } else if (lane < nr) {
        for (int g = 0; g < rgl; ++g) {
          unsigned char* dst = st + x_off + ((int64_t)lane * rgl + g) * 4 * XR;
          if constexpr (!TR) {
            bulk_copy_g2s(dst, xp + g * plane + 4 * (int64_t)(src.x >> 2) * NBP * W, 4 * XR, &full[s]);
          } else {
            const int32_t fr[4] = {src.x, src.y, src.z, src.w};
            const int own = (int)((R0 + lane) & 3);
#pragma unroll
            for (int f = 0; f < 4; ++f)
              if (f != own) bulk_copy_g2s(dst + f * XR, xp + g * plane + (int64_t)fr[f] * NBP * W, XR, &full[s]);
          }
        }
      }
      issued = i + 1;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    // drain: every issued stage must have landed before the block's shared memory goes away
    if (lane == 0)
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j)
        mbar_wait_bounded(&full[j % stages], (unsigned)((j / stages) & 1));
    return;
  }
  // ---------------- consumers: two groups of warps take alternate tiles ----------------
  const int cgrp = (warp - 1) / kFragGroupWarps;
  const int cw = (warp - 1) % kFragGroupWarps;
  const int g8 = lane >> 2, t4 = lane & 3;
  for (int64_t i = cgrp; i < mine; i += kFragGroups) {
    const int s = (int)(i % stages);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((i / stages) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const unsigned char* st = stage0 + s * stage_bytes;
    const int64_t R0 = tile_first_row(i);
    const int nr = (int)std::min<int64_t>(rpt, nrows - R0);
    const int items = nr * rgl;
    for (int it = cw; it < items; it += kFragGroupWarps) {
      const int r = it / rgl;
      const int gl = it - r * rgl;
      const unsigned char* brow = st + (int64_t)r * ROW;
      const __half* xs = reinterpret_cast<const __half*>(st + x_off + ((int64_t)r * rgl + gl) * 4 * XR);
      const int lp = s_lp[s * 32 + r];
      // one right-hand side: the three blocks accumulate apart (three
      // independent MMA chains per row instead of one), summed at the end
      constexpr int NACC = W == 1 ? 3 : 1;
      float acc[NACC][MT][4];
#pragma unroll
      for (int q = 0; q < NACC; ++q)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) acc[q][mt][0] = acc[q][mt][1] = acc[q][mt][2] = acc[q][mt][3] = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int l = k + (k >= lp ? 1 : 0);
        const __half* xl = xs + l * NBP * W;
        const unsigned char* bk = brow + k * NB * NBP * EB;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
          uint32_t b0, b1;
          if constexpr (W == 8) {
            ldmatrix_x2_trans(b0, b1, smem_addr(xl + (kt * 16 + (lane & 15)) * 8));
          } else {
            b0 = g8 == 0 ? *reinterpret_cast<const uint32_t*>(xl + kt * 16 + 2 * t4) : 0u;
            b1 = g8 == 0 ? *reinterpret_cast<const uint32_t*>(xl + kt * 16 + 8 + 2 * t4) : 0u;
          }
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            uint32_t a0, a1, a2, a3;
            load_a<E, NB, NBP>(bk, mt, kt, lane, a0, a1, a2, a3);
            mma_16816(acc[k % NACC][mt], a0, a1, a2, a3, b0, b1);
          }
        }
      }
#pragma unroll
      for (int q = 1; q < NACC; ++q)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[0][mt][e] += acc[q][mt][e];
      float scale = 1.f;
      if constexpr (FragFmt<E>::kScaled) scale = *reinterpret_cast<const float*>(brow + BODY);
      const float as = alpha * scale;
      const __half* x0s = reinterpret_cast<const __half*>(st + x0_off + ((int64_t)gl * rpt + r) * XR);
      const int64_t row = R0 + r;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int a = 16 * mt + g8 + 8 * h;
          if constexpr (W == 8) {
            const float2 x0v = __half22float2(*reinterpret_cast<const __half2*>(x0s + a * 8 + 2 * t4));
            const float o0 = x0v.x + as * acc[0][mt][2 * h], o1 = x0v.y + as * acc[0][mt][2 * h + 1];
            if constexpr (OUTP) {
              *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(yv) + gl * plane + (row * NBP + a) * 8 + 2 * t4) =
                  __floats2half2_rn(o0, o1);
            } else if (a < NB) {
              const int q = gl * 8 + 2 * t4;
              float* yf = reinterpret_cast<float*>(yv);
              if (q < rhs_here) yf[((int64_t)q * nrows + row) * NB + a] = o0 * out_scale;
              if (q + 1 < rhs_here) yf[((int64_t)(q + 1) * nrows + row) * NB + a] = o1 * out_scale;
            }
          } else if (t4 == 0) {
            const float o = __half2float(x0s[a]) + as * acc[0][mt][2 * h];
            if constexpr (OUTP)
              reinterpret_cast<__half*>(yv)[row * NBP + a] = __float2half_rn(o);
            else if (a < NB)
              reinterpret_cast<float*>(yv)[row * NB + a] = o * out_scale;
          }
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// One hop launch on op's fragment-ordered copy (trans: the transposed copy)
// for one right-hand side (w = 1) or rgl groups of 8 (w = 8); rhs_here
// bounds the FP32 output's right-hand sides.  rpt_req / stages_req: tile
// rows and pipeline stages (0: the geometry's default).
template <typename E>
int launch_hop_frag(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int w, int rgl, int rhs_here,
                    bool outp, float out_scale, int trans, int rpt_req, int stages_req, cudaStream_t st) {
  const void* copy = lowp_of(op, trans).vals;
  const int nb = op->nb;
  const geom::Frag g = geom::frag_geometry(nb, FragFmt<E>::kEB, FragFmt<E>::kScaled, w, rgl, rpt_req, stages_req);
  if (g.stages < 2 || g.stages % kFragGroups)
    return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: a tile does not fit shared memory");
  const size_t smem = geom::frag_smem_bytes(g);
  int dev = 0, nsm = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 32 * (1 + kFragGroups * kFragGroupWarps);
  auto go = [&](auto kernel) -> int {
    DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (op->nrows + g.rpt - 1) / g.rpt;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    const int64_t row_bytes = geom::hop_row_bytes(nb, FragFmt<E>::kEB, FragFmt<E>::kScaled);
    const int64_t keep_from = std::max<int64_t>(0, ntiles - kFragL2KeepBytes / (g.rpt * row_bytes));
    {
      ::dfm::KernelTimer timer_(trans ? DFM_KERNEL_SPMV16_T : DFM_KERNEL_SPMV16, st);
      kernel<<<(unsigned)grid, threads, smem, st>>>(reinterpret_cast<const unsigned char*>(copy), op->mesh->recv,
                                                    op->nrows, xp, x0p, y, rgl, rhs_here, 1.0f, out_scale, g.rpt,
                                                    g.stages, next_sweep_direction(copy), keep_from, op->dev_err);
    }
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    return DFM_OK;
  };
  auto pick = [&](auto nbc) -> int {
    constexpr int NBC = decltype(nbc)::value;
    if (w == 1) {
      if (outp) return trans ? go(hop_frag_kernel<NBC, E, 1, true, true>) : go(hop_frag_kernel<NBC, E, 1, true, false>);
      return trans ? go(hop_frag_kernel<NBC, E, 1, false, true>) : go(hop_frag_kernel<NBC, E, 1, false, false>);
    }
    if (outp) return trans ? go(hop_frag_kernel<NBC, E, 8, true, true>) : go(hop_frag_kernel<NBC, E, 8, true, false>);
    return trans ? go(hop_frag_kernel<NBC, E, 8, false, true>) : go(hop_frag_kernel<NBC, E, 8, false, false>);
  };
  switch (nb) {
    case 10: return pick(std::integral_constant<int, 10>{});
    case 15: return pick(std::integral_constant<int, 15>{});
    case 28: return pick(std::integral_constant<int, 28>{});
    case 45: return pick(std::integral_constant<int, 45>{});
    default: return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: no fragment-ordered layout for this basis");
  }
}

}  // namespace fragk

// entry points per copy format (hop_launch_*.cu)
int hop_frag_launch_fp8(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int w, int rgl, int rhs_here,
                        bool outp, float out_scale, int trans, int rpt, int stages, cudaStream_t st);
int hop_frag_launch_f16(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int w, int rgl, int rhs_here,
                        bool outp, float out_scale, int trans, int rpt, int stages, cudaStream_t st);

}  // namespace dfm
