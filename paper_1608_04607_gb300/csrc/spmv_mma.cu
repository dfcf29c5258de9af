// Forward application y = x0 + alpha B x of a BF16 operator to several FP32
// right-hand sides on tensor cores (the Krylov operator of the batched solves
// on the 45-function workload).
//
// Per operator row the product is Y (NB x R) = sum_k B_k X_k over the row's
// three blocks, a dense contraction.  The blocks are BF16 (exact as MMA
// operands); each FP32 coefficient x is split exactly into three BF16 parts
// x = x1 + x2 + x3 (8 significant bits each, 24 together), so the three
// mma.sync.m16n8k16 products per tile with FP32 accumulators give B x to
// FP32 accuracy.  A fragments come from the row-major BF16 blocks in shared
// memory (two 16-bit loads per pair: rows of an odd basis are not 4-byte
// aligned); B fragments from the staged FP32 coefficients, split on the fly.
//
// Pipeline as in the other applications: a producer warp streams tiles of
// consecutive operator rows by bulk copy and gathers each row's source-tet
// coefficients of every right-hand side by one bulk copy per (row,
// right-hand side), the lanes issuing them in parallel; eight consumer warps in two groups
// take alternate tiles (an even number of stages keeps the barrier phases
// unambiguous) and own whole (row, group of 8 right-hand sides) items.
// Waits are bounded; a time-out sets the operator's error flag.
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "dfm_internal.cuh"
#include "tma_pipe.cuh"
#include "tune.h"

namespace dfm {
namespace {

using namespace pipe;
constexpr int kGroups = 2;      // consumer groups taking alternate tiles
constexpr int kGroupWarps = 4;  // warps per consumer group
constexpr int kMaxStages = 8;
constexpr int kMaxRhs = 16;     // right-hand sides per launch
constexpr int64_t kBudget = 200 * 1024 - 2048;

__device__ __forceinline__ void mma_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// the BF16 pair (B[a][b], B[a][b + 1]) of a row-major NB x NB block; zero
// outside the block
template <int NB>
__device__ __forceinline__ uint32_t pair_at(const uint16_t* blk, int a, int b) {
  const uint32_t lo = (a < NB && b < NB) ? blk[a * NB + b] : 0u;
  const uint32_t hi = (a < NB && b + 1 < NB) ? blk[a * NB + b + 1] : 0u;
  return lo | (hi << 16);
}

// exact three-way BF16 split of two FP32 values, packed per part
__device__ __forceinline__ void split3(float x0, float x1, uint32_t out[3]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    memcpy(&out[p], &h, 4);
    const float2 f = __bfloat1622float2(h);
    x0 -= f.x;
    x1 -= f.y;
  }
}

template <int NB>
__global__ void __launch_bounds__(32 * (1 + kGroups * kGroupWarps), 1)
spmv_mma_kernel(const __nv_bfloat16* __restrict__ vals, int64_t row_stride, const int32_t* __restrict__ recv,
                int64_t nrows, const float* __restrict__ x, const float* x0, float* y, int R, float alpha, int rpt,
                int stages, int reverse, int64_t keep_from, int* __restrict__ err) {
  constexpr int NBP = (NB + 7) / 8 * 8;
  constexpr int MT = NBP / 16, KT = NBP / 16;
  constexpr int XB = 4 * NB * 4;  // bytes of one source tet's coefficients (one right-hand side)
  static_assert(NBP % 16 == 0, "tensor-core application needs NBP % 16 == 0");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kMaxStages;
  int32_t* s_lp = reinterpret_cast<int32_t*>(smem_raw + 128);
  unsigned char* stage0 = smem_raw + 128 + ((kMaxStages * 32 * 4 + 127) / 128) * 128;
  const int64_t row_bytes = row_stride * 2;
  const int64_t x_off = (int64_t)rpt * row_bytes;
  const int64_t stage_bytes = x_off + (int64_t)rpt * R * XB;
  const int ng = (R + 7) / 8;
  const int64_t ntiles = (nrows + rpt - 1) / rpt;
  const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);  // the producer's arrive.expect_tx; every copy is a bulk copy
      mbar_init(&empty[s], kGroupWarps);
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
    int32_t next_src = 0;
    if (mine > 0) {
      const int64_t R0 = tile_first_row(0);
      if (lane < rpt && R0 + lane < nrows) next_src = recv[R0 + lane];
    }
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      const int64_t R0 = tile_first_row(i);
      const int nr = (int)std::min<int64_t>(rpt, nrows - R0);
      const int32_t src = next_src;
      if (i + 1 < mine) {
        const int64_t R1 = tile_first_row(i + 1);
        if (lane < rpt && R1 + lane < nrows) next_src = recv[R1 + lane];
      }
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      if (lane < nr) s_lp[s * 32 + lane] = src & 3;  // the source tet's exit face, skipped
      __syncwarp();  // the map is written before lane 0's arrive publishes the stage
      if (lane == 0) {
        mbar_arrive_expect_tx(&full[s], (unsigned)(nr * row_bytes + (int64_t)nr * R * XB));
        const uint64_t pol = (blockIdx.x + i * (int64_t)gridDim.x) >= keep_from ? pol_last : pol_first;
        bulk_copy_g2s_hint(st, vals + R0 * row_stride, (unsigned)(nr * row_bytes), &full[s], pol);
      }
      // one bulk copy per (row, right-hand side): the source tet's 4 NB coefficients
      for (int base = 0; base < nr * R; base += 32) {  // uniform trip count for the shuffle
        const int item = base + lane;
        const int it = item < nr * R ? item : 0;
        const int r = it / R, q = it - (it / R) * R;
        const int32_t sr = __shfl_sync(0xffffffffu, src, r);
        if (item < nr * R)
          bulk_copy_g2s(st + x_off + (int64_t)it * XB, x + ((int64_t)q * nrows + 4 * (int64_t)(sr >> 2)) * NB, XB,
                        &full[s]);
      }
      issued = i + 1;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    if (lane == 0)
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j)
        mbar_wait_bounded(&full[j % stages], (unsigned)((j / stages) & 1));
    return;
  }
  // ---------------- consumers ----------------
  const int cgrp = (warp - 1) / kGroupWarps;
  const int cw = (warp - 1) % kGroupWarps;
  const int g8 = lane >> 2, t4 = lane & 3;
  for (int64_t i = cgrp; i < mine; i += kGroups) {
    const int s = (int)(i % stages);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((i / stages) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const unsigned char* st = stage0 + s * stage_bytes;
    const int64_t R0 = tile_first_row(i);
    const int nr = (int)std::min<int64_t>(rpt, nrows - R0);
    const int items = nr * ng;
    for (int it = cw; it < items; it += kGroupWarps) {
      const int r = it / ng;
      const int gq = it - r * ng;
      const uint16_t* brow = reinterpret_cast<const uint16_t*>(st + (int64_t)r * row_bytes);
      const int lp = s_lp[s * 32 + r];
      const int q = gq * 8 + g8;  // this lane's right-hand side in the B fragments
      const float* xq = reinterpret_cast<const float*>(st + x_off + ((int64_t)r * R + (q < R ? q : 0)) * XB);
      const int64_t row = R0 + r;
      // x0 of this lane's outputs, loaded before the products so that the
      // global-memory latency hides behind them
      float x0v[MT][2][2];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int a = 16 * mt + g8 + 8 * h;
            const int qq = gq * 8 + 2 * t4 + e;
            x0v[mt][h][e] = (x0 && a < NB && qq < R) ? x0[((int64_t)qq * nrows + row) * NB + a] : 0.f;
          }
      float acc[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int l = k + (k >= lp ? 1 : 0);
        const float* xl = xq + l * NB;
        const uint16_t* bk = brow + k * NB * NB;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
          const int c0 = kt * 16 + 2 * t4, c1 = c0 + 8;
          const bool live = q < R;
          uint32_t blo[3], bhi[3];
          split3(live && c0 < NB ? xl[c0] : 0.f, live && c0 + 1 < NB ? xl[c0 + 1] : 0.f, blo);
          split3(live && c1 < NB ? xl[c1] : 0.f, live && c1 + 1 < NB ? xl[c1 + 1] : 0.f, bhi);
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const int a = mt * 16 + g8;
            const uint32_t a0 = pair_at<NB>(bk, a, c0), a1 = pair_at<NB>(bk, a + 8, c0);
            const uint32_t a2 = pair_at<NB>(bk, a, c1), a3 = pair_at<NB>(bk, a + 8, c1);
#pragma unroll
            for (int p = 0; p < 3; ++p) mma_bf16(acc[mt], a0, a1, a2, a3, blo[p], bhi[p]);
          }
        }
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int a = 16 * mt + g8 + 8 * h;
          if (a >= NB) continue;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int qq = gq * 8 + 2 * t4 + e;
            if (qq >= R) continue;
            y[((int64_t)qq * nrows + row) * NB + a] = x0v[mt][h][e] + alpha * acc[mt][2 * h + e];
          }
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

struct Geo {
  int rpt, stages;
  int64_t stage_bytes;
};

// tile rows in multiples of the rows that give each warp of a group one
// (row, group of 8) item; stages even (consumer groups alternate) and within
// the shared-memory budget
Geo geometry(int nb, int R, int rpt, int stages) {
  const int64_t row = (int64_t)((3 * nb * nb + 7) / 8 * 8) * 2 + (int64_t)R * 16 * nb;
  Geo g{};
  g.rpt = std::max(1, std::min(rpt, 32));
  while (g.rpt > 1 && 2 * g.rpt * row > kBudget) --g.rpt;
  g.stage_bytes = g.rpt * row;
  int64_t st = std::min<int64_t>(kMaxStages, kBudget / g.stage_bytes);
  if (stages > 0) st = std::min<int64_t>(st, stages);
  st -= st % kGroups;
  g.stages = (int)st;
  return g;
}

template <int NB>
int launch_nb(const dfm_op* op, const float* x, const float* x0, float* y, int R, float alpha, int rpt, int stages,
              cudaStream_t st) {
  const Geo g = geometry(NB, R, rpt, stages);
  if (g.stages < 2) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: tensor-core tile does not fit shared memory");
  const size_t smem = 128 + ((kMaxStages * 32 * 4 + 127) / 128) * 128 + (size_t)g.stages * g.stage_bytes;
  int dev = 0, nsm = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 32 * (1 + kGroups * kGroupWarps);
  auto kernel = spmv_mma_kernel<NB>;
  DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (op->nrows + g.rpt - 1) / g.rpt;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
  const int64_t keep_from = std::max<int64_t>(0, ntiles - (64ll << 20) / (g.rpt * op->row_stride * 2));
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_SPMV, st);
    kernel<<<(unsigned)grid, threads, smem, st>>>(reinterpret_cast<const __nv_bfloat16*>(op->vals), op->row_stride,
                                                  op->recv ? op->recv : op->mesh->recv, op->nrows, x, x0, y, R,
                                                  alpha, g.rpt, g.stages,
                                                  next_sweep_direction(op->vals), keep_from, op->dev_err);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

int launch_any(const dfm_op* op, const float* x, const float* x0, float* y, int R, float alpha, int rpt, int stages,
               cudaStream_t st) {
  switch (op->nb) {
    case 10: return launch_nb<10>(op, x, x0, y, R, alpha, rpt, stages, st);
    case 15: return launch_nb<15>(op, x, x0, y, R, alpha, rpt, stages, st);
    case 28: return launch_nb<28>(op, x, x0, y, R, alpha, rpt, stages, st);
    case 45: return launch_nb<45>(op, x, x0, y, R, alpha, rpt, stages, st);
    default: return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: no tensor-core application for this basis");
  }
}

}  // namespace

bool apply_mma_supported(const dfm_op* op, int R) {
  return op->precision == DFM_BF16 && R >= 4 && geom::frag_basis(op->nb);
}

// y = x0 + alpha B x for R >= 4 FP32 right-hand sides on a BF16 operator,
// kMaxRhs per launch, each launch shape with its autotuned tile geometry
int apply_mma(const dfm_op* op, const float* x, const float* x0, float* y, int R, double alpha, cudaStream_t st) {
  const int64_t stride = op->nrows * (int64_t)op->nb;
  int dev = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  for (int r0 = 0; r0 < R; r0 += kMaxRhs) {
    const int Rl = std::min(kMaxRhs, R - r0);
    const float* xr = x + r0 * stride;
    const float* x0r = x0 ? x0 + r0 * stride : nullptr;
    float* yr = y + r0 * stride;
    auto go = [&](int rpt, int stages) { return launch_any(op, xr, x0r, yr, Rl, (float)alpha, rpt, stages, st); };
    const int unit = std::max(1, kGroupWarps / ((Rl + 7) / 8));
    // tile rows: a full round of items per consumer group and multiples, or
    // half of one (smaller stages: two blocks per SM)
    std::vector<tune::Geometry> cands;
    for (int rpt : {std::max(1, unit / 2), unit, 2 * unit, 3 * unit, 4 * unit})
      for (int s : {2, 4, 6}) {
        const Geo g = geometry(op->nb, Rl, rpt, s);
        bool dup = false;
        for (const tune::Geometry& c : cands) dup = dup || (c.rpt == g.rpt && c.stages == g.stages);
        if (g.rpt == rpt && g.stages == s && !dup) cands.push_back(tune::Geometry{g.rpt, g.stages, 0.f});
      }
    const Geo d = geometry(op->nb, Rl, unit, 0);
    const tune::Key key{1, op->nb, op->precision, Rl, 1, 0, op->nrows, dev};
    tune::Geometry chosen;
    int rc = tune::choose(key, st, cands, tune::Geometry{d.rpt, d.stages, 0.f}, go, &chosen);
    if (rc) return rc;
    rc = go(chosen.rpt, chosen.stages);
    if (rc) return rc;
  }
  return DFM_OK;
}

}  // namespace dfm
