// Block-sparse application of the transfer operator: y = x0 + alpha B x and
// y = x0 + alpha B^T x (Sec. 2: B couples a face only to the faces of one tet,
// so every block row and every block column holds exactly three blocks).
//
// Forward: row R receives three blocks, all from tet t = recv[R]/4, whose
// source faces are the three faces of t other than l' = recv[R]%4.  Tiles of
// consecutive rows (contiguous in memory, 32-byte aligned rows) stream into
// shared memory through a TMA bulk-copy pipeline; one thread per (row, test
// index) forms its dot products against the source tet's coefficients (read
// through the read-only cache); a staged tile serves every right-hand side.
//
// Transpose: column J = 4t + l owns the blocks (t, l) -> l' received by rows
// recv[4t + l'] in slot l - (l > l'); one thread per (column, trial index)
// walks the three blocks with coalesced reads along the trial index.
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include <mutex>
#include <unordered_map>

#include "dfm_internal.cuh"
#include "tma_pipe.cuh"

namespace dfm {
namespace {

using namespace pipe;

constexpr int kThreads = 128;

template <typename TV, typename TX, typename TA>
__global__ void __launch_bounds__(kThreads)
spmv_t_kernel(const TV* __restrict__ vals, int64_t row_stride, const int32_t* __restrict__ recv, int64_t nrows, int nb,
              const TX* __restrict__ x, const TX* x0, TX* y, int R, TA alpha) {
  const int64_t total = nrows * nb;
  const int nb2 = nb * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total * R; i += (int64_t)gridDim.x * blockDim.x) {
    const int rhs = (int)(i / total);
    const int64_t e = i - rhs * total;
    const int64_t J = e / nb;
    const int b = (int)(e - J * nb);
    const int64_t t = J >> 2;
    const int l = (int)(J & 3);
    const TX* xr = x + (int64_t)rhs * total;
    TA acc = TA(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int lp = k + (k >= l ? 1 : 0);
      const int64_t Rw = recv[4 * t + lp];
      const int slot = l - (l > lp ? 1 : 0);
      const TV* blk = vals + Rw * row_stride + (int64_t)slot * nb2 + b;
      const TX* xw = xr + Rw * nb;
      for (int a = 0; a < nb; ++a) acc = fma((TA)__ldg(blk + a * nb), (TA)xw[a], acc);
    }
    const TA base = x0 ? (TA)x0[i] : TA(0);
    y[i] = (TX)(base + alpha * acc);
  }
}

// ---------------------------------------------------------------------------
// Forward application with a TMA bulk-copy pipeline.
//
// Each block walks its tiles (consecutive rows, one contiguous range of the
// operator) with kStages shared-memory buffers: one thread issues a 1-D
// cp.async.bulk copy per tile, completion is tracked by a per-stage mbarrier
// (expect_tx), and the block computes tile i while tiles i+1..i+kStages-1 are
// in flight.  Every wait is bounded; on a time-out the block records an error,
// waits (bounded) for its own copies and leaves.
// ---------------------------------------------------------------------------
constexpr int kStages = 4;
constexpr int kMaxStagedRhs = 16;  // right-hand sides staged per operator pass
constexpr int kConsumerWarps = 4;  // computing warps per block (plus one producer warp)

// Operators applied together: y_r = x0_r + alpha * sum_k coef[r][k] B_k x_r,
// for the right-hand sides of one launch (k < K <= kMaxCombo, r < kMaxStagedRhs).
constexpr int kMaxCombo = 4;
struct Combo {
  const void* vals[kMaxCombo];
  int K;
  double coef[kMaxStagedRhs][kMaxCombo];
};

// Output a of one operator row: sum over the row's three blocks k of
// sum_b B_k[a][b] x_l[b], l = the k-th face of the source tet other than lp.
// blk points at B_0[a][0]; xs at the source tet's 4 x NB coefficients.
template <int NB, typename TV, typename TX, typename TA>
__device__ __forceinline__ TA row_times_x(const TV* blk, const TX* xs, int lp) {
  TA acc[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int l = k + (k >= lp ? 1 : 0);
    const TV* bk = blk + k * NB * NB;
    const TX* xl = xs + l * NB;
    TA a0 = TA(0);
#pragma unroll
    for (int b = 0; b < NB; ++b) a0 = fma((TA)bk[b], (TA)xl[b], a0);
    acc[k] = a0;
  }
  return (acc[0] + acc[1]) + acc[2];
}

// The same with FP64 vectors on an FP32 or BF16 operator (the FP64 residual of
// iterative refinement) without FP64 arithmetic, whose rate on this GPU is a
// small fraction of the FP32 rate: each x = xh + xl is held as a pair of
// floats (xh = fl32(x), xl = fl32(x - xh)); the product b xh is split exactly
// into p + e (e = fma(b, xh, -p)), p is summed by Knuth's two-sum into s with
// its rounding error, e and b xl are added to a compensation c, and the row
// sum s + c carries about twice the FP32 precision, ample for a residual
// that cancels to 1e-10 of the terms.
template <int NB, typename TV>
__device__ __forceinline__ double row_times_x_split(const TV* blk, const float2* xs, int lp) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int l = k + (k >= lp ? 1 : 0);
    const TV* bk = blk + k * NB * NB;
    const float2* xl = xs + l * NB;
#pragma unroll 5
    for (int b = 0; b < NB; ++b) {
      const float bv = (float)bk[b];
      const float2 xv = xl[b];
      const float p = __fmul_rn(bv, xv.x);
      const float e = __fmaf_rn(bv, xv.x, -p);
      const float t = __fadd_rn(s, p);
      const float z = __fsub_rn(t, s);
      const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
      c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(bv, xv.y, e)));
      s = t;
    }
  }
  return (double)s + (double)c;
}

// The same for QN <= 4 right-hand sides at once (their staged coefficients
// xstride float2 apart): the QN independent two-sum chains interleave, which
// keeps the FP32 pipes busy with few warps, and each block entry is read once.
template <int NB, typename TV, int QN>
__device__ __forceinline__ void row_times_x_split_q(const TV* blk, const float2* xs, int64_t xstride, int lp,
                                                    double out[QN]) {
  float s[QN], c[QN];
#pragma unroll
  for (int q = 0; q < QN; ++q) s[q] = c[q] = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int l = k + (k >= lp ? 1 : 0);
    const TV* bk = blk + k * NB * NB;
    const float2* xl = xs + l * NB;
#pragma unroll 3
    for (int b = 0; b < NB; ++b) {
      const float bv = (float)bk[b];
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const float2 xv = xl[q * xstride + b];
        const float p = __fmul_rn(bv, xv.x);
        const float e = __fmaf_rn(bv, xv.x, -p);
        const float t = __fadd_rn(s[q], p);
        const float z = __fsub_rn(t, s[q]);
        const float err = __fadd_rn(__fsub_rn(s[q], __fsub_rn(t, z)), __fsub_rn(p, z));
        c[q] = __fadd_rn(c[q], __fadd_rn(err, __fmaf_rn(bv, xv.y, e)));
        s[q] = t;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QN; ++q) out[q] = (double)s[q] + (double)c[q];
}

// Warp-specialised pipeline.  Warp 0 is the producer: for each of the block's
// tiles it waits until the stage is free (`empty` barrier, one arrival per
// consumer warp), reads the tile's row map (one coalesced load by the lanes),
// and issues the bulk copies (operator rows; per row and right-hand side the
// source tet's 4 x NB coefficients), all completing on the stage's `full`
// barrier.  Warps 1..kConsumerWarps compute.  All waits are bounded; the
// producer drains its outstanding copies (bounded) before the block exits.
// KC = 1: a single operator (cb.K must be 1), compiled without the combination
// loop; KC = 0: cb.K operators combined with per-right-hand-side weights.
template <int NB, int KC, typename TV, typename TX, typename TA>
__global__ void __launch_bounds__(32 * (kConsumerWarps + 1))
spmv_tma_kernel(const Combo cb, int64_t row_stride, const int32_t* __restrict__ recv, int64_t nrows,
                int rows_per_tile, int stages, const TX* __restrict__ x, const TX* x0, TX* y, int R, TA alpha,
                int stage_x0, int reverse, int64_t keep_from, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kStages;
  int32_t* s_recv = reinterpret_cast<int32_t*>(smem_raw + 128);
  const int K = KC ? KC : cb.K;
  const int64_t op_tile_bytes = (int64_t)rows_per_tile * row_stride * (int64_t)sizeof(TV);
  const int64_t vals_bytes = K * op_tile_bytes;
  const int64_t xblk = 4 * NB * (int64_t)sizeof(TX);
  const int64_t x0_bytes = stage_x0 ? (int64_t)R * rows_per_tile * NB * (int64_t)sizeof(TX) : 0;
  const int64_t stage_bytes = vals_bytes + (int64_t)R * rows_per_tile * xblk + ((x0_bytes + 15) / 16) * 16;
  unsigned char* stage0 = smem_raw + 128 + ((stages * rows_per_tile * 4 + 127) / 128) * 128;
  const int64_t ntiles = (nrows + rows_per_tile - 1) / rows_per_tile;
  const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    // ---------------- producer ----------------
    // lane r handles tile row r (rows_per_tile <= 32); the row map of the next
    // tile is loaded one iteration ahead so its latency overlaps this tile's issue
    int64_t issued = 0;
    bool ok = true;
    auto tile_rows = [&](int64_t i, int64_t* R0, int* nr) {
      const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
      *R0 = (reverse ? ntiles - 1 - tile : tile) * rows_per_tile;
      const int64_t left = nrows - *R0;
      *nr = left < rows_per_tile ? (int)left : rows_per_tile;
    };
    // operator tiles late in this sweep are kept in L2 (evict_last) for the
    // next application, which sweeps in the opposite direction and reads them
    // first; the rest stream through (evict_first)
    const uint64_t pol_last = l2_policy_evict_last();
    const uint64_t pol_first = l2_policy_evict_first();
    int32_t next_src = 0;
    if (mine > 0) {
      int64_t R0;
      int nr;
      tile_rows(0, &R0, &nr);
      if (lane < nr) next_src = recv[R0 + lane];
    }
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      int64_t R0;
      int nr;
      tile_rows(i, &R0, &nr);
      const int32_t src = next_src;
      if (i + 1 < mine) {
        int64_t R1;
        int n1;
        tile_rows(i + 1, &R1, &n1);
        if (lane < n1) next_src = recv[R1 + lane];
      }
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      int32_t* rs = s_recv + s * rows_per_tile;
      if (lane < nr) rs[lane] = src;
      __syncwarp();  // the row map is written before lane 0's arrive publishes the stage
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const unsigned x0b = stage_x0 ? (unsigned)((int64_t)R * nr * NB * (int64_t)sizeof(TX)) : 0u;
      if (lane == 0) {
        const unsigned vb = (unsigned)(nr * row_stride * (int64_t)sizeof(TV));
        mbar_arrive_expect_tx(&full[s], K * vb + (unsigned)(R * nr * xblk) + x0b);
        const uint64_t pol = (blockIdx.x + i * (int64_t)gridDim.x) >= keep_from ? pol_last : pol_first;
        for (int k = 0; k < K; ++k)
          bulk_copy_g2s_hint(st + k * op_tile_bytes, reinterpret_cast<const TV*>(cb.vals[k]) + R0 * row_stride, vb,
                             &full[s], pol);
        for (int rhs = 0; rhs < R && stage_x0; ++rhs)
          bulk_copy_g2s(st + vals_bytes + (int64_t)R * rows_per_tile * xblk +
                            (int64_t)rhs * rows_per_tile * NB * (int64_t)sizeof(TX),
                        x0 + ((int64_t)rhs * nrows + R0) * NB, (unsigned)(nr * NB * sizeof(TX)), &full[s]);
      }
      if (lane < nr)
        for (int rhs = 0; rhs < R; ++rhs)
          bulk_copy_g2s(st + vals_bytes + ((int64_t)rhs * rows_per_tile + lane) * xblk,
                        x + ((int64_t)rhs * nrows + 4 * (int64_t)(src >> 2)) * NB, (unsigned)xblk, &full[s]);
      issued = i + 1;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    // drain: every issued stage must have landed before the block's shared memory goes away
    if (lane == 0)
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j)
        mbar_wait_bounded(&full[j % stages], (unsigned)((j / stages) & 1));
    return;
  }
  // ---------------- consumers ----------------
  // FP64 vectors on a 32- or 16-bit operator: compensated FP32 sums
  constexpr bool kSplit = std::is_same<TX, double>::value && !std::is_same<TV, double>::value;
  const int ctid = threadIdx.x - 32;
  const int nthreads = 32 * kConsumerWarps;
  for (int64_t i = 0; i < mine; ++i) {
    const int s = (int)(i % stages);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((i / stages) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const unsigned char* st = stage0 + s * stage_bytes;
    if constexpr (kSplit) {
      // each staged coefficient (a double) becomes its (hi, lo) float pair in
      // place, once per tile, before any consumer reads it
      double* xd = reinterpret_cast<double*>(stage0 + s * stage_bytes + vals_bytes);
      const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
      const int64_t left = nrows - (reverse ? ntiles - 1 - tile : tile) * rows_per_tile;
      const int nr = left < rows_per_tile ? (int)left : rows_per_tile;
      const int per = 4 * NB;
      for (int e = ctid; e < R * rows_per_tile * per; e += nthreads) {
        if ((e / per) % rows_per_tile >= nr) continue;  // rows past the mesh end are not staged
        const double v = xd[e];
        const float hi = (float)v;
        reinterpret_cast<float2*>(xd)[e] = make_float2(hi, (float)(v - (double)hi));
      }
      asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
    }
    const TV* tv = reinterpret_cast<const TV*>(st);
    const TX* tx = reinterpret_cast<const TX*>(st + vals_bytes);
    const TX* tx0 = reinterpret_cast<const TX*>(st + vals_bytes + (int64_t)R * rows_per_tile * xblk);
    const int32_t* rs = s_recv + s * rows_per_tile;
    const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
    const int64_t R0 = (reverse ? ntiles - 1 - tile : tile) * rows_per_tile;
    const int64_t left = nrows - R0;
    const int nr = left < rows_per_tile ? (int)left : rows_per_tile;
    for (int e = ctid; e < nr * NB; e += nthreads) {
      const int r = e / NB;
      const int a = e - r * NB;
      const int lp = rs[r] & 3;
      const TV* blk0 = tv + (int64_t)r * row_stride + a * NB;
      if constexpr (kSplit) {
        if (KC == 1) {  // four right-hand sides per pass of the block row
          const int64_t xstride = (int64_t)rows_per_tile * 4 * NB;  // float2 pairs between right-hand sides
          for (int q0 = 0; q0 < R; q0 += 4) {
            double tot[4];
            const float2* xs = reinterpret_cast<const float2*>(tx + ((int64_t)q0 * rows_per_tile + r) * 4 * NB);
            if (R - q0 >= 4)
              row_times_x_split_q<NB, TV, 4>(blk0, xs, xstride, lp, tot);
            else if (R - q0 == 3)
              row_times_x_split_q<NB, TV, 3>(blk0, xs, xstride, lp, tot);
            else if (R - q0 == 2)
              row_times_x_split_q<NB, TV, 2>(blk0, xs, xstride, lp, tot);
            else
              row_times_x_split_q<NB, TV, 1>(blk0, xs, xstride, lp, tot);
            for (int q = 0; q < 4 && q0 + q < R; ++q) {
              const int rhs = q0 + q;
              const int64_t o = ((int64_t)rhs * nrows + R0 + r) * NB + a;
              const TA base =
                  stage_x0 ? (TA)tx0[((int64_t)rhs * rows_per_tile + r) * NB + a] : (x0 ? (TA)x0[o] : TA(0));
              y[o] = (TX)(base + alpha * (TA)tot[q]);
            }
          }
          continue;
        }
      }
      for (int rhs = 0; rhs < R; ++rhs) {
        const TX* xs = tx + ((int64_t)rhs * rows_per_tile + r) * 4 * NB;
        TA total;
        if constexpr (kSplit) {
          if (KC == 1) {
            total = (TA)row_times_x_split<NB, TV>(blk0, reinterpret_cast<const float2*>(xs), lp);
          } else {
            total = TA(0);
            for (int kk = 0; kk < K; ++kk)
              total = fma((TA)cb.coef[rhs][kk],
                          (TA)row_times_x_split<NB, TV>(blk0 + kk * (op_tile_bytes / (int64_t)sizeof(TV)),
                                                        reinterpret_cast<const float2*>(xs), lp),
                          total);
          }
        } else if (KC == 1) {
          total = row_times_x<NB, TV, TX, TA>(blk0, xs, lp);
        } else {
          total = TA(0);
          for (int kk = 0; kk < K; ++kk)
            total = fma((TA)cb.coef[rhs][kk],
                        row_times_x<NB, TV, TX, TA>(blk0 + kk * (op_tile_bytes / (int64_t)sizeof(TV)), xs, lp), total);
        }
        const int64_t o = ((int64_t)rhs * nrows + R0 + r) * NB + a;
        const TA base = stage_x0 ? (TA)tx0[((int64_t)rhs * rows_per_tile + r) * NB + a] : (x0 ? (TA)x0[o] : TA(0));
        y[o] = (TX)(base + alpha * total);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}


// Transposed application y = x0 + alpha B^T x with the same pipeline.  A tile
// is a run of consecutive source tets; the blocks leaving tet t are the rows
// recv[4t + l'] (l' = 0..3, one full row each, all three slots come from t), so
// every operator row is copied exactly once over the whole grid.  Producer lane
// r of a tile copies row r by TMA and stages x of that row (NB values, loaded
// one tile ahead into registers).  Consumers form, for column J = 4t + l,
//   (B^T x)_J[b] = sum_{l' != l} sum_a B_{recv[4t+l'], slot(l,l')}[a][b] x_{recv[4t+l']}[a],
// slot(l, l') = l - (l > l').  One right-hand side per launch.
template <int NB, typename TV, typename TX, typename TA>
__global__ void __launch_bounds__(32 * (kConsumerWarps + 1))
spmv_t_tma_kernel(const TV* __restrict__ vals, int64_t row_stride, const int32_t* __restrict__ recv, int64_t nt,
                  int tets_per_tile, int stages, const TX* __restrict__ x, const TX* x0, TX* y, TA alpha,
                  int reverse, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + kStages;
  const int rpt = 4 * tets_per_tile;  // rows per tile (<= 32)
  constexpr int NB2 = NB * NB;
  const int64_t row_bytes = row_stride * (int64_t)sizeof(TV);
  const int64_t xs_bytes = ((int64_t)rpt * NB * sizeof(TA) + 15) / 16 * 16;
  const int64_t stage_bytes = rpt * row_bytes + xs_bytes;
  unsigned char* stage0 = smem_raw + 128;
  const int64_t ntiles = (nt + tets_per_tile - 1) / tets_per_tile;
  const int64_t mine = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto tile_tets = [&](int64_t i, int64_t* T0, int* ntt) {
    const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
    *T0 = (reverse ? ntiles - 1 - tile : tile) * tets_per_tile;
    const int64_t left = nt - *T0;
    *ntt = left < tets_per_tile ? (int)left : tets_per_tile;
  };
  if (warp == 0) {
    // ---------------- producer ----------------
    int64_t issued = 0;
    bool ok = true;
    int32_t next_row = 0;
    TA next_x[NB];
    auto fetch = [&](int64_t i, int32_t* row, TA* xv) {
      int64_t T0;
      int ntt;
      tile_tets(i, &T0, &ntt);
      if (lane < 4 * ntt) {
        *row = recv[4 * T0 + lane];
        const TX* xr = x + (int64_t)(*row) * NB;
#pragma unroll
        for (int a = 0; a < NB; ++a) xv[a] = (TA)__ldg(xr + a);
      }
    };
    if (mine > 0) fetch(0, &next_row, next_x);
    for (int64_t i = 0; i < mine && ok; ++i) {
      const int s = (int)(i % stages);
      int64_t T0;
      int ntt;
      tile_tets(i, &T0, &ntt);
      const int32_t row = next_row;
      TA xv[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a) xv[a] = next_x[a];
      if (i + 1 < mine) fetch(i + 1, &next_row, next_x);
      if (i >= stages) ok = mbar_wait_bounded(&empty[s], (unsigned)(((i / stages) - 1) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      unsigned char* st = stage0 + s * stage_bytes;
      TA* xs = reinterpret_cast<TA*>(st + rpt * row_bytes);
      const int nr = 4 * ntt;
      if (lane < nr) {
#pragma unroll
        for (int a = 0; a < NB; ++a) xs[lane * NB + a] = xv[a];
      }
      __syncwarp();  // staged x is written before lane 0's arrive publishes the stage
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) mbar_arrive_expect_tx(&full[s], (unsigned)(nr * row_bytes));
      if (lane < nr) bulk_copy_g2s(st + lane * row_bytes, vals + (int64_t)row * row_stride, (unsigned)row_bytes, &full[s]);
      issued = i + 1;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    if (lane == 0)
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j)
        mbar_wait_bounded(&full[j % stages], (unsigned)((j / stages) & 1));
    return;
  }
  // ---------------- consumers ----------------
  const int ctid = threadIdx.x - 32;
  const int nthreads = 32 * kConsumerWarps;
  for (int64_t i = 0; i < mine; ++i) {
    const int s = (int)(i % stages);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (unsigned)((i / stages) & 1)));
    if (!ok) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const unsigned char* st = stage0 + s * stage_bytes;
    const TV* tv = reinterpret_cast<const TV*>(st);
    const TA* xs = reinterpret_cast<const TA*>(st + rpt * row_bytes);
    int64_t T0;
    int ntt;
    tile_tets(i, &T0, &ntt);
    for (int e = ctid; e < ntt * 4 * NB; e += nthreads) {
      const int lt = e / (4 * NB);
      const int rem = e - lt * 4 * NB;
      const int l = rem / NB;
      const int b = rem - l * NB;
      TA acc = TA(0);
#pragma unroll
      for (int lp = 0; lp < 4; ++lp) {
        if (lp == l) continue;
        const int slot = l - (l > lp ? 1 : 0);
        const TV* blk = tv + (int64_t)(lt * 4 + lp) * row_stride + slot * NB2 + b;
        const TA* xr = xs + (lt * 4 + lp) * NB;
#pragma unroll
        for (int a = 0; a < NB; ++a) acc = fma((TA)blk[a * NB], xr[a], acc);
      }
      const int64_t o = (4 * (T0 + lt) + l) * NB + b;
      const TA base = x0 ? (TA)x0[o] : TA(0);
      y[o] = (TX)(base + alpha * acc);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// Consecutive applications of one operator sweep its rows in alternating
// directions: a sweep that starts where the previous one ended finds that
// sweep's last rows still in L2.  The parity is kept per values buffer (the
// FP32 blocks and their 16-bit copy are separate streams of bytes).  Results
// do not depend on the direction: every output row is formed by one warp in a
// fixed order either way.
std::mutex g_sweep_mu;
std::unordered_map<const void*, unsigned> g_sweep;

}  // namespace

int next_sweep_direction(const void* vals) {
  std::lock_guard<std::mutex> lk(g_sweep_mu);
  unsigned& p = g_sweep[vals];
  const int dir = (int)(p & 1u);
  ++p;
  return dir;
}

void forget_sweep(const void* vals) {
  if (!vals) return;
  std::lock_guard<std::mutex> lk(g_sweep_mu);
  g_sweep.erase(vals);
}

namespace {

// Operator bytes per application kept in L2 for the next one (of the 129 MB
// L2; the rest holds the vectors and the row map).
constexpr int64_t kL2KeepBytes = 64ll << 20;

template <typename TV, typename TX, typename TA>
int launch(const dfm_op* op, const TX* x, const TX* x0, TX* y, int R, double alpha, int trans, cudaStream_t st,
           const dfm_op* const* combo_ops = nullptr, int K = 1, const double* coef = nullptr) {
  const TV* vals = reinterpret_cast<const TV*>(op->vals);
  const int32_t* recv = op->recv ? op->recv : op->mesh->recv;
  int dev = 0, nsm = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!trans) {
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(op->vals) & 15))
      return set_error(DFM_ERR_ARG, "dfm_apply: x must be 16-byte aligned");
    // bases above N_p = 8 and linear-spatial-basis sizes: a block row per warp,
    // no staged row tiles (wide.cu)
    if (!narrow_nb(op->nb)) {
      if constexpr (std::is_same<TV, float>::value && std::is_same<TX, TA>::value) {
        if (K != 1 || combo_ops)
          return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply_combo: combined operators need a basis of the per-warp kernels");
        return apply_wide(op, x, x0, y, R, alpha, st);
      }
      return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: bases above Np = 8 need FP32 blocks");
    }
    // BF16 blocks with several FP32 right-hand sides: a dense contraction per
    // row, on tensor cores (spmv_mma.cu)
    if constexpr (std::is_same<TV, __nv_bfloat16>::value && std::is_same<TX, float>::value)
      if (K == 1 && !combo_ops && apply_mma_supported(op, R)) return apply_mma(op, x, x0, y, R, alpha, st);
    if (R > kMaxStagedRhs) {  // several passes, each staging up to kMaxStagedRhs right-hand sides
      const int64_t stride = op->nrows * (int64_t)op->nb;
      for (int r0 = 0; r0 < R; r0 += kMaxStagedRhs) {
        const int rc = launch<TV, TX, TA>(op, x + r0 * stride, x0 ? x0 + r0 * stride : nullptr, y + r0 * stride,
                                          std::min(kMaxStagedRhs, R - r0), alpha, 0, st, combo_ops, K,
                                          coef ? coef + (int64_t)r0 * K : nullptr);
        if (rc) return rc;
      }
      return DFM_OK;
    }
    const geom::Fwd g = geom::fwd_geometry(op->nb, (int)sizeof(TV), (int)sizeof(TX), K, R, op->nrows,
                                           x0 && !(reinterpret_cast<uintptr_t>(x0) & 15), kStages);
    const int rpt = g.rpt, stage_x0 = g.stage_x0, stages = g.stages;
    const int64_t row_bytes = g.row_bytes;
    Combo cb{};
    cb.K = K;
    for (int k = 0; k < K; ++k) cb.vals[k] = combo_ops ? combo_ops[k]->vals : op->vals;
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < K; ++k) cb.coef[r][k] = coef ? coef[(int64_t)r * K + k] : 1.0;
    if (stages < 1) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: an operator row does not fit shared memory");
    const size_t smem = 128 + ((stages * rpt * 4 + 127) / 128) * 128 + (size_t)stages * (rpt * row_bytes + 16);
    int rc = DFM_OK;
    auto go = [&](auto kernel) -> int {
      DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * (kConsumerWarps + 1), smem));
      if (per_sm < 1) per_sm = 1;
      const int64_t ntiles = (op->nrows + rpt - 1) / rpt;
      const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
      {
        ::dfm::KernelTimer timer_(sizeof(TX) == 8 ? DFM_KERNEL_SPMV64 : DFM_KERNEL_SPMV, st);
        const int64_t op_tile = (int64_t)K * rpt * op->row_stride * (int64_t)sizeof(TV);
        const int64_t keep_from = std::max<int64_t>(0, ntiles - kL2KeepBytes / op_tile);
        kernel<<<(unsigned)grid, 32 * (kConsumerWarps + 1), smem, st>>>(cb, op->row_stride, recv, op->nrows, rpt,
                                                                         stages, x, x0, y, R, (TA)alpha, stage_x0,
                                                                         next_sweep_direction(op->vals), keep_from,
                                                                         op->dev_err);
      }
      DFM_LAUNCHED();
      return DFM_OK;
    };
    auto by_nb = [&](auto kc) -> int {
      constexpr int KC = decltype(kc)::value;
      switch (op->nb) {
        case 1: return go(spmv_tma_kernel<1, KC, TV, TX, TA>);
        case 3: return go(spmv_tma_kernel<3, KC, TV, TX, TA>);
        case 6: return go(spmv_tma_kernel<6, KC, TV, TX, TA>);
        case 10: return go(spmv_tma_kernel<10, KC, TV, TX, TA>);
        case 15: return go(spmv_tma_kernel<15, KC, TV, TX, TA>);
        case 21: return go(spmv_tma_kernel<21, KC, TV, TX, TA>);
        case 28: return go(spmv_tma_kernel<28, KC, TV, TX, TA>);
        case 36: return go(spmv_tma_kernel<36, KC, TV, TX, TA>);
        case 45: return go(spmv_tma_kernel<45, KC, TV, TX, TA>);
        default: return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: unsupported basis size");
      }
    };
    if (K == 1)
      rc = by_nb(std::integral_constant<int, 1>{});
    else if constexpr (std::is_same<TV, float>::value)  // combinations are of FP32 operators only
      rc = by_nb(std::integral_constant<int, 0>{});
    else
      return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply_combo: operators must be FP32");
    if (rc) return rc;
  } else if (combo_ops == nullptr && !(reinterpret_cast<uintptr_t>(op->vals) & 15) && narrow_nb(op->nb) &&
             (200 * 1024 - 512) / (8 * op->row_stride * (int64_t)sizeof(TV) +
                                   ((int64_t)8 * op->nb * (int64_t)sizeof(TA) + 15) / 16 * 16) >= 2) {
    // (two stages of two tets' rows fit; larger rows take the gather below)
    // pipelined transposed application, one right-hand side per launch
    const int64_t nt = op->nrows / 4;
    const int64_t row_bytes = op->row_stride * (int64_t)sizeof(TV);
    int tpt = 2;  // tets per tile (8 rows)
    const int64_t xs_bytes = ((int64_t)4 * tpt * op->nb * (int64_t)sizeof(TA) + 15) / 16 * 16;
    const int64_t budget = 200 * 1024 - 512;
    const int64_t stage_bytes = 4 * tpt * row_bytes + xs_bytes;
    const int stages = (int)std::min<int64_t>(kStages, budget / stage_bytes);
    if (stages < 2) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: operator rows too large for the transposed pipeline");
    const size_t smem = 128 + (size_t)stages * stage_bytes;
    const int64_t stride = op->nrows * (int64_t)op->nb;
    auto go = [&](auto kernel) -> int {
      DFM_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * (kConsumerWarps + 1), smem));
      if (per_sm < 1) per_sm = 1;
      const int64_t ntiles = (nt + tpt - 1) / tpt;
      const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
      for (int r = 0; r < R; ++r) {
        {
          ::dfm::KernelTimer timer_(sizeof(TX) == 8 ? DFM_KERNEL_SPMV64_T : DFM_KERNEL_SPMV_T, st);
          kernel<<<(unsigned)grid, 32 * (kConsumerWarps + 1), smem, st>>>(
              vals, op->row_stride, recv, nt, tpt, stages, x + r * stride, x0 ? x0 + r * stride : nullptr,
              y + r * stride, (TA)alpha, next_sweep_direction(op->vals), op->dev_err);
        }
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
      }
      return DFM_OK;
    };
    int rc = DFM_OK;
    switch (op->nb) {
      case 1: rc = go(spmv_t_tma_kernel<1, TV, TX, TA>); break;
      case 3: rc = go(spmv_t_tma_kernel<3, TV, TX, TA>); break;
      case 6: rc = go(spmv_t_tma_kernel<6, TV, TX, TA>); break;
      case 10: rc = go(spmv_t_tma_kernel<10, TV, TX, TA>); break;
      case 15: rc = go(spmv_t_tma_kernel<15, TV, TX, TA>); break;
      case 21: rc = go(spmv_t_tma_kernel<21, TV, TX, TA>); break;
      case 28: rc = go(spmv_t_tma_kernel<28, TV, TX, TA>); break;
      case 36: rc = go(spmv_t_tma_kernel<36, TV, TX, TA>); break;
      case 45: rc = go(spmv_t_tma_kernel<45, TV, TX, TA>); break;
      default: return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: unsupported basis size");
    }
    if (rc) return rc;
  } else {
    const int64_t total = op->nrows * op->nb * (int64_t)R;
    const int64_t grid = std::min<int64_t>((total + kThreads - 1) / kThreads, (int64_t)nsm * 16);
    {
      ::dfm::KernelTimer timer_(sizeof(TX) == 8 ? DFM_KERNEL_SPMV64_T : DFM_KERNEL_SPMV_T, st);
      spmv_t_kernel<TV, TX, TA><<<(unsigned)grid, kThreads, 0, st>>>(vals, op->row_stride, recv, op->nrows, op->nb,
                                                                     x, x0, y, R, (TA)alpha);
    }
    DFM_LAUNCHED();
  }
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

}  // namespace

int apply_one(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
              cudaStream_t st);

// y = x0 + alpha (B x), B with its reflected part (heterogeneous media) if any:
// the first part with x0, then the reflected part accumulated onto y
int apply_impl(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
               cudaStream_t st) {
  int rc = apply_one(op, x, x0, y, R, alpha, trans, xtype, st);
  if (rc || !op->rop) return rc;
  return apply_one(op->rop, x, y, y, R, alpha, trans, xtype, st);
}

int apply_one(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
              cudaStream_t st) {
  if (!op || !x || !y || R < 1) return set_error(DFM_ERR_ARG, "dfm_apply: NULL operator/vector or R < 1");
  if (x == y) return set_error(DFM_ERR_ARG, "dfm_apply: y must not alias x");
  if (xtype == DFM_F64) {
    if (op->precision == DFM_F64)
      return launch<double, double, double>(op, (const double*)x, (const double*)x0, (double*)y, R, alpha, trans, st);
    if (op->precision == DFM_F32)
      return launch<float, double, double>(op, (const double*)x, (const double*)x0, (double*)y, R, alpha, trans, st);
    if (op->precision == DFM_BF16)
      return launch<__nv_bfloat16, double, double>(op, (const double*)x, (const double*)x0, (double*)y, R, alpha,
                                                   trans, st);
  } else if (xtype == DFM_F32) {
    if (op->precision == DFM_F32)
      return launch<float, float, float>(op, (const float*)x, (const float*)x0, (float*)y, R, alpha, trans, st);
    if (op->precision == DFM_F64)
      return launch<double, float, double>(op, (const float*)x, (const float*)x0, (float*)y, R, alpha, trans, st);
    if (op->precision == DFM_BF16)
      return launch<__nv_bfloat16, float, float>(op, (const float*)x, (const float*)x0, (float*)y, R, alpha, trans,
                                                 st);
  }
  return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: unsupported operator/vector precision");
}

int apply_combo_impl(const dfm_op* const* ops, int K, const double* coef, const void* x, const void* x0, void* y,
                     int R, double alpha, int xtype, cudaStream_t st) {
  if (!ops || K < 1 || K > kMaxCombo || !coef || !x || !y || R < 1)
    return set_error(DFM_ERR_ARG, "dfm_apply_combo: bad argument (1 <= K <= 4)");
  if (x == y) return set_error(DFM_ERR_ARG, "dfm_apply_combo: y must not alias x");
  for (int k = 0; k < K; ++k) {
    if (!ops[k] || ops[k]->mesh != ops[0]->mesh || ops[k]->Np != ops[0]->Np || ops[k]->precision != DFM_F32)
      return set_error(DFM_ERR_ARG, "dfm_apply_combo: operators must be FP32 and share mesh and Np");
    if (ops[k]->rop)
      return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply_combo: operators with a reflected part are not combined");
  }
  if (xtype == DFM_F64)
    return launch<float, double, double>(ops[0], (const double*)x, (const double*)x0, (double*)y, R, alpha, 0, st, ops,
                                         K, coef);
  if (xtype == DFM_F32)
    return launch<float, float, float>(ops[0], (const float*)x, (const float*)x0, (float*)y, R, alpha, 0, st, ops, K,
                                       coef);
  return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply_combo: unsupported vector precision");
}

}  // namespace dfm

extern "C" int dfm_apply_combo(const dfm_op* const* ops, int K, const double* coef_host, const void* x, const void* x0,
                               void* y, int R, double alpha, int xtype, void* stream) {
  return dfm::apply_combo_impl(ops, K, coef_host, x, x0, y, R, alpha, xtype, dfm::as_stream(stream));
}

extern "C" int dfm_apply(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans,
                         int xtype, void* stream) {
  return dfm::apply_impl(op, x, x0, y, R, alpha, trans, xtype, dfm::as_stream(stream));
}

namespace dfm {
namespace {
// One barrier that expects a single arrival nobody makes: the bounded wait of
// the pipelines runs out after `polls` polls and takes the same exit as a
// stalled copy (flag the operator, end the kernel).  No copy is in flight.
__global__ void wait_timeout_selftest_kernel(long long polls, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    pipe::mbar_init(&bar, 1);
    pipe::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (long long i = 0; i < polls && !done; ++i) done = pipe::mbar_try_wait(&bar, 0);
    if (!done) atomicExch(err, 1);
  }
}
}  // namespace

int read_timeout_flag(const dfm_op* op, cudaStream_t st, const char* who) {
  if (!op->dev_err) return DFM_OK;
  int e = 0;
  DFM_CUDA_CHECK(cudaMemcpyAsync(&e, op->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(st));
  if (!e) return DFM_OK;
  DFM_CUDA_CHECK(cudaMemsetAsync(op->dev_err, 0, sizeof(int), st));
  return set_error(DFM_ERR_TIMEOUT, std::string(who) + ": a kernel timed out waiting for its data");
}
}  // namespace dfm

extern "C" int dfm_op_check_error(const dfm_op* op, void* stream) {
  if (!op) return dfm::set_error(DFM_ERR_ARG, "dfm_op_check_error: NULL operator");
  return dfm::read_timeout_flag(op, dfm::as_stream(stream), "dfm_op_check_error");
}

extern "C" int dfm_selftest_timeout(const dfm_op* op, int polls, void* stream) {
  if (!op || !op->dev_err || polls < 1 || polls > 1000000)
    return dfm::set_error(DFM_ERR_ARG, "dfm_selftest_timeout: bad argument (1 <= polls <= 1000000)");
  dfm::wait_timeout_selftest_kernel<<<1, 32, 0, dfm::as_stream(stream)>>>((long long)polls, op->dev_err);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}
