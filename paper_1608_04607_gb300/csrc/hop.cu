// Polynomial-preconditioner hops on a 16-bit copy of the blocks.
//
// The flexible inner solver evaluates z = p(B~) v = sum_{k<d} B~^k v by
// Horner's rule, z <- v + B~ z, with B~ the FP16 (or BF16) rounding of the
// FP32 blocks.  A hop reads half the operator bytes of an FP32 application;
// the result only preconditions (the Arnoldi relation uses the FP32 operator),
// so the rounding costs accuracy of the preconditioner, not of the solution.
//
// Layouts, chosen so that a consumer thread reads 16-byte vectors only:
//  - the 16-bit copy: per operator row, per block k (3), per column chunk c
//    (NBP / 8 chunks, NBP = NB rounded up to 8), per test index a (NB): the 8
//    trial values b = 8c .. 8c+7 of B_k[a][.] (zero for b >= NB).  The
//    threads forming outputs a = 0..NB-1 of a row read consecutive 16-byte
//    chunks (no shared-memory bank conflicts).
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
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

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

template <typename T16>
__device__ __forceinline__ float2 widen2(uint32_t w) {
  if constexpr (std::is_same<T16, __half>::value) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
  } else {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    return __bfloat1622float2(h);
  }
}

// y = x0 + alpha B~ x for R right-hand sides; x, x0 padded (NBP per face
// row), y padded (OUTP) or unpadded (NB per face row).
template <int NB, typename T16, bool OUTP>
__global__ void __launch_bounds__(32 * (kHopConsumerWarps + 1))
hop_kernel(const T16* __restrict__ vals, const int32_t* __restrict__ recv, int64_t nrows, const float* __restrict__ xp,
           const float* __restrict__ x0p, float* __restrict__ y, int R, float alpha, int stages, int reverse,
           int64_t keep_from, int* __restrict__ err) {
  constexpr int NBP = (NB + 7) / 8 * 8;
  constexpr int NC = NBP / 8;
  constexpr int RPT = (32 * kHopConsumerWarps) / NBP;  // rows per tile
  constexpr int64_t ROW_ELEMS = 3 * NB * NBP;
  constexpr unsigned ROW_BYTES = (unsigned)(ROW_ELEMS * 2);
  constexpr unsigned XBLK = 4 * NBP * 4;
  constexpr unsigned X0ROW = NBP * 4;
  static_assert(RPT >= 1 && RPT <= 32, "rows per tile");
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
        bulk_copy_g2s_hint(st, vals + R0 * ROW_ELEMS, (unsigned)nr * ROW_BYTES, &full[s], pol);
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
      const T16* brow = reinterpret_cast<const T16*>(st) + r * ROW_ELEMS;
      for (int rhs = 0; rhs < R; ++rhs) {
        const float* xs = reinterpret_cast<const float*>(st + (int64_t)RPT * ROW_BYTES + ((int64_t)rhs * RPT + r) * XBLK);
        const float* x0s =
            reinterpret_cast<const float*>(st + (int64_t)RPT * ROW_BYTES + (int64_t)R * RPT * XBLK + (int64_t)rhs * RPT * X0ROW);
        float out = 0.f;
        if (a < NB) {
          float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                           make_float2(0.f, 0.f)};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int l = k + (k >= lp ? 1 : 0);
            const float* xl = xs + l * NBP;
            const T16* bk = brow + k * NB * NBP;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const uint4 bv = *reinterpret_cast<const uint4*>(bk + (c * NB + a) * 8);
              const float4 xa = *reinterpret_cast<const float4*>(xl + c * 8);
              const float4 xb = *reinterpret_cast<const float4*>(xl + c * 8 + 4);
              acc[0] = __ffma2_rn(widen2<T16>(bv.x), make_float2(xa.x, xa.y), acc[0]);
              acc[1] = __ffma2_rn(widen2<T16>(bv.y), make_float2(xa.z, xa.w), acc[1]);
              acc[2] = __ffma2_rn(widen2<T16>(bv.z), make_float2(xb.x, xb.y), acc[2]);
              acc[3] = __ffma2_rn(widen2<T16>(bv.w), make_float2(xb.z, xb.w), acc[3]);
            }
          }
          const float sum = ((acc[0].x + acc[0].y) + (acc[1].x + acc[1].y)) + ((acc[2].x + acc[2].y) + (acc[3].x + acc[3].y));
          out = x0s[r * NBP + a] + alpha * sum;
        }
        const int64_t row = (int64_t)rhs * nrows + R0 + r;
        if (OUTP)
          y[row * NBP + a] = out;  // pads (a >= NB) written as 0
        else if (a < NB)
          y[row * NB + a] = out;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <typename T16>
__global__ void to_hop_layout_kernel(const float* __restrict__ src, int64_t row_stride, T16* __restrict__ dst,
                                     int64_t nrows, int nb, int nbp) {
  const int64_t row_elems = 3 * (int64_t)nb * nbp;
  const int64_t total = nrows * row_elems;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / row_elems;
    int64_t rem = i - row * row_elems;
    const int k = (int)(rem / ((int64_t)nb * nbp));
    rem -= (int64_t)k * nb * nbp;
    const int c = (int)(rem / (nb * 8));
    rem -= (int64_t)c * nb * 8;
    const int a = (int)(rem / 8);
    const int b = c * 8 + (int)(rem - a * 8);
    const float v = b < nb ? src[row * row_stride + (int64_t)k * nb * nb + (int64_t)a * nb + b] : 0.f;
    if constexpr (std::is_same<T16, __half>::value)
      dst[i] = __float2half_rn(v);
    else
      dst[i] = __float2bfloat16_rn(v);
  }
}

__global__ void hop_pack_kernel(const float* __restrict__ v, float* __restrict__ vp, int64_t rows, int nb, int nbp) {
  const int64_t total = rows * nbp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / nbp;
    const int a = (int)(i - row * nbp);
    vp[i] = a < nb ? v[row * nb + a] : 0.f;
  }
}

int grid_for_elems(int64_t n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)std::max(nsm, 1) * 8));
}

template <typename T16, bool OUTP>
int launch_hop(const dfm_op* op, const float* xp, const float* x0p, float* y, int R, cudaStream_t st) {
  const int nb = op->nb;
  const int nbp = hop_nbp(nb);
  const int rpt = (32 * kHopConsumerWarps) / nbp;
  const int64_t row_bytes = 3 * (int64_t)nb * nbp * 2;
  const int64_t stage_bytes = rpt * row_bytes + (int64_t)R * rpt * (4 * nbp * 4 + nbp * 4);
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
          reinterpret_cast<const T16*>(op->lp_vals), op->mesh->recv, op->nrows, xp, x0p, y, R, 1.0f, stages,
          next_sweep_direction(op->lp_vals), keep_from, op->dev_err);
    }
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    return DFM_OK;
  };
  switch (nb) {
    case 1: return go(hop_kernel<1, T16, OUTP>);
    case 3: return go(hop_kernel<3, T16, OUTP>);
    case 6: return go(hop_kernel<6, T16, OUTP>);
    case 10: return go(hop_kernel<10, T16, OUTP>);
    case 15: return go(hop_kernel<15, T16, OUTP>);
    case 21: return go(hop_kernel<21, T16, OUTP>);
    case 28: return go(hop_kernel<28, T16, OUTP>);
    case 36: return go(hop_kernel<36, T16, OUTP>);
    case 45: return go(hop_kernel<45, T16, OUTP>);
    default: return set_error(DFM_ERR_UNSUPPORTED, "preconditioner hop: unsupported basis size");
  }
}

}  // namespace

int prepare_lowp(const dfm_op* cop, int precision, cudaStream_t st) {
  dfm_op* op = const_cast<dfm_op*>(cop);
  if (op->precision != DFM_F32 || (precision != DFM_F16 && precision != DFM_BF16))
    return set_error(DFM_ERR_UNSUPPORTED, "preconditioner copy: needs an FP32 operator and DFM_F16 or DFM_BF16");
  const int nbp = hop_nbp(op->nb);
  const int64_t elems = op->nrows * 3 * (int64_t)op->nb * nbp;
  if (!op->lp_vals) {
    DFM_CUDA_CHECK(cudaMalloc(&op->lp_vals, elems * 2));
  }
  if (!op->lp_valid || op->lp_precision != precision) {
    const int grid = grid_for_elems(elems);
    if (precision == DFM_F16)
      to_hop_layout_kernel<__half><<<grid, 256, 0, st>>>((const float*)op->vals, op->row_stride,
                                                         (__half*)op->lp_vals, op->nrows, op->nb, nbp);
    else
      to_hop_layout_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const float*)op->vals, op->row_stride,
                                                                (__nv_bfloat16*)op->lp_vals, op->nrows, op->nb, nbp);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    op->lp_precision = precision;
    op->lp_valid = true;
  }
  return DFM_OK;
}

int hop_pack(const float* v, float* vp, int64_t rows, int nb, cudaStream_t st) {
  hop_pack_kernel<<<grid_for_elems(rows * hop_nbp(nb)), 256, 0, st>>>(v, vp, rows, nb, hop_nbp(nb));
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

int hop_apply(const dfm_op* op, const float* xp, const float* x0p, float* y, int R, int out_padded, cudaStream_t st) {
  if (!op || !op->lp_valid || !xp || !x0p || !y || R < 1)
    return set_error(DFM_ERR_ARG, "preconditioner hop: no 16-bit copy or NULL vector");
  if ((reinterpret_cast<uintptr_t>(xp) | reinterpret_cast<uintptr_t>(x0p) | reinterpret_cast<uintptr_t>(op->lp_vals)) &
      15)
    return set_error(DFM_ERR_ARG, "preconditioner hop: vectors and copy must be 16-byte aligned");
  const int64_t stride_p = op->nrows * (int64_t)hop_nbp(op->nb);
  const int64_t stride_y = out_padded ? stride_p : op->nrows * (int64_t)op->nb;
  for (int r0 = 0; r0 < R; r0 += kHopMaxRhs) {
    const int Rp = std::min(kHopMaxRhs, R - r0);
    int rc;
    const float* x = xp + r0 * stride_p;
    const float* x0 = x0p + r0 * stride_p;
    float* yy = y + r0 * stride_y;
    if (op->lp_precision == DFM_F16)
      rc = out_padded ? launch_hop<__half, true>(op, x, x0, yy, Rp, st) : launch_hop<__half, false>(op, x, x0, yy, Rp, st);
    else
      rc = out_padded ? launch_hop<__nv_bfloat16, true>(op, x, x0, yy, Rp, st)
                      : launch_hop<__nv_bfloat16, false>(op, x, x0, yy, Rp, st);
    if (rc) return rc;
  }
  return DFM_OK;
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
  if (degree == 1) {
    DFM_CUDA_CHECK(cudaMemcpyAsync(z, x, sizeof(float) * rows * op->nb, cudaMemcpyDeviceToDevice, st));
    return DFM_OK;
  }
  const int64_t elems = rows * hop_nbp(op->nb);
  float* scratch = nullptr;
  DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&scratch), 3 * elems * sizeof(float), st));
  float* vp = scratch;
  float* h[2] = {scratch + elems, scratch + 2 * elems};
  rc = hop_pack(x, vp, rows, op->nb, st);
  const float* src = vp;
  for (int k = 1; k < degree && rc == DFM_OK; ++k) {
    const bool last = (k == degree - 1);
    float* dst = last ? z : h[k & 1];
    rc = hop_apply(op, src, vp, dst, R, last ? 0 : 1, st);
    src = dst;
  }
  const cudaError_t e = cudaFreeAsync(scratch, st);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_error(e, "dfm_precond_apply: cudaFreeAsync");
  return DFM_OK;
}
