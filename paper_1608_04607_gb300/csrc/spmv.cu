// Block-sparse application of the transfer operator: y = x0 + alpha B x and
// y = x0 + alpha B^T x (Sec. 2: B couples a face only to the faces of one tet,
// so every block row and every block column holds exactly three blocks).
//
// Forward: row R receives three blocks, all from tet t = recv[R]/4, whose
// source faces are the three faces of t other than l' = recv[R]%4.  A thread
// block stages a tile of consecutive rows of the operator (contiguous in
// memory, 16-byte aligned rows) and the coefficients of each row's source tet
// in shared memory with vector loads, then one thread per (row, test index)
// forms its dot products; the staged tile is reused for every right-hand side.
//
// Transpose: column J = 4t + l owns the blocks (t, l) -> l' received by rows
// recv[4t + l'] in slot l - (l > l'); one thread per (column, trial index)
// walks the three blocks with coalesced reads along the trial index.
#include <algorithm>

#include "dfm_internal.cuh"

namespace dfm {
namespace {

constexpr int kThreads = 128;

template <typename TV, typename TX, typename TA>
__global__ void __launch_bounds__(kThreads)
spmv_kernel(const TV* __restrict__ vals, int64_t row_stride, const int32_t* __restrict__ recv, int64_t nrows, int nb,
            int rows_per_tile, const TX* __restrict__ x, const TX* x0, TX* y, int R,
            TA alpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TV* s_vals = reinterpret_cast<TV*>(smem_raw);
  TA* s_x = reinterpret_cast<TA*>(smem_raw + sizeof(TV) * rows_per_tile * row_stride);
  const int64_t ntiles = (nrows + rows_per_tile - 1) / rows_per_tile;
  const int nb2 = nb * nb;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t R0 = tile * rows_per_tile;
    const int64_t left = nrows - R0;
    const int nr = left < rows_per_tile ? (int)left : rows_per_tile;
    // stage the tile's operator rows (contiguous, 16-byte vectors)
    const int4* src = reinterpret_cast<const int4*>(vals + R0 * row_stride);
    int4* dst = reinterpret_cast<int4*>(s_vals);
    const int64_t nvec = (int64_t)nr * row_stride * sizeof(TV) / 16;
    for (int64_t i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
    for (int rhs = 0; rhs < R; ++rhs) {
      const TX* xr = x + (int64_t)rhs * nrows * nb;
      // stage the four rows of each tile row's source tet
      for (int i = threadIdx.x; i < nr * 4 * nb; i += blockDim.x) {
        const int r = i / (4 * nb);
        const int j = i - r * 4 * nb;
        const int64_t t = recv[R0 + r] >> 2;
        s_x[i] = (TA)xr[4 * t * nb + j];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nr * nb; i += blockDim.x) {
        const int r = i / nb;
        const int a = i - r * nb;
        const int lp = recv[R0 + r] & 3;
        const TV* blk = s_vals + (int64_t)r * row_stride + a * nb;
        const TA* xs = s_x + r * 4 * nb;
        TA acc = TA(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int l = k + (k >= lp ? 1 : 0);
          const TV* bk = blk + k * nb2;
          const TA* xl = xs + l * nb;
          for (int b = 0; b < nb; ++b) acc = fma((TA)bk[b], xl[b], acc);
        }
        const int64_t o = ((int64_t)rhs * nrows + R0 + r) * nb + a;
        const TA base = x0 ? (TA)x0[o] : TA(0);
        y[o] = (TX)(base + alpha * acc);
      }
      __syncthreads();
    }
  }
}

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

int rows_per_tile_for(int nb) {
  int r = kThreads / nb;
  if (r < 1) r = 1;
  return r;
}

template <typename TV, typename TX, typename TA>
int launch(const dfm_op* op, const TX* x, const TX* x0, TX* y, int R, double alpha, int trans, cudaStream_t st) {
  const TV* vals = reinterpret_cast<const TV*>(op->vals);
  const int32_t* recv = op->mesh->recv;
  int dev = 0, nsm = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!trans) {
    const int rpt = rows_per_tile_for(op->nb);
    const size_t smem = sizeof(TV) * rpt * op->row_stride + sizeof(TA) * rpt * 4 * op->nb;
    if (smem > 200 * 1024) return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: tile does not fit shared memory");
    DFM_CUDA_CHECK(cudaFuncSetAttribute(spmv_kernel<TV, TX, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    int per_sm = 0;
    DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv_kernel<TV, TX, TA>, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = (op->nrows + rpt - 1) / rpt;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    {
      ::dfm::KernelTimer timer_(sizeof(TX) == 8 ? DFM_KERNEL_SPMV64 : DFM_KERNEL_SPMV, st);
      spmv_kernel<TV, TX, TA><<<(unsigned)grid, kThreads, smem, st>>>(vals, op->row_stride, recv, op->nrows, op->nb,
                                                                      rpt, x, x0, y, R, (TA)alpha);
    }
    DFM_LAUNCHED();
  } else {
    const int64_t total = op->nrows * op->nb * (int64_t)R;
    const int64_t grid = std::min<int64_t>((total + kThreads - 1) / kThreads, (int64_t)nsm * 16);
    {
      ::dfm::KernelTimer timer_(DFM_KERNEL_SPMV_T, st);
      spmv_t_kernel<TV, TX, TA><<<(unsigned)grid, kThreads, 0, st>>>(vals, op->row_stride, recv, op->nrows, op->nb,
                                                                     x, x0, y, R, (TA)alpha);
    }
    DFM_LAUNCHED();
  }
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

}  // namespace

int apply_impl(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
               cudaStream_t st) {
  if (!op || !x || !y || R < 1) return set_error(DFM_ERR_ARG, "dfm_apply: NULL operator/vector or R < 1");
  if (x == y) return set_error(DFM_ERR_ARG, "dfm_apply: y must not alias x");
  if (xtype == DFM_F64) {
    if (op->precision == DFM_F64)
      return launch<double, double, double>(op, (const double*)x, (const double*)x0, (double*)y, R, alpha, trans, st);
    if (op->precision == DFM_F32)
      return launch<float, double, double>(op, (const double*)x, (const double*)x0, (double*)y, R, alpha, trans, st);
  } else if (xtype == DFM_F32) {
    if (op->precision == DFM_F32)
      return launch<float, float, float>(op, (const float*)x, (const float*)x0, (float*)y, R, alpha, trans, st);
    if (op->precision == DFM_F64)
      return launch<double, float, double>(op, (const float*)x, (const float*)x0, (float*)y, R, alpha, trans, st);
  }
  return set_error(DFM_ERR_UNSUPPORTED, "dfm_apply: unsupported operator/vector precision");
}

}  // namespace dfm

extern "C" int dfm_apply(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans,
                         int xtype, void* stream) {
  return dfm::apply_impl(op, x, x0, y, R, alpha, trans, xtype, dfm::as_stream(stream));
}
