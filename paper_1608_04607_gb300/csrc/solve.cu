// Stationary solve (I - B) rho = rho0 (Sec. 2, Eqs. NSum and GovIE).
//
//  - Neumann: the series rho = sum_n B^n rho0 summed as x <- rho0 + B x, FP64,
//    stopped on the relative increment.
//  - GMRES: restarted GMRES(m) in the operator's precision; Arnoldi by
//    classical Gram-Schmidt with one conditional re-orthogonalisation pass,
//    Givens rotations on the host.
//  - GMRES_IR: iterative refinement; the residual r = rho0 - (I - B) x is
//    formed in FP64 (FP32 blocks widened exactly, FP64 accumulation) and each
//    correction solves (I - B) d = r / |r| by FP32 GMRES to a loose tolerance.
//    Since the FP64 residual, not the FP32 inner solve, decides convergence,
//    the final accuracy is that of the FP64 residual.
//
// Vector kernels use fixed grids and a deterministic two-stage reduction.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "dfm_internal.cuh"

namespace dfm {
namespace {

constexpr int kRedBlocks = 512;  // partial-sum blocks of the reductions
constexpr int kRedThreads = 256;
constexpr int kDotChunk = 8;     // dot products per pass over the vector
constexpr int kMaxKrylov = 256;  // largest GMRES restart length

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : T(0);
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}

// partial[b][j] = sum over block b's slice of V[j][i] * w[i], j < k (V rows of length n, stride ld)
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
multi_dot_kernel(const T* __restrict__ V, int64_t ld, int k, const T* __restrict__ w, int64_t n, T* __restrict__ partial) {
  __shared__ T sh[32];
  for (int j0 = 0; j0 < k; j0 += kDotChunk) {
    T acc[kDotChunk];
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) acc[c] = T(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const T wi = w[i];
#pragma unroll
      for (int c = 0; c < kDotChunk; ++c)
        if (j0 + c < k) acc[c] = fma(V[(int64_t)(j0 + c) * ld + i], wi, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) {
      if (j0 + c >= k) break;
      const T s = block_sum(acc[c], sh);
      if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + j0 + c] = s;
    }
  }
}

// out[j] = sum_b partial[b][j]
template <typename T>
__global__ void reduce_partials_kernel(const T* __restrict__ partial, int nblk, int k, T* __restrict__ out) {
  __shared__ T sh[32];
  for (int j = blockIdx.x; j < k; j += gridDim.x) {
    T s = T(0);
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(int64_t)b * k + j];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[j] = s;
  }
}

// w[i] += sum_j coef_sign * h[j] * V[j][i]; partial[b] = sum of squares of the new w over block b
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
multi_axpy_kernel(const T* __restrict__ V, int64_t ld, int k, const T* __restrict__ h, T coef_sign, T* w, int64_t n,
                  T* __restrict__ partial) {
  __shared__ T sh[32];
  __shared__ T hs[kMaxKrylov + 8];
  for (int j = threadIdx.x; j < k && j < kMaxKrylov + 8; j += blockDim.x) hs[j] = coef_sign * h[j];
  __syncthreads();
  T sq = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // four independent chains keep several loads in flight per thread
    T v0 = w[i], v1 = T(0), v2 = T(0), v3 = T(0);
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      v0 = fma(hs[j], V[(int64_t)j * ld + i], v0);
      v1 = fma(hs[j + 1], V[(int64_t)(j + 1) * ld + i], v1);
      v2 = fma(hs[j + 2], V[(int64_t)(j + 2) * ld + i], v2);
      v3 = fma(hs[j + 3], V[(int64_t)(j + 3) * ld + i], v3);
    }
    for (; j < k; ++j) v0 = fma(hs[j], V[(int64_t)j * ld + i], v0);
    const T v = (v0 + v1) + (v2 + v3);
    w[i] = v;
    sq = fma(v, v, sq);
  }
  if (partial) {
    const T s = block_sum(sq, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

template <typename T>
__global__ void scale_kernel(T* __restrict__ y, const T* __restrict__ x, T s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

// y = a * x + b * z
template <typename T>
__global__ void axpby_kernel(T* __restrict__ y, T a, const T* __restrict__ x, T b, const T* __restrict__ z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * z[i];
}

// y = a - b (all FP64)
__global__ void sub_kernel(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] - b[i];
}

// partial[b] = (sum (a-b)^2, sum a^2)
__global__ void __launch_bounds__(kRedThreads)
diff_norm_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double d2 = 0.0, a2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = a[i] - b[i];
    d2 = fma(d, d, d2);
    a2 = fma(a[i], a[i], a2);
  }
  const double s1 = block_sum(d2, sh);
  if (threadIdx.x == 0) partial[2 * blockIdx.x] = s1;
  const double s2 = block_sum(a2, sh);
  if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = s2;
}

// rf = (float)(r * s)
__global__ void to_f32_kernel(float* __restrict__ y, const double* __restrict__ x, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)(x[i] * s);
}

// x += s * (double)d
__global__ void add_f32_kernel(double* __restrict__ x, const float* __restrict__ d, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)d[i], x[i]);
}


// ---------------------------------------------------------------------------
// Batched kernels: R right-hand sides in lockstep (blockIdx.y = right-hand
// side).  Vector r of Krylov step j lives at V + j * ldj + r * ldr.
// ---------------------------------------------------------------------------
constexpr int kBRedBlocks = 128;  // partial-sum blocks per right-hand side

// partial[(r * gridDim.x + b) * k + j] = slice of V[j]_r . w_r
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
bdot_kernel(const T* __restrict__ V, int64_t ldj, int64_t ldr, int k, const T* __restrict__ w, int64_t wldr, int64_t n,
            T* __restrict__ partial) {
  __shared__ T sh[32];
  const int r = blockIdx.y;
  const T* wr = w + r * wldr;
  for (int j0 = 0; j0 < k; j0 += kDotChunk) {
    T acc[kDotChunk];
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) acc[c] = T(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const T wi = wr[i];
#pragma unroll
      for (int c = 0; c < kDotChunk; ++c)
        if (j0 + c < k) acc[c] = fma(V[(int64_t)(j0 + c) * ldj + r * ldr + i], wi, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kDotChunk; ++c) {
      if (j0 + c >= k) break;
      const T sum = block_sum(acc[c], sh);
      if (threadIdx.x == 0) partial[((int64_t)r * gridDim.x + blockIdx.x) * k + j0 + c] = sum;
    }
  }
}

// out[r * ldo + j] = sum_b partial[(r * nblk + b) * k + j]; grid (k, R)
template <typename T>
__global__ void breduce_kernel(const T* __restrict__ partial, int nblk, int k, int64_t ldo, T* __restrict__ out) {
  __shared__ T sh[32];
  const int j = blockIdx.x, r = blockIdx.y;
  T sum = T(0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) sum += partial[((int64_t)r * nblk + b) * k + j];
  sum = block_sum(sum, sh);
  if (threadIdx.x == 0) out[r * ldo + j] = sum;
}

// w_r += sign * sum_j h[r * hld + j] V[j]_r;  partial[r * gridDim.x + b] = slice of |w_r|^2
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
baxpy_kernel(const T* __restrict__ V, int64_t ldj, int64_t ldr, int k, const T* __restrict__ h, int hld, T sign, T* w,
             int64_t wldr, int64_t n, T* __restrict__ partial) {
  __shared__ T sh[32];
  __shared__ T hs[kMaxKrylov + 8];
  const int r = blockIdx.y;
  for (int j = threadIdx.x; j < k && j < kMaxKrylov + 8; j += blockDim.x) hs[j] = sign * h[(int64_t)r * hld + j];
  __syncthreads();
  T* wr = w + r * wldr;
  const T* Vr = V + r * ldr;
  T sq = T(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T v0 = wr[i], v1 = T(0), v2 = T(0), v3 = T(0);
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      v0 = fma(hs[j], Vr[(int64_t)j * ldj + i], v0);
      v1 = fma(hs[j + 1], Vr[(int64_t)(j + 1) * ldj + i], v1);
      v2 = fma(hs[j + 2], Vr[(int64_t)(j + 2) * ldj + i], v2);
      v3 = fma(hs[j + 3], Vr[(int64_t)(j + 3) * ldj + i], v3);
    }
    for (; j < k; ++j) v0 = fma(hs[j], Vr[(int64_t)j * ldj + i], v0);
    const T v = (v0 + v1) + (v2 + v3);
    wr[i] = v;
    sq = fma(v, v, sq);
  }
  if (partial) {
    const T sum = block_sum(sq, sh);
    if (threadIdx.x == 0) partial[(int64_t)r * gridDim.x + blockIdx.x] = sum;
  }
}

// w_r *= s[r]
template <typename T>
__global__ void bscale_kernel(T* w, int64_t wldr, const T* __restrict__ s, int64_t n) {
  const int r = blockIdx.y;
  const T f = s[r];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[r * wldr + i] *= f;
}

// y_r = (float)(x_r * s[r])  (FP64 residual -> FP32 right-hand side)
__global__ void bto_f32_kernel(float* __restrict__ y, const double* __restrict__ x, const double* __restrict__ s,
                               int64_t n) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[r * n + i] = (float)(x[r * n + i] * s[r]);
}

// x_r += s[r] * (double)d_r
__global__ void badd_f32_kernel(double* __restrict__ x, const float* __restrict__ d, const double* __restrict__ s,
                                int64_t n) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[r * n + i] = fma(s[r], (double)d[r * n + i], x[r * n + i]);
}

__global__ void source_kernel(const FaceGeom* __restrict__ geom, const int64_t* __restrict__ rows, int n_src,
                              int64_t nrows, int nb, double* __restrict__ rho0) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int64_t r = rows[s];
  rho0[((int64_t)s * nrows + r) * nb] = sqrt(geom[r].area);
}

// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------

struct Ctx {
  const dfm_op* op;
  cudaStream_t st;
  int nsm;
  int64_t n;      // rows * nb
  int trans = 0;  // 1: the operator is applied transposed (adjoint solves)
  // per-right-hand-side operators sum_k coef[r][k] B_k (K > 1), coef already
  // offset to the first right-hand side of the current group
  const dfm_op* const* combo = nullptr;
  int K = 1;
  const double* coef = nullptr;
};

// y = x0 + alpha * A x for the R right-hand sides of the current group
inline int ctx_apply(const Ctx& c, const void* x, const void* x0, void* y, int R, double alpha, int xtype) {
  if (c.combo) return apply_combo_impl(c.combo, c.K, c.coef, x, x0, y, R, alpha, xtype, c.st);
  return apply_impl(c.op, x, x0, y, R, alpha, c.trans, xtype, c.st);
}

inline unsigned grid_for(int64_t n, int nsm) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)nsm * 8));
}

template <typename T>
int dots(const Ctx& c, const T* V, int64_t ld, int k, const T* w, T* partial, T* out_dev, T* out_host) {
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_DOT, c.st);
    multi_dot_kernel<T><<<kRedBlocks, kRedThreads, 0, c.st>>>(V, ld, k, w, c.n, partial);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  reduce_partials_kernel<T><<<std::min(k, 64), kRedThreads, 0, c.st>>>(partial, kRedBlocks, k, out_dev);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  DFM_CUDA_CHECK(cudaMemcpyAsync(out_host, out_dev, sizeof(T) * k, cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  return DFM_OK;
}

// w += sign * V h; returns |w|^2 in *sq_host (synchronises)
template <typename T>
int axpy_norm(const Ctx& c, const T* V, int64_t ld, int k, const T* h_dev, T sign, T* w, T* partial, T* red_dev,
              double* sq_host) {
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
    multi_axpy_kernel<T><<<kRedBlocks, kRedThreads, 0, c.st>>>(V, ld, k, h_dev, sign, w, c.n, partial);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  reduce_partials_kernel<T><<<1, kRedThreads, 0, c.st>>>(partial, kRedBlocks, 1, red_dev);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  T s;
  DFM_CUDA_CHECK(cudaMemcpyAsync(&s, red_dev, sizeof(T), cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  *sq_host = (double)s;
  return DFM_OK;
}

template <typename T>
int norm2(const Ctx& c, const T* v, T* partial, T* red_dev, double* out) {
  T s;
  int rc = dots<T>(c, v, 0, 1, v, partial, red_dev, &s);
  *out = sqrt((double)s);
  return rc;
}

// workspace carving
struct Work {
  char* base;
  int64_t off = 0;
  template <typename T>
  T* take(int64_t count) {
    off = (off + 255) & ~int64_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * (int64_t)sizeof(T);
    return p;
  }
};

int ensure_work(const dfm_op* cop, int64_t bytes) {
  dfm_op* op = const_cast<dfm_op*>(cop);
  if (op->swork_bytes >= bytes) return DFM_OK;
  cudaFree(op->swork);
  op->swork = nullptr;
  op->swork_bytes = 0;
  DFM_CUDA_CHECK(cudaMalloc(&op->swork, bytes));
  op->swork_bytes = bytes;
  return DFM_OK;
}

// GMRES(m) on (I - B) x = b in precision T (operator applied as TV with TX = T),
// right-preconditioned by the Neumann polynomial p(B) = sum_{k<d} B^k:
//   (I - B) p(B) = I - B^d,  so the Arnoldi process runs on I - B^d and the
//   update is x += p(B) (V y), p(B) z evaluated by Horner (s <- z + B s).
// The polynomial shrinks the Krylov dimension about d-fold for a modest
// increase in operator applications, which keeps the quadratic Gram-Schmidt
// cost small.  x holds the initial guess; tol is relative to |b|; operator
// applications are added to *iters, capped by max_iter.  *est returns the
// last relative residual estimate.  t1, t2: scratch vectors of length n.
// Flexible variant: the preconditioner's hops run on the operator's 16-bit
// copy (hop_apply) through zero-padded FP32 vectors vp (the packed v_j), ha,
// hb ([R][rows][NBP] each); the result z_j = p~(B) v_j lands in Z.
struct Hop {
  const dfm_op* op = nullptr;
  float* vp = nullptr;
  float* ha = nullptr;
  float* hb = nullptr;
};

// z = sum_{k<d} B~^k v for R unit-norm vectors v ([R][n]) by Horner on the
// low-precision copy; unit norm keeps |v| <= 1, so the FP16 hop vectors hold
// v 2^-8.
inline int precond_hops(const Ctx& c, const Hop& hp, int R, int d, const float* v, float* z) {
  return ::dfm::hop_horner(hp.op, R, d, v, z, hp.vp, hp.ha, hp.hb, 1.0f / 256.0f, c.st, c.trans);
}

#include "block_gmres.cuh"

// Two-level correction of the flexible preconditioner (dfm_solve_opts.coarse;
// not in the paper, the solver acceleration its slow modes call for): the
// slowest mode of I - B at small loss is the isotropic density, so a coarse
// space V of the (0,0) slot weighted by sqrt|T| on g^3 spatial aggregates of
// tets (by centroid, boxes of the bounding box) is solved exactly and the
// polynomial handles the rest:
//   z = Q v + p~(B) (v - A Q v),  Q = V E^{-1} V^T,  E = V^T A V,  A = I - B.
// A V is formed once per solve (nc operator applications), so each
// preconditioner call costs nc-long dot and update passes, not an extra
// application: A Q v = (A V) E^{-1} V^T v.
struct Coarse {
  int nc = 0;
  float* V = nullptr;   // [nc][n]
  float* AV = nullptr;  // [nc][n]
  float* r = nullptr;   // [n] v - A Q v
  float* y = nullptr;   // [nc] E^{-1} V^T v (device)
  int32_t* agg = nullptr;  // [n_tets] aggregate of each tet
  std::vector<double> Einv;  // nc x nc
};

// V[agg(t)][R nb] = sqrt|T_R| for row R = 4t + f (the (0,0) slot)
__global__ void coarse_basis_kernel(const FaceGeom* __restrict__ geom, const int32_t* __restrict__ agg, int64_t nrows,
                                    int nb, int64_t n, float* __restrict__ V) {
  for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < nrows; R += (int64_t)gridDim.x * blockDim.x)
    V[(int64_t)agg[R >> 2] * n + R * nb] = (float)sqrt(geom[R].area);
}

// Builds V, A V and E^{-1} for g aggregates per axis; counts the nc
// applications in *iters.  Empty aggregates are dropped; a singular E (or
// g = 0) leaves nc = 0 (no correction).
inline int coarse_setup(const Ctx& c, const dfm_mesh* mesh, int g, Coarse& cs, float* partial, float* h_dev,
                        int* iters) {
  cs.nc = 0;
  if (g < 1) return DFM_OK;
  std::vector<double> verts((size_t)mesh->nv * 3);
  std::vector<int32_t> tets((size_t)mesh->nt * 4);
  DFM_CUDA_CHECK(cudaMemcpyAsync(verts.data(), mesh->verts, sizeof(double) * verts.size(), cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaMemcpyAsync(tets.data(), mesh->tets, sizeof(int32_t) * tets.size(), cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < mesh->nv; ++v)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], verts[3 * v + k]);
      hi[k] = std::max(hi[k], verts[3 * v + k]);
    }
  std::vector<int32_t> box((size_t)mesh->nt);
  std::vector<int> count((size_t)g * g * g, 0);
  for (int64_t t = 0; t < mesh->nt; ++t) {
    int idx[3];
    for (int k = 0; k < 3; ++k) {
      double cen = 0;
      for (int j = 0; j < 4; ++j) cen += 0.25 * verts[3 * (int64_t)tets[4 * t + j] + k];
      const double ext = hi[k] - lo[k];
      int i = ext > 0 ? (int)std::floor(g * (cen - lo[k]) / ext) : 0;
      idx[k] = std::max(0, std::min(g - 1, i));
    }
    box[t] = idx[0] + g * (idx[1] + g * idx[2]);
    ++count[box[t]];
  }
  std::vector<int> remap(count.size(), -1);
  int nc = 0;
  for (size_t b = 0; b < count.size(); ++b)
    if (count[b] > 0) remap[b] = nc++;
  for (auto& b : box) b = remap[b];
  DFM_CUDA_CHECK(cudaMemcpyAsync(cs.agg, box.data(), sizeof(int32_t) * box.size(), cudaMemcpyHostToDevice, c.st));
  const int64_t n = c.n;
  DFM_CUDA_CHECK(cudaMemsetAsync(cs.V, 0, sizeof(float) * nc * n, c.st));
  coarse_basis_kernel<<<grid_for(mesh->nrows, c.nsm), 256, 0, c.st>>>(mesh->geom, cs.agg, mesh->nrows, c.op->nb, n,
                                                                        cs.V);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  for (int k = 0; k < nc; ++k) {
    const int rc = ctx_apply(c, cs.V + (int64_t)k * n, cs.V + (int64_t)k * n, cs.AV + (int64_t)k * n, 1, -1.0,
                             DFM_F32);
    if (rc) return rc;
    ++*iters;
  }
  // E[i][k] = V_i . (A V)_k, inverted by Gauss-Jordan with partial pivoting
  std::vector<double> E((size_t)nc * nc), col(nc);
  std::vector<float> colf(nc);
  for (int k = 0; k < nc; ++k) {
    const int rc = dots<float>(c, cs.V, n, nc, cs.AV + (int64_t)k * n, partial, h_dev, colf.data());
    if (rc) return rc;
    for (int i = 0; i < nc; ++i) E[(size_t)i * nc + k] = colf[i];
  }
  std::vector<double> inv((size_t)nc * nc, 0.0);
  for (int i = 0; i < nc; ++i) inv[(size_t)i * nc + i] = 1.0;
  double emax = 0;
  for (double e : E) emax = std::max(emax, std::fabs(e));
  for (int k = 0; k < nc; ++k) {
    int p = k;
    for (int i = k + 1; i < nc; ++i)
      if (std::fabs(E[(size_t)i * nc + k]) > std::fabs(E[(size_t)p * nc + k])) p = i;
    if (!(std::fabs(E[(size_t)p * nc + k]) > 1e-12 * emax)) return DFM_OK;  // singular: no correction
    for (int j = 0; j < nc; ++j) {
      std::swap(E[(size_t)k * nc + j], E[(size_t)p * nc + j]);
      std::swap(inv[(size_t)k * nc + j], inv[(size_t)p * nc + j]);
    }
    const double piv = E[(size_t)k * nc + k];
    for (int j = 0; j < nc; ++j) {
      E[(size_t)k * nc + j] /= piv;
      inv[(size_t)k * nc + j] /= piv;
    }
    for (int i = 0; i < nc; ++i) {
      if (i == k) continue;
      const double f = E[(size_t)i * nc + k];
      if (f == 0.0) continue;
      for (int j = 0; j < nc; ++j) {
        E[(size_t)i * nc + j] -= f * E[(size_t)k * nc + j];
        inv[(size_t)i * nc + j] -= f * inv[(size_t)k * nc + j];
      }
    }
  }
  cs.Einv = inv;
  cs.nc = nc;
  return DFM_OK;
}

// z = Q v + p~(B) (v - A Q v) (see Coarse)
inline int coarse_hops(const Ctx& c, const Coarse& cs, const Hop& hp, int d, const float* v, float* z, float* partial,
                       float* h_dev) {
  const int nc = cs.nc;
  std::vector<float> cv(nc), y(nc);
  int rc = dots<float>(c, cs.V, c.n, nc, v, partial, h_dev, cv.data());
  if (rc) return rc;
  for (int i = 0; i < nc; ++i) {
    double s = 0;
    for (int j = 0; j < nc; ++j) s += cs.Einv[(size_t)i * nc + j] * cv[j];
    y[i] = (float)s;
  }
  DFM_CUDA_CHECK(cudaMemcpyAsync(cs.y, y.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, c.st));
  DFM_CUDA_CHECK(cudaMemcpyAsync(cs.r, v, sizeof(float) * c.n, cudaMemcpyDeviceToDevice, c.st));
  multi_axpy_kernel<float><<<kRedBlocks, kRedThreads, 0, c.st>>>(cs.AV, c.n, nc, cs.y, -1.f, cs.r, c.n, nullptr);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  rc = precond_hops(c, hp, 1, d, cs.r, z);
  if (rc) return rc;
  multi_axpy_kernel<float><<<kRedBlocks, kRedThreads, 0, c.st>>>(cs.V, c.n, nc, cs.y, 1.f, z, c.n, nullptr);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

template <typename T>
int gmres(const Ctx& c, const T* b, T* x, double tol, int m, int d, int max_iter, int* iters, double* est, T* V,
          T* tmp, T* t1, T* t2, T* h_dev, T* partial, T* red_dev, const Hop* lp = nullptr, T* Z = nullptr,
          const Coarse* coarse = nullptr) {
  const int64_t n = c.n;
  const int xtype = sizeof(T) == 8 ? DFM_F64 : DFM_F32;
  if (d < 1) d = 1;
  std::vector<T> hh(m + 2);
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  double bnorm;
  int rc = norm2<T>(c, b, partial, red_dev, &bnorm);
  if (rc) return rc;
  if (!(bnorm == bnorm) || isinf(bnorm)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite right-hand side");
  if (bnorm == 0.0) {
    DFM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(T) * n, c.st));
    *est = 0.0;
    return DFM_OK;
  }
  double prev_beta = -1.0;
  // w = v - B^d v  (d operator applications, ping-pong through t1/t2)
  auto apply_poly_op = [&](const T* v, T* w) -> int {
    const T* src = v;
    for (int k = 1; k < d; ++k) {
      T* dst = (k & 1) ? t1 : t2;
      int r = ctx_apply(c, src, nullptr, dst, 1, 1.0, xtype);
      if (r) return r;
      src = dst;
    }
    *iters += d;
    return ctx_apply(c, src, v, w, 1, -1.0, xtype);
  };
  while (true) {
    // r = b - (I - B) x = (b - x) + B x   -> V[0]
    axpby_kernel<T><<<grid_for(n, c.nsm), 256, 0, c.st>>>(tmp, T(1), b, T(-1), x, n);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    rc = ctx_apply(c, x, tmp, V, 1, 1.0, xtype);
    if (rc) return rc;
    ++*iters;
    double beta;
    rc = norm2<T>(c, V, partial, red_dev, &beta);
    if (rc) return rc;
    if (!(beta == beta) || isinf(beta)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite residual");
    *est = beta / bnorm;
    if (beta <= tol * bnorm) return DFM_OK;
    if (*iters >= max_iter) return DFM_ERR_NOT_CONVERGED;
    // a restart cycle that gained less than 10% means the working precision is
    // exhausted: stop and let the caller's FP64 refinement take over
    if (prev_beta > 0 && beta > 0.9 * prev_beta) return DFM_ERR_NOT_CONVERGED;
    prev_beta = beta;
    scale_kernel<T><<<grid_for(n, c.nsm), 256, 0, c.st>>>(V, V, T(1.0 / beta), n);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kdone = 0;
    for (int j = 0; j < m; ++j) {
      T* vj = V + (int64_t)j * n;
      T* w = V + (int64_t)(j + 1) * n;
      if (lp) {
        // flexible step: z_j = p~(B) v_j by Horner on the 16-bit copy, w = z_j - B z_j
        T* zj = Z + (int64_t)j * n;
        if constexpr (std::is_same<T, float>::value) {
          rc = (coarse && coarse->nc > 0) ? coarse_hops(c, *coarse, *lp, d, vj, zj, partial, h_dev)
                                          : precond_hops(c, *lp, 1, d, vj, zj);
        } else {
          rc = set_error(DFM_ERR_UNSUPPORTED, "dfm_solve: 16-bit preconditioner hops need FP32 Krylov vectors");
        }
        if (rc) return rc;
        *iters += d;
        rc = ctx_apply(c, zj, zj, w, 1, -1.0, xtype);
      } else {
        rc = apply_poly_op(vj, w);
      }
      if (rc) return rc;
      // classical Gram-Schmidt: h = V^T w (plus |w|^2 as the last entry)
      rc = dots<T>(c, V, n, j + 2, w, partial, h_dev, hh.data());
      if (rc) return rc;
      const double wnorm_before = sqrt(std::max(0.0, (double)hh[j + 1]));
      double sq;
      rc = axpy_norm<T>(c, V, n, j + 1, h_dev, T(-1), w, partial, red_dev, &sq);
      if (rc) return rc;
      for (int i = 0; i <= j; ++i) H[i * m + j] = (double)hh[i];
      if (sqrt(sq) < 0.5 * wnorm_before) {  // re-orthogonalise once
        rc = dots<T>(c, V, n, j + 1, w, partial, h_dev, hh.data());
        if (rc) return rc;
        rc = axpy_norm<T>(c, V, n, j + 1, h_dev, T(-1), w, partial, red_dev, &sq);
        if (rc) return rc;
        for (int i = 0; i <= j; ++i) H[i * m + j] += (double)hh[i];
      }
      double hn = sqrt(sq);
      if (!(hn == hn)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite Krylov vector");
      H[(j + 1) * m + j] = hn;
      if (hn > 0) {
        scale_kernel<T><<<grid_for(n, c.nsm), 256, 0, c.st>>>(w, w, T(1.0 / hn), n);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
      }
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = den > 0 ? H[j * m + j] / den : 1.0;
      sn[j] = den > 0 ? H[(j + 1) * m + j] / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      kdone = j + 1;
      *est = fabs(g[j + 1]) / bnorm;
      if (fabs(g[j + 1]) <= 0.5 * tol * bnorm || *iters + d >= max_iter || hn == 0.0) break;
    }
    // y = H^{-1} g (upper triangular); z = V y; x += p(B) z
    for (int i = kdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < kdone; ++k) s -= H[i * m + k] * y[k];
      y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
    }
    for (int i = 0; i < kdone; ++i) hh[i] = (T)y[i];
    DFM_CUDA_CHECK(cudaMemcpyAsync(h_dev, hh.data(), sizeof(T) * kdone, cudaMemcpyHostToDevice, c.st));
    if (lp) {  // flexible update: x += Z y
      {
        ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
        multi_axpy_kernel<T><<<kRedBlocks, kRedThreads, 0, c.st>>>(Z, n, kdone, h_dev, T(1), x, n, nullptr);
      }
      DFM_LAUNCHED();
      DFM_CUDA_CHECK(cudaGetLastError());
      continue;
    }
    DFM_CUDA_CHECK(cudaMemsetAsync(tmp, 0, sizeof(T) * n, c.st));
    {
      ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
      multi_axpy_kernel<T><<<kRedBlocks, kRedThreads, 0, c.st>>>(V, n, kdone, h_dev, T(1), tmp, n, nullptr);
    }
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    const T* s_src = tmp;
    for (int k = 1; k < d; ++k) {  // Horner: s <- z + B s
      T* dst = (k & 1) ? t1 : t2;
      rc = ctx_apply(c, s_src, tmp, dst, 1, 1.0, xtype);
      if (rc) return rc;
      s_src = dst;
    }
    *iters += d - 1;
    axpby_kernel<T><<<grid_for(n, c.nsm), 256, 0, c.st>>>(x, T(1), x, T(1), s_src, n);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
  }
}

// FP64 relative residual |rho0 - (I - B) x| / |rho0| with FP64 vectors
int residual64(const Ctx& c, const double* rho0, const double* x, double* r, double* partial, double* red_dev,
               double* out, double* rnorm_abs) {
  sub_kernel<<<grid_for(c.n, c.nsm), 256, 0, c.st>>>(r, rho0, x, c.n);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  // r = (rho0 - x) + B x, written to a second half of r
  double* r2 = r + c.n;
  int rc = ctx_apply(c, x, r, r2, 1, 1.0, DFM_F64);
  if (rc) return rc;
  double rn, bn;
  rc = norm2<double>(c, r2, partial, red_dev, &rn);
  if (rc) return rc;
  rc = norm2<double>(c, rho0, partial, red_dev, &bn);
  if (rc) return rc;
  *rnorm_abs = rn;
  *out = bn > 0 ? rn / bn : rn;
  return DFM_OK;
}


// ---------------------------------------------------------------------------
// Batched host helpers
// ---------------------------------------------------------------------------

// host[r * k + j] = V[j]_r . w_r  (synchronises)
template <typename T>
int bdots(const Ctx& c, int R, const T* V, int64_t ldj, int64_t ldr, int k, const T* w, int64_t wldr, T* partial,
          T* out_dev, T* out_host) {
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_DOT, c.st);
    bdot_kernel<T><<<dim3(kBRedBlocks, R), kRedThreads, 0, c.st>>>(V, ldj, ldr, k, w, wldr, c.n, partial);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  breduce_kernel<T><<<dim3(k, R), 128, 0, c.st>>>(partial, kBRedBlocks, k, k, out_dev);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  DFM_CUDA_CHECK(cudaMemcpyAsync(out_host, out_dev, sizeof(T) * k * R, cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  return DFM_OK;
}

// w_r += sign * V h_r (h_dev [R][hld]); sq_host[r] = |w_r|^2  (synchronises when sq_host)
template <typename T>
int baxpy(const Ctx& c, int R, const T* V, int64_t ldj, int64_t ldr, int k, const T* h_dev, int hld, T sign, T* w,
          int64_t wldr, T* partial, T* red_dev, std::vector<double>* sq_host) {
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
    baxpy_kernel<T><<<dim3(kBRedBlocks, R), kRedThreads, 0, c.st>>>(V, ldj, ldr, k, h_dev, hld, sign, w, wldr, c.n,
                                                                     sq_host ? partial : nullptr);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  if (!sq_host) return DFM_OK;
  breduce_kernel<T><<<dim3(1, R), 128, 0, c.st>>>(partial, kBRedBlocks, 1, 1, red_dev);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  std::vector<T> tmp(R);
  DFM_CUDA_CHECK(cudaMemcpyAsync(tmp.data(), red_dev, sizeof(T) * R, cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  sq_host->resize(R);
  for (int r = 0; r < R; ++r) (*sq_host)[r] = (double)tmp[r];
  return DFM_OK;
}

template <typename T>
int bscale(const Ctx& c, int R, T* w, int64_t wldr, const std::vector<double>& f, T* s_dev) {
  std::vector<T> fh(R);
  for (int r = 0; r < R; ++r) fh[r] = (T)f[r];
  DFM_CUDA_CHECK(cudaMemcpyAsync(s_dev, fh.data(), sizeof(T) * R, cudaMemcpyHostToDevice, c.st));
  bscale_kernel<T><<<dim3(grid_for(c.n, c.nsm), R), 256, 0, c.st>>>(w, wldr, s_dev, c.n);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

// GMRES(m) for R right-hand sides in lockstep, right-preconditioned by
// p(B) = sum_{k<d} B^k (see gmres()); every operator application is one
// launch over all R vectors, so the operator is read once per hop for all of
// them.  Each right-hand side keeps its own Hessenberg matrix and stops
// contributing once its residual estimate meets tol (relative to |b_r|).
// b, x: [R][n]; V: [(m+1)][R][n]; tmp, t1, t2: [R][n].
template <typename T>
int gmres_batched(const Ctx& c, int R, const T* b, T* x, double tol, int m, int d, int max_iter, int* iters,
                  std::vector<double>* est, T* V, T* tmp, T* t1, T* t2, T* h_dev, T* partial, T* red_dev,
                  const Hop* lp = nullptr, T* Z = nullptr) {
  const int64_t n = c.n;
  const int64_t Rn = (int64_t)R * n;
  const int xtype = sizeof(T) == 8 ? DFM_F64 : DFM_F32;
  const int hld = m + 2;
  std::vector<T> hh((size_t)R * hld);
  std::vector<std::vector<double>> H(R, std::vector<double>((m + 1) * m)), cs(R, std::vector<double>(m)),
      sn(R, std::vector<double>(m)), g(R, std::vector<double>(m + 1));
  std::vector<double> bnorm(R), beta(R), sq, f(R);
  std::vector<int> kdone(R), active(R);
  est->assign(R, 0.0);
  int rc = bdots<T>(c, R, b, 0, n, 1, b, n, partial, h_dev, hh.data());
  if (rc) return rc;
  for (int r = 0; r < R; ++r) {
    bnorm[r] = sqrt(std::max(0.0, (double)hh[r]));
    if (!(bnorm[r] == bnorm[r]) || isinf(bnorm[r]))
      return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite right-hand side");
  }
  double prev_worst = -1.0;
  auto poly_op = [&](const T* v, T* w) -> int {
    const T* src = v;
    for (int k = 1; k < d; ++k) {
      T* dst = (k & 1) ? t1 : t2;
      int r2 = ctx_apply(c, src, nullptr, dst, R, 1.0, xtype);
      if (r2) return r2;
      src = dst;
    }
    *iters += d;
    return ctx_apply(c, src, v, w, R, -1.0, xtype);
  };
  while (true) {
    axpby_kernel<T><<<grid_for(Rn, c.nsm), 256, 0, c.st>>>(tmp, T(1), b, T(-1), x, Rn);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    rc = ctx_apply(c, x, tmp, V, R, 1.0, xtype);
    if (rc) return rc;
    ++*iters;
    rc = bdots<T>(c, R, V, 0, n, 1, V, n, partial, h_dev, hh.data());
    if (rc) return rc;
    int nact = 0;
    for (int r = 0; r < R; ++r) {
      beta[r] = sqrt(std::max(0.0, (double)hh[r]));
      if (!(beta[r] == beta[r]) || isinf(beta[r])) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite residual");
      (*est)[r] = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
      active[r] = beta[r] > tol * bnorm[r] && bnorm[r] > 0;
      nact += active[r];
      f[r] = active[r] ? 1.0 / beta[r] : 0.0;
      g[r].assign(m + 1, 0.0);
      g[r][0] = active[r] ? beta[r] : 0.0;
      kdone[r] = 0;
    }
    if (nact == 0) return DFM_OK;
    if (*iters >= max_iter) return DFM_ERR_NOT_CONVERGED;
    {
      double worst = 0.0;
      for (int r = 0; r < R; ++r)
        if (active[r]) worst = std::max(worst, (*est)[r]);
      if (prev_worst > 0 && worst > 0.9 * prev_worst) return DFM_ERR_NOT_CONVERGED;  // precision exhausted
      prev_worst = worst;
    }
    rc = bscale<T>(c, R, V, n, f, red_dev);
    if (rc) return rc;
    for (int j = 0; j < m; ++j) {
      T* vj = V + (int64_t)j * Rn;
      T* w = V + (int64_t)(j + 1) * Rn;
      if (lp) {
        // flexible step: z_j = p~(B) v_j on the 16-bit copy, w = z_j - B z_j
        T* zj = Z + (int64_t)j * Rn;
        if constexpr (std::is_same<T, float>::value) {
          rc = precond_hops(c, *lp, R, d, vj, zj);
        } else {
          rc = set_error(DFM_ERR_UNSUPPORTED, "dfm_solve: 16-bit preconditioner hops need FP32 Krylov vectors");
        }
        if (rc) return rc;
        *iters += d;
        rc = ctx_apply(c, zj, zj, w, R, -1.0, xtype);
      } else {
        rc = poly_op(vj, w);
      }
      if (rc) return rc;
      rc = bdots<T>(c, R, V, Rn, n, j + 2, w, n, partial, h_dev, hh.data());
      if (rc) return rc;
      std::vector<double> before(R);
      for (int r = 0; r < R; ++r) before[r] = sqrt(std::max(0.0, (double)hh[(size_t)r * (j + 2) + j + 1]));
      // pack h_r[0..j] with stride hld for the update
      std::vector<T> hp((size_t)R * hld, T(0));
      for (int r = 0; r < R; ++r)
        for (int i = 0; i <= j; ++i) {
          hp[(size_t)r * hld + i] = hh[(size_t)r * (j + 2) + i];
          H[r][i * m + j] = (double)hh[(size_t)r * (j + 2) + i];
        }
      DFM_CUDA_CHECK(cudaMemcpyAsync(h_dev, hp.data(), sizeof(T) * R * hld, cudaMemcpyHostToDevice, c.st));
      rc = baxpy<T>(c, R, V, Rn, n, j + 1, h_dev, hld, T(-1), w, n, partial, red_dev, &sq);
      if (rc) return rc;
      bool reorth = false;
      for (int r = 0; r < R; ++r) reorth |= (active[r] && sqrt(sq[r]) < 0.5 * before[r]);
      if (reorth) {
        rc = bdots<T>(c, R, V, Rn, n, j + 1, w, n, partial, h_dev, hh.data());
        if (rc) return rc;
        std::fill(hp.begin(), hp.end(), T(0));
        for (int r = 0; r < R; ++r)
          for (int i = 0; i <= j; ++i) {
            hp[(size_t)r * hld + i] = hh[(size_t)r * (j + 1) + i];
            H[r][i * m + j] += (double)hh[(size_t)r * (j + 1) + i];
          }
        DFM_CUDA_CHECK(cudaMemcpyAsync(h_dev, hp.data(), sizeof(T) * R * hld, cudaMemcpyHostToDevice, c.st));
        rc = baxpy<T>(c, R, V, Rn, n, j + 1, h_dev, hld, T(-1), w, n, partial, red_dev, &sq);
        if (rc) return rc;
      }
      int still = 0;
      for (int r = 0; r < R; ++r) {
        const double hn = sqrt(std::max(0.0, sq[r]));
        if (!(hn == hn)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite Krylov vector");
        f[r] = (active[r] && hn > 0) ? 1.0 / hn : 0.0;
        if (!active[r]) continue;
        std::vector<double>& Hr = H[r];
        Hr[(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = Hr[i * m + j], bb = Hr[(i + 1) * m + j];
          Hr[i * m + j] = cs[r][i] * a + sn[r][i] * bb;
          Hr[(i + 1) * m + j] = -sn[r][i] * a + cs[r][i] * bb;
        }
        const double den = hypot(Hr[j * m + j], Hr[(j + 1) * m + j]);
        cs[r][j] = den > 0 ? Hr[j * m + j] / den : 1.0;
        sn[r][j] = den > 0 ? Hr[(j + 1) * m + j] / den : 0.0;
        Hr[j * m + j] = den;
        Hr[(j + 1) * m + j] = 0.0;
        g[r][j + 1] = -sn[r][j] * g[r][j];
        g[r][j] = cs[r][j] * g[r][j];
        kdone[r] = j + 1;
        (*est)[r] = fabs(g[r][j + 1]) / bnorm[r];
        if (fabs(g[r][j + 1]) <= 0.5 * tol * bnorm[r] || hn == 0.0) active[r] = 0;
        still += active[r];
      }
      rc = bscale<T>(c, R, w, n, f, red_dev);
      if (rc) return rc;
      if (still == 0 || *iters + d >= max_iter) break;
    }
    // per right-hand side: y_r = H_r^{-1} g_r; x_r += p(B) V y_r
    int kmax = 0;
    std::vector<T> yp((size_t)R * hld, T(0));
    for (int r = 0; r < R; ++r) {
      const int kd = kdone[r];
      kmax = std::max(kmax, kd);
      std::vector<double> y(kd);
      for (int i = kd - 1; i >= 0; --i) {
        double acc = g[r][i];
        for (int k2 = i + 1; k2 < kd; ++k2) acc -= H[r][i * m + k2] * y[k2];
        y[i] = H[r][i * m + i] != 0.0 ? acc / H[r][i * m + i] : 0.0;
      }
      for (int i = 0; i < kd; ++i) yp[(size_t)r * hld + i] = (T)y[i];
    }
    if (kmax == 0) continue;
    DFM_CUDA_CHECK(cudaMemcpyAsync(h_dev, yp.data(), sizeof(T) * R * hld, cudaMemcpyHostToDevice, c.st));
    if (lp) {  // flexible update: x_r += Z_r y_r
      rc = baxpy<T>(c, R, Z, Rn, n, kmax, h_dev, hld, T(1), x, n, partial, red_dev, nullptr);
      if (rc) return rc;
      continue;
    }
    DFM_CUDA_CHECK(cudaMemsetAsync(tmp, 0, sizeof(T) * Rn, c.st));
    rc = baxpy<T>(c, R, V, Rn, n, kmax, h_dev, hld, T(1), tmp, n, partial, red_dev, nullptr);
    if (rc) return rc;
    const T* s_src = tmp;
    for (int k = 1; k < d; ++k) {  // Horner: s <- z + B s
      T* dst = (k & 1) ? t1 : t2;
      rc = ctx_apply(c, s_src, tmp, dst, R, 1.0, xtype);
      if (rc) return rc;
      s_src = dst;
    }
    *iters += d - 1;
    axpby_kernel<T><<<grid_for(Rn, c.nsm), 256, 0, c.st>>>(x, T(1), x, T(1), s_src, Rn);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
  }
}

// FP64 residuals r_r = rho0_r - (I - B) x_r for R right-hand sides:
// rel[r] = |r_r| / |rho0_r|, abs[r] = |r_r|; the residuals are left in r + R n.
int bresidual64(const Ctx& c, int R, const double* rho0, const double* x, double* r, double* partial, double* red_dev,
                std::vector<double>* rel, std::vector<double>* absn) {
  const int64_t Rn = (int64_t)R * c.n;
  sub_kernel<<<grid_for(Rn, c.nsm), 256, 0, c.st>>>(r, rho0, x, Rn);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  double* r2 = r + Rn;
  int rc = ctx_apply(c, x, r, r2, R, 1.0, DFM_F64);
  if (rc) return rc;
  std::vector<double> rn(R), bn(R);
  rc = bdots<double>(c, R, r2, 0, c.n, 1, r2, c.n, partial, red_dev, rn.data());
  if (rc) return rc;
  rc = bdots<double>(c, R, rho0, 0, c.n, 1, rho0, c.n, partial, red_dev, bn.data());
  if (rc) return rc;
  rel->resize(R);
  absn->resize(R);
  for (int i = 0; i < R; ++i) {
    (*absn)[i] = sqrt(std::max(0.0, rn[i]));
    const double b = sqrt(std::max(0.0, bn[i]));
    (*rel)[i] = b > 0 ? (*absn)[i] / b : (*absn)[i];
  }
  return DFM_OK;
}
}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_source(const dfm_mesh* mesh, int Np, const int64_t* rows_host, int n_src, double* rho0,
                          void* stream) {
  if (!mesh || !rows_host || !rho0 || n_src < 1 || !basis_ok(Np, geom::kWideMaxNp))
    return set_error(DFM_ERR_ARG, "dfm_source: bad argument");
  for (int s = 0; s < n_src; ++s)
    if (rows_host[s] < 0 || rows_host[s] >= mesh->nrows) return set_error(DFM_ERR_ARG, "dfm_source: row out of range");
  cudaStream_t st = as_stream(stream);
  // the linear functions of the linear spatial basis have zero mean: the
  // coefficient sits on index 0 (constant function, Zernike (0, 0)) either way
  const int nb = basis_size(Np);
  int64_t* rows_d = nullptr;
  DFM_CUDA_CHECK(cudaMallocAsync(&rows_d, sizeof(int64_t) * n_src, st));
  DFM_CUDA_CHECK(cudaMemcpyAsync(rows_d, rows_host, sizeof(int64_t) * n_src, cudaMemcpyHostToDevice, st));
  DFM_CUDA_CHECK(cudaMemsetAsync(rho0, 0, sizeof(double) * n_src * mesh->nrows * nb, st));
  source_kernel<<<(n_src + 127) / 128, 128, 0, st>>>(mesh->geom, rows_d, n_src, mesh->nrows, nb, rho0);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  DFM_CUDA_CHECK(cudaFreeAsync(rows_d, st));
  return DFM_OK;
}

namespace dfm {
namespace {
int solve_impl(const dfm_op* op, const dfm_op* const* combo, int K, const double* coef, const double* rho0, int R,
               double* rho, const dfm_solve_opts* opts, void* stream, dfm_solve_info* info) {
  if (!op || !rho0 || !rho || !opts || R < 1) return set_error(DFM_ERR_ARG, "dfm_solve: bad argument");
  if (rho == rho0) return set_error(DFM_ERR_ARG, "dfm_solve: rho must not alias rho0");
  if (!(opts->tol > 0)) return set_error(DFM_ERR_ARG, "dfm_solve: tol must be > 0");
  const int method = opts->method;
  const int max_iter = opts->max_iter > 0 ? opts->max_iter : 20000;
  const int m = opts->restart > 0 ? std::min(opts->restart, kMaxKrylov) : 128;
  const double inner_tol = opts->inner_tol > 0 ? opts->inner_tol : 1e-6;
  // default degree: 48 when the hops run on a low-precision copy (a half or a
  // quarter of the bytes per hop moves the balance between hops and
  // Gram-Schmidt work towards more hops per Krylov step), else 16
  const int poly = opts->poly_degree > 0 ? std::min(opts->poly_degree, 64) : (opts->precond_precision ? 48 : 16);
  // with combined operators the preconditioner's copy is made from ops[0]
  // (B_0, e.g. B(mu_c)): one p(B~_0) serves every right-hand side's B_r
  // a transposed solve preconditions with p(B~^T) on the transposed copy
  const bool use_lp = opts->precond_precision != 0 && method == DFM_SOLVE_GMRES_IR;
  if (opts->precond_precision != 0 && opts->precond_precision != DFM_F16 && opts->precond_precision != DFM_BF16 &&
      opts->precond_precision != DFM_FP8E4M3)
    return set_error(DFM_ERR_ARG, "dfm_solve: precond_precision must be 0, DFM_F16, DFM_BF16 or DFM_FP8E4M3");
  Ctx c;
  c.op = op;
  c.st = as_stream(stream);
  c.n = op->nrows * op->nb;
  c.trans = opts->transpose ? 1 : 0;
  c.combo = combo;
  c.K = K;
  c.coef = coef;
  if (combo && (c.trans || opts->method != DFM_SOLVE_GMRES_IR))
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_solve_combo: only GMRES_IR without transpose");
  int dev = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  DFM_CUDA_CHECK(cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t n = c.n;
  if (method == DFM_SOLVE_NEUMANN && op->precision != DFM_F64 && op->precision != DFM_F32)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_solve: Neumann needs an FP64 or FP32 operator");
  if (method == DFM_SOLVE_GMRES_IR && op->precision != DFM_F32 && op->precision != DFM_BF16)
    return set_error(DFM_ERR_UNSUPPORTED, "dfm_solve: GMRES_IR needs an FP32 or BF16 operator");
  if (method < 0 || method > 2) return set_error(DFM_ERR_ARG, "dfm_solve: unknown method");
  // right-hand sides solved in lockstep (GMRES_IR with R > 1): group size
  // capped so that a group's FP32 Krylov vectors take at most half of the
  // device memory that is free (plus what this operator's solver workspace
  // already holds), and at least 24 GiB
  const bool batched = (method == DFM_SOLVE_GMRES_IR && R > 1);
  int Rg = 1;
  if (batched) {
    const int64_t per_rhs =
        (int64_t)(m + 6 + (use_lp ? m : 0)) * n * 4 + (use_lp ? 3 * op->nrows * hop_nbp(op->nb) * 4 : 0);
    const int64_t cap = opts->batch > 0 ? opts->batch : 16;
    size_t free_b = 0, total_b = 0;
    DFM_CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
    const int64_t budget = std::max<int64_t>(int64_t(24) << 30, ((int64_t)free_b + op->swork_bytes) / 2);
    Rg = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)R, cap, budget / per_rhs}));
  }
  // workspace: FP64 vectors (x scratch, residual x2), Krylov basis in the inner precision
  const bool inner64 = (method == DFM_SOLVE_GMRES && op->precision == DFM_F64);
  const int64_t es = inner64 ? 8 : 4;
  const int64_t hcap = (int64_t)Rg * (kMaxKrylov + 8);
  int64_t bytes = 0;
  const bool gather = combo && K > 1 && batched && R > Rg;
  bytes += (2 * (int64_t)Rg + 2 + (gather ? 2 * (int64_t)Rg : 0)) * n * 8 + 8192;  // r, tmp64, xold [, gather b/x]
  const int64_t hop_elems = use_lp ? (int64_t)Rg * op->nrows * hop_nbp(op->nb) : 0;  // one padded hop vector
  const int64_t inner_bytes = (int64_t)(m + 7 + (use_lp ? m : 0)) * Rg * n * es + 3 * hop_elems * 4 +
                              12 * 256;  // V (m+1), tmp, t1, t2, b, x [, Z (m), vp, ha, hb]
  bytes += inner_bytes + 4096;
  const int64_t part_elems = std::max<int64_t>((int64_t)kRedBlocks * (kMaxKrylov + 8), (int64_t)kBRedBlocks * hcap);
  bytes += (part_elems + 2 * hcap + 2 * Rg + 256) * 8 + 4096;  // partials, h, red
  // block flexible GMRES: restart in block steps, (mb + 1) Rg basis vectors at most 512
  // (one operator for the whole group: not with per-right-hand-side combinations)
  const bool block = batched && use_lp && opts->block && Rg > 1 && !combo;
  const int mb = block ? std::max(1, std::min(m, 512 / Rg - 1)) : 0;
  const int64_t bpart = block ? (int64_t)kGMaxSplits * (mb + 1) * Rg * Rg : 0;
  const int64_t bsmall = block ? (int64_t)(mb + 3) * Rg * Rg : 0;
  if (block) bytes += (bpart + bsmall) * 4 + 1024;
  // two-level correction (single right-hand-side flexible solves): V, A V, r, y, aggregates
  if (opts->coarse < 0 || opts->coarse > 4) return set_error(DFM_ERR_ARG, "dfm_solve: coarse must be in 0..4");
  const bool use_coarse = opts->coarse > 0 && !batched && use_lp && method == DFM_SOLVE_GMRES_IR && !combo;
  const int g_coarse = use_coarse ? opts->coarse : 0;
  const int nc_max = g_coarse * g_coarse * g_coarse;
  if (use_coarse) bytes += ((2 * (int64_t)nc_max + 1) * n + 64) * 4 + op->mesh->nt * 4 + 5 * 256;
  int rc = ensure_work(op, bytes + 8 * 256);
  if (rc) return rc;
  Work W{reinterpret_cast<char*>(op->swork)};
  double* r64 = W.take<double>(2 * (int64_t)Rg * n);
  double* tmp64 = W.take<double>(n);
  double* xold = W.take<double>(n);
  double* gather_b = gather ? W.take<double>((int64_t)Rg * n) : nullptr;
  double* gather_x = gather ? W.take<double>((int64_t)Rg * n) : nullptr;
  double* part64 = W.take<double>(part_elems);
  double* h64 = W.take<double>(2 * hcap);
  double* red64 = W.take<double>(std::max(8, 2 * Rg));
  char* inner_base = W.take<char>(inner_bytes);
  BlockScratch bscr;
  if (block) {
    bscr.part = W.take<float>(bpart);
    bscr.part_elems = bpart;
    bscr.small = W.take<float>(bsmall);
  }
  Coarse coarse;
  if (use_coarse) {
    coarse.V = W.take<float>((int64_t)nc_max * n);
    coarse.AV = W.take<float>((int64_t)nc_max * n);
    coarse.r = W.take<float>(n);
    coarse.y = W.take<float>(64);
    coarse.agg = W.take<int32_t>(op->mesh->nt);
  }
  Hop hop;
  const Hop* lp = nullptr;
  if (use_lp) {
    rc = prepare_lowp(op, opts->precond_precision, c.st, opts->transpose ? 1 : 0, batched ? Rg : 1);
    if (rc) return rc;
    hop.op = op;
    lp = &hop;
  }
  if (batched) {
    Work Wi{inner_base};
    float* V = Wi.take<float>((int64_t)(m + 1) * Rg * n);
    float* tmp = Wi.take<float>((int64_t)Rg * n);
    float* t1 = Wi.take<float>((int64_t)Rg * n);
    float* t2 = Wi.take<float>((int64_t)Rg * n);
    float* bf = Wi.take<float>((int64_t)Rg * n);
    float* xf = Wi.take<float>((int64_t)Rg * n);
    float* Zb = use_lp ? Wi.take<float>((int64_t)m * Rg * n) : nullptr;
    if (use_lp) {
      hop.vp = Wi.take<float>(hop_elems);
      hop.ha = Wi.take<float>(hop_elems);
      hop.hb = Wi.take<float>(hop_elems);
    }
    float* part32 = reinterpret_cast<float*>(part64);
    float* h32 = reinterpret_cast<float*>(h64);
    float* red32 = reinterpret_cast<float*>(red64);
    dfm_solve_info ai{0, 0, 0.0};
    int status = DFM_OK;
    // right-hand sides with their own damping converge at different rates and a
    // lockstep group runs at its slowest member's pace: order them by the first
    // damping moment weight (mu_r - mu_c) so that each group holds similar ones
    std::vector<int> order(R);
    for (int r = 0; r < R; ++r) order[r] = r;
    const bool reorder = combo && K > 1 && R > Rg;
    if (reorder)
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int b2) { return coef[(int64_t)a * K + 1] < coef[(int64_t)b2 * K + 1]; });
    std::vector<double> grp_coef;
    for (int g0 = 0; g0 < R; g0 += Rg) {
      const int Rc = std::min(Rg, R - g0);
      const double* b = rho0 + (int64_t)g0 * n;
      double* x = rho + (int64_t)g0 * n;
      if (reorder) {  // gather the group into contiguous buffers
        b = gather_b;
        x = gather_x;
        grp_coef.resize((size_t)Rc * K);
        for (int r = 0; r < Rc; ++r) {
          const int src = order[g0 + r];
          DFM_CUDA_CHECK(cudaMemcpyAsync(gather_b + (int64_t)r * n, rho0 + (int64_t)src * n, sizeof(double) * n,
                                         cudaMemcpyDeviceToDevice, c.st));
          if (opts->use_x0)
            DFM_CUDA_CHECK(cudaMemcpyAsync(gather_x + (int64_t)r * n, rho + (int64_t)src * n, sizeof(double) * n,
                                           cudaMemcpyDeviceToDevice, c.st));
          for (int k = 0; k < K; ++k) grp_coef[(size_t)r * K + k] = coef[(int64_t)src * K + k];
        }
        c.coef = grp_coef.data();
      } else if (combo) {
        c.coef = coef + (int64_t)g0 * K;
      }
      if (!opts->use_x0) DFM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * Rc * n, c.st));
      int iters = 0, outer = 0;
      std::vector<double> rel, absn, est;
      int gs = DFM_OK;
      while (true) {
        rc = bresidual64(c, Rc, b, x, r64, part64, red64, &rel, &absn);
        if (rc) return rc;
        double worst = 0.0;
        bool bad = false;
        for (int r = 0; r < Rc; ++r) {
          bad |= !(rel[r] == rel[r]) || isinf(rel[r]);
          worst = std::max(worst, rel[r]);
        }
        if (bad) {
          gs = set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite residual");
          break;
        }
        if (worst <= opts->tol) break;
        if (iters >= max_iter || outer > 200) {
          gs = set_error(DFM_ERR_NOT_CONVERGED, "dfm_solve: batched refinement reached max_iter");
          break;
        }
        std::vector<double> sdown(Rc), sup(Rc);
        for (int r = 0; r < Rc; ++r) {
          const bool act = rel[r] > opts->tol && absn[r] > 0;
          sdown[r] = act ? 1.0 / absn[r] : 0.0;
          sup[r] = act ? absn[r] : 0.0;
        }
        DFM_CUDA_CHECK(cudaMemcpyAsync(red64, sdown.data(), sizeof(double) * Rc, cudaMemcpyHostToDevice, c.st));
        bto_f32_kernel<<<dim3(grid_for(n, c.nsm), Rc), 256, 0, c.st>>>(bf, r64 + (int64_t)Rc * n, red64, n);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
        DFM_CUDA_CHECK(cudaMemsetAsync(xf, 0, sizeof(float) * Rc * n, c.st));
        const double itol = std::max(inner_tol, 0.3 * opts->tol / std::max(worst, 1e-300));
        int gi = (block && Rc > 1)
                     ? gmres_block(c, Rc, bf, xf, itol, mb, poly, max_iter, &iters, &est, V, Zb, tmp, *lp, bscr)
                     : gmres_batched<float>(c, Rc, bf, xf, itol, m, poly, max_iter, &iters, &est, V, tmp, t1, t2,
                                            h32, part32, red32, lp, Zb);
        if (gi != DFM_OK && gi != DFM_ERR_NOT_CONVERGED) return gi;
        DFM_CUDA_CHECK(cudaMemcpyAsync(red64, sup.data(), sizeof(double) * Rc, cudaMemcpyHostToDevice, c.st));
        badd_f32_kernel<<<dim3(grid_for(n, c.nsm), Rc), 256, 0, c.st>>>(x, xf, red64, n);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
        ++outer;
      }
      if (reorder)  // scatter the group's solutions back
        for (int r = 0; r < Rc; ++r)
          DFM_CUDA_CHECK(cudaMemcpyAsync(rho + (int64_t)order[g0 + r] * n, gather_x + (int64_t)r * n,
                                         sizeof(double) * n, cudaMemcpyDeviceToDevice, c.st));
      double worst = 0.0;
      for (double v : rel) worst = std::max(worst, v);
      ai.iters += iters;
      ai.outer += outer;
      ai.resid = std::max(ai.resid, worst);
      if (gs != DFM_OK && status == DFM_OK) status = gs;
    }
    if (info) *info = ai;
    return status;
  }
  dfm_solve_info acc_info{0, 0, 0.0};
  int status = DFM_OK;
  for (int s = 0; s < R && status != DFM_ERR_NONFINITE; ++s) {
    if (combo) c.coef = coef + (int64_t)s * K;
    const double* b = rho0 + (int64_t)s * n;
    double* x = rho + (int64_t)s * n;
    int iters = 0, outer = 0;
    double resid = 0.0, rabs = 0.0;
    if (!opts->use_x0) DFM_CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, c.st));
    int rs = DFM_OK;
    if (method == DFM_SOLVE_NEUMANN) {
      // x <- rho0 + B x until |x_new - x| <= tol |x_new|
      std::vector<double> ph(2 * kRedBlocks);
      while (true) {
        DFM_CUDA_CHECK(cudaMemcpyAsync(xold, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.st));
        rs = ctx_apply(c, xold, b, x, 1, 1.0, DFM_F64);
        if (rs) return rs;
        ++iters;
        diff_norm_kernel<<<kRedBlocks, kRedThreads, 0, c.st>>>(x, xold, n, part64);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
        DFM_CUDA_CHECK(cudaMemcpyAsync(ph.data(), part64, sizeof(double) * 2 * kRedBlocks, cudaMemcpyDeviceToHost, c.st));
        DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
        double d2 = 0, a2 = 0;
        for (int i = 0; i < kRedBlocks; ++i) {
          d2 += ph[2 * i];
          a2 += ph[2 * i + 1];
        }
        if (!(d2 == d2) || isinf(d2)) {
          rs = set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite Neumann iterate");
          break;
        }
        if (sqrt(d2) <= opts->tol * sqrt(a2)) break;
        if (iters >= max_iter) {
          rs = set_error(DFM_ERR_NOT_CONVERGED, "dfm_solve: Neumann series reached max_iter");
          break;
        }
      }
      if (rs != DFM_ERR_NONFINITE) {
        int r2 = residual64(c, b, x, r64, part64, red64, &resid, &rabs);
        if (r2) return r2;
      }
    } else if (method == DFM_SOLVE_GMRES && inner64) {
      Work Wi{inner_base};
      double* V = Wi.take<double>((int64_t)(m + 1) * n);
      double* tmp = Wi.take<double>(n);
      double* t1 = Wi.take<double>(n);
      double* t2 = Wi.take<double>(n);
      double est = 0;
      rs = gmres<double>(c, b, x, opts->tol, m, opts->poly_degree > 0 ? poly : 1, max_iter, &iters, &est, V, tmp,
                         t1, t2, h64, part64, red64);
      if (rs == DFM_ERR_NOT_CONVERGED) set_error(rs, "dfm_solve: GMRES reached max_iter");
      if (rs == DFM_OK || rs == DFM_ERR_NOT_CONVERGED) {
        int r2 = residual64(c, b, x, r64, part64, red64, &resid, &rabs);
        if (r2) return r2;
      }
    } else {
      // FP32 Krylov: plain GMRES (tol on the FP32 residual) or refinement around it
      Work Wi{inner_base};
      float* V = Wi.take<float>((int64_t)(m + 1) * n);
      float* tmp = Wi.take<float>(n);
      float* t1 = Wi.take<float>(n);
      float* t2 = Wi.take<float>(n);
      float* bf = Wi.take<float>(n);
      float* xf = Wi.take<float>(n);
      float* Zs = use_lp ? Wi.take<float>((int64_t)m * n) : nullptr;
      if (use_lp) {
        hop.vp = Wi.take<float>(hop_elems);
        hop.ha = Wi.take<float>(hop_elems);
        hop.hb = Wi.take<float>(hop_elems);
      }
      float* part32 = reinterpret_cast<float*>(part64);
      float* h32 = reinterpret_cast<float*>(h64);
      float* red32 = reinterpret_cast<float*>(red64);
      if (use_coarse && s == 0) {  // one coarse space for every right-hand side of the call
        rs = coarse_setup(c, op->mesh, g_coarse, coarse, part32, h32, &iters);
        if (rs) return rs;
      }
      while (true) {
        int r2 = residual64(c, b, x, r64, part64, red64, &resid, &rabs);
        if (r2) return r2;
        if (!(resid == resid) || isinf(resid)) {
          rs = set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite residual");
          break;
        }
        if (resid <= opts->tol) break;
        if (iters >= max_iter) {
          rs = set_error(DFM_ERR_NOT_CONVERGED, "dfm_solve: refinement reached max_iter");
          break;
        }
        // correction: (I - B) d = r / |r| in FP32
        to_f32_kernel<<<grid_for(n, c.nsm), 256, 0, c.st>>>(bf, r64 + n, 1.0 / rabs, n);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
        DFM_CUDA_CHECK(cudaMemsetAsync(xf, 0, sizeof(float) * n, c.st));
        double est = 0;
        // inner tolerance: what this refinement step still has to gain, floored
        // at what FP32 Krylov vectors can deliver
        const double need = opts->tol / std::max(resid, 1e-300);
        const double itol = method == DFM_SOLVE_GMRES_IR ? std::max(inner_tol, 0.3 * need)
                                                         : std::max(opts->tol, 1e-6);
        int gi = gmres<float>(c, bf, xf, itol, m, poly, max_iter, &iters, &est, V, tmp, t1, t2, h32, part32, red32,
                              method == DFM_SOLVE_GMRES_IR ? lp : nullptr, Zs, use_coarse ? &coarse : nullptr);
        if (gi != DFM_OK && gi != DFM_ERR_NOT_CONVERGED) return gi;
        add_f32_kernel<<<grid_for(n, c.nsm), 256, 0, c.st>>>(x, xf, rabs, n);
        DFM_LAUNCHED();
        DFM_CUDA_CHECK(cudaGetLastError());
        ++outer;
        if (outer > 200) {
          rs = set_error(DFM_ERR_NOT_CONVERGED, "dfm_solve: refinement stalled");
          break;
        }
      }
    }
    acc_info.iters += iters;
    acc_info.outer += outer;
    acc_info.resid = std::max(acc_info.resid, resid);
    if (rs != DFM_OK && status == DFM_OK) status = rs;
  }
  if (info) *info = acc_info;
  // a pipelined operator application or hop that gave up waiting for its data
  const int te = read_timeout_flag(op, c.st, "dfm_solve");
  if (te) return te;
  return status;
}
}  // namespace
}  // namespace dfm

extern "C" int dfm_solve(const dfm_op* op, const double* rho0, int R, double* rho, const dfm_solve_opts* opts,
                         void* stream, dfm_solve_info* info) {
  return dfm::solve_impl(op, nullptr, 1, nullptr, rho0, R, rho, opts, stream, info);
}

extern "C" int dfm_solve_combo(const dfm_op* const* ops, int K, const double* coef_host, const double* rho0, int R,
                               double* rho, const dfm_solve_opts* opts, void* stream, dfm_solve_info* info) {
  if (!ops || K < 1 || K > 4 || !coef_host) return dfm::set_error(DFM_ERR_ARG, "dfm_solve_combo: bad argument");
  for (int k = 0; k < K; ++k)
    if (!ops[k] || ops[k]->mesh != ops[0]->mesh || ops[k]->Np != ops[0]->Np || ops[k]->ns != ops[0]->ns ||
        ops[k]->precision != DFM_F32)
      return dfm::set_error(DFM_ERR_ARG, "dfm_solve_combo: operators must be FP32 and share mesh and Np");
  return dfm::solve_impl(ops[0], ops, K, coef_host, rho0, R, rho, opts, stream, info);
}

extern "C" int dfm_solve_damped(const dfm_op* const* moments, int K, const double* mu_rhs_host, const double* rho0,
                                int R, double* rho, const dfm_solve_opts* opts, void* stream, dfm_solve_info* info) {
  if (!moments || K < 1 || K > 4 || !mu_rhs_host || R < 1)
    return dfm::set_error(DFM_ERR_ARG, "dfm_solve_damped: bad argument");
  for (int k = 0; k < K; ++k) {
    const dfm_op* o = moments[k];
    if (!o || o->mesh != moments[0]->mesh || o->Np != moments[0]->Np || o->ns != moments[0]->ns ||
        o->precision != DFM_F32)
      return dfm::set_error(DFM_ERR_ARG, "dfm_solve_damped: moments must be FP32 and share mesh and Np");
    if (o->moment != k)
      return dfm::set_error(DFM_ERR_ARG, "dfm_solve_damped: moments[k] must be assembled with moment = k");
    if (!(o->mu_uniform >= 0.0) || o->mu_uniform != moments[0]->mu_uniform)
      return dfm::set_error(DFM_ERR_ARG, "dfm_solve_damped: moments must share one uniform damping mu_c");
  }
  const double mu_c = moments[0]->mu_uniform;
  // Taylor weights of B(mu_r) = sum_k (mu_r - mu_c)^k / k! B^(k) about the
  // damping the moments were assembled at (the damping factor exp(-mu L) of
  // Sec. 2 is analytic in mu)
  std::vector<double> coef((size_t)R * K);
  for (int r = 0; r < R; ++r) {
    const double mr = mu_rhs_host[r];
    if (!(mr >= 0.0) || isinf(mr)) return dfm::set_error(DFM_ERR_ARG, "dfm_solve_damped: mu_rhs must be finite, >= 0");
    double c = 1.0;
    for (int k = 0; k < K; ++k) {
      coef[(size_t)r * K + k] = c;
      c *= (mr - mu_c) / (k + 1);
    }
  }
  return dfm::solve_impl(moments[0], moments, K, coef.data(), rho0, R, rho, opts, stream, info);
}
