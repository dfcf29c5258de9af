// Boundary densities with one ray direction (Sec. 4.1, Eq. RhoNeumann).
//
// The paper's cuboid verification prescribes a constant density on the x = 0
// face travelling along the inward normal, rho0 = delta(rho)/(2 pi rho) in the
// polar momentum coordinates of the face, and projects it onto the finite
// basis of Eq. FBApprox.  The same projection holds for any inward direction
// d: the unit-mass delta at p_d = (d.e1, d.e2) has inner product Z_n^m(p_d)
// with each Zernike polynomial, the Galerkin coefficient divides by the
// polynomial's norm pi eps_m/(2n+2) and the spatial basis function
// 1/sqrt(|T|) of the face contributes |T|/sqrt(|T|).  One thread per source
// evaluates the Zernike recursion once in FP64 and writes its row.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dfm_internal.cuh"
#include "node.cuh"

namespace dfm {
namespace {

template <int NP>
__global__ void directed_source_kernel(const FaceGeom* __restrict__ geom, const int64_t* __restrict__ rows,
                                       const double* __restrict__ dirs, int n_src, int64_t nrows, int combine,
                                       double* __restrict__ rho0, int* __restrict__ bad) {
  constexpr int NB = (NP + 1) * (NP + 2) / 2;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  const int64_t r = rows[s];
  const FaceGeom F = geom[r];
  double px = 0.0, py = 0.0;  // the inward normal: p = 0
  if (dirs) {
    double d[3] = {dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2]};
    const double inv = 1.0 / sqrt(dot3(d, d));  // the host rejected zero directions
    for (int c = 0; c < 3; ++c) d[c] *= inv;
    if (!(dot3(d, F.n) > 0.0)) {  // the ray must enter the tet
      atomicOr(bad, 1);
      return;
    }
    px = dot3(d, F.e1);
    py = dot3(d, F.e2);
  }
  double Z[NB];
  zernike<NP, double>(px, py, Z);
  const double sa = sqrt(F.area);
  double* out = rho0 + ((combine ? 0 : (int64_t)s * nrows) + r) * NB;
  int i = 0;
#pragma unroll
  for (int n = 0; n <= NP; ++n)
#pragma unroll
    for (int m = -n; m <= n; m += 2, ++i) out[i] = (2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI) * Z[i] * sa;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_source_directed(const dfm_mesh* mesh, int Np, const int64_t* rows_host, const double* dirs_host,
                                   int n_src, int combine, double* rho0, void* stream) {
  if (!mesh || !rows_host || !rho0 || n_src < 1 || Np < 0 || Np > 8 || (combine != 0 && combine != 1))
    return set_error(DFM_ERR_ARG, "dfm_source_directed: bad argument");
  for (int s = 0; s < n_src; ++s)
    if (rows_host[s] < 0 || rows_host[s] >= mesh->nrows)
      return set_error(DFM_ERR_ARG, "dfm_source_directed: row out of range");
  if (dirs_host)
    for (int s = 0; s < n_src; ++s) {
      const double* d = dirs_host + 3 * (int64_t)s;
      const double l2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(l2 > 0.0) || !std::isfinite(l2))
        return set_error(DFM_ERR_ARG, "dfm_source_directed: zero or non-finite direction");
    }
  if (combine) {
    std::vector<int64_t> v(rows_host, rows_host + n_src);
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end())
      return set_error(DFM_ERR_ARG, "dfm_source_directed: repeated row in a combined source");
  }
  cudaStream_t st = as_stream(stream);
  const int nb = nbasis(Np);
  // stream-ordered scratch: rows, directions, the direction check flag
  char* buf = nullptr;
  const size_t bytes = sizeof(int64_t) * n_src + 3 * sizeof(double) * n_src + 16;
  DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, st));
  int64_t* rows_d = reinterpret_cast<int64_t*>(buf);
  double* dirs_d = reinterpret_cast<double*>(buf + sizeof(int64_t) * n_src);
  int* bad_d = reinterpret_cast<int*>(buf + sizeof(int64_t) * n_src + 3 * sizeof(double) * n_src);
  DFM_CUDA_CHECK(cudaMemcpyAsync(rows_d, rows_host, sizeof(int64_t) * n_src, cudaMemcpyHostToDevice, st));
  if (dirs_host)
    DFM_CUDA_CHECK(cudaMemcpyAsync(dirs_d, dirs_host, 3 * sizeof(double) * n_src, cudaMemcpyHostToDevice, st));
  DFM_CUDA_CHECK(cudaMemsetAsync(bad_d, 0, sizeof(int), st));
  DFM_CUDA_CHECK(cudaMemsetAsync(rho0, 0, sizeof(double) * (combine ? 1 : n_src) * mesh->nrows * nb, st));
  const unsigned blocks = (unsigned)((n_src + 127) / 128);
  const double* dp = dirs_host ? dirs_d : nullptr;
#define CASE(N)                                                                                                  \
  case N:                                                                                                        \
    directed_source_kernel<N><<<blocks, 128, 0, st>>>(mesh->geom, rows_d, dp, n_src, mesh->nrows, combine, rho0, \
                                                      bad_d);                                                    \
    break;
  switch (Np) { CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) }
#undef CASE
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  int bad = 0;
  if (dirs_host) DFM_CUDA_CHECK(cudaMemcpyAsync(&bad, bad_d, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFM_CUDA_CHECK(cudaFreeAsync(buf, st));
  if (dirs_host) {
    DFM_CUDA_CHECK(cudaStreamSynchronize(st));
    if (bad) return set_error(DFM_ERR_ARG, "dfm_source_directed: a direction does not point into its tet");
  }
  return DFM_OK;
}
