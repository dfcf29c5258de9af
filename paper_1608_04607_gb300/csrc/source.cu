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
#include "interior_rule.cuh"
#include "node.cuh"

namespace dfm {
namespace {

template <int NP>
__global__ void directed_source_kernel(const FaceGeom* __restrict__ geom, const int64_t* __restrict__ rows,
                                       const double* __restrict__ dirs, int n_src, int64_t nrows, int combine,
                                       double* __restrict__ rho0, int* __restrict__ bad, int stride) {
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
  double* out = rho0 + ((combine ? 0 : (int64_t)s * nrows) + r) * stride;
  int i = 0;
#pragma unroll
  for (int n = 0; n <= NP; ++n)
#pragma unroll
    for (int m = -n; m <= n; m += 2, ++i) out[i] = (2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI) * Z[i] * sa;
}


// Point sources (Sec. 4.2, Eq. SourceRho) in uniform media.  Rays leave r0 in
// every direction, cross the tet that holds r0 and enter the next tet through
// a face F of it that does not contain r0, carrying the density
//   strength cos(theta) exp(-mu R) / R^2 delta(u - unit(s - r0))
// at the face point s (R = |s - r0|, theta the angle between the ray and F's
// normal).  The row across F receives it (on the boundary: F's own row with
// weight refl and the specularly reflected direction, whose tangential
// components are the ray's), so its Galerkin coefficients are
//   a[rec][(n,m)] = N_nm / sqrt|F| Int_F strength cos exp(-mu R)/R^2 Z_n^m(p(u)) ds,
// p(u) the tangential part of u in the receiving face's frame.  cos/R^2 ds is
// the solid-angle element seen from r0, the same measure as the interior
// density's integral, so the split polar rule of that integral applies with
// the direction reversed.  A point on a face, an edge or a vertex lies in the
// closure of several tets; each of them sends through its faces that do not
// contain the point.

// Barycentric tolerance: r0 counts as inside a tet when no coordinate is below
// -kBaryTol and as lying on face l when coordinate l is at most kBaryTol.
constexpr double kBaryTol = 1e-12;

struct PointTask {
  int s;     // source
  int mask;  // faces (bits l < 4) whose plane does not hold r0
  int64_t k; // tet
};

__device__ __forceinline__ double vol6(const double* a, const double* b, const double* c, const double* d) {
  const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double w[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
  return u[0] * (v[1] * w[2] - v[2] * w[1]) + u[1] * (v[2] * w[0] - v[0] * w[2]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
}

// One thread per tet, looping over the sources: the barycentric coordinates
// of each r0 as ratios of signed volumes; every (source, tet) whose closure
// holds r0 becomes a task.  Overflow of the task list and per-source hit
// counts are reported to the host.
__global__ void point_locate_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets, int64_t nt,
                                    const double* __restrict__ r0, int n_src, PointTask* __restrict__ tasks, int cap,
                                    int* __restrict__ count, int* __restrict__ hits) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nt) return;
  double P[4][3];
  for (int v = 0; v < 4; ++v)
    for (int c = 0; c < 3; ++c) P[v][c] = V[3 * (int64_t)tets[4 * k + v] + c];
  const double vol = vol6(P[0], P[1], P[2], P[3]);
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = fmin(fmin(P[0][c], P[1][c]), fmin(P[2][c], P[3][c]));
    hi[c] = fmax(fmax(P[0][c], P[1][c]), fmax(P[2][c], P[3][c]));
  }
  const double slack = 1e-9 * fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
  for (int s = 0; s < n_src; ++s) {
    const double* r = r0 + 3 * s;
    bool box = true;
    for (int c = 0; c < 3; ++c) box = box && r[c] >= lo[c] - slack && r[c] <= hi[c] + slack;
    if (!box) continue;
    double lam[4];
    lam[0] = vol6(r, P[1], P[2], P[3]) / vol;
    lam[1] = vol6(P[0], r, P[2], P[3]) / vol;
    lam[2] = vol6(P[0], P[1], r, P[3]) / vol;
    lam[3] = vol6(P[0], P[1], P[2], r) / vol;
    if (fmin(fmin(lam[0], lam[1]), fmin(lam[2], lam[3])) < -kBaryTol) continue;
    int mask = 0;
    for (int l = 0; l < 4; ++l)
      if (lam[l] > kBaryTol) mask |= 1 << l;
    atomicAdd(&hits[s], 1);
    const int i = atomicAdd(count, 1);
    if (i < cap) tasks[i] = PointTask{s, mask, k};
  }
}

// One block of four warps per task, warp l integrating face l: lanes stride
// over the rule's nodes, accumulate w exp(-mu R) Z(p) in FP64 and reduce by
// shuffles; lane 0 adds the row into rho0 (the receiving rows of different
// tasks and faces are distinct, so each entry gets one addition onto zero).
// polar: the split polar rule with nq points per direction (6 nq^2 nodes);
// otherwise the collapsed tensor Gauss-Legendre rule of order nq on the flat
// triangle (nq^2 nodes).
template <int NP>
__global__ void __launch_bounds__(128) point_face_kernel(
    const double* __restrict__ V, const int32_t* __restrict__ tets, const int32_t* __restrict__ recv,
    const double* __restrict__ refl, const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet,
    double mu_uniform, const double* __restrict__ r0, const PointTask* __restrict__ tasks,
    const int* __restrict__ count, int cap, int polar, int nq, const double* __restrict__ gl_x,
    const double* __restrict__ gl_w, double strength, int64_t nrows, double* __restrict__ rho0) {
  constexpr int NB = (NP + 1) * (NP + 2) / 2;
  const int lane = threadIdx.x & 31;
  const int l = threadIdx.x >> 5;
  if ((int)blockIdx.x >= min(*count, cap)) return;
  const PointTask task = tasks[blockIdx.x];
  if (!((task.mask >> l) & 1)) return;  // r0 lies on face l: no ray crosses it
  const int64_t row = 4 * task.k + l;
  const int64_t rec = recv[row];
  const double wgt = rec == row ? refl[row] : 1.0;
  const FaceGeom F = geom[row];
  const FaceGeom G = geom[rec];
  const double r[3] = {r0[3 * task.s], r0[3 * task.s + 1], r0[3 * task.s + 2]};
  double p[3][3];
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) p[v][c] = V[3 * (int64_t)tets[4 * task.k + ((l + 1 + v) & 3)] + c];
  const double mu = mu_tet ? mu_tet[task.k] : mu_uniform;
  const double h = (r[0] - p[0][0]) * F.n[0] + (r[1] - p[0][1]) * F.n[1] + (r[2] - p[0][2]) * F.n[2];
  double acc[NB], Z[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) acc[a] = 0.0;
  const int nodes = polar ? 6 * nq * nq : nq * nq;
  for (int k = lane; k < nodes; k += 32) {
    double u[3], w, R;
    if (polar) {
      const rule::PolarNode q = rule::polar_node(p, F.n, F.e1, F.e2, r, nq, k, gl_x, gl_w);
      if (q.w == 0.0) continue;
      // q.(dx, dy) is the tangential part of unit(r0 - s); the ray runs the other way
      const double cz = h / q.R;
      for (int c = 0; c < 3; ++c) u[c] = -(q.dx * F.e1[c] + q.dy * F.e2[c] + cz * F.n[c]);
      w = q.w;
      R = q.R;
    } else {
      const int i = k / nq, j = k - i * nq;
      const double a = 0.5 * (1.0 + gl_x[i]);
      const double b = (1.0 - a) * 0.5 * (1.0 + gl_x[j]);
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = p[0][c] + a * (p[1][c] - p[0][c]) + b * (p[2][c] - p[0][c]) - r[c];
      R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int c = 0; c < 3; ++c) u[c] = d[c] / R;
      const double cs = -(u[0] * F.n[0] + u[1] * F.n[1] + u[2] * F.n[2]);  // F.n points into tet k
      w = gl_w[i] * gl_w[j] * 0.25 * (1.0 - a) * 2.0 * F.area * cs / (R * R);
    }
    const double ker = w * exp(-mu * R);
    zernike<NP, double>(u[0] * G.e1[0] + u[1] * G.e1[1] + u[2] * G.e1[2],
                        u[0] * G.e2[0] + u[1] * G.e2[1] + u[2] * G.e2[2], Z);
#pragma unroll
    for (int a = 0; a < NB; ++a) acc[a] = fma(ker, Z[a], acc[a]);
  }
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
  if (lane == 0) {
    const double sc = wgt * strength / sqrt(F.area);
    double* out = rho0 + ((int64_t)task.s * nrows + rec) * NB;
    int i = 0;
#pragma unroll
    for (int n = 0; n <= NP; ++n)
#pragma unroll
      for (int m = -n; m <= n; m += 2, ++i)
        atomicAdd(&out[i], sc * (2.0 * n + 2.0) / ((m == 0 ? 2.0 : 1.0) * M_PI) * acc[i]);
  }
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_source_directed(const dfm_mesh* mesh, int Np, const int64_t* rows_host, const double* dirs_host,
                                   int n_src, int combine, double* rho0, void* stream) {
  if (!mesh || !rows_host || !rho0 || n_src < 1 || !basis_ok(Np, geom::kWideMaxNp) || (combine != 0 && combine != 1))
    return set_error(DFM_ERR_ARG, "dfm_source_directed: bad argument");
  // a constant density on the face projects onto the constant spatial
  // function only: the first (Np+1)(Np+2)/2 entries of each row
  const int stride = basis_size(Np);
  Np = basis_np(Np);
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
  DFM_CUDA_CHECK(cudaMemsetAsync(rho0, 0, sizeof(double) * (combine ? 1 : n_src) * mesh->nrows * stride, st));
  const unsigned blocks = (unsigned)((n_src + 127) / 128);
  const double* dp = dirs_host ? dirs_d : nullptr;
#define CASE(N)                                                                                                  \
  case N:                                                                                                        \
    directed_source_kernel<N><<<blocks, 128, 0, st>>>(mesh->geom, rows_d, dp, n_src, mesh->nrows, combine, rho0, \
                                                      bad_d, stride);                                            \
    break;
  switch (Np) {
    CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    default: {  // Np = 9..20 (wide.cu)
      const int rc = launch_directed_source_wide(Np, mesh->geom, rows_d, dp, n_src, mesh->nrows, combine, rho0, bad_d,
                                                 stride, st);
      if (rc) {
        cudaFreeAsync(buf, st);
        return rc;
      }
    }
  }
#undef CASE
  if (Np <= 8) DFM_LAUNCHED();
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

extern "C" int dfm_point_source(const dfm_mesh* mesh, int Np, const double* r0_host, int n_src, const double* mu,
                                double mu_uniform, double strength, int nq, double* rho0, void* stream) {
  if (!mesh || !r0_host || !rho0 || n_src < 1 || Np < 0 || Np > 8)
    return set_error(DFM_ERR_ARG, "dfm_point_source: bad argument");
  if (nq == 0) nq = -24;
  const bool polar = nq < 0;
  if (polar) nq = -nq;
  if (nq < 2 || nq > 64) return set_error(DFM_ERR_ARG, "dfm_point_source: |nq| must be in 2..64");
  if (!mu && !(mu_uniform >= 0)) return set_error(DFM_ERR_ARG, "dfm_point_source: mu_uniform must be >= 0");
  if (!std::isfinite(strength)) return set_error(DFM_ERR_ARG, "dfm_point_source: strength must be finite");
  for (int64_t i = 0; i < 3 * (int64_t)n_src; ++i)
    if (!std::isfinite(r0_host[i])) return set_error(DFM_ERR_ARG, "dfm_point_source: non-finite source position");
  cudaStream_t st = as_stream(stream);
  const int nb = nbasis(Np);
  // stream-ordered scratch: positions, hit counts, the task counter, the Gauss table
  char* buf = nullptr;
  const size_t head = 3 * sizeof(double) * n_src + 2 * 64 * sizeof(double);
  const size_t bytes = head + sizeof(int) * (n_src + 1) + 16;
  DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, st));
  double* r0_d = reinterpret_cast<double*>(buf);
  double* glx = r0_d + 3 * n_src;
  double* glw = glx + 64;
  int* hits = reinterpret_cast<int*>(buf + head);
  int* count = hits + n_src;
  DFM_CUDA_CHECK(cudaMemcpyAsync(r0_d, r0_host, 3 * sizeof(double) * n_src, cudaMemcpyHostToDevice, st));
  DFM_CUDA_CHECK(cudaMemsetAsync(rho0, 0, sizeof(double) * n_src * mesh->nrows * nb, st));
  int rc = gauss_legendre_device(nq, glx, glw, st);
  if (rc) {
    cudaFreeAsync(buf, st);
    return rc;
  }
  // locate (twice if the first task list was too short: the count is exact)
  int cap = 64 * n_src, n_tasks = 0;
  std::vector<int> hits_h(n_src);
  PointTask* tasks = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&tasks), sizeof(PointTask) * cap, st));
    DFM_CUDA_CHECK(cudaMemsetAsync(hits, 0, sizeof(int) * (n_src + 1), st));
    point_locate_kernel<<<(unsigned)((mesh->nt + 127) / 128), 128, 0, st>>>(mesh->verts, mesh->tets, mesh->nt, r0_d,
                                                                           n_src, tasks, cap, count, hits);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    DFM_CUDA_CHECK(cudaMemcpyAsync(&n_tasks, count, sizeof(int), cudaMemcpyDeviceToHost, st));
    DFM_CUDA_CHECK(cudaMemcpyAsync(hits_h.data(), hits, sizeof(int) * n_src, cudaMemcpyDeviceToHost, st));
    DFM_CUDA_CHECK(cudaStreamSynchronize(st));
    if (n_tasks <= cap) break;
    DFM_CUDA_CHECK(cudaFreeAsync(tasks, st));
    cap = n_tasks;
  }
  if (n_tasks > 0) {
#define CASE(N)                                                                                                  \
  case N:                                                                                                        \
    point_face_kernel<N><<<(unsigned)n_tasks, 128, 0, st>>>(mesh->verts, mesh->tets, mesh->recv, mesh->refl,     \
                                                            mesh->geom, mu, mu_uniform, r0_d, tasks, count, cap, \
                                                            polar ? 1 : 0, nq, glx, glw, strength, mesh->nrows,  \
                                                            rho0);                                               \
    break;
    switch (Np) { CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) }
#undef CASE
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
  }
  DFM_CUDA_CHECK(cudaFreeAsync(tasks, st));
  DFM_CUDA_CHECK(cudaFreeAsync(buf, st));
  for (int s = 0; s < n_src; ++s)
    if (hits_h[s] == 0) return set_error(DFM_ERR_ARG, "dfm_point_source: a source lies outside the mesh");
  return DFM_OK;
}
