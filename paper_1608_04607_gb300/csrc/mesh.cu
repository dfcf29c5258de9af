// Mesh set-up: face matching on the device and per-face geometry.
//
// The operator couples a tet face only to the faces of the same tet and,
// through an interior face, to the neighbour across it (Sec. 2: the flow map
// phi_ij only reaches neighbouring tetrahedra, so B is sparse).  The
// neighbour of every face is found with an open-addressing hash on the sorted
// vertex triple; the face frames of Sec. 3.3 are built in FP64.
#include <math.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "dfm_internal.cuh"

namespace dfm {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  return set_error(e == cudaErrorMemoryAllocation ? DFM_ERR_OOM : DFM_ERR_CUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kVertBits = 21;  // vertex ids < 2^21 packed three to a 63-bit key

// error bits written by the kernels
constexpr int kErrIndex = 1;      // vertex index out of range
constexpr int kErrRepeat = 2;     // repeated vertex in a tet
constexpr int kErrManifold = 4;   // face shared by more than two tets
constexpr int kErrTable = 8;      // hash probe limit reached

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool face_key(const int32_t* __restrict__ tets, int64_t nv, int64_t row,
                                         unsigned long long* key, int* err) {
  const int64_t t = row >> 2;
  const int f = (int)(row & 3);
  int a = tets[4 * t + ((f + 1) & 3)], b = tets[4 * t + ((f + 2) & 3)], c = tets[4 * t + ((f + 3) & 3)];
  if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
    *err |= kErrIndex;
    return false;
  }
  if (a > b) { int s = a; a = b; b = s; }
  if (b > c) { int s = b; b = c; c = s; }
  if (a > b) { int s = a; a = b; b = s; }
  if (a == b || b == c) {
    *err |= kErrRepeat;
    return false;
  }
  *key = ((unsigned long long)a << (2 * kVertBits)) | ((unsigned long long)b << kVertBits) | (unsigned long long)c;
  return true;
}

__global__ void face_insert_kernel(const int32_t* __restrict__ tets, int64_t nv, int64_t nrows,
                                   unsigned long long* keys, int32_t* rowA, int32_t* rowB, uint64_t mask,
                                   int* err_flag) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int err = 0;
  unsigned long long key;
  if (face_key(tets, nv, r, &key, &err)) {
    uint64_t h = mix64(key) & mask;
    bool placed = false;
    for (uint64_t probe = 0; probe <= mask; ++probe) {  // bounded: at most the table size
      unsigned long long prev = atomicCAS(&keys[h], kEmpty, key);
      if (prev == kEmpty || prev == key) {
        if (atomicCAS(&rowA[h], -1, (int32_t)r) != -1 && atomicCAS(&rowB[h], -1, (int32_t)r) != -1)
          err |= kErrManifold;
        placed = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!placed) err |= kErrTable;
  }
  if (err) atomicOr(err_flag, err);
}

__global__ void face_match_kernel(const int32_t* __restrict__ tets, int64_t nv, int64_t nrows,
                                  const unsigned long long* __restrict__ keys, const int32_t* __restrict__ rowA,
                                  const int32_t* __restrict__ rowB, uint64_t mask, int32_t* recv,
                                  unsigned long long* nboundary, int* err_flag) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int err = 0;
  unsigned long long key;
  int32_t other = -1;
  if (face_key(tets, nv, r, &key, &err)) {
    uint64_t h = mix64(key) & mask;
    bool found = false;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      if (keys[h] == key) {
        found = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (found) {
      const int32_t a = rowA[h], b = rowB[h];
      other = (a == (int32_t)r) ? b : a;
    } else {
      err |= kErrTable;
    }
  }
  recv[r] = other >= 0 ? other : (int32_t)r;
  if (other < 0) atomicAdd(nboundary, 1ull);
  if (err) atomicOr(err_flag, err);
}

__device__ __forceinline__ void load3(const double* V, int64_t i, double* p) {
  p[0] = V[3 * i];
  p[1] = V[3 * i + 1];
  p[2] = V[3 * i + 2];
}

// One thread per row: FP64 face frame and area; the f == 0 thread also
// stores the tet volume.
__global__ void face_geometry_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets, int64_t nrows,
                                     FaceGeom* __restrict__ geom, double* __restrict__ vol) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t t = r >> 2;
  const int f = (int)(r & 3);
  double p0[3], p1[3], p2[3], ap[3];
  load3(V, tets[4 * t + ((f + 1) & 3)], p0);
  load3(V, tets[4 * t + ((f + 2) & 3)], p1);
  load3(V, tets[4 * t + ((f + 3) & 3)], p2);
  load3(V, tets[4 * t + f], ap);
  double a[3], b[3], h[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = p1[k] - p0[k];
    b[k] = p2[k] - p0[k];
    h[k] = ap[k] - p0[k];
  }
  double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  const double det = c[0] * h[0] + c[1] * h[1] + c[2] * h[2];
  const double s = (det < 0 ? -1.0 : 1.0) / cn;
  const double an = 1.0 / sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  FaceGeom g;
  for (int k = 0; k < 3; ++k) {
    g.o[k] = p0[k];
    g.n[k] = c[k] * s;
    g.e1[k] = a[k] * an;
  }
  g.e2[0] = g.n[1] * g.e1[2] - g.n[2] * g.e1[1];
  g.e2[1] = g.n[2] * g.e1[0] - g.n[0] * g.e1[2];
  g.e2[2] = g.n[0] * g.e1[1] - g.n[1] * g.e1[0];
  g.area = 0.5 * cn;
  g.pad[0] = g.pad[1] = g.pad[2] = 0.0;
  geom[r] = g;
  if (f == 0) vol[t] = det / 6.0;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" const char* dfm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* dfm_version(void) { return "dfm-gb300 0.1 (sm_103a)"; }

extern "C" void dfm_mesh_destroy(dfm_mesh* m) {
  if (!m) return;
  cudaFree(m->verts);
  cudaFree(m->tets);
  cudaFree(m->recv);
  cudaFree(m->refl);
  cudaFree(m->geom);
  delete m;
}

extern "C" int dfm_mesh_create(const double* verts, int64_t n_verts, const int32_t* tets, int64_t n_tets,
                               const double* refl, double refl_default, void* stream, dfm_mesh** out) {
  if (!out) return set_error(DFM_ERR_ARG, "dfm_mesh_create: out is NULL");
  *out = nullptr;
  if (!verts || !tets) return set_error(DFM_ERR_ARG, "dfm_mesh_create: verts/tets is NULL");
  if (n_verts < 4 || n_tets < 1) return set_error(DFM_ERR_ARG, "dfm_mesh_create: need >= 4 vertices and >= 1 tet");
  if (n_verts >= (int64_t(1) << kVertBits))
    return set_error(DFM_ERR_ARG, "dfm_mesh_create: at most 2^21 - 1 vertices are supported");
  if (n_tets > (int64_t(1) << 28)) return set_error(DFM_ERR_ARG, "dfm_mesh_create: too many tets");
  const int64_t nrows = 4 * n_tets;
  std::vector<double> refl_h(nrows, refl_default);
  if (refl)
    for (int64_t i = 0; i < nrows; ++i) refl_h[i] = refl[i];
  for (int64_t i = 0; i < nrows; ++i)
    if (!(refl_h[i] >= 0.0 && refl_h[i] <= 1.0))
      return set_error(DFM_ERR_ARG, "dfm_mesh_create: reflection coefficients must lie in [0, 1]");
  for (int64_t i = 0; i < 3 * n_verts; ++i)
    if (!isfinite(verts[i])) return set_error(DFM_ERR_NONFINITE, "dfm_mesh_create: non-finite vertex coordinate");

  cudaStream_t st = as_stream(stream);
  dfm_mesh* m = new dfm_mesh();
  m->nv = n_verts;
  m->nt = n_tets;
  m->nrows = nrows;
  unsigned long long* keys = nullptr;
  int32_t *rowA = nullptr, *rowB = nullptr;
  int* err_d = nullptr;
  unsigned long long* nb_d = nullptr;
  double* vol_d = nullptr;
  uint64_t tsize = 1;
  while (tsize < (uint64_t)(2 * nrows)) tsize <<= 1;
  auto fail = [&](int code) {
    cudaFree(keys); cudaFree(rowA); cudaFree(rowB); cudaFree(err_d); cudaFree(nb_d); cudaFree(vol_d);
    dfm_mesh_destroy(m);
    return code;
  };
#define TRY(expr)                                              \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return fail(cuda_error(e_, #expr)); \
  } while (0)
  TRY(cudaMalloc(&m->verts, sizeof(double) * 3 * n_verts));
  TRY(cudaMalloc(&m->tets, sizeof(int32_t) * 4 * n_tets));
  TRY(cudaMalloc(&m->recv, sizeof(int32_t) * nrows));
  TRY(cudaMalloc(&m->refl, sizeof(double) * nrows));
  TRY(cudaMalloc(&m->geom, sizeof(FaceGeom) * nrows));
  TRY(cudaMalloc(&keys, sizeof(unsigned long long) * tsize));
  TRY(cudaMalloc(&rowA, sizeof(int32_t) * tsize));
  TRY(cudaMalloc(&rowB, sizeof(int32_t) * tsize));
  TRY(cudaMalloc(&err_d, sizeof(int)));
  TRY(cudaMalloc(&nb_d, sizeof(unsigned long long)));
  TRY(cudaMalloc(&vol_d, sizeof(double) * n_tets));
  TRY(cudaMemcpyAsync(m->verts, verts, sizeof(double) * 3 * n_verts, cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(m->tets, tets, sizeof(int32_t) * 4 * n_tets, cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(m->refl, refl_h.data(), sizeof(double) * nrows, cudaMemcpyHostToDevice, st));
  TRY(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * tsize, st));
  TRY(cudaMemsetAsync(rowA, 0xFF, sizeof(int32_t) * tsize, st));
  TRY(cudaMemsetAsync(rowB, 0xFF, sizeof(int32_t) * tsize, st));
  TRY(cudaMemsetAsync(err_d, 0, sizeof(int), st));
  TRY(cudaMemsetAsync(nb_d, 0, sizeof(unsigned long long), st));
  const int bs = 256;
  const unsigned grid = (unsigned)((nrows + bs - 1) / bs);
  face_insert_kernel<<<grid, bs, 0, st>>>(m->tets, n_verts, nrows, keys, rowA, rowB, tsize - 1, err_d);
  DFM_LAUNCHED();
  TRY(cudaGetLastError());
  face_match_kernel<<<grid, bs, 0, st>>>(m->tets, n_verts, nrows, keys, rowA, rowB, tsize - 1, m->recv, nb_d, err_d);
  DFM_LAUNCHED();
  TRY(cudaGetLastError());
  face_geometry_kernel<<<grid, bs, 0, st>>>(m->verts, m->tets, nrows, m->geom, vol_d);
  DFM_LAUNCHED();
  TRY(cudaGetLastError());
  int err_h = 0;
  unsigned long long nb_h = 0;
  std::vector<double> vol_h(n_tets);
  TRY(cudaMemcpyAsync(&err_h, err_d, sizeof(int), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&nb_h, nb_d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(vol_h.data(), vol_d, sizeof(double) * n_tets, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (err_h & kErrIndex) return fail(set_error(DFM_ERR_MESH, "dfm_mesh_create: vertex index out of range"));
  if (err_h & kErrRepeat) return fail(set_error(DFM_ERR_MESH, "dfm_mesh_create: a tet repeats a vertex"));
  if (err_h & kErrManifold)
    return fail(set_error(DFM_ERR_MESH, "dfm_mesh_create: a face is shared by more than two tets"));
  if (err_h & kErrTable) return fail(set_error(DFM_ERR_MESH, "dfm_mesh_create: face hash probe limit reached"));
  double vmin = INFINITY, vsum = 0.0;
  for (int64_t t = 0; t < n_tets; ++t) {
    vmin = fmin(vmin, fabs(vol_h[t]));
    vsum += fabs(vol_h[t]);
  }
  if (!(vmin > 1e-14 * vsum / (double)n_tets))
    return fail(set_error(DFM_ERR_MESH, "dfm_mesh_create: a tet has (near) zero volume"));
  m->nboundary = (int64_t)nb_h;
  m->min_abs_volume = vmin;
  m->total_volume = vsum;
  cudaFree(keys); cudaFree(rowA); cudaFree(rowB); cudaFree(err_d); cudaFree(nb_d); cudaFree(vol_d);
  *out = m;
  return DFM_OK;
#undef TRY
}

extern "C" int dfm_mesh_info(const dfm_mesh* m, dfm_mesh_info_t* info) {
  if (!m || !info) return set_error(DFM_ERR_ARG, "dfm_mesh_info: NULL argument");
  info->n_verts = m->nv;
  info->n_tets = m->nt;
  info->n_rows = m->nrows;
  info->n_boundary_rows = m->nboundary;
  info->min_abs_volume = m->min_abs_volume;
  info->total_volume = m->total_volume;
  return DFM_OK;
}

extern "C" int dfm_mesh_recv(const dfm_mesh* m, int32_t* recv_host) {
  if (!m || !recv_host) return set_error(DFM_ERR_ARG, "dfm_mesh_recv: NULL argument");
  DFM_CUDA_CHECK(cudaMemcpy(recv_host, m->recv, sizeof(int32_t) * m->nrows, cudaMemcpyDeviceToHost));
  return DFM_OK;
}
