// Face matching without any device allocation.
//
// dfm_mesh_create allocates its hash table with cudaMalloc.  Some callers
// cannot allocate device memory when they need the face matching:
// applications that reserve all device memory for their own pool or arena up
// front (an untracked cudaMalloc then fails or fragments the pool), and code
// that runs where the host must not enter the CUDA allocator at all.  This
// variant keeps its hash table in a fixed file-scope device array; the caller
// passes the tets and the output buffer.
//
// The array is a module-level __device__ object: every GPU that loads the
// library holds it (kStaticFaceSlots slots, 16 bytes each, 16 MiB plus a few
// words) until the process exits.  Every call shares it and it keeps the last
// call's contents, so each call re-initialises the table before use; two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the table and must be serialised by the
// caller.
#include <mutex>

#include "dfm_internal.cuh"

namespace dfm {
namespace {

constexpr int64_t kStaticFaceSlots = int64_t(1) << 20;  // hash slots (power of two)
constexpr int64_t kStaticMaxTets = kStaticFaceSlots / 8;  // 4 faces per tet, load factor <= 1/2
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kVertBitsStatic = 21;

struct StaticFaceTable {
  unsigned long long keys[kStaticFaceSlots];
  int32_t rowA[kStaticFaceSlots];
  int32_t rowB[kStaticFaceSlots];
  unsigned long long n_boundary;
  int err;
};

// The scratch itself.  Host code must not pass &g_face_table: in host code the
// name denotes a host-side stand-in, not the device address.
static __device__ __align__(256) StaticFaceTable g_face_table;

constexpr int kErrIndexS = 1, kErrRepeatS = 2, kErrManifoldS = 4, kErrTableS = 8;

__device__ __forceinline__ unsigned long long mix64s(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool face_key_s(const int32_t* __restrict__ tets, int64_t nv, int64_t row,
                                           unsigned long long* key, int* err) {
  const int64_t t = row >> 2;
  const int f = (int)(row & 3);
  int a = tets[4 * t + ((f + 1) & 3)], b = tets[4 * t + ((f + 2) & 3)], c = tets[4 * t + ((f + 3) & 3)];
  if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
    *err |= kErrIndexS;
    return false;
  }
  if (a > b) { int s = a; a = b; b = s; }
  if (b > c) { int s = b; b = c; c = s; }
  if (a > b) { int s = a; a = b; b = s; }
  if (a == b || b == c) {
    *err |= kErrRepeatS;
    return false;
  }
  *key = ((unsigned long long)a << (2 * kVertBitsStatic)) | ((unsigned long long)b << kVertBitsStatic) |
         (unsigned long long)c;
  return true;
}

// Resets the first `slots` entries of the table and its counters.
__global__ void static_table_clear_kernel(StaticFaceTable* T, int64_t slots) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < slots) {
    T->keys[i] = kEmptyKey;
    T->rowA[i] = -1;
    T->rowB[i] = -1;
  }
  if (i == 0) {
    T->n_boundary = 0;
    T->err = 0;
  }
}

__global__ void static_insert_kernel(StaticFaceTable* T, const int32_t* __restrict__ tets, int64_t nv, int64_t nrows,
                                     uint64_t mask) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int err = 0;
  unsigned long long key;
  if (face_key_s(tets, nv, r, &key, &err)) {
    uint64_t h = mix64s(key) & mask;
    bool placed = false;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(&T->keys[h], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) {
        if (atomicCAS(&T->rowA[h], -1, (int32_t)r) != -1 && atomicCAS(&T->rowB[h], -1, (int32_t)r) != -1)
          err |= kErrManifoldS;
        placed = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (!placed) err |= kErrTableS;
  }
  if (err) atomicOr(&T->err, err);
}

__global__ void static_match_kernel(StaticFaceTable* T, const int32_t* __restrict__ tets, int64_t nv, int64_t nrows,
                                    uint64_t mask, int32_t* __restrict__ recv) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int err = 0;
  unsigned long long key;
  int32_t other = -1;
  if (face_key_s(tets, nv, r, &key, &err)) {
    uint64_t h = mix64s(key) & mask;
    bool found = false;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      if (T->keys[h] == key) {
        found = true;
        break;
      }
      h = (h + 1) & mask;
    }
    if (found) {
      const int32_t a = T->rowA[h], b = T->rowB[h];
      other = (a == (int32_t)r) ? b : a;
    } else {
      err |= kErrTableS;
    }
  }
  recv[r] = other >= 0 ? other : (int32_t)r;
  if (other < 0) atomicAdd(&T->n_boundary, 1ull);
  if (err) atomicOr(&T->err, err);
}

// Device address of g_face_table, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
StaticFaceTable* g_addr[kMaxDevices] = {};

int static_table_address(StaticFaceTable** out) {
  int dev = 0;
  DFM_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(DFM_ERR_UNSUPPORTED, "dfm_face_match_static: device id >= 64");
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_face_table);
    if (e != cudaSuccess) return cuda_error(e, "dfm_face_match_static: cudaGetSymbolAddress");
    g_addr[dev] = static_cast<StaticFaceTable*>(p);
  }
  *out = g_addr[dev];
  return DFM_OK;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_face_match_static(const int32_t* tets, int64_t n_verts, int64_t n_tets, int32_t* recv,
                                     int64_t* n_boundary, void* stream) {
  if (!tets || !recv) return set_error(DFM_ERR_ARG, "dfm_face_match_static: tets/recv is NULL");
  if (n_tets < 1 || n_verts < 4) return set_error(DFM_ERR_ARG, "dfm_face_match_static: need >= 1 tet and >= 4 vertices");
  if (n_tets > kStaticMaxTets)
    return set_error(DFM_ERR_ARG, "dfm_face_match_static: at most 131072 tets (fixed 2^20-slot table); use "
                                  "dfm_mesh_create for larger meshes");
  if (n_verts >= (int64_t(1) << kVertBitsStatic))
    return set_error(DFM_ERR_ARG, "dfm_face_match_static: at most 2^21 - 1 vertices are supported");
  StaticFaceTable* T = nullptr;
  int rc = static_table_address(&T);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  const int64_t nrows = 4 * n_tets;
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * nrows)) slots <<= 1;
  const int bs = 256;
  static_table_clear_kernel<<<(unsigned)((slots + bs - 1) / bs), bs, 0, st>>>(T, (int64_t)slots);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  const unsigned grid = (unsigned)((nrows + bs - 1) / bs);
  static_insert_kernel<<<grid, bs, 0, st>>>(T, tets, n_verts, nrows, slots - 1);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  static_match_kernel<<<grid, bs, 0, st>>>(T, tets, n_verts, nrows, slots - 1, recv);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  int err_h = 0;
  unsigned long long nb_h = 0;
  DFM_CUDA_CHECK(cudaMemcpyAsync(&err_h, &T->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFM_CUDA_CHECK(cudaMemcpyAsync(&nb_h, &T->n_boundary, sizeof(nb_h), cudaMemcpyDeviceToHost, st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(st));
  if (err_h & kErrIndexS) return set_error(DFM_ERR_MESH, "dfm_face_match_static: vertex index out of range");
  if (err_h & kErrRepeatS) return set_error(DFM_ERR_MESH, "dfm_face_match_static: a tet repeats a vertex");
  if (err_h & kErrManifoldS)
    return set_error(DFM_ERR_MESH, "dfm_face_match_static: a face is shared by more than two tets");
  if (err_h & kErrTableS) return set_error(DFM_ERR_MESH, "dfm_face_match_static: hash probe limit reached");
  if (n_boundary) *n_boundary = (int64_t)nb_h;
  return DFM_OK;
}
