// Internal declarations shared by the CUDA translation units of libdfm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dfm.h"
#include "launch_geometry.h"

namespace dfm {

// Sets the thread-local error message and returns code.
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* where);

#define DFM_CUDA_CHECK(expr)                                  \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return ::dfm::cuda_error(e_, #expr); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int nbasis(int Np) { return (Np + 1) * (Np + 2) / 2; }

// basis codes of the C ABI (DFM_BASIS): momentum order, spatial functions
// per face, unknowns per row
inline int basis_np(int code) { return code & 0xff; }
inline int basis_ns(int code) { return (code >> 8) == 1 ? 3 : 1; }
inline int basis_size(int code) { return basis_ns(code) * nbasis(basis_np(code)); }
// a valid code: order 0..max_np, spatial basis 0 or 1 (the linear one up to order 8)
inline bool basis_ok(int code, int max_np) {
  const int s = code >> 8, np = code & 0xff;
  return code >= 0 && (s == 0 || s == 1) && np <= max_np && (s == 0 || np <= 8);
}
// the basis sizes the per-warp kernels and preconditioner copies are built for
inline bool narrow_nb(int nb) {
  return nb == 1 || nb == 3 || nb == 6 || nb == 10 || nb == 15 || nb == 21 || nb == 28 || nb == 36 || nb == 45;
}

// Per-row face geometry (FP64), row = 4 t + f.
struct FaceGeom {
  double o[3];   // frame origin (first face vertex)
  double e1[3];  // tangent axis along the first edge
  double e2[3];  // n x e1
  double n[3];   // inward unit normal
  double area;
  double pad[3];
};

}  // namespace dfm

struct dfm_mesh {
  int64_t nv = 0, nt = 0, nrows = 0, nboundary = 0;
  double min_abs_volume = 0, total_volume = 0;
  double* verts = nullptr;        // device [nv][3]
  int32_t* tets = nullptr;        // device [nt][4]
  int32_t* recv = nullptr;        // device [4 nt]
  double* refl = nullptr;         // device [4 nt] reflection coefficient per row
  dfm::FaceGeom* geom = nullptr;  // device [4 nt]
};

struct dfm_op {
  const dfm_mesh* mesh = nullptr;
  int Np = 0, nb = 0, precision = DFM_F32;
  int ns = 1;  // spatial functions per face (1 constant, 3 linear); nb = ns (Np+1)(Np+2)/2
  int64_t nrows = 0, row_stride = 0;
  void* vals = nullptr;  // device
  int64_t bytes = 0;
  // damping of the last assembly: the uniform mu (or -1 for a per-tet field)
  // and the moment k of d^k B / d mu^k it holds
  double mu_uniform = -1.0;
  int moment = 0;
  int* dev_err = nullptr;  // device flag set by kernels whose bounded waits time out
  // heterogeneous media (Sec. 3.3): the blocks reflected at interfaces between
  // different media, an operator of its own whose row R receives from R's own
  // tet (recv = the identity map); applied after this one.  recv: the row map
  // of the applications (NULL: mesh->recv)
  dfm_op* rop = nullptr;
  const int32_t* recv = nullptr;
  int32_t* own_recv = nullptr;  // owned identity map of a reflection operator
  // 16-bit copy of the blocks for inexact preconditioner hops (same layout)
  void* lp_vals = nullptr;
  int64_t lp_bytes = 0;
  int lp_precision = 0;
  bool lp_valid = false;
  bool lp_frag = false;  // fragment-ordered (tensor-core hops) rather than chunk-ordered
  // the same for B^T (transposed solves): row J = 4t + l holds the blocks that
  // column J sends, transposed, in the order of the receiving faces l' != l
  void* lpT_vals = nullptr;
  int64_t lpT_bytes = 0;
  int lpT_precision = 0;
  bool lpT_valid = false;
  bool lpT_frag = false;
  // CUDA graphs of the preconditioner's hop chains, keyed by their shape and
  // buffers (hop.cu); destroyed with the operator
  void* hop_graphs = nullptr;
  // assembly scratch (per-pair constants, Gauss table), grown on demand
  void* work = nullptr;
  int64_t work_bytes = 0;
  // solver workspace (Krylov basis and vectors), grown on demand
  void* swork = nullptr;
  int64_t swork_bytes = 0;
};

namespace dfm {
// launch accounting (stats.cu): every kernel launch site calls count_launch();
// timed sites wrap the launch in a KernelTimer (event pair when enabled).
// Under stream capture (set_capturing) neither counts nor times: a replayed
// graph is counted with count_launches and timed as one span of `weight`
// launches.
void count_launch();
void count_launches(long long n);
void set_capturing(bool on);
class KernelTimer {
 public:
  KernelTimer(int kernel, cudaStream_t st, int weight = 1);
  ~KernelTimer();
 private:
  int kernel_;
  cudaStream_t st_;
  int e0_;
  int weight_;
};
#define DFM_LAUNCHED() ::dfm::count_launch()

// row stride (elements) of the block storage: 3 nb^2 rounded up to 8 elements
inline int64_t op_row_stride(int nb) { return geom::op_row_stride(nb); }
inline int elem_size(int precision) { return precision == DFM_F64 ? 8 : (precision == DFM_F32 ? 4 : 2); }

// implemented in spmv.cu
int apply_impl(const dfm_op* op, const void* x, const void* x0, void* y, int R, double alpha, int trans, int xtype,
               cudaStream_t st);
int apply_combo_impl(const dfm_op* const* ops, int K, const double* coef, const void* x, const void* x0, void* y,
                     int R, double alpha, int xtype, cudaStream_t st);
// 16-bit copy of op's blocks (made on first use after each assembly); returns a
// view operator that applies it (same mesh, layout and error flag)
// Consecutive applications of one operator alternate the direction in which
// they sweep its rows (0 or 1 for this launch; state kept per values buffer);
// forget_sweep drops the state of a buffer that is being freed.
int next_sweep_direction(const void* vals);
void forget_sweep(const void* vals);
// Polynomial-preconditioner hops on a 16-bit copy of the blocks (hop.cu).
// Padded width of a face's coefficients in hop vectors and in the copy.
inline int hop_nbp(int nb) { return geom::hop_nbp(nb); }
// (re)builds op->lp_vals (trans: op->lpT_vals) in precision DFM_F16, DFM_BF16
// or DFM_FP8E4M3 from the FP32 or BF16 blocks, in the layout that hops with R
// right-hand sides per launch group run fastest on
int prepare_lowp(const dfm_op* op, int precision, cudaStream_t st, int trans, int R);
// the forward (trans = 0) or transposed copy of op
struct LowpView {
  const void* vals;
  int precision;
  bool valid;
  bool frag;
};
inline LowpView lowp_of(const dfm_op* op, int trans) {
  return trans ? LowpView{op->lpT_vals, op->lpT_precision, op->lpT_valid, op->lpT_frag}
               : LowpView{op->lp_vals, op->lp_precision, op->lp_valid, op->lp_frag};
}
// z = sum_{k<d} B~^k v for R vectors ([R][rows][nb] FP32) by Horner on the
// low-precision copy (trans: B~^T on the transposed copy); vp, ha, hb: 16-byte-aligned scratch of R rows NBP floats
// each.  FP16/e4m3 copies run on FP16 vectors holding v * vscale (a power of
// two that keeps |v| vscale <= 2^-8).
int hop_horner(const dfm_op* op, int R, int d, const float* v, float* z, void* vp, void* ha, void* hb, float vscale,
               cudaStream_t st, int trans = 0);
// frees the operator's cached hop-chain graphs (hop.cu)
void destroy_hop_graphs(dfm_op* op);
// tensor-core forward application of a BF16 operator to R >= 4 FP32
// right-hand sides (spmv_mma.cu)
bool apply_mma_supported(const dfm_op* op, int R);
int apply_mma(const dfm_op* op, const float* x, const float* x0, float* y, int R, double alpha, cudaStream_t st);
// reads and clears op's time-out flag (waits on st): DFM_ERR_TIMEOUT if set
int read_timeout_flag(const dfm_op* op, cudaStream_t st, const char* who);
// bases above N_p = 8 (wide.cu).  pairs: the assembly's per-pair constants
// (PairConst of node.cuh); vals FP32.
int launch_assemble_wide(int Np, const void* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                         float cos_max, float* vals, int64_t row_stride, unsigned long long* nodes, int moment,
                         cudaStream_t st);
// the linear spatial basis (3 functions per face, N_p <= 8): pos_scratch holds
// 8 bytes per pair (vertex positions), 8-byte aligned
int launch_assemble_p1(const dfm_mesh* mesh, int Np, const void* pairs, void* pos_scratch, int64_t npairs,
                       const double* glx, const double* glw, int q, float cos_max, float* vals, int64_t row_stride,
                       unsigned long long* nodes, cudaStream_t st);
int apply_wide(const dfm_op* op, const float* x, const float* x0, float* y, int R, double alpha, cudaStream_t st);
int apply_wide(const dfm_op* op, const double* x, const double* x0, double* y, int R, double alpha, cudaStream_t st);
// stride: unknowns per row of rho0 (3 (Np+1)(Np+2)/2 with the linear spatial basis)
int launch_directed_source_wide(int Np, const FaceGeom* geom, const int64_t* rows, const double* dirs, int n_src,
                                int64_t nrows, int combine, double* rho0, int* bad, int stride, cudaStream_t st);
// ns spatial functions per face (1, or 3 for the linear spatial basis)
int launch_interior_density_wide(int Np, int ns, bool polar, const dfm_mesh* mesh, const double* mu,
                                 double mu_uniform, const int64_t* list, const double* weights, int n,
                                 const double* glx, const double* glw, int nq, double* gvec, double* dgvec,
                                 cudaStream_t st);
// implemented in quad.cu
int gauss_legendre_device(int q, double* x, double* w, cudaStream_t st);
}  // namespace dfm
