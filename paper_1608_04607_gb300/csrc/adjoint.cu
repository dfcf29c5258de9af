// Adjoint gradient of a receiver functional with respect to per-tet damping,
// and the interior density functional it is built from (Sec. 4.1, Eq. IntDens).
//
// J(rho) = g . rho with (I - B) rho = rho0.  With (I - B)^T lambda = g,
//   dJ/dmu_t = lambda^T (dB/dmu_t) rho + (dg/dmu_t) . rho.
// B depends on mu_t only through the damped areas S = 2 |OBC| phi2(mu L_O) of
// the 12 face pairs of tet t (Sec. 3.3), so
//   dB/dmu_t (pair) = lambda_pair N_{n'm'} / sqrt(|T_l||T_l'|) sum_nodes w J 2|OBC| L_O phi2'(mu L_O) Z(p') Z(p)^T.
// The contraction lambda_R^T dB rho_J is computed on the fly: per node the
// scalar c = w' (Z(p') . lambda_s) is accumulated into u = sum c Z(p), and the
// pair contributes u . rho_J for every right-hand side; dB is never formed.
#include <math.h>

#include <algorithm>
#include <vector>

#include "dfm_internal.cuh"
#include "interior_rule.cuh"
#include "node.cuh"

namespace dfm {
namespace {

constexpr int kCWarps = 4;  // face pairs per block in the contraction kernel

template <int NP>
__global__ void __launch_bounds__(kCWarps * 32)
contract_kernel(const PairConst* __restrict__ pairs, int64_t npairs, const double* __restrict__ gl_x,
                const double* __restrict__ gl_w, int q, float cos_max, const double* __restrict__ lam,
                const double* __restrict__ rho, int R, int64_t nrows, int64_t nt, double* __restrict__ dJ) {
  constexpr int NB = (NP + 1) * (NP + 2) / 2;
  __shared__ PatchSmem smem[kCWarps];
  __shared__ float s_lam[kCWarps][NB];
  __shared__ float s_x[kMaxQ], s_w[kMaxQ];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  PatchSmem& S = smem[wid];
  if (threadIdx.x < q) {
    s_x[threadIdx.x] = (float)gl_x[threadIdx.x];
    s_w[threadIdx.x] = (float)gl_w[threadIdx.x];
  }
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * kCWarps + wid;
  if (p >= npairs) return;  // no block-wide barrier follows
  const PairConst pc = pairs[p];
  if (pc.kind < 0) return;  // no block for this pair in this part
  const int64_t t = p / 12;
  const int f = (int)((p % 12) / 3);
  const int64_t J = 4 * t + f;
  // lambda of the receiving row, scaled by the test-side normalisation
  for (int a = lane; a < NB; a += 32)
    s_lam[wid][a] = (float)(lam[(int64_t)pc.out_row * NB + a] * (double)pc.scale * (double)zernike_invnorm(a));
  if (lane == 0) {
    S.sp = 0;
    for (int r = 3; r >= 0; --r) region_poly(pc, r, S.stack[S.sp++]);
  }
  __syncwarp();
  const float mu = pc.mu;
  const int qq = q * q;
  float u[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) u[b] = 0.f;
  while (true) {
    if (lane == 0) fill_patches(S, cos_max);
    __syncwarp();
    const int npatch = S.npatch;
    if (npatch == 0) break;
    const int nodes = npatch * qq;
    for (int k = lane; k < nodes; k += 32) {
      const int pi = k / qq;
      const int rem = k - pi * qq;
      const int i = rem / q;
      const int j = rem - i * q;
      const NodeGeom<float> g = node_geom<float>(S.patch[pi], s_x[i], s_x[j], pc);
      if (!g.valid) continue;
      const float wd = s_w[i] * s_w[j] * g.jac * 2.f * g.Anab * g.LO * phi2_prime<float>(mu * g.LO) *
                       media_weight<float>(pc, g.d0, g.d1, g.d2);
      float Zp[NB], Zq[NB];
      zernike<NP, float>(g.d0, g.d1, Zp);
      const float qx = pc.qscale * (g.d0 * pc.R1[0] + g.d1 * pc.R1[1] + g.d2 * pc.R1[2]);
      const float qy = pc.qscale * (g.d0 * pc.R2[0] + g.d1 * pc.R2[1] + g.d2 * pc.R2[2]);
      zernike<NP, float>(qx, qy, Zq);
      float sq = 0.f;
#pragma unroll
      for (int a = 0; a < NB; ++a) sq = fmaf(Zq[a], s_lam[wid][a], sq);
      const float c = wd * sq;
#pragma unroll
      for (int b = 0; b < NB; ++b) u[b] = fmaf(c, Zp[b], u[b]);
    }
    __syncwarp();
  }
  // butterfly reduction: every lane ends with the warp's u
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u[b] += __shfl_xor_sync(0xffffffffu, u[b], o);
  for (int r = lane; r < R; r += 32) {
    const double* x = rho + ((int64_t)r * nrows + J) * NB;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < NB; ++b) s = fma((double)u[b], x[b], s);
    atomicAdd(&dJ[(int64_t)r * nt + t], s);
  }
}

// dJ[r][t] += sum_{l,a} dg[4t+l][a] rho_r[4t+l][a]  (rows with dg == 0 are skipped)
__global__ void explicit_term_kernel(const double* __restrict__ dg, const double* __restrict__ rho, int R, int nb,
                                     int64_t nrows, int64_t nt, double* __restrict__ dJ) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* d = dg + 4 * t * nb;
  bool any = false;
  for (int i = 0; i < 4 * nb; ++i) any |= (d[i] != 0.0);
  if (!any) return;
  for (int r = 0; r < R; ++r) {
    const double* x = rho + ((int64_t)r * nrows + 4 * t) * nb;
    double s = 0.0;
    for (int i = 0; i < 4 * nb; ++i) s = fma(d[i], x[i], s);
    dJ[(int64_t)r * nt + t] += s;
  }
}

// Interior density coefficients at the centroid of tet e (Eq. IntDens), FP64.
// One warp per (listed tet, face): collapsed tensor Gauss on the face.
template <int NP>
__global__ void interior_density_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets,
                                        const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet,
                                        double mu_uniform, const int64_t* __restrict__ list,
                                        const double* __restrict__ weights, int n, const double* __restrict__ gl_x,
                                        const double* __restrict__ gl_w, int nq, double* __restrict__ gvec,
                                        double* __restrict__ dgvec) {
  constexpr int NB = (NP + 1) * (NP + 2) / 2;
  const int lane = threadIdx.x & 31;
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wg >= 4 * (int64_t)n) return;
  const int i = (int)(wg >> 2);
  const int l = (int)(wg & 3);
  const int64_t e = list[i];
  const double wt = weights ? weights[i] : 1.0;
  const int32_t* tv = tets + 4 * e;
  double r[3] = {0, 0, 0};
  for (int v = 0; v < 4; ++v)
    for (int c = 0; c < 3; ++c) r[c] += 0.25 * V[3 * (int64_t)tv[v] + c];
  const FaceGeom F = geom[4 * e + l];
  double p[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) p[k][c] = V[3 * (int64_t)tv[(l + 1 + k) & 3] + c];
  const double mu = mu_tet ? mu_tet[e] : mu_uniform;
  double g[NB], dg[NB], Z[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) g[a] = dg[a] = 0.0;
  for (int k = lane; k < nq * nq; k += 32) {
    const int ii = k / nq, jj = k - ii * nq;
    const double u = 0.5 * (1.0 + gl_x[ii]);
    const double v = (1.0 - u) * 0.5 * (1.0 + gl_x[jj]);
    const double w = gl_w[ii] * gl_w[jj] * 0.25 * (1.0 - u) * 2.0 * F.area;
    double rs[3];
    for (int c = 0; c < 3; ++c) rs[c] = r[c] - (p[0][c] + u * (p[1][c] - p[0][c]) + v * (p[2][c] - p[0][c]));
    const double dist = sqrt(rs[0] * rs[0] + rs[1] * rs[1] + rs[2] * rs[2]);
    const double id = 1.0 / dist;
    const double d0 = rs[0] * id, d1 = rs[1] * id, d2 = rs[2] * id;
    const double cosv = d0 * F.n[0] + d1 * F.n[1] + d2 * F.n[2];
    const double ker = w * cosv * exp(-mu * dist) * id * id;
    zernike<NP, double>(d0 * F.e1[0] + d1 * F.e1[1] + d2 * F.e1[2], d0 * F.e2[0] + d1 * F.e2[1] + d2 * F.e2[2], Z);
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      g[a] = fma(ker, Z[a], g[a]);
      dg[a] = fma(-dist * ker, Z[a], dg[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g[a] += __shfl_xor_sync(0xffffffffu, g[a], o);
      dg[a] += __shfl_xor_sync(0xffffffffu, dg[a], o);
    }
  if (lane == 0) {
    const double s = wt / sqrt(F.area);
    for (int a = 0; a < NB; ++a) {
      atomicAdd(&gvec[(4 * e + l) * NB + a], s * g[a]);
      if (dgvec) atomicAdd(&dgvec[(4 * e + l) * NB + a], s * dg[a]);
    }
  }
}

int launch_contract(int Np, const PairConst* pairs, int64_t npairs, const double* glx, const double* glw, int q,
                    float cos_max, const double* lam, const double* rho, int R, int64_t nrows, int64_t nt, double* dJ,
                    cudaStream_t st) {
  const unsigned blocks = (unsigned)((npairs + kCWarps - 1) / kCWarps);
  ::dfm::KernelTimer timer_(DFM_KERNEL_CONTRACT, st);
#define CASE(N)                                                                                                \
  case N:                                                                                                      \
    contract_kernel<N><<<blocks, kCWarps * 32, 0, st>>>(pairs, npairs, glx, glw, q, cos_max, lam, rho, R, nrows, \
                                                        nt, dJ);                                               \
    break;
  switch (Np) {
    CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    default: return set_error(DFM_ERR_ARG, "dfm_adjoint: Np must be in 0..8");
  }
#undef CASE
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

// The same functional with the split polar rule of interior_rule.cuh (6 nq^2
// nodes per face), which stays accurate when the centroid is close to a face.
template <int NP>
__global__ void interior_density_polar_kernel(const double* __restrict__ V, const int32_t* __restrict__ tets,
                                              const FaceGeom* __restrict__ geom, const double* __restrict__ mu_tet,
                                              double mu_uniform, const int64_t* __restrict__ list,
                                              const double* __restrict__ weights, int n,
                                              const double* __restrict__ gl_x, const double* __restrict__ gl_w,
                                              int nq, double* __restrict__ gvec, double* __restrict__ dgvec) {
  constexpr int NB = (NP + 1) * (NP + 2) / 2;
  const int lane = threadIdx.x & 31;
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wg >= 4 * (int64_t)n) return;
  const int i = (int)(wg >> 2);
  const int l = (int)(wg & 3);
  const int64_t e = list[i];
  const double wt = weights ? weights[i] : 1.0;
  const int32_t* tv = tets + 4 * e;
  double r[3] = {0, 0, 0};
  for (int v = 0; v < 4; ++v)
    for (int c = 0; c < 3; ++c) r[c] += 0.25 * V[3 * (int64_t)tv[v] + c];
  const FaceGeom F = geom[4 * e + l];
  double p[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) p[k][c] = V[3 * (int64_t)tv[(l + 1 + k) & 3] + c];
  const double mu = mu_tet ? mu_tet[e] : mu_uniform;
  double g[NB], dg[NB], Z[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) g[a] = dg[a] = 0.0;
  const int nodes = 6 * nq * nq;
  for (int k = lane; k < nodes; k += 32) {
    const rule::PolarNode q = rule::polar_node(p, F.n, F.e1, F.e2, r, nq, k, gl_x, gl_w);
    if (q.w == 0.0) continue;
    const double ker = q.w * exp(-mu * q.R);
    zernike<NP, double>(q.dx, q.dy, Z);
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      g[a] = fma(ker, Z[a], g[a]);
      dg[a] = fma(-q.R * ker, Z[a], dg[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g[a] += __shfl_xor_sync(0xffffffffu, g[a], o);
      dg[a] += __shfl_xor_sync(0xffffffffu, dg[a], o);
    }
  if (lane == 0) {
    const double s = wt / sqrt(F.area);
    for (int a = 0; a < NB; ++a) {
      atomicAdd(&gvec[(4 * e + l) * NB + a], s * g[a]);
      if (dgvec) atomicAdd(&dgvec[(4 * e + l) * NB + a], s * dg[a]);
    }
  }
}

// out[r][e] = sum over tet e's four rows of gvec . rho_r: one warp per (r, e),
// the lanes striding over the 4 nb contiguous coefficients of the tet
__global__ void tet_density_kernel(const double* __restrict__ g, const double* __restrict__ rho, int64_t nt,
                                   int nb, int64_t units, double* __restrict__ out) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= units) return;  // blockDim is a multiple of 32: whole warps leave together
  const int64_t r = w / nt, e = w - r * nt;
  const double* gp = g + 4 * e * nb;
  const double* xp = rho + (r * 4 * nt + 4 * e) * nb;
  double acc = 0.0;
  for (int k = lane; k < 4 * nb; k += 32) acc = fma(gp[k], xp[k], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[w] = acc;
}

}  // namespace
}  // namespace dfm

using namespace dfm;

extern "C" int dfm_interior_density(const dfm_mesh* mesh, int Np, const double* mu, double mu_uniform,
                                    const int64_t* tets_host, const double* weights_host, int n, int nq, double* gvec,
                                    double* dgvec, void* stream) {
  if (!mesh || !tets_host || !gvec || n < 1 || !basis_ok(Np, geom::kWideMaxNp))
    return set_error(DFM_ERR_ARG, "dfm_interior_density: bad argument");
  const int ns = basis_ns(Np);
  Np = basis_np(Np);
  // nq < 0: the split polar rule with |nq| points per direction; nq = 0: the
  // same rule with 24 points (accurate for centroids close to a face, as on
  // thin tets); nq > 0: the flat collapsed Gauss rule of that order
  if (nq == 0) nq = -24;
  const bool polar = nq < 0;
  if (polar) nq = -nq;
  if (nq < 2 || nq > 64) return set_error(DFM_ERR_ARG, "dfm_interior_density: |nq| must be in 2..64");
  if (!mu && !(mu_uniform >= 0)) return set_error(DFM_ERR_ARG, "dfm_interior_density: mu_uniform must be >= 0");
  for (int i = 0; i < n; ++i)
    if (tets_host[i] < 0 || tets_host[i] >= mesh->nt) return set_error(DFM_ERR_ARG, "dfm_interior_density: bad tet id");
  cudaStream_t st = as_stream(stream);
  // small stream-ordered scratch: tet list, weights, Gauss table
  char* buf = nullptr;
  const size_t bytes = sizeof(int64_t) * n + sizeof(double) * n + 2 * 64 * sizeof(double) + 256;
  DFM_CUDA_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, st));
  int64_t* list = reinterpret_cast<int64_t*>(buf);
  double* w = reinterpret_cast<double*>(buf + sizeof(int64_t) * n);
  double* glx = w + n;
  double* glw = glx + 64;
  DFM_CUDA_CHECK(cudaMemcpyAsync(list, tets_host, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  if (weights_host) DFM_CUDA_CHECK(cudaMemcpyAsync(w, weights_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  int rc = gauss_legendre_device(nq, glx, glw, st);
  if (rc) return rc;
  const int64_t threads = 4 * (int64_t)n * 32;
  const unsigned blocks = (unsigned)((threads + 127) / 128);
  const double* wp = weights_host ? w : nullptr;
#define CASE(N)                                                                                                  \
  case N:                                                                                                        \
    if (polar)                                                                                                   \
      interior_density_polar_kernel<N><<<blocks, 128, 0, st>>>(mesh->verts, mesh->tets, mesh->geom, mu,         \
                                                               mu_uniform, list, wp, n, glx, glw, nq, gvec,     \
                                                               dgvec);                                           \
    else                                                                                                         \
      interior_density_kernel<N><<<blocks, 128, 0, st>>>(mesh->verts, mesh->tets, mesh->geom, mu, mu_uniform, list, \
                                                         wp, n, glx, glw, nq, gvec, dgvec);                      \
    break;
  switch (ns == 1 ? Np : -1) {
    CASE(0) CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    default:  // Np = 9..20, and the linear spatial basis (wide.cu)
      rc = launch_interior_density_wide(Np, ns, polar, mesh, mu, mu_uniform, list, wp, n, glx, glw, nq, gvec, dgvec,
                                        st);
      if (rc) {
        cudaFreeAsync(buf, st);
        return rc;
      }
  }
#undef CASE
  if (Np <= 8 && ns == 1) DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  DFM_CUDA_CHECK(cudaFreeAsync(buf, st));
  return DFM_OK;
}

extern "C" int dfm_tet_density(const dfm_mesh* mesh, int Np, const double* gvec, const double* rho, int R,
                               double* out, void* stream) {
  if (!mesh || !gvec || !rho || !out || R < 1 || !basis_ok(Np, geom::kWideMaxNp))
    return set_error(DFM_ERR_ARG, "dfm_tet_density: bad argument");
  const int64_t units = (int64_t)R * mesh->nt;
  const int64_t blocks = (units + 7) / 8;  // 8 warps per block
  if (blocks > 0x7fffffff) return set_error(DFM_ERR_ARG, "dfm_tet_density: too many right-hand sides");
  cudaStream_t st = as_stream(stream);
  tet_density_kernel<<<(unsigned)blocks, 256, 0, st>>>(gvec, rho, mesh->nt, basis_size(Np), units, out);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

extern "C" int dfm_adjoint(const dfm_op* op, const dfm_params* params, const double* rho, int R, const double* gvec,
                           const double* dgvec, double* lambda_out, double* dJ_dmu, const dfm_solve_opts* opts,
                           void* stream, dfm_solve_info* info) {
  if (!op || !params || !rho || !gvec || !lambda_out || !dJ_dmu || !opts || R < 1)
    return set_error(DFM_ERR_ARG, "dfm_adjoint: bad argument");
  if (basis_np(params->Np) != op->Np || basis_ns(params->Np) != op->ns)
    return set_error(DFM_ERR_ARG, "dfm_adjoint: params->Np differs from the operator's");
  if (op->Np > 8 || op->ns > 1)
    return set_error(DFM_ERR_UNSUPPORTED,
                     "dfm_adjoint: the dB/dmu contraction is built for Np <= 8 and the piecewise-constant basis");
  const dfm_mesh* mesh = op->mesh;
  cudaStream_t st = as_stream(stream);
  // 1. adjoint equation (I - B)^T lambda = g
  dfm_solve_opts o = *opts;
  o.transpose = 1;
  o.use_x0 = opts->use_x0 ? 1 : 0;  // lambda_out holds the initial guess
  int rc = dfm_solve(op, gvec, 1, lambda_out, &o, stream, info);
  if (rc != DFM_OK && rc != DFM_ERR_NOT_CONVERGED) return rc;
  const int solve_rc = rc;
  // 2. per-pair constants for the operator's damping, then the fused contraction
  const int q = params->quad_order ? params->quad_order : params->Np + 6;
  if (q < 1 || q > kMaxQ) return set_error(DFM_ERR_ARG, "dfm_adjoint: quad_order must be in 1..32");
  const double deg = params->max_patch_deg > 0 ? params->max_patch_deg : 60.0;
  const float cos_max = (float)cos(deg * M_PI / 180.0);
  const int64_t npairs = 12 * mesh->nt;
  dfm_op* mop = const_cast<dfm_op*>(op);
  const int64_t need = npairs * (int64_t)sizeof(PairConst) + 2 * 64 * (int64_t)sizeof(double) + 256;
  if (mop->work_bytes < need) return set_error(DFM_ERR_ARG, "dfm_adjoint: operator has no assembly workspace");
  PairConst* pairs = reinterpret_cast<PairConst*>(mop->work);
  double* glx = reinterpret_cast<double*>(reinterpret_cast<char*>(mop->work) + npairs * sizeof(PairConst));
  double* glw = glx + 64;
  rc = gauss_legendre_device(q, glx, glw, st);
  if (rc) return rc;
  DFM_CUDA_CHECK(cudaMemsetAsync(dJ_dmu, 0, sizeof(double) * R * mesh->nt, st));
  // part 0: the blocks received across each exit face; part 1 (heterogeneous
  // media): the blocks reflected at interfaces; both cross tet t
  const bool media = params->c || params->rho_f;
  if (media != (op->rop != nullptr))
    return set_error(DFM_ERR_ARG, "dfm_adjoint: params->c / rho_f differ from the operator's assembly");
  for (int part = 0; part < (media ? 2 : 1); ++part) {
    pair_setup_kernel<<<(unsigned)((npairs + 127) / 128), 128, 0, st>>>(mesh->verts, mesh->tets, mesh->recv,
                                                                       mesh->refl, mesh->geom, params->mu,
                                                                       params->mu_uniform, npairs, pairs, params->c,
                                                                       params->rho_f, part);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    rc = launch_contract(op->Np, pairs, npairs, glx, glw, q, cos_max, lambda_out, rho, R, op->nrows, mesh->nt,
                         dJ_dmu, st);
    if (rc) return rc;
  }
  if (dgvec) {
    explicit_term_kernel<<<(unsigned)((mesh->nt + 127) / 128), 128, 0, st>>>(dgvec, rho, R, op->nb, op->nrows,
                                                                              mesh->nt, dJ_dmu);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
  }
  return solve_rc;
}
