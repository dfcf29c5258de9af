// Block flexible GMRES for a group of right-hand sides sharing one Krylov
// space (included by solve.cu inside its anonymous namespace, after Ctx, Hop,
// ctx_apply and precond_hops).
//
// The paper gives no solver.  The lockstep solver iterates each right-hand
// side in its own Krylov space and shares only the operator passes; the slow
// directional modes of I - B are common to all sources of one operator, so
// one block space spanned by all of them converges in fewer passes.  Per
// block step j (R columns):
//   Z_j = p~(B) V_j (the same low-precision hops as the lockstep solver),
//   W = (I - B) Z_j,
//   [V_0 .. V_j]^T W and W^T W in one pass (gdot_kernel: a tall-skinny
//   product, every basis vector and W read once), then W <- (W - V C) S^-1 with S
//   the Cholesky factor of W^T W - C^T C (gtrans_kernel in place; 9..16 columns
//   on tensor cores, gtrans_mma_kernel), then a
//   second pass: against the basis again where the first lost more than half
//   of a column's norm, else Cholesky QR of the block alone (block classical
//   Gram-Schmidt with Cholesky QR and selective re-orthogonalisation), so
//   H_(:,j) = C1 + C2 S1 and H_(j+1,j) = S2 S1;
//   the block Hessenberg least-squares problem min |E1 S0 - H Y| is kept in
//   upper-triangular form by Givens rotations on the host (FP64), its
//   residual rows giving every right-hand side's residual estimate;
// at the end of a cycle x += [Z_0 .. Z_k] Y (gtrans_kernel).
// A Gram matrix pivot below 1e-14 of the largest diagonal marks a column with
// no new direction (a zero right-hand side, or a block that has become
// invariant): its basis vector is set to zero and stays zero.

// basis vectors per warp of gdot_kernel (its registers hold kGQ x RM sums)
template <int RM>
struct GdotQ {
  static constexpr int value = RM >= 16 ? 4 : 8;
};
constexpr int kGMaxSplits = 512;  // element ranges of gdot_kernel
constexpr int kBlockMaxR = 16;    // largest block

// partial[(s * K + q) * R + r] = sum over element range s of V_q . W_r,
// q < K, r < R; V_q = V + q n, W_r = W + r n (n a multiple of 4, 16-byte
// aligned vectors).  One CTA per element range s: the range's W is staged in
// shared memory chunk by chunk; each warp takes kGQ basis vectors at a time
// and its lanes stream consecutive 16-byte pieces of them (coalesced), each
// piece multiplied with the R staged W pieces; the warp's kGQ x R sums are
// reduced by shuffles once per group of basis vectors.  W is staged once per
// group of (warps x kGQ) basis vectors.
template <int RM>
__global__ void __launch_bounds__(256)
gdot_kernel(const float* __restrict__ V, int K, const float* __restrict__ W, int R, int64_t n,
            float* __restrict__ partial) {
  constexpr int CH = 2048 / RM;  // float4 elements of W per staged chunk (32 KB)
  constexpr int kGQ = GdotQ<RM>::value;
  __shared__ float4 ws[RM * CH];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t n4 = n >> 2;
  const int64_t per = (n4 + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * per, e1 = min(n4, e0 + per);
  const float4* W4 = reinterpret_cast<const float4*>(W);
  const float4* V4 = reinterpret_cast<const float4*>(V);
  for (int qg = 0; qg < K; qg += nw * kGQ) {
    const int q0 = qg + wid * kGQ;
    float acc[kGQ][RM];
#pragma unroll
    for (int u = 0; u < kGQ; ++u)
#pragma unroll
      for (int r = 0; r < RM; ++r) acc[u][r] = 0.f;
    for (int64_t c0 = e0; c0 < e1; c0 += CH) {
      const int len = (int)(e1 - c0 < (int64_t)CH ? e1 - c0 : (int64_t)CH);
      __syncthreads();
      for (int i = threadIdx.x; i < R * CH; i += blockDim.x) {
        const int r = i / CH, j = i - r * CH;
        ws[r * CH + j] = j < len ? W4[r * n4 + c0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      if (q0 >= K) continue;
      for (int j = lane; j < len; j += 32) {
        float4 v[kGQ];
#pragma unroll
        for (int u = 0; u < kGQ; ++u)
          v[u] = q0 + u < K ? V4[(int64_t)(q0 + u) * n4 + c0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < RM; ++r) {
          if (r >= R) break;
          const float4 w = ws[r * CH + j];
#pragma unroll
          for (int u = 0; u < kGQ; ++u)
            acc[u][r] = fmaf(v[u].x, w.x, fmaf(v[u].y, w.y, fmaf(v[u].z, w.z, fmaf(v[u].w, w.w, acc[u][r]))));
        }
      }
    }
    if (q0 >= K) continue;
#pragma unroll
    for (int u = 0; u < kGQ; ++u)
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        float v = acc[u][r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && q0 + u < K && r < R) partial[((int64_t)blockIdx.x * K + q0 + u) * R + r] = v;
      }
  }
}

// out[q * R + r] = sum_s partial[(s * K + q) * R + r] (fixed order)
__global__ void gdot_reduce_kernel(const float* __restrict__ partial, int S, int KR, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= KR) return;
  float s = 0.f;
  for (int k = 0; k < S; ++k) s += partial[(int64_t)k * KR + i];
  out[i] = s;
}

// In place, per element: W_r <- sum_i W_i T[i][r] + sum_q V_q H[q][r]
// (T = the identity when Tm is NULL); coef = [H (K x R) | T (R x R)] in FP32;
// partial[b * R + r] = block b's share of |W_r|^2 when partial is given.
template <int RM>
__global__ void __launch_bounds__(256, RM >= 16 ? 2 : 3)
gtrans_kernel(const float* __restrict__ V, int K, const float* __restrict__ coef, int has_t, float* W, int R,
              int64_t n, float* __restrict__ partial) {
  extern __shared__ float cs[];  // K R + R R
  for (int i = threadIdx.x; i < K * R + (has_t ? R * R : 0); i += blockDim.x) cs[i] = coef[i];
  __syncthreads();
  const float* Hs = cs;
  const float* Ts = cs + K * R;
  const int64_t n4 = n >> 2;
  float4* W4 = reinterpret_cast<float4*>(W);
  const float4* V4 = reinterpret_cast<const float4*>(V);
  float sq[RM];
#pragma unroll
  for (int r = 0; r < RM; ++r) sq[r] = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    float4 acc[RM];
    if (has_t) {
      // acc = W T, one W column at a time (all R loads precede the stores below)
#pragma unroll
      for (int r = 0; r < RM; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        if (i >= R) break;
        const float4 wi = W4[i * n4 + e];
#pragma unroll
        for (int r = 0; r < RM; ++r) {
          if (r >= R) break;
          const float t = Ts[i * R + r];
          acc[r].x = fmaf(wi.x, t, acc[r].x);
          acc[r].y = fmaf(wi.y, t, acc[r].y);
          acc[r].z = fmaf(wi.z, t, acc[r].z);
          acc[r].w = fmaf(wi.w, t, acc[r].w);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < RM; ++r) acc[r] = r < R ? W4[r * n4 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // four basis vectors per round: four independent 16-byte loads in flight
    // per thread keep enough bytes moving to stream at the HBM rate
    int q = 0;
    for (; q + 4 <= K; q += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = V4[(int64_t)(q + u) * n4 + e];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int r = 0; r < RM; ++r) {
          if (r >= R) break;
          const float h = Hs[(q + u) * R + r];
          acc[r].x = fmaf(v[u].x, h, acc[r].x);
          acc[r].y = fmaf(v[u].y, h, acc[r].y);
          acc[r].z = fmaf(v[u].z, h, acc[r].z);
          acc[r].w = fmaf(v[u].w, h, acc[r].w);
        }
    }
    for (; q < K; ++q) {
      const float4 v = V4[(int64_t)q * n4 + e];
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        if (r >= R) break;
        const float h = Hs[q * R + r];
        acc[r].x = fmaf(v.x, h, acc[r].x);
        acc[r].y = fmaf(v.y, h, acc[r].y);
        acc[r].z = fmaf(v.z, h, acc[r].z);
        acc[r].w = fmaf(v.w, h, acc[r].w);
      }
    }
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      if (r >= R) break;
      W4[r * n4 + e] = acc[r];
      sq[r] = fmaf(acc[r].x, acc[r].x, fmaf(acc[r].y, acc[r].y, fmaf(acc[r].z, acc[r].z, fmaf(acc[r].w, acc[r].w, sq[r]))));
    }
  }
  if (!partial) return;
  __shared__ float sh[8][RM];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    float v = sq[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][r] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < R) {
    float s = 0.f;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) s += sh[w8][threadIdx.x];
    partial[(int64_t)blockIdx.x * R + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Tensor-core block update for blocks of 9..16 columns.  The update is a dense
// contraction (K basis vectors into 16 columns over n elements, 8 FLOP per
// byte of basis, close to the FP32 ridge), so it runs as mma.sync m16n8k8
// TF32 products with every FP32 operand split into two TF32 parts,
// x = hi + lo, and the three products lo hi + hi lo + hi hi accumulated in
// FP32 (the lo lo term lies below FP32 rounding): about 22 significant bits
// per product.  The contraction index of a product may be assigned to the
// MMA's k slots in any order used alike for both operands; here a lane's k
// slots hold consecutive elements of one float4 of its operand rows, so every
// operand moves as coalesced 16-byte vectors.  Fragment layout of m16n8k8
// (g = lane / 4, t = lane % 4): A a0..a3 = (g, t), (g + 8, t), (g, t + 4),
// (g + 8, t + 4); B b0, b1 = (k t, n g), (k t + 4, n g); C c0..c3 = (g, 2t),
// (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1).
// The tall-skinny product [V_0 .. V_j]^T W stays on CUDA cores (gdot_kernel):
// in the same form on tensor cores its three-product chains per accumulator
// tile serialised and it ran 60% slower at 16 columns (892 against 557 ms per
// step of the 45-function benchmark), while this update ran 13% faster.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_round(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return h;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// c += A B from the hi / lo parts of both (three products, smallest first)
__device__ __forceinline__ void mma3_tf32(float* c, const uint32_t* ah, const uint32_t* al, uint32_t bh0, uint32_t bh1,
                                          uint32_t bl0, uint32_t bl1) {
  mma_tf32(c, al, bh0, bh1);
  mma_tf32(c, ah, bl0, bl1);
  mma_tf32(c, ah, bh0, bh1);
}
__device__ __forceinline__ void split4(float x0, float x1, float x2, float x3, uint32_t* hi, uint32_t* lo) {
  tf32_split(x0, hi[0], lo[0]);
  tf32_split(x1, hi[1], lo[1]);
  tf32_split(x2, hi[2], lo[2]);
  tf32_split(x3, hi[3], lo[3]);
}

// In place, per element: W_r <- sum_i W_i T[i][r] + sum_q V_q H[q][r] as
// gtrans_kernel (no norm partials), R <= 16, on tensor cores: the rows of
// X = [V; W] (W only with T) contract with B = [H; T] (coefficients split once
// into shared memory, zero-padded to 16 columns and to a multiple of 8 rows).
// A warp owns tiles of 32 elements: lane (g, t) loads float4 g of the tile
// from X rows k0 + t and k0 + t + 4, so MMA rows g, g + 8 are the float4's
// elements 0, 1 (first M tile) or 2, 3 (second), and its C fragment holds, for
// columns 2t and 2t + 1, the four elements of that float4.
__global__ void __launch_bounds__(256, 2)
gtrans_mma_kernel(const float* __restrict__ V, int K, const float* __restrict__ coef, int has_t, float* W, int R,
                  int64_t n) {
  extern __shared__ uint32_t cfs[];  // [K8][16] hi, then [K8][16] lo
  const int KX = K + (has_t ? R : 0);
  const int K8 = (KX + 7) / 8 * 8;
  uint32_t* chi = cfs;
  uint32_t* clo = cfs + K8 * 16;
  for (int i = threadIdx.x; i < K8 * 16; i += blockDim.x) {
    const int k = i >> 4, r = i & 15;
    float v = 0.f;
    if (r < R) {
      if (k < K) v = coef[k * R + r];
      else if (k < KX) v = coef[K * R + (k - K) * R + r];
    }
    tf32_split(v, chi[i], clo[i]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int64_t n4 = n >> 2;
  float4* W4 = reinterpret_cast<float4*>(W);
  const float4* V4 = reinterpret_cast<const float4*>(V);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t ntile = (n4 + 7) / 8;
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); tile < ntile; tile += nwarp) {
    const int64_t e4 = tile * 8 + g;
    const bool valid = e4 < n4;
    float acc[2][2][4];  // [M tile][N tile][c]
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int r0 = nt * 8 + 2 * t, r1 = r0 + 1;
      float4 w0 = zero, w1 = zero;
      if (!has_t && valid) {
        if (r0 < R) w0 = W4[(int64_t)r0 * n4 + e4];
        if (r1 < R) w1 = W4[(int64_t)r1 * n4 + e4];
      }
      acc[0][nt][0] = w0.x; acc[0][nt][1] = w1.x; acc[0][nt][2] = w0.y; acc[0][nt][3] = w1.y;
      acc[1][nt][0] = w0.z; acc[1][nt][1] = w1.z; acc[1][nt][2] = w0.w; acc[1][nt][3] = w1.w;
    }
    for (int k0 = 0; k0 < K8; k0 += 8) {
      const int ka = k0 + t, kb = ka + 4;
      float4 xa = zero, xb = zero;
      if (valid) {
        if (ka < K) xa = V4[(int64_t)ka * n4 + e4];
        else if (ka < KX) xa = W4[(int64_t)(ka - K) * n4 + e4];
        if (kb < K) xb = V4[(int64_t)kb * n4 + e4];
        else if (kb < KX) xb = W4[(int64_t)(kb - K) * n4 + e4];
      }
      uint32_t ah[2][4], al[2][4];
      split4(xa.x, xa.y, xb.x, xb.y, ah[0], al[0]);
      split4(xa.z, xa.w, xb.z, xb.w, ah[1], al[1]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int col = nt * 8 + g;
        const uint32_t bh0 = chi[ka * 16 + col], bh1 = chi[kb * 16 + col];
        const uint32_t bl0 = clo[ka * 16 + col], bl1 = clo[kb * 16 + col];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma3_tf32(acc[mt][nt], ah[mt], al[mt], bh0, bh1, bl0, bl1);
      }
    }
    if (valid) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int r0 = nt * 8 + 2 * t, r1 = r0 + 1;
        if (r0 < R) W4[(int64_t)r0 * n4 + e4] = make_float4(acc[0][nt][0], acc[0][nt][2], acc[1][nt][0], acc[1][nt][2]);
        if (r1 < R) W4[(int64_t)r1 * n4 + e4] = make_float4(acc[0][nt][1], acc[0][nt][3], acc[1][nt][1], acc[1][nt][3]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct BlockScratch {
  float* part = nullptr;  // gdot partials: kGMaxSplits * kmax * R floats
  int64_t part_elems = 0;
  float* small = nullptr;  // device coefficients / reduced products (>= (kmax + R) * R + R * R floats)
  float* sq = nullptr;     // gtrans norm partials (grid * R floats)
};

inline int gdot_splits(int64_t n, int nsm) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min(2 * nsm, kGMaxSplits), (n >> 2) / 2048));
}

// G[q][r] = V_q . W_r for q < K (host, FP64 copies of the FP32 products)
inline int block_dot(const Ctx& c, const float* V, int K, const float* W, int R, const BlockScratch& bs,
                     std::vector<double>* G) {
  const int S = gdot_splits(c.n, c.nsm);
  if ((int64_t)S * K * R > bs.part_elems) return set_error(DFM_ERR_ARG, "block solve: Gram partials overflow");
  {
    ::dfm::KernelTimer timer_(DFM_KERNEL_DOT, c.st);
    if (R <= 2) gdot_kernel<2><<<S, 256, 0, c.st>>>(V, K, W, R, c.n, bs.part);
    else if (R <= 4) gdot_kernel<4><<<S, 256, 0, c.st>>>(V, K, W, R, c.n, bs.part);
    else if (R <= 8) gdot_kernel<8><<<S, 256, 0, c.st>>>(V, K, W, R, c.n, bs.part);
    else gdot_kernel<16><<<S, 256, 0, c.st>>>(V, K, W, R, c.n, bs.part);
  }
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  gdot_reduce_kernel<<<(K * R + 127) / 128, 128, 0, c.st>>>(bs.part, S, K * R, bs.small);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  std::vector<float> h((size_t)K * R);
  DFM_CUDA_CHECK(cudaMemcpyAsync(h.data(), bs.small, sizeof(float) * K * R, cudaMemcpyDeviceToHost, c.st));
  DFM_CUDA_CHECK(cudaStreamSynchronize(c.st));
  G->assign(h.begin(), h.end());
  return DFM_OK;
}

// W <- W T + sign V H (T: R x R or empty for the identity; H: K x R)
inline int block_update(const Ctx& c, const float* V, int K, const std::vector<double>& H, double sign,
                        const std::vector<double>& T, float* W, int R, const BlockScratch& bs) {
  const bool has_t = !T.empty();
  std::vector<float> coef((size_t)K * R + (has_t ? R * R : 0));
  for (int64_t i = 0; i < (int64_t)K * R; ++i) coef[i] = (float)(sign * H[i]);
  if (has_t)
    for (int i = 0; i < R * R; ++i) coef[(size_t)K * R + i] = (float)T[i];
  DFM_CUDA_CHECK(cudaMemcpyAsync(bs.small, coef.data(), sizeof(float) * coef.size(), cudaMemcpyHostToDevice, c.st));
  const size_t smem = sizeof(float) * coef.size();
  if (smem > 48 * 1024) return set_error(DFM_ERR_ARG, "block solve: too many basis vectors for one update");
  int rc = DFM_OK;
  // one resident wave of CTAs, each striding over the elements
  auto go = [&](auto kernel) -> int {
    int per_sm = 0;
    DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((c.n >> 2) + 255) / 256, (int64_t)std::max(per_sm, 1) * c.nsm));
    ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
    kernel<<<grid, 256, smem, c.st>>>(V, K, bs.small, has_t, W, R, c.n, nullptr);
    return DFM_OK;
  };
  if (R <= 2) rc = go(gtrans_kernel<2>);
  else if (R <= 4) rc = go(gtrans_kernel<4>);
  else if (R <= 8) rc = go(gtrans_kernel<8>);
  else {  // 9..16 columns: tensor cores, coefficients split into TF32 parts in shared memory
    const int K8 = (K + (has_t ? R : 0) + 7) / 8 * 8;
    const size_t msmem = (size_t)K8 * 16 * 2 * sizeof(uint32_t);
    if (msmem > 200 * 1024) return set_error(DFM_ERR_ARG, "block solve: too many basis vectors for one update");
    DFM_CUDA_CHECK(cudaFuncSetAttribute(gtrans_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem));
    int per_sm = 0;
    DFM_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gtrans_mma_kernel, 256, msmem));
    const int64_t tiles = ((c.n >> 2) + 7) / 8;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((tiles + 7) / 8, (int64_t)std::max(per_sm, 1) * c.nsm));
    ::dfm::KernelTimer timer_(DFM_KERNEL_AXPY, c.st);
    gtrans_mma_kernel<<<grid, 256, msmem, c.st>>>(V, K, bs.small, has_t ? 1 : 0, W, R, c.n);
  }
  if (rc) return rc;
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

// Cholesky M = S^T S (M: R x R symmetric, row-major) with pivots below
// 1e-14 of the largest diagonal entry marked dead; Sinv maps W' to W1 = W' Sinv
// (dead columns of W1 zero) and S (rows of dead columns zero) gives
// W' ~ W1 S.  Returns false on a non-finite entry.
inline bool chol_block(const std::vector<double>& M, int R, std::vector<double>* S, std::vector<double>* Sinv) {
  double mx = 0.0;
  for (int i = 0; i < R; ++i) {
    if (!std::isfinite(M[i * R + i])) return false;
    mx = std::max(mx, M[i * R + i]);
  }
  S->assign((size_t)R * R, 0.0);
  Sinv->assign((size_t)R * R, 0.0);
  std::vector<char> dead(R, 0);
  const double floor_ = 1e-14 * mx;
  for (int j = 0; j < R; ++j) {
    // S[k][j] = (M[k][j] - sum_{l<k} S[l][k] S[l][j]) / S[k][k] for live k < j
    for (int k = 0; k < j; ++k) {
      if (dead[k]) continue;
      double a = M[k * R + j];
      for (int l = 0; l < k; ++l) a -= (*S)[l * R + k] * (*S)[l * R + j];
      (*S)[k * R + j] = a / (*S)[k * R + k];
    }
    double d = M[j * R + j];
    for (int l = 0; l < j; ++l) d -= (*S)[l * R + j] * (*S)[l * R + j];
    if (!std::isfinite(d)) return false;
    if (!(d > floor_) || mx == 0.0) {
      dead[j] = 1;
      continue;
    }
    (*S)[j * R + j] = sqrt(d);
  }
  // Sinv column j = (e_j - sum_{live k < j} Sinv[:, k] S[k][j]) / S[j][j] for live j
  for (int j = 0; j < R; ++j) {
    if (dead[j]) continue;
    for (int i = 0; i < R; ++i) {
      double a = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < j; ++k)
        if (!dead[k]) a -= (*Sinv)[i * R + k] * (*S)[k * R + j];
      (*Sinv)[i * R + j] = a / (*S)[j * R + j];
    }
  }
  return true;
}

// Orthonormalise the R vectors W (stored right after the K orthonormal basis
// vectors V, so that [V, W] is contiguous) against V and among themselves:
// W_in = V Hc + W_out Rs, Hc K x R, Rs R x R upper triangular.
inline int block_orth(const Ctx& c, float* V, int K, int R, const BlockScratch& bs, std::vector<double>* Hc,
                      std::vector<double>* Rs) {
  float* W = V + (int64_t)K * c.n;
  Hc->assign((size_t)K * R, 0.0);
  std::vector<double> Sacc((size_t)R * R, 0.0);
  for (int i = 0; i < R; ++i) Sacc[i * R + i] = 1.0;
  // The second pass projects against the basis again only when the first
  // lost more than half of some column's norm to it (the cancellation that
  // leaves rounding-size components along the basis); otherwise it
  // re-orthonormalises the block within itself (Cholesky QR on W alone,
  // reading R vectors instead of K + R).
  bool full = true;
  for (int pass = 0; pass < 2; ++pass) {
    const int Kp = full ? K : 0;
    float* Vp = W - (int64_t)Kp * c.n;  // [Vp, W] contiguous
    std::vector<double> G;
    int rc = block_dot(c, Vp, Kp + R, W, R, bs, &G);
    if (rc) return rc;
    // M = W^T W - C^T C, C = G[0..Kp)
    std::vector<double> M((size_t)R * R);
    for (int a = 0; a < R; ++a)
      for (int b = 0; b < R; ++b) {
        double s = 0.5 * (G[(size_t)(Kp + a) * R + b] + G[(size_t)(Kp + b) * R + a]);
        for (int q = 0; q < Kp; ++q) s -= G[(size_t)q * R + a] * G[(size_t)q * R + b];
        M[a * R + b] = s;
      }
    if (pass == 0) {
      full = false;
      for (int a = 0; a < R; ++a) full |= M[a * R + a] < 0.25 * G[(size_t)(Kp + a) * R + a];
    }
    std::vector<double> S, Sinv;
    if (!chol_block(M, R, &S, &Sinv)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite Krylov block");
    // W <- (W - Vp C) Sinv = W Sinv - Vp (C Sinv)
    std::vector<double> CS((size_t)Kp * R, 0.0);
    for (int q = 0; q < Kp; ++q)
      for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s += G[(size_t)q * R + i] * Sinv[i * R + r];
        CS[(size_t)q * R + r] = s;
      }
    rc = block_update(c, Vp, Kp, CS, -1.0, Sinv, W, R, bs);
    if (rc) return rc;
    // W_in = V (Hc + C Sacc) + W_new (S Sacc)
    for (int q = 0; q < Kp; ++q)
      for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s += G[(size_t)q * R + i] * Sacc[i * R + r];
        (*Hc)[(size_t)q * R + r] += s;
      }
    std::vector<double> SS((size_t)R * R, 0.0);
    for (int a = 0; a < R; ++a)
      for (int b = 0; b < R; ++b) {
        double s = 0.0;
        for (int i = 0; i < R; ++i) s += S[a * R + i] * Sacc[i * R + b];
        SS[a * R + b] = s;
      }
    Sacc.swap(SS);
  }
  *Rs = Sacc;
  return DFM_OK;
}

// Block flexible GMRES(m) for the R (<= kBlockMaxR) right-hand sides b
// ([R][n]) of one group, x ([R][n]) holding the initial guess; tol is relative
// to each |b_r|.  V: (m + 1) R vectors, Z: m R vectors, tmp: R vectors.
// Operator applications are added to *iters (one per pass over the group).
inline int gmres_block(const Ctx& c, int R, const float* b, float* x, double tol, int m, int d, int max_iter,
                       int* iters, std::vector<double>* est, float* V, float* Z, float* tmp, const Hop& lp,
                       const BlockScratch& bs) {
  const int64_t n = c.n;
  const int64_t Rn = (int64_t)R * n;
  est->assign(R, 0.0);
  std::vector<double> G;
  int rc = block_dot(c, b, R, b, R, bs, &G);
  if (rc) return rc;
  std::vector<double> bnorm(R);
  for (int r = 0; r < R; ++r) {
    bnorm[r] = sqrt(std::max(0.0, G[(size_t)r * R + r]));
    if (!std::isfinite(bnorm[r])) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite right-hand side");
  }
  const int rows = (m + 1) * R, cols = m * R;
  double prev_worst = -1.0;
  while (true) {
    // block residual V_0 = b - (I - B) x
    axpby_kernel<float><<<grid_for(Rn, c.nsm), 256, 0, c.st>>>(tmp, 1.f, b, -1.f, x, Rn);
    DFM_LAUNCHED();
    DFM_CUDA_CHECK(cudaGetLastError());
    rc = ctx_apply(c, x, tmp, V, R, 1.0, DFM_F32);
    if (rc) return rc;
    ++*iters;
    std::vector<double> Hc, S0;
    rc = block_orth(c, V, 0, R, bs, &Hc, &S0);
    if (rc) return rc;
    // least-squares state: Hm (rows x cols), Gm = E1 S0 (rows x R), rotations
    std::vector<double> Hm((size_t)rows * cols, 0.0), Gm((size_t)rows * R, 0.0);
    for (int a = 0; a < R; ++a)
      for (int r = 0; r < R; ++r) Gm[(size_t)a * R + r] = S0[a * R + r];
    struct Rot {
      int i, k;
      double c, s;
    };
    std::vector<Rot> rots;
    double worst = 0.0;
    for (int r = 0; r < R; ++r) {
      double rn = 0.0;
      for (int a = 0; a < R; ++a) rn += Gm[(size_t)a * R + r] * Gm[(size_t)a * R + r];
      (*est)[r] = bnorm[r] > 0 ? sqrt(rn) / bnorm[r] : 0.0;
      worst = std::max(worst, (*est)[r]);
    }
    if (worst <= tol) return DFM_OK;
    if (*iters >= max_iter) return DFM_ERR_NOT_CONVERGED;
    if (prev_worst > 0 && worst > 0.9 * prev_worst) return DFM_ERR_NOT_CONVERGED;  // precision exhausted
    prev_worst = worst;
    int kdone = 0;
    for (int j = 0; j < m; ++j) {
      float* vj = V + (int64_t)j * Rn;
      float* zj = Z + (int64_t)j * Rn;
      float* w = V + (int64_t)(j + 1) * Rn;
      rc = precond_hops(c, lp, R, d, vj, zj);
      if (rc) return rc;
      *iters += d;
      rc = ctx_apply(c, zj, zj, w, R, -1.0, DFM_F32);
      if (rc) return rc;
      std::vector<double> Rs;
      rc = block_orth(c, V, (j + 1) * R, R, bs, &Hc, &Rs);
      if (rc) return rc;
      // new block column: rows [0, (j+1)R) = Hc, rows [(j+1)R, (j+2)R) = Rs
      const int c0 = j * R;
      for (int q = 0; q < (j + 1) * R; ++q)
        for (int r = 0; r < R; ++r) Hm[(size_t)q * cols + c0 + r] = Hc[(size_t)q * R + r];
      for (int a = 0; a < R; ++a)
        for (int r = 0; r < R; ++r) Hm[(size_t)((j + 1) * R + a) * cols + c0 + r] = Rs[a * R + r];
      for (const Rot& g : rots)
        for (int r = 0; r < R; ++r) {
          double& hi = Hm[(size_t)g.i * cols + c0 + r];
          double& hk = Hm[(size_t)g.k * cols + c0 + r];
          const double a = hi, bb = hk;
          hi = g.c * a + g.s * bb;
          hk = -g.s * a + g.c * bb;
        }
      for (int r = 0; r < R; ++r) {
        const int col = c0 + r;
        const int last = (j + 1) * R + r;  // lowest non-zero row of this column
        for (int k = col + 1; k <= last; ++k) {
          const double a = Hm[(size_t)col * cols + col], bb = Hm[(size_t)k * cols + col];
          if (bb == 0.0) continue;
          const double den = hypot(a, bb);
          const Rot g{col, k, a / den, bb / den};
          for (int cc = col; cc < c0 + R; ++cc) {
            double& hi = Hm[(size_t)g.i * cols + cc];
            double& hk = Hm[(size_t)g.k * cols + cc];
            const double x1 = hi, x2 = hk;
            hi = g.c * x1 + g.s * x2;
            hk = -g.s * x1 + g.c * x2;
          }
          for (int rr = 0; rr < R; ++rr) {
            double& gi = Gm[(size_t)g.i * R + rr];
            double& gk = Gm[(size_t)g.k * R + rr];
            const double x1 = gi, x2 = gk;
            gi = g.c * x1 + g.s * x2;
            gk = -g.s * x1 + g.c * x2;
          }
          rots.push_back(g);
        }
      }
      kdone = j + 1;
      worst = 0.0;
      for (int r = 0; r < R; ++r) {
        double rn = 0.0;
        for (int a = 0; a < R; ++a) {
          const double v = Gm[(size_t)((j + 1) * R + a) * R + r];
          rn += v * v;
        }
        if (!std::isfinite(rn)) return set_error(DFM_ERR_NONFINITE, "dfm_solve: non-finite Krylov block");
        (*est)[r] = bnorm[r] > 0 ? sqrt(rn) / bnorm[r] : 0.0;
        worst = std::max(worst, (*est)[r]);
      }
      if (worst <= 0.5 * tol || *iters + d >= max_iter) break;
    }
    // Y = U^-1 Gm (upper triangular kdone R), x += [Z_0 .. Z_kdone) Y
    const int kc = kdone * R;
    std::vector<double> Y((size_t)kc * R, 0.0);
    for (int r = 0; r < R; ++r)
      for (int i = kc - 1; i >= 0; --i) {
        double a = Gm[(size_t)i * R + r];
        for (int k = i + 1; k < kc; ++k) a -= Hm[(size_t)i * cols + k] * Y[(size_t)k * R + r];
        const double dg = Hm[(size_t)i * cols + i];
        Y[(size_t)i * R + r] = dg != 0.0 ? a / dg : 0.0;
      }
    if (kc > 0) {
      rc = block_update(c, Z, kc, Y, 1.0, std::vector<double>(), x, R, bs);
      if (rc) return rc;
    }
  }
}
