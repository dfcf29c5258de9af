// Instantiation of the preconditioner hop kernels for the FP16 copy: the
// CUDA-core hop (bases whose padded width is not a multiple of 16) and the
// tensor-core hop on the fragment-ordered copy (the others).
#include "hop_frag.cuh"
#include "hop_kernel.cuh"

namespace dfm {

int hop_launch_f16(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int R, float out_scale,
                   bool outp, int trans, cudaStream_t st) {
  using namespace hopk;
  if (R == 1)
    return outp ? launch_hop<__half, __half, true, 1>(op, xp, x0p, y, R, out_scale, trans, st)
                : launch_hop<__half, __half, false, 1>(op, xp, x0p, y, R, out_scale, trans, st);
  return outp ? launch_hop<__half, __half, true, kHopRhsInner>(op, xp, x0p, y, R, out_scale, trans, st)
              : launch_hop<__half, __half, false, kHopRhsInner>(op, xp, x0p, y, R, out_scale, trans, st);
}

int hop_frag_launch_f16(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int w, int rgl, int rhs_here,
                        bool outp, float out_scale, int trans, int rpt, int stages, cudaStream_t st) {
  return fragk::launch_hop_frag<__half>(op, xp, x0p, y, w, rgl, rhs_here, outp, out_scale, trans, rpt, stages, st);
}

}  // namespace dfm
