// Instantiation of the preconditioner hop kernel for the FP16 copy.
#include "hop_kernel.cuh"

namespace dfm {

int hop_launch_f16(const dfm_op* op, const __half* xp, const __half* x0p, void* y, int R, float out_scale,
                   bool outp, int trans, cudaStream_t st) {
  using namespace hopk;
  if (R == 1)
    return outp ? launch_hop<__half, __half, true, 1>(op, xp, x0p, y, R, out_scale, trans, st)
                : launch_hop<__half, __half, false, 1>(op, xp, x0p, y, R, out_scale, trans, st);
  if (hop_uses_mma(op->nb, R))  // several right-hand sides on tensor cores
    return outp ? launch_hop<__half, __half, true, 1, true>(op, xp, x0p, y, R, out_scale, trans, st)
                : launch_hop<__half, __half, false, 1, true>(op, xp, x0p, y, R, out_scale, trans, st);
  return outp ? launch_hop<__half, __half, true, kHopRhsInner>(op, xp, x0p, y, R, out_scale, trans, st)
              : launch_hop<__half, __half, false, kHopRhsInner>(op, xp, x0p, y, R, out_scale, trans, st);
}

}  // namespace dfm
