// Instantiation of the preconditioner hop kernel for the BF16 copy.
#include "hop_kernel.cuh"

namespace dfm {

int hop_launch_bf16(const dfm_op* op, const float* xp, const float* x0p, void* y, int R, float out_scale,
                    bool outp, int trans, cudaStream_t st) {
  using namespace hopk;
  // FP32 hop vectors loop over the right-hand sides outside the chunks
  return outp ? launch_hop<__nv_bfloat16, float, true, 1>(op, xp, x0p, y, R, out_scale, trans, st)
              : launch_hop<__nv_bfloat16, float, false, 1>(op, xp, x0p, y, R, out_scale, trans, st);
}

}  // namespace dfm
