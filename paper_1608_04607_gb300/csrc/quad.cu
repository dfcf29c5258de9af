// Gauss-Legendre rules on the device, FP64.
//
// The direction integral of Sec. 3.4 is reduced to integrals over [-1,1]^2
// per direction patch; each uses a tensor Gauss-Legendre rule of order q.
// Nodes are the roots of the Legendre polynomial P_q, found by Newton's method
// with P_q and P_{q-1} from the three-term recurrence
//   (k+1) P_{k+1}(x) = (2k+1) x P_k(x) - k P_{k-1}(x),
// and weights w = 2 / ((1 - x^2) P_q'(x)^2), P_q' = q (x P_q - P_{q-1})/(x^2 - 1).
#include <math.h>

#include "dfm_internal.cuh"

namespace dfm {
namespace {

__global__ void gauss_legendre_kernel(int q, double* __restrict__ x, double* __restrict__ w) {
  const int i = threadIdx.x;  // i-th root counted from the largest
  if (i >= q) return;
  double z = cos(M_PI * (i + 0.75) / (q + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < q; ++k) {
      const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    // p1 = P_q(z), p0 = P_{q-1}(z)
    if (q == 1) {
      p1 = z;
      p0 = 1.0;
    }
    dp = q * (z * p1 - p0) / (z * z - 1.0);
    const double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  // final derivative at the converged root
  double p0 = 1.0, p1 = z;
  for (int k = 1; k < q; ++k) {
    const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  if (q == 1) p0 = 1.0, p1 = z;
  dp = q * (z * p1 - p0) / (z * z - 1.0);
  x[q - 1 - i] = z;
  w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

}  // namespace

int gauss_legendre_device(int q, double* x, double* w, cudaStream_t st) {
  if (q < 1 || q > 64 || !x || !w) return set_error(DFM_ERR_ARG, "gauss_legendre: need 1 <= q <= 64 and buffers");
  gauss_legendre_kernel<<<1, 64, 0, st>>>(q, x, w);
  DFM_LAUNCHED();
  DFM_CUDA_CHECK(cudaGetLastError());
  return DFM_OK;
}

}  // namespace dfm

extern "C" int dfm_gauss_legendre(int q, double* x, double* w, void* stream) {
  return dfm::gauss_legendre_device(q, x, w, dfm::as_stream(stream));
}
