// Population observables on the device (Sec. 2: the magnetisation M = (1/D) sum_x phi_x
// and its moments; App. F: the mode balance), reduced in FP64 in one CTA.
//   out[0] = <M>, out[1] = <|M|>, out[2] = <M^2>, out[3] = chi = D (<M^2> - <M>^2),
//   out[4] = mode balance = (weight of M > 0) / (weight of M < 0), zeros ignored,
//            +inf when nothing is negative, NaN when both sides are empty,
//   out[5] = the total weight,
// with weights w_i (uniform when w is NULL) normalised by their sum. Each thread sums
// a strided subset, then a fixed-order warp and CTA tree: the result is deterministic.
#include <math.h>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int kObsThreads = 1024;
}

__global__ void __launch_bounds__(kObsThreads) obs_reduce_kernel(const double* __restrict__ M,
                                                                 const double* __restrict__ w, int N, int D,
                                                                 double* __restrict__ out) {
  __shared__ double red[64];
  double sw = 0.0, s1 = 0.0, sa = 0.0, s2 = 0.0, sp = 0.0, sn = 0.0;
  for (int i = threadIdx.x; i < N; i += kObsThreads) {
    const double m = M[i], wi = w ? w[i] : 1.0;
    sw += wi;
    s1 += wi * m;
    sa += wi * fabs(m);
    s2 += wi * m * m;
    if (m > 0.0) sp += wi;
    else if (m < 0.0) sn += wi;
  }
  sw = block_sum(sw, red);
  s1 = block_sum(s1, red);
  sa = block_sum(sa, red);
  s2 = block_sum(s2, red);
  sp = block_sum(sp, red);
  sn = block_sum(sn, red);
  if (threadIdx.x == 0) {
    const double mean = s1 / sw, m2 = s2 / sw;
    out[0] = mean;
    out[1] = sa / sw;
    out[2] = m2;
    out[3] = (double)D * (m2 - mean * mean);
    out[4] = sn > 0.0 ? sp / sn : (sp > 0.0 ? INFINITY : NAN);
    out[5] = sw;
  }
}

cudaError_t launch_observables(const void* phi, int dtype, int N, int D, const double* w, double* M, double* out,
                               cudaStream_t s) {
  if (N <= 0 || D <= 0) return cudaErrorInvalidValue;
  cudaError_t e = launch_magnetisation(phi, dtype, N, D, M, s);
  if (e != cudaSuccess) return e;
  obs_reduce_kernel<<<1, kObsThreads, 0, s>>>(M, w, N, D, out);
  return cudaGetLastError();
}

}  // namespace phi4
