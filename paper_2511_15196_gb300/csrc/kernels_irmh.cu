// SMC-IRMH (Sec. 2 sampler (ii)): the independent Gaussian proposal phi' = mu + L z of
// the population's mean and covariance needs, for the Hastings factor q(phi) / q(phi'),
// every particle's whitened squared norm r = |L^{-1}(phi - mu)|^2 (once per temperature,
// after the refit; an accepted proposal's r is |z|^2) and the proposals' |z|^2.
#include "internal.h"
#include "common.cuh"

namespace phi4 {

// One warp per particle: x = phi - mu in registers (site k = lane + 32 i in slot i),
// right-looking forward substitution w_j = x_j / L_jj, x_k -= L_kj w_j for k > j, and
// r = sum_j w_j^2 (every lane holds the same w_j; lane 0 keeps the sum).
template <int NR>
__global__ void __launch_bounds__(256) whitened_sq_norm_kernel(const double* __restrict__ phi,
                                                               const double* __restrict__ mu,
                                                               const double* __restrict__ Lf, int ld, int N, int D,
                                                               double* __restrict__ r) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= N) return;
  double x[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int k = lane + 32 * i;
    x[i] = k < D ? phi[(size_t)n * D + k] - mu[k] : 0.0;
  }
  double acc = 0.0;
#pragma unroll
  for (int sg = 0; sg < NR; ++sg) {
#pragma unroll 1
    for (int jj = 0; jj < 32; ++jj) {
      const int j = 32 * sg + jj;
      if (j >= D) break;
      const double w = __shfl_sync(0xffffffffu, x[sg], jj) / Lf[(size_t)j * ld + j];
      acc = fma(w, w, acc);
#pragma unroll
      for (int i = sg; i < NR; ++i) {
        const int k = lane + 32 * i;
        if (k > j && k < D) x[i] = fma(-Lf[(size_t)k * ld + j], w, x[i]);
      }
    }
  }
  if (lane == 0) r[n] = acc;
}

__global__ void __launch_bounds__(256) row_sq_norm_kernel(const double* __restrict__ Z, int N, int D,
                                                          double* __restrict__ zz) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= N) return;
  double s = 0.0;
  for (int k = lane; k < D; k += 32) {
    const double z = Z[(size_t)n * D + k];
    s = fma(z, z, s);
  }
  s = warp_sum(s);
  if (lane == 0) zz[n] = s;
}

cudaError_t launch_whitened_sq_norm(const double* phi, const double* mu, const double* Lf, int ld, int N, int D,
                                    double* r, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((N + 7) / 8);
  const int nr = (D + 31) / 32;
  if (nr <= 1) whitened_sq_norm_kernel<1><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else if (nr <= 2) whitened_sq_norm_kernel<2><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else if (nr <= 4) whitened_sq_norm_kernel<4><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else if (nr <= 8) whitened_sq_norm_kernel<8><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else if (nr <= 16) whitened_sq_norm_kernel<16><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else if (nr <= 32) whitened_sq_norm_kernel<32><<<grid, 256, 0, s>>>(phi, mu, Lf, ld, N, D, r);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_row_sq_norm(const double* Z, int N, int D, double* zz, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  row_sq_norm_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(Z, N, D, zz);
  return cudaGetLastError();
}

}  // namespace phi4
