// Adaptive tempering on the device (Sec. 2 sampler (i); App. A target ESS): the next
// temperature by bisection on the ESS of the incremental weights, then the weights and
// the log-evidence increment, in one cooperative launch (the bisection itself is in
// bisect.cuh), and the Kahan-compensated running log Z.
#include <math.h>
#include "internal.h"
#include "bisect.cuh"

namespace phi4 {

namespace {
constexpr int kMaxGrid = 256;
}  // namespace

template <int EPT>
__global__ void __launch_bounds__(kBisectThreads) bisect_kernel(const double* __restrict__ ell, int N,
                                                                const double* __restrict__ beta_in, double rho,
                                                                int iters, double* __restrict__ w_out,
                                                                double* __restrict__ out, GridSync gs) {
  bisect_body<EPT>(ell, N, beta_in, rho, iters, w_out, out, gs, (int)gridDim.x, (int)blockIdx.x);
}

__global__ void logz_accumulate_kernel(const double* __restrict__ out, double* __restrict__ kahan,
                                       double* __restrict__ beta) {
  logz_accumulate(out, kahan, beta);
}

size_t bisect_scratch_bytes(int N) {
  (void)N;
  return 256 + sizeof(double) * 2 * 2 * kMaxGrid;
}

template <int EPT>
static cudaError_t launch_bisect_t(int G, const double* ell, int N, const double* beta_in, double rho, int iters,
                                   double* w, double* out, GridSync gs, cudaStream_t s) {
  void* args[] = {(void*)&ell, (void*)&N, (void*)&beta_in, (void*)&rho, (void*)&iters, (void*)&w, (void*)&out,
                  (void*)&gs};
  return cudaLaunchCooperativeKernel((const void*)bisect_kernel<EPT>, dim3(G), dim3(kBisectThreads), args, 0, s);
}

// One CTA: the grid barrier degenerates to the CTA's own arrival (nothing waits on
// another CTA), so an ordinary launch is safe next to other streams' work.
template <int EPT>
static cudaError_t launch_bisect_one(const double* ell, int N, const double* beta_in, double rho, int iters,
                                     double* w, double* out, GridSync gs, cudaStream_t s) {
  bisect_kernel<EPT><<<1, kBisectThreads, 0, s>>>(ell, N, beta_in, rho, iters, w, out, gs);
  return cudaGetLastError();
}

cudaError_t launch_bisect(const double* ell, int N, const double* beta_in, double rho, int iters, double* w,
                          double* out, void* scratch, uint32_t* status, cudaStream_t s, bool single_cta) {
  if (N <= 0) return cudaErrorInvalidValue;
  unsigned char* base = (unsigned char*)scratch;
  GridSync gs{(unsigned*)base, (unsigned*)(base + 4), (double*)(base + 256), status};
  cudaError_t e = cudaMemsetAsync(base, 0, 8, s);
  if (e != cudaSuccess) return e;
  if (single_cta) {
    const int ept = (N + kBisectThreads - 1) / kBisectThreads;
    if (ept <= 8) return launch_bisect_one<8>(ell, N, beta_in, rho, iters, w, out, gs, s);
    if (ept <= 16) return launch_bisect_one<16>(ell, N, beta_in, rho, iters, w, out, gs, s);
    if (ept <= 32) return launch_bisect_one<32>(ell, N, beta_in, rho, iters, w, out, gs, s);
    return cudaErrorInvalidValue;
  }
  int G = (N + kBisectThreads - 1) / kBisectThreads;
  const int sms = sm_count();
  if (G > sms) G = sms;
  if (G > kMaxGrid) G = kMaxGrid;
  if (G < 1) G = 1;
  const int ept = (N + G * kBisectThreads - 1) / (G * kBisectThreads);
  if (ept <= 1) return launch_bisect_t<1>(G, ell, N, beta_in, rho, iters, w, out, gs, s);
  if (ept <= 2) return launch_bisect_t<2>(G, ell, N, beta_in, rho, iters, w, out, gs, s);
  if (ept <= 4) return launch_bisect_t<4>(G, ell, N, beta_in, rho, iters, w, out, gs, s);
  if (ept <= 8) return launch_bisect_t<8>(G, ell, N, beta_in, rho, iters, w, out, gs, s);
  return cudaErrorInvalidValue;
}

PHI4_SPIN_LIMIT_SETTER(set_spin_limit_temper)

cudaError_t launch_logz_accumulate(const double* out, double* logz_kahan, double* beta, cudaStream_t s) {
  logz_accumulate_kernel<<<1, 1, 0, s>>>(out, logz_kahan, beta);
  return cudaGetLastError();
}

}  // namespace phi4
