// Adaptive tempering on the device (Sec. 2 sampler (i); App. A target ESS):
// the next temperature by bisection on the ESS of the incremental weights,
// then the weights and the log-evidence increment, in one cooperative launch.
// Every bisection step needs two sums over all N particles, so the grid meets
// at a software barrier (one atomic counter, a bounded acquire-spin) once per
// step; each CTA then adds the per-CTA partials in the same fixed order, so all
// CTAs take identical decisions and the result is deterministic.
#include <math.h>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int kThreads = 128;
constexpr int kMaxGrid = 256;

struct GridSync {
  unsigned* bar;       // arrival counter (zeroed before launch)
  unsigned* abort;     // set by a CTA whose wait gave up
  double* part;        // [2][gridDim][2] per-CTA partials, double-buffered by phase parity
  uint32_t* status;
};

PHI4_DEV bool spin_until(const unsigned* bar, unsigned target, const unsigned* abort) {
  const long long t0 = clock64(), lim = spin_limit();
  for (;;) {
    unsigned v, a;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
    if (v >= target) return true;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(a) : "l"(abort) : "memory");
    if (a) return false;
    if (clock64() - t0 > lim) return false;
    __nanosleep(32);
  }
}

// Grid-wide (sum or max) of two doubles. Returns false if the barrier gave up.
template <bool kMax>
PHI4_DEV bool grid_reduce2(GridSync& gs, unsigned& phase, double& v0, double& v1, double* red) {
  const int G = gridDim.x;
  if (kMax) {
    v0 = block_max(v0, red);
    v1 = block_max(v1, red);
  } else {
    v0 = block_sum(v0, red);
    v1 = block_sum(v1, red);
  }
  __shared__ int ok_s;
  double* part = gs.part + (size_t)(phase & 1u) * G * 2;
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = v0;
    part[2 * blockIdx.x + 1] = v1;
    __threadfence();
    atomicAdd(gs.bar, 1u);
    const bool ok = spin_until(gs.bar, (phase + 1u) * (unsigned)G, gs.abort);
    if (!ok) {
      atomicExch(gs.abort, 1u);
      atomicOr(gs.status, ST_TIMEOUT);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  if (!ok_s) return false;
  if (threadIdx.x < 32) {
    double a = kMax ? -INFINITY : 0.0, b = kMax ? -INFINITY : 0.0;
    for (int j = threadIdx.x; j < G; j += 32) {
      const double x0 = __ldcg(part + 2 * j), x1 = __ldcg(part + 2 * j + 1);
      if (kMax) { a = fmax(a, x0); b = fmax(b, x1); } else { a += x0; b += x1; }
    }
    if (kMax) { a = warp_max(a); b = warp_max(b); } else { a = warp_sum(a); b = warp_sum(b); }
    if (threadIdx.x == 0) { red[0] = a; red[1] = b; }
  }
  __syncthreads();
  v0 = red[0];
  v1 = red[1];
  __syncthreads();
  ++phase;
  return true;
}
}  // namespace

template <int EPT>
__global__ void __launch_bounds__(kThreads) bisect_kernel(const double* __restrict__ ell, int N,
                                                          const double* __restrict__ beta_in, double rho, int iters,
                                                          double* __restrict__ w_out, double* __restrict__ out,
                                                          GridSync gs) {
  __shared__ double red[64];
  const int stride = gridDim.x * kThreads;
  const int gid = blockIdx.x * kThreads + threadIdx.x;
  double l[EPT];
  int nonfinite = 0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = gid + e * stride;
    l[e] = i < N ? ell[i] : -INFINITY;
    if (i < N && !isfinite(l[e])) nonfinite = 1;
  }
  double lmax = -INFINITY, nf = (double)nonfinite;
#pragma unroll
  for (int e = 0; e < EPT; ++e) lmax = fmax(lmax, l[e]);
  unsigned phase = 0;
  if (!grid_reduce2<true>(gs, phase, lmax, nf, red)) return;
  if (nf > 0.0 && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(gs.status, ST_NONFINITE);
  // a_i = ell_i - max ell (<= 0; exactly 0 at the maximiser)
  double a[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) a[e] = (gid + e * stride < N) ? (l[e] - lmax) : -INFINITY;

  const double beta = *beta_in;
  const double target = rho * (double)N;
  auto ess_sums = [&](double d, double& s1, double& s2) {
    s1 = 0.0;
    s2 = 0.0;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      if (gid + e * stride < N) {
        const double w = exp(d * a[e]);
        s1 += w;
        s2 += w * w;
      }
    }
  };
  double hi = 1.0 - beta, lo = 0.0, d = hi;
  double s1, s2;
  ess_sums(hi, s1, s2);
  if (!grid_reduce2<false>(gs, phase, s1, s2, red)) return;
  int used = 0;
  bool to_one = (s1 * s1 / s2 >= target);
  if (!to_one) {
    for (int k = 0; k < iters; ++k) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      ++used;
      ess_sums(mid, s1, s2);
      if (!grid_reduce2<false>(gs, phase, s1, s2, red)) return;
      if (s1 * s1 / s2 >= target) lo = mid; else hi = mid;
    }
    if (lo == 0.0) {
      d = hi;
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(gs.status, ST_BISECT_FLOOR);
    } else {
      d = lo;
    }
  }
  // weights and the evidence increment at the chosen dbeta
  s1 = 0.0;
  s2 = 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = gid + e * stride;
    if (i < N) {
      const double w = exp(d * a[e]);
      w_out[i] = w;
      s1 += w;
      s2 += w * w;
    }
  }
  if (!grid_reduce2<false>(gs, phase, s1, s2, red)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = d;
    out[1] = to_one ? 1.0 : beta + d;
    out[2] = s1 * s1 / s2;
    out[3] = d * lmax + log(s1) - log((double)N);
    out[4] = (double)used;
  }
}

__global__ void logz_accumulate_kernel(const double* __restrict__ out, double* __restrict__ kahan,
                                       double* __restrict__ beta) {
  // Kahan-compensated running log Z over temperatures: kahan[0] = sum, kahan[1] = compensation.
  const double y = out[3] - kahan[1];
  const double t = kahan[0] + y;
  kahan[1] = (t - kahan[0]) - y;
  kahan[0] = t;
  *beta = out[1];
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
  return cudaLaunchCooperativeKernel((const void*)bisect_kernel<EPT>, dim3(G), dim3(kThreads), args, 0, s);
}

// One CTA: the grid barrier degenerates to the CTA's own arrival (nothing waits on
// another CTA), so an ordinary launch is safe next to other streams' work.
template <int EPT>
static cudaError_t launch_bisect_one(const double* ell, int N, const double* beta_in, double rho, int iters,
                                     double* w, double* out, GridSync gs, cudaStream_t s) {
  bisect_kernel<EPT><<<1, kThreads, 0, s>>>(ell, N, beta_in, rho, iters, w, out, gs);
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
    const int ept = (N + kThreads - 1) / kThreads;
    if (ept <= 8) return launch_bisect_one<8>(ell, N, beta_in, rho, iters, w, out, gs, s);
    if (ept <= 16) return launch_bisect_one<16>(ell, N, beta_in, rho, iters, w, out, gs, s);
    if (ept <= 32) return launch_bisect_one<32>(ell, N, beta_in, rho, iters, w, out, gs, s);
    return cudaErrorInvalidValue;
  }
  int G = (N + kThreads - 1) / kThreads;
  const int sms = sm_count();
  if (G > sms) G = sms;
  if (G > kMaxGrid) G = kMaxGrid;
  if (G < 1) G = 1;
  const int ept = (N + G * kThreads - 1) / (G * kThreads);
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
