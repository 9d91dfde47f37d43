// ESS bisection and reweighting of one population (Sec. 2 sampler (i); App. A target
// ESS) as a device function over G cooperating CTAs (bid = this CTA's index among them):
// the next temperature by bisection on the ESS of the incremental weights, the weights
// and the log-evidence increment. Every bisection step needs two sums over all N
// particles, so the CTAs meet at a software barrier (one atomic counter, a bounded
// acquire-spin) once per step; each CTA then adds the per-CTA partials in the same fixed
// order, so all CTAs take identical decisions and the result is deterministic. With G = 1
// the barrier is the CTA's own arrival. Used by the single-run kernel (G = gridDim.x) and
// by the batched kernel (one CTA per run, G = 1).
#pragma once
#include <math.h>
#include "common.cuh"

namespace phi4 {

constexpr int kBisectThreads = 128;

struct GridSync {
  unsigned* bar;       // arrival counter (zeroed before launch)
  unsigned* abort;     // set by a CTA whose wait gave up
  double* part;        // [2][G][2] per-CTA partials, double-buffered by phase parity
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

// Sum (or max) over the G CTAs of two doubles. Returns false if the barrier gave up.
template <bool kMax>
PHI4_DEV bool grid_reduce2(GridSync& gs, int G, int bid, unsigned& phase, double& v0, double& v1, double* red) {
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
    part[2 * bid] = v0;
    part[2 * bid + 1] = v1;
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

// out[0] = dbeta, out[1] = new beta, out[2] = ESS, out[3] = log Z increment,
// out[4] = halvings; w_out[i] = exp(dbeta (ell_i - max ell)).
template <int EPT>
PHI4_DEV void bisect_body(const double* __restrict__ ell, int N, const double* __restrict__ beta_in, double rho,
                          int iters, double* __restrict__ w_out, double* __restrict__ out, GridSync& gs, int G,
                          int bid) {
  __shared__ double red[64];
  const int stride = G * kBisectThreads;
  const int gid = bid * kBisectThreads + threadIdx.x;
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
  if (!grid_reduce2<true>(gs, G, bid, phase, lmax, nf, red)) return;
  if (nf > 0.0 && bid == 0 && threadIdx.x == 0) atomicOr(gs.status, ST_NONFINITE);
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
  if (!grid_reduce2<false>(gs, G, bid, phase, s1, s2, red)) return;
  int used = 0;
  bool to_one = (s1 * s1 / s2 >= target);
  if (!to_one) {
    for (int k = 0; k < iters; ++k) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      ++used;
      ess_sums(mid, s1, s2);
      if (!grid_reduce2<false>(gs, G, bid, phase, s1, s2, red)) return;
      if (s1 * s1 / s2 >= target) lo = mid; else hi = mid;
    }
    if (lo == 0.0) {
      d = hi;
      if (bid == 0 && threadIdx.x == 0) atomicOr(gs.status, ST_BISECT_FLOOR);
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
  if (!grid_reduce2<false>(gs, G, bid, phase, s1, s2, red)) return;
  if (bid == 0 && threadIdx.x == 0) {
    out[0] = d;
    out[1] = to_one ? 1.0 : beta + d;
    out[2] = s1 * s1 / s2;
    out[3] = d * lmax + log(s1) - log((double)N);
    out[4] = (double)used;
  }
}

// Kahan-compensated running log Z over temperatures: kahan[0] = sum, kahan[1] =
// compensation; the new beta is out[1].
PHI4_DEV void logz_accumulate(const double* __restrict__ out, double* __restrict__ kahan, double* __restrict__ beta) {
  const double y = out[3] - kahan[1];
  const double t = kahan[0] + y;
  kahan[1] = (t - kahan[0]) - y;
  kahan[0] = t;
  *beta = out[1];
}

}  // namespace phi4
