// Shared device helpers of the phi4smc kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include "internal.h"

#define PHI4_DEV __device__ __forceinline__

namespace phi4 {

// Bits of the device status word.
enum : uint32_t {
  ST_NONFINITE = 1u,     // NaN/Inf in log-weights or the action
  ST_NOT_PD = 2u,        // non-positive Cholesky pivot
  ST_TIMEOUT = 4u,       // a bounded device wait gave up
  ST_BISECT_FLOOR = 8u,  // no positive dbeta kept ESS >= rho N
};

// Every spin-wait in this library gives up after about one second of SM clock.
constexpr long long kSpinLimitCycles = kSpinLimitCyclesDefault;

// Limit of the software waits (grid barriers, flags between CTAs, hand-offs between
// warps), in SM clock cycles, kSpinLimitCycles unless phi4_set_spin_limit changed it.
// Each translation unit holds its own copy of this variable; phi4_set_spin_limit sets
// every copy (see PHI4_SPIN_LIMIT_SETTER). The waits on TMA copies and tensor-core
// commits keep kSpinLimitCycles: they wait on hardware that completes by itself, and
// leaving them early would leave copies in flight into the CTA's shared memory.
static __device__ long long g_spin_limit = kSpinLimitCycles;
PHI4_DEV long long spin_limit() { return *(volatile long long*)&g_spin_limit; }
#define PHI4_SPIN_LIMIT_SETTER(fn) \
  cudaError_t fn(long long cycles) { return cudaMemcpyToSymbol(g_spin_limit, &cycles, sizeof(cycles)); }

// CTA-scope mbarrier helpers (shared-memory barrier objects, phase parity waits).
PHI4_DEV uint32_t cta_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation waits here until the previous kernel of its stream has completed and
// its writes are visible (immediately when launched without it); `pdl_trigger` lets
// the next such kernel be launched before this one ends.
PHI4_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
PHI4_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
PHI4_DEV void cta_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cta_smem_addr(bar)), "r"(count) : "memory");
}
PHI4_DEV void cta_mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cta_smem_addr(bar)) : "memory");
}
PHI4_DEV bool cta_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(cta_smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity (a hand-off between warps); false
// after spin_limit() cycles or once another warp has raised *abort_flag.
PHI4_DEV bool cta_mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (cta_mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64(), lim = spin_limit();
  for (;;) {
    if (cta_mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > lim) return false;
  }
}

// Shared-memory progress counters between warps of one CTA: the producer publishes with
// a release store, consumers poll with acquire loads (cheaper than an mbarrier round
// trip when the value is already there). Waits are bounded like every spin here.
PHI4_DEV void cta_flag_release(int* f, int v) {
  asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(cta_smem_addr(f)), "r"(v) : "memory");
}
PHI4_DEV int cta_flag_acquire(const int* f) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(cta_smem_addr(f)) : "memory");
  return v;
}
PHI4_DEV bool cta_flag_wait_geq(const int* f, int target, volatile int* abort_flag) {
  if (cta_flag_acquire(f) >= target) return true;
  const long long t0 = clock64(), lim = spin_limit();
  for (;;) {
    if (cta_flag_acquire(f) >= target) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > lim) return false;
  }
}

// Progress counter in global memory between CTAs of one (co-resident) grid: release
// store after the producer's writes, acquire loads by the consumers.
PHI4_DEV void gpu_flag_release(int* f, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
PHI4_DEV int gpu_flag_acquire(const int* f) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}

PHI4_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
PHI4_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
PHI4_DEV double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
PHI4_DEV unsigned long long warp_incl_scan(unsigned long long v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide sum of one double per thread; every thread gets the result.
// `red` is shared scratch of >= 32 doubles. Deterministic order.
PHI4_DEV double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}
PHI4_DEV double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : -INFINITY;
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// Compensated float accumulator (Kahan): cheap on the FP32 pipes, keeps the
// per-thread partial sums of float site terms close to their exact value.
struct KahanF {
  float s = 0.f, c = 0.f;
  PHI4_DEV void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  PHI4_DEV double value() const { return (double)s - (double)c; }
};

// Error-free transformations in float (Knuth's two-sum; the two-product through one
// fused multiply-add): a + b = s + e and a * b = p + e exactly, with s, p the rounded
// results. They let the float forms sum float site terms to about 2^-48 relative.
PHI4_DEV void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
PHI4_DEV void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// A float pair hi + lo accumulating (hi, lo) terms: the running sum's rounding errors are
// collected exactly by two_sum and added, with the terms' low parts, into lo.
struct AccF2 {
  float hi = 0.f, lo = 0.f;
  PHI4_DEV void add(float th, float tl) {
    float s, e;
    two_sum(hi, th, s, e);
    hi = s;
    lo += e + tl;
  }
  PHI4_DEV void add(const AccF2& o) {
    add(o.hi, o.lo);
  }
  PHI4_DEV double value() const { return (double)hi + (double)lo; }
};

// Sum of an AccF2 over the 32 lanes (the same tree on every lane).
PHI4_DEV AccF2 warp_sum_f2(AccF2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    AccF2 b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a.add(b);
  }
  return a;
}

// The float site terms of Eq. (1), split so that every product is exact: the kinetic
// sum sum_x sum_mu (phi_{x+mu} - phi_x)^2 (the site form summed over the periodic lattice)
// equals 4 sum_x phi_x^2 - 2 sum_x phi_x (phi_right + phi_down), so each site contributes
// phi^2 to P2, phi^4 to P4 and phi phi_right + phi phi_down to C, each an exact product
// (two_prod) added to a compensated float pair. Then, in double,
//   S = (4 c_kin + c_mass m2) P2 - 2 c_kin C + lambda P4  and  |phi|^2 = P2;
// the pairs are exact to about 2^-48 of the summed terms, so S is exact to that order of
// the site terms' magnitude (the difference 4 P2 - 2 C may cancel; its absolute error does
// not grow). Dropped parts: squares of the low halves.
PHI4_DEV void site_terms_f2(float f, float fr, float fd, AccF2& C, AccF2& P2, AccF2& P4) {
  float ph, pl, qh, ql;
  two_prod(f, fr, ph, pl);
  C.add(ph, pl);
  two_prod(f, fd, ph, pl);
  C.add(ph, pl);
  two_prod(f, f, qh, ql);
  P2.add(qh, ql);
  two_prod(qh, qh, ph, pl);
  P4.add(ph, fmaf(2.f * qh, ql, pl));
}
// S and |phi|^2 from the three sums (double).
PHI4_DEV double action_from_sums(double C, double P2, double P4, double c_kin, double cm2, double lam) {
  return (4.0 * c_kin + cm2) * P2 - 2.0 * c_kin * C + lam * P4;
}

template <typename T> PHI4_DEV T to_t(float x);
template <> PHI4_DEV float to_t<float>(float x) { return x; }
template <> PHI4_DEV __nv_bfloat16 to_t<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

}  // namespace phi4
