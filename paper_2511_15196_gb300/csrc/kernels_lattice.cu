// Periodic 4-neighbour stencil of Eq. (1): action, squared norm, Metropolis
// accept step and magnetisation. A particle's row is staged in shared memory
// (coalesced loads), each thread evaluates a strided set of sites, and the
// per-particle sums are reduced in a fixed order (deterministic).
//   D >= 1024: one particle per 256-thread CTA;  D < 1024: one particle per warp.
#include <math.h>
#include "internal.h"
#include <cuda_fp16.h>
#include "philox.cuh"
#include "batch.h"

namespace phi4 {

template <typename T>
struct SiteCoef {
  double ck, cm, lm;
};

// Per-thread partial sums of the site terms and of phi^2 over sites x = t, t+TPP, ...
template <typename T, int TPP>
PHI4_DEV void site_sums(const T* __restrict__ row, int L, int D, int t, SiteCoef<T> k, double& s_out,
                        double& q_out) {
  const int dr = TPP / L, dc = TPP % L;
  int r = t / L, c = t - (t / L) * L;
  if constexpr (sizeof(T) == 8) {
    double s = 0.0, q = 0.0;
    for (int x = t; x < D; x += TPP) {
      const int cl = c == 0 ? L - 1 : c - 1, cr = c == L - 1 ? 0 : c + 1;
      const int ru = r == 0 ? L - 1 : r - 1, rd = r == L - 1 ? 0 : r + 1;
      const double f = row[x];
      const double nb = row[r * L + cl] + row[r * L + cr] + row[ru * L + c] + row[rd * L + c];
      const double f2 = f * f;
      s += k.ck * (f * (4.0 * f - nb)) + k.cm * f2 + k.lm * (f2 * f2);
      q += f2;
      c += dc; r += dr;
      if (c >= L) { c -= L; ++r; }
    }
    s_out = s; q_out = q;
  } else {
    // float fields: exact products and compensated sums (site_terms_f2), the three partial
    // sums combined in double (K here is the neighbour-product sum C)
    AccF2 K, P2, P4;
    for (int x = t; x < D; x += TPP) {
      const int cr = c == L - 1 ? 0 : c + 1, rd = r == L - 1 ? 0 : r + 1;
      site_terms_f2(row[x], row[r * L + cr], row[rd * L + c], K, P2, P4);
      c += dc; r += dr;
      if (c >= L) { c -= L; ++r; }
    }
    const double p2 = P2.value();
    s_out = action_from_sums(K.value(), p2, P4.value(), k.ck, k.cm, k.lm);
    q_out = p2;
  }
}

// Reduce (a, b) over the TPP threads of a group; result valid in thread t == 0 of the group.
template <int TPP>
PHI4_DEV void group_sum2(double& a, double& b, double* red) {
  if constexpr (TPP == 32) {
    a = warp_sum(a);
    b = warp_sum(b);
  } else {
    a = block_sum(a, red);
    b = block_sum(b, red + 32);
  }
}

template <typename T>
PHI4_DEV SiteCoef<T> coefs(const ActionParams& p) {
  return SiteCoef<T>{p.c_kin, p.c_mass * p.m2, p.lam};
}

template <typename T, int PPB, int TPP>
__global__ void __launch_bounds__(PPB* TPP) action_kernel(const T* __restrict__ phi, ActionParams p,
                                                          double* __restrict__ S, double* __restrict__ sq,
                                                          double* __restrict__ ell, int keep_ref) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  T* rows = reinterpret_cast<T*>(smem_raw);
  const int g = threadIdx.x / TPP, t = threadIdx.x % TPP;
  const int i = blockIdx.x * PPB + g;
  T* row = rows + (size_t)g * p.D;
  if (i < p.N)
    for (int x = t; x < p.D; x += TPP) row[x] = phi[(size_t)i * p.D + x];
  __syncthreads();
  double s = 0.0, q = 0.0;
  if (i < p.N) site_sums<T, TPP>(row, p.L, p.D, t, coefs<T>(p), s, q);
  group_sum2<TPP>(s, q, red);
  if (i < p.N && t == 0) {
    S[i] = s;
    sq[i] = q;
    if (ell) ell[i] = keep_ref ? -s : (-s + 0.5 * q + p.half_d_log2pi);
  }
}

template <typename T, int PPB, int TPP>
__global__ void __launch_bounds__(PPB* TPP) accept_kernel(T* __restrict__ phi, const T* __restrict__ prop,
                                                          ActionParams p, int keep_ref, double* __restrict__ S,
                                                          double* __restrict__ sq, double* __restrict__ ell,
                                                          const double* __restrict__ beta_ptr, PhiloxKey key,
                                                          uint32_t w0, uint32_t sweep,
                                                          uint32_t* __restrict__ acc_count,
                                                          uint32_t* __restrict__ status,
                                                          const double* __restrict__ irmh_zz,
                                                          double* __restrict__ irmh_r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ int accept_flag[PPB];
  T* rows = reinterpret_cast<T*>(smem_raw);
  const int g = threadIdx.x / TPP, t = threadIdx.x % TPP;
  const int i = blockIdx.x * PPB + g;
  T* row = rows + (size_t)g * p.D;
  if (i < p.N)
    for (int x = t; x < p.D; x += TPP) row[x] = prop[(size_t)i * p.D + x];
  __syncthreads();
  double s = 0.0, q = 0.0;
  if (i < p.N) site_sums<T, TPP>(row, p.L, p.D, t, coefs<T>(p), s, q);
  group_sum2<TPP>(s, q, red);
  if (i < p.N && t == 0) {
    const double beta = *beta_ptr;
    const double dS = s - S[i], dq = q - sq[i];
    double log_alpha = keep_ref ? (-beta * dS - 0.5 * dq) : (-beta * dS - (1.0 - beta) * 0.5 * dq);
    if (irmh_zz) log_alpha += 0.5 * (irmh_zz[i] - irmh_r[i]);  // log q(phi) - log q(phi')
    const uint4 w = philox4x32_10(make_uint4(w0, sweep, (uint32_t)i, 0u), key);
    const double u = uniform53(w.x, w.y);
    int acc = log(u) < log_alpha;
    if (!isfinite(s) || !isfinite(q)) {
      atomicOr(status, ST_NONFINITE);
      acc = 0;
    }
    accept_flag[g] = acc;
    if (acc) {
      S[i] = s;
      sq[i] = q;
      ell[i] = keep_ref ? -s : (-s + 0.5 * q + p.half_d_log2pi);
      if (irmh_zz) irmh_r[i] = irmh_zz[i];
      atomicAdd(acc_count, 1u);
    }
  }
  __syncthreads();
  if (i < p.N && accept_flag[g])
    for (int x = t; x < p.D; x += TPP) phi[(size_t)i * p.D + x] = row[x];
}

// SMC-HMC transition (Sec. 2 sampler (iii)). Inverse mass v_s = Sigma_ss + ridge (the
// refit's covariance diagonal), momenta p = z / sqrt(v). The kernel integrates in the
// whitened momentum y = sqrt(v) p (y = z at the start, kinetic energy |y|^2 / 2), so with
// e_s = eps sqrt(v_s) a leapfrog step is x += e y, y += e g(x) and the first and last
// momentum steps are half steps. g is the gradient of the tempered log target,
//   g_s = -beta (c_kin (8 x_s - 2 sum of neighbours) + 2 c_mass m2 x_s + 4 lam x_s^3) - a x_s
//       = A x_s + B nb_s + C x_s^3,
// a = 1 - beta (1 with the reference kept). Accept when log u < H(start) - H(end) with
// H = beta S + a |x|^2 / 2 + |y|^2 / 2, the sums in double.

// e_s = eps sqrt(Sigma_ss + ridge), once per temperature
__global__ void hmc_scale_kernel(const double* __restrict__ sigma, int D, const double* __restrict__ ridge,
                                 double eps, double* __restrict__ e) {
  const double dl = *ridge;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < D; s += gridDim.x * blockDim.x)
    e[s] = eps * sqrt(sigma[(size_t)s * D + s] + dl);
}

// Sum (a, b) over the TPP threads of each particle's group; valid in the group's thread 0.
template <int TPP>
PHI4_DEV void hmc_group_sum2(double& a, double& b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  if constexpr (TPP > 32) {
    constexpr int WPG = TPP / 32;
    const int w = threadIdx.x >> 5, g = threadIdx.x / TPP;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      red[2 * w] = a;
      red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x % TPP == 0) {
      a = b = 0.0;
      for (int k = 0; k < WPG; ++k) {
        a += red[2 * (g * WPG + k)];
        b += red[2 * (g * WPG + k) + 1];
      }
    }
  }
}

// TPP threads per particle, max(TPP, 256) threads per CTA; thread t of a group owns sites
// t + k TPP (k < K) in registers: its field, y and e, and the four neighbour indices. The
// field also lives in a double-buffered shared row so neighbours can read it: one barrier
// per leapfrog step (the buffer written at step l was last read at step l - 2, before the
// barrier of step l - 1).
template <typename T, int TPP, int K>
__global__ void __launch_bounds__(TPP < 256 ? 256 : TPP)
    hmc_kernel(T* __restrict__ phi, const T* __restrict__ Z, const double* __restrict__ escale, ActionParams p,
               int keep_ref, double* __restrict__ S, double* __restrict__ sq, double* __restrict__ ell,
               const double* __restrict__ beta_ptr, int n_leap, PhiloxKey key, uint32_t w0, uint32_t sweep,
               uint32_t* __restrict__ acc_count, uint32_t* __restrict__ status) {
  constexpr int NT = TPP < 256 ? 256 : TPP;
  constexpr int PPB = NT / TPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ int accept_flag[PPB];
  const int L = p.L, D = p.D;
  const int g = threadIdx.x / TPP, t = threadIdx.x % TPP;
  const int i = blockIdx.x * PPB + g;
  const bool live = i < p.N;
  T* buf0 = reinterpret_cast<T*>(smem_raw) + (size_t)g * 2 * D;
  T* buf1 = buf0 + D;
  const double beta = *beta_ptr, a = keep_ref ? 1.0 : 1.0 - beta;
  const T A = (T)(-beta * (8.0 * p.c_kin + 2.0 * p.c_mass * p.m2) - a);
  const T B = (T)(2.0 * beta * p.c_kin);
  const T C = (T)(-4.0 * beta * p.lam);
  T x[K], y[K], e[K];
  uint32_t lr[K], ud[K];
  double kin0 = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int s = t + k * TPP;
    x[k] = y[k] = e[k] = T(0);
    lr[k] = ud[k] = 0u;
    if (live && s < D) {
      const int r = s / L, c = s - r * L;
      const int cl = c == 0 ? L - 1 : c - 1, cr = c == L - 1 ? 0 : c + 1;
      const int ru = r == 0 ? L - 1 : r - 1, rd = r == L - 1 ? 0 : r + 1;
      lr[k] = (uint32_t)(r * L + cl) | ((uint32_t)(r * L + cr) << 16);
      ud[k] = (uint32_t)(ru * L + c) | ((uint32_t)(rd * L + c) << 16);
      x[k] = phi[(size_t)i * D + s];
      buf0[s] = x[k];
      y[k] = Z[(size_t)i * D + s];
      e[k] = (T)escale[s];
      kin0 += (double)y[k] * (double)y[k];
    }
  }
  auto sync = [&]() {
    if constexpr (NT == 32) __syncwarp();
    else __syncthreads();
  };
  // y += h e g(x) over the own sites, neighbours from the row `cur`
  auto kick = [&](const T* __restrict__ cur, T h) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k * TPP < D) {
        const int s = t + k * TPP;
        if (live && s < D) {
          const T nb = (cur[lr[k] & 0xffffu] + cur[lr[k] >> 16]) + (cur[ud[k] & 0xffffu] + cur[ud[k] >> 16]);
          const T f = x[k];
          const T gr = fma(C, f * f * f, fma(A, f, B * nb));
          y[k] = fma(h * e[k], gr, y[k]);
        }
      }
    }
  };
  sync();
  kick(buf0, T(0.5));
  T* cur = buf0;
  for (int l = 0; l < n_leap; ++l) {
    T* nxt = cur == buf0 ? buf1 : buf0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int s = t + k * TPP;
      if (k * TPP < D && live && s < D) {
        x[k] = fma(e[k], y[k], x[k]);
        nxt[s] = x[k];
      }
    }
    sync();
    cur = nxt;
    kick(cur, l + 1 < n_leap ? T(1) : T(0.5));
  }
  double s_new = 0.0, q_new = 0.0, kin1 = 0.0;
  if (live) site_sums<T, TPP>(cur, L, D, t, coefs<T>(p), s_new, q_new);
#pragma unroll
  for (int k = 0; k < K; ++k) kin1 += (double)y[k] * (double)y[k];
  hmc_group_sum2<TPP>(s_new, q_new, red);
  hmc_group_sum2<TPP>(kin0, kin1, red);
  if (live && t == 0) {
    const double dS = s_new - S[i], dq = q_new - sq[i];
    const double log_alpha = (keep_ref ? (-beta * dS - 0.5 * dq) : (-beta * dS - (1.0 - beta) * 0.5 * dq)) -
                             0.5 * (kin1 - kin0);
    const uint4 w = philox4x32_10(make_uint4(w0, sweep, (uint32_t)i, 0u), key);
    int acc = log(uniform53(w.x, w.y)) < log_alpha;
    if (!isfinite(s_new) || !isfinite(q_new)) {
      atomicOr(status, ST_NONFINITE);
      acc = 0;
    }
    accept_flag[g] = acc;
    if (acc) {
      S[i] = s_new;
      sq[i] = q_new;
      ell[i] = keep_ref ? -s_new : (-s_new + 0.5 * q_new + p.half_d_log2pi);
      atomicAdd(acc_count, 1u);
    }
  }
  sync();
  if (live && accept_flag[g]) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int s = t + k * TPP;
      if (k * TPP < D && s < D) phi[(size_t)i * D + s] = x[k];
    }
  }
}

namespace {
template <typename T, int TPP, int K>
cudaError_t hmc_go(T* phi, const T* Z, const double* escale, const ActionParams& p, int keep, double* S, double* sq,
                   double* ell, const double* beta, int n_leap, PhiloxKey key, uint32_t w0, uint32_t sweep,
                   uint32_t* acc_count, uint32_t* status, cudaStream_t s) {
  constexpr int NT = TPP < 256 ? 256 : TPP;
  constexpr int PPB = NT / TPP;
  const size_t sm = (size_t)PPB * 2 * p.D * sizeof(T);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(hmc_kernel<T, TPP, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  hmc_kernel<T, TPP, K><<<(unsigned)((p.N + PPB - 1) / PPB), NT, sm, s>>>(
      phi, Z, escale, p, keep, S, sq, ell, beta, n_leap, key, w0, sweep, acc_count, status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_hmc_scale(const double* sigma, int D, const double* ridge, double eps, double* escale,
                             cudaStream_t s) {
  hmc_scale_kernel<<<(unsigned)((D + 255) / 256), 256, 0, s>>>(sigma, D, ridge, eps, escale);
  return cudaGetLastError();
}

// Layouts: each thread owns at most 4 sites (float) or 8 (double), so the float form keeps
// about 64 registers and 1024-thread CTAs at D = 4096 (32 warps per SM).
cudaError_t launch_hmc(void* phi, const void* Z, int dtype, const double* escale, const ActionParams& p,
                       int keep_reference, double* S, double* sq, double* ell, const double* beta, int n_leap,
                       uint64_t seed, uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count,
                       uint32_t* status, cudaStream_t s) {
  if (p.N <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(RNG_ACCEPT, step);
  const int D = p.D;
#define PHI4_HMC_GO(T, TPP, K)                                                                                   \
  return hmc_go<T, TPP, K>((T*)phi, (const T*)Z, escale, p, keep_reference, S, sq, ell, beta, n_leap, key, w0, \
                           sweep, acc_count, status, s)
  if (dtype == 0) {
    if (D <= 256) PHI4_HMC_GO(double, 32, 8);
    if (D <= 512) PHI4_HMC_GO(double, 64, 8);
    if (D <= 1024) PHI4_HMC_GO(double, 128, 8);
    if (D <= 2048) PHI4_HMC_GO(double, 256, 8);
    if (D <= 4096) PHI4_HMC_GO(double, 512, 8);
  } else if (dtype == 1) {
    if (D <= 128) PHI4_HMC_GO(float, 32, 4);
    if (D <= 256) PHI4_HMC_GO(float, 64, 4);
    if (D <= 512) PHI4_HMC_GO(float, 128, 4);
    if (D <= 1024) PHI4_HMC_GO(float, 256, 4);
    if (D <= 2048) PHI4_HMC_GO(float, 512, 4);
    if (D <= 4096) PHI4_HMC_GO(float, 1024, 4);
  }
#undef PHI4_HMC_GO
  return cudaErrorInvalidValue;
}

// Metropolis decision log u < log alpha for u in (0, 1] (53-bit), taken exactly as in
// double precision but mostly without the double log: log u lies in [log 2^-53, 0],
// so log alpha > 0 accepts and log alpha < -40 rejects; otherwise logf of the
// float-rounded u is within 1e-5 of log u (float rounding of u and logf's error
// bound), so only draws inside that margin need the double log.
PHI4_DEV int accept_decision(double u, double log_alpha) {
  if (!(log_alpha == log_alpha)) return 0;
  if (log_alpha > 0.0) return 1;
  if (log_alpha == 0.0) return u < 1.0;
  if (log_alpha < -40.0) return 0;
  const double lf = (double)logf((float)u);
  if (lf < log_alpha - 2e-5) return 1;
  if (lf > log_alpha + 2e-5) return 0;
  return log(u) < log_alpha;
}

// The same decision from the raw Philox words of u = (x + 1) 2^-53, x = (w0 << 21) |
// (w1 >> 11), with no FP64 instruction on the common path (an FP64 instruction holds
// its sub-partition's FP64 unit for 64 cycles on this part): the special cases of
// log alpha are read from its bit pattern, u and log alpha are truncated to float with
// integer operations (relative error <= 2^-23 each), and logf of the float u is within
// 5e-6 of log u for |log u| <= 37; outside a 2e-5 band the float comparison decides,
// inside it the double one does (rare).
PHI4_DEV int accept_decision_bits(uint32_t w0, uint32_t w1, double log_alpha) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(log_alpha);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long x = ((unsigned long long)w0 << 21) | (unsigned long long)(w1 >> 11);
  if (mag > 0x7FF0000000000000ull) return 0;                // NaN
  if (mag == 0ull) return x != (1ull << 53) - 1ull;          // log alpha = 0: accept iff u < 1
  if ((b >> 63) == 0ull) return 1;                           // log alpha > 0 (or +inf)
  if (mag > 0x4044000000000000ull) return 0;                 // log alpha < -40 (or -inf) <= log 2^-53
  // float of u (truncated): the top 24 bits of x + 1 <= 2^53 with its exponent
  const unsigned long long x1 = x + 1ull;
  const int lz = __clzll((long long)x1);                     // 11 .. 63
  const int top = 63 - lz;                                   // x1 in [2^top, 2^(top+1))
  const uint32_t man = top >= 23 ? (uint32_t)(x1 >> (top - 23)) : (uint32_t)(x1 << (23 - top));
  const float uf = __uint_as_float(((uint32_t)(top - 53 + 127) << 23) | (man & 0x7FFFFFu));
  // float of log alpha (truncated, negative, |log alpha| <= 40; tiny values flush to -0)
  const int ex = (int)(mag >> 52) - 1023 + 127;
  const float la = ex <= 0 ? -0.0f : __uint_as_float(0x80000000u | ((uint32_t)ex << 23) | (uint32_t)((mag >> 29) & 0x7FFFFFull));
  const float lf = logf(uf);
  if (lf < la - 2e-5f) return 1;
  if (lf > la + 2e-5f) return 0;
  return log((double)x1 * 0x1p-53) < log_alpha;
}

// Float fields with L % 4 == 0: each thread owns float4 groups of four sites of one
// lattice row (kept in registers), reads the down neighbour group and the right end
// neighbour from the staged row, and sums the site terms with exact products and
// compensated float sums (site_terms_f2); the sums travel as float pairs through the
// warp and CTA trees and are combined into S and |phi|^2 in double, so S of the float
// fields is exact to about 2^-48 relative. The proposal is either a float row `prop` or
// phi + delta with delta an fp16 increment (the tensor-core proposal's epilogue output). The block holds PPB particles of TPP threads each (PPB <= 8,
// TPP <= 256, TPP a multiple of 32, PPB * TPP = blockDim.x); particle g of the block is
// i = i0 + g, and `rot` rotates the decision warp over the block's warps.
constexpr int kVecMaxPPB = 8, kVecMaxWarps = 8;
template <bool kDelta, int kMaxG>
PHI4_DEV void accept_vec_body(int PPB, int TPP, int i0, int N, int rot, float* __restrict__ phi,
                              const float* __restrict__ prop, const __half* __restrict__ delta,
                              const ActionParams& p, int keep_ref, double* __restrict__ S, double* __restrict__ sq,
                              double* __restrict__ ell, const double* __restrict__ beta_ptr, PhiloxKey key,
                              uint32_t w0, uint32_t sweep, uint32_t* __restrict__ acc_count,
                              uint32_t* __restrict__ status, float* __restrict__ rows) {
  __shared__ float red[kVecMaxPPB][kVecMaxWarps][6];
  __shared__ int accept_flag[kVecMaxPPB];
  __shared__ uint2 uwords[kVecMaxPPB];
  const int g = threadIdx.x / TPP, t = threadIdx.x % TPP;
  const int i = i0 + g;
  const int L = p.L, D = p.D, ng = D >> 2;
  float* row = rows + (size_t)g * D;
  float4 v[kMaxG];
  if (i < N) {
#pragma unroll
    for (int k = 0; k < kMaxG; ++k) {
      const int q = t + k * TPP;
      if (q < ng) {
        float4 f;
        if constexpr (kDelta) {
          f = reinterpret_cast<const float4*>(phi + (size_t)i * D)[q];
          const uint2 hv = reinterpret_cast<const uint2*>(delta + (size_t)i * D)[q];
          const float2 d01 = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
          const float2 d23 = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
          f.x += d01.x; f.y += d01.y; f.z += d23.x; f.w += d23.y;
        } else {
          f = reinterpret_cast<const float4*>(prop + (size_t)i * D)[q];
        }
        v[k] = f;
        reinterpret_cast<float4*>(row)[q] = f;
      }
    }
  }
  // the particle's decision is taken by warp wd (rotating with the block so the serial
  // double work lands on every sub-partition in turn); another warp draws its uniform's
  // words while the others start the stencil
  const int kWarps = TPP / 32;
  const int wd = (rot + g) % kWarps;
  if (i < N && t == ((wd + kWarps / 2) % kWarps) * 32) {
    const uint4 w = philox4x32_10(make_uint4(w0, sweep, (uint32_t)i, 0u), key);
    uwords[g] = make_uint2(w.x, w.y);
  }
  __syncthreads();
  // exact products and compensated float sums of the site terms (site_terms_f2; K holds the
  // neighbour-product sum C):
  // per thread, then per warp in float pairs; the decision warp adds the warps' pairs and
  // forms S and |phi|^2 in double
  AccF2 K, P2, P4;
  if (i < N) {
#pragma unroll
    for (int k = 0; k < kMaxG; ++k) {
      const int q = t + k * TPP;
      if (q < ng) {
        const int x0 = q << 2;
        const int r = x0 / L, c0 = x0 - r * L;
        const int rd = r == L - 1 ? 0 : r + 1;
        const float4 dn = reinterpret_cast<const float4*>(row + rd * L)[c0 >> 2];
        const float rt = row[r * L + (c0 + 4 == L ? 0 : c0 + 4)];
        const float4 f = v[k];
        site_terms_f2(f.x, f.y, dn.x, K, P2, P4);
        site_terms_f2(f.y, f.z, dn.y, K, P2, P4);
        site_terms_f2(f.z, f.w, dn.z, K, P2, P4);
        site_terms_f2(f.w, rt, dn.w, K, P2, P4);
      }
    }
  }
  K = warp_sum_f2(K);
  P2 = warp_sum_f2(P2);
  P4 = warp_sum_f2(P4);
  const int lane = t & 31, wg = t >> 5;
  if (lane == 0) {
    float* rr = red[g][wg];
    rr[0] = K.hi; rr[1] = K.lo; rr[2] = P2.hi; rr[3] = P2.lo; rr[4] = P4.hi; rr[5] = P4.lo;
  }
  __syncthreads();
  if (i < N && wg == wd) {
    AccF2 k2, q2, f2;
    if (lane < kWarps) {
      const float* rr = red[g][lane];
      k2.hi = rr[0]; k2.lo = rr[1]; q2.hi = rr[2]; q2.lo = rr[3]; f2.hi = rr[4]; f2.lo = rr[5];
    }
    k2 = warp_sum_f2(k2);
    q2 = warp_sum_f2(q2);
    f2 = warp_sum_f2(f2);
    if (lane == 0) {
      const double Qp = q2.value();
      const double Sp = action_from_sums(k2.value(), Qp, f2.value(), p.c_kin, p.c_mass * p.m2, p.lam);
      const double beta = *beta_ptr;
      const double dS = Sp - S[i], dq2 = Qp - sq[i];
      const double log_alpha = keep_ref ? (-beta * dS - 0.5 * dq2) : (-beta * dS - (1.0 - beta) * 0.5 * dq2);
      const uint2 uw = uwords[g];
      int acc = accept_decision_bits(uw.x, uw.y, log_alpha);
      const unsigned long long bs = (unsigned long long)__double_as_longlong(Sp),
                               bq = (unsigned long long)__double_as_longlong(Qp);
      if (((bs >> 52) & 0x7FF) == 0x7FF || ((bq >> 52) & 0x7FF) == 0x7FF) {  // not finite
        atomicOr(status, ST_NONFINITE);
        acc = 0;
      }
      accept_flag[g] = acc;
      if (acc) {
        S[i] = Sp;
        sq[i] = Qp;
        ell[i] = keep_ref ? -Sp : (-Sp + 0.5 * Qp + p.half_d_log2pi);
        atomicAdd(acc_count, 1u);
      }
    }
  }
  __syncthreads();
  if (i < N && accept_flag[g]) {
#pragma unroll
    for (int k = 0; k < kMaxG; ++k) {
      const int q = t + k * TPP;
      if (q < ng) reinterpret_cast<float4*>(phi + (size_t)i * D)[q] = v[k];
    }
  }
}

template <int PPB, int TPP, bool kDelta, int kMaxG>
__global__ void __launch_bounds__(PPB* TPP) accept_vec_kernel(float* __restrict__ phi, const float* __restrict__ prop,
                                                              const __half* __restrict__ delta, ActionParams p,
                                                              int keep_ref, double* __restrict__ S,
                                                              double* __restrict__ sq, double* __restrict__ ell,
                                                              const double* __restrict__ beta_ptr, PhiloxKey key,
                                                              uint32_t w0, uint32_t sweep,
                                                              uint32_t* __restrict__ acc_count,
                                                              uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  accept_vec_body<kDelta, kMaxG>(PPB, TPP, (int)blockIdx.x * PPB, p.N, (int)blockIdx.x, phi, prop, delta, p,
                                 keep_ref, S, sq, ell, beta_ptr, key, w0, sweep, acc_count, status,
                                 reinterpret_cast<float*>(smem_raw));
}

// Batched form: one launch over the blocks of every member run (mixed form, L % 4 == 0).
// Block b belongs to the run r with blk0[r] <= b < blk0[r + 1] (binary search over the
// runs' block offsets); its particles and block shape (PPB, TPP) are that run's, the same
// as a single run's launch picks, so the results equal the single-run kernel's. Runs that
// are done (scal[SC_ACTIVE] == 0) or whose sweeps are fewer than `sweep` + 1 are skipped;
// the temperature index comes from the run's device counter. Every shape the single-run
// launcher picks fills the 256 threads (PPB * TPP = 256).
__global__ void __launch_bounds__(256) batch_accept_kernel(const BatchRun* __restrict__ runs, int R,
                                                           const int* __restrict__ blk0, uint32_t sweep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk0[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const BatchRun& b = runs[lo];
  if (b.scal[SC_ACTIVE] == 0.0 || (int)sweep >= b.n_mcmc) return;
  const int local = (int)blockIdx.x - blk0[lo];
  const uint32_t t = (uint32_t)b.scal[SC_T];
  accept_vec_body<true, 8>(b.ppb, b.tpp, local * b.ppb, b.ap.N, local, (float*)b.phi_dst, nullptr, b.delta, b.ap,
                           b.keep_ref, b.S_dst, b.sq_dst, b.ell_dst, b.scal + SC_BETA, b.key,
                           counter_word0(RNG_ACCEPT, t), sweep, b.acc, b.status, reinterpret_cast<float*>(smem_raw));
}

cudaError_t batch_accept_prepare(size_t smem) { return set_smem_bytes((const void*)batch_accept_kernel, smem); }

cudaError_t launch_batch_accept(const BatchRun* runs, int R, const int* blk0, int n_blocks, size_t smem,
                                uint32_t sweep, cudaStream_t s) {
  if (n_blocks <= 0) return cudaSuccess;
  batch_accept_kernel<<<n_blocks, 256, smem, s>>>(runs, R, blk0, sweep);
  return cudaGetLastError();
}

// The block shape the single-run launcher picks for a mixed run of D sites (see accept_vec).
void accept_vec_shape(int D, int* ppb, int* tpp) {
  if (D >= 1024) { *ppb = 1; *tpp = 256; } else { *ppb = 8; *tpp = 32; }
}

template <typename T>
__global__ void magnetisation_kernel(const T* __restrict__ phi, int N, int D, double* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= N) return;
  double s = 0.0;
  for (int x = lane; x < D; x += 32) s += (double)phi[(size_t)i * D + x];
  s = warp_sum(s);
  if (lane == 0) M[i] = s / D;
}

cudaError_t set_smem_bytes(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

namespace {
template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
constexpr int kBigD = 1024;
}  // namespace

template <typename T>
static cudaError_t action_t(const T* phi, const ActionParams& p, double* S, double* sq, double* ell, int keep_ref,
                            cudaStream_t s) {
  if (p.D >= kBigD) {
    const size_t sm = (size_t)p.D * sizeof(T);
    cudaError_t e = set_smem(action_kernel<T, 1, 256>, sm);
    if (e != cudaSuccess) return e;
    action_kernel<T, 1, 256><<<p.N, 256, sm, s>>>(phi, p, S, sq, ell, keep_ref);
  } else {
    const size_t sm = (size_t)8 * p.D * sizeof(T);
    cudaError_t e = set_smem(action_kernel<T, 8, 32>, sm);
    if (e != cudaSuccess) return e;
    action_kernel<T, 8, 32><<<(p.N + 7) / 8, 256, sm, s>>>(phi, p, S, sq, ell, keep_ref);
  }
  return cudaGetLastError();
}

cudaError_t launch_action(const void* phi, int dtype, const ActionParams& p, double* S, double* sq, double* ell,
                          int keep_reference, cudaStream_t s) {
  if (p.N <= 0) return cudaSuccess;
  if (dtype == 0) return action_t<double>((const double*)phi, p, S, sq, ell, keep_reference, s);
  if (dtype == 1) return action_t<float>((const float*)phi, p, S, sq, ell, keep_reference, s);
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t accept_t(T* phi, const T* prop, const ActionParams& p, int keep_ref, double* S, double* sq,
                            double* ell, const double* beta, PhiloxKey key, uint32_t w0, uint32_t sweep,
                            uint32_t* acc, uint32_t* status, cudaStream_t s, const double* irmh_zz = nullptr,
                            double* irmh_r = nullptr) {
  if (p.D >= kBigD) {
    const size_t sm = (size_t)p.D * sizeof(T);
    cudaError_t e = set_smem(accept_kernel<T, 1, 256>, sm);
    if (e != cudaSuccess) return e;
    accept_kernel<T, 1, 256><<<p.N, 256, sm, s>>>(phi, prop, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc,
                                                  status, irmh_zz, irmh_r);
  } else {
    const size_t sm = (size_t)8 * p.D * sizeof(T);
    cudaError_t e = set_smem(accept_kernel<T, 8, 32>, sm);
    if (e != cudaSuccess) return e;
    accept_kernel<T, 8, 32><<<(p.N + 7) / 8, 256, sm, s>>>(phi, prop, p, keep_ref, S, sq, ell, beta, key, w0,
                                                           sweep, acc, status, irmh_zz, irmh_r);
  }
  return cudaGetLastError();
}

template <int PPB, int TPP, bool kDelta, int G>
static cudaError_t accept_vec_g(float* phi, const float* prop, const __half* delta, const ActionParams& p, int keep_ref,
                                double* S, double* sq, double* ell, const double* beta, PhiloxKey key, uint32_t w0,
                                uint32_t sweep, uint32_t* acc, uint32_t* status, cudaStream_t s) {
  const size_t sm = (size_t)PPB * p.D * sizeof(float);
  cudaError_t e = set_smem(accept_vec_kernel<PPB, TPP, kDelta, G>, sm);
  if (e != cudaSuccess) return e;
  accept_vec_kernel<PPB, TPP, kDelta, G><<<(p.N + PPB - 1) / PPB, PPB * TPP, sm, s>>>(
      phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status);
  return cudaGetLastError();
}

template <bool kDelta>
static cudaError_t accept_vec(float* phi, const float* prop, const __half* delta, const ActionParams& p, int keep_ref,
                              double* S, double* sq, double* ell, const double* beta, PhiloxKey key, uint32_t w0,
                              uint32_t sweep, uint32_t* acc, uint32_t* status, cudaStream_t s) {
  // float4 groups per thread: D / 4 / threads-per-particle
  if (p.D >= kBigD) {
    const int g = (p.D / 4 + 255) / 256;
    if (g <= 1) return accept_vec_g<1, 256, kDelta, 1>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
    if (g <= 2) return accept_vec_g<1, 256, kDelta, 2>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
    if (g <= 4) return accept_vec_g<1, 256, kDelta, 4>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
    return accept_vec_g<1, 256, kDelta, 8>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
  }
  const int g = (p.D / 4 + 31) / 32;
  if (g <= 2) return accept_vec_g<8, 32, kDelta, 2>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
  if (g <= 4) return accept_vec_g<8, 32, kDelta, 4>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
  return accept_vec_g<8, 32, kDelta, 8>(phi, prop, delta, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc, status, s);
}

static bool vec_ok(const ActionParams& p) { return p.L % 4 == 0 && p.D <= 8 * 4 * 256; }

cudaError_t launch_accept_delta(float* phi, const void* delta_f16, const ActionParams& p, int keep_reference,
                                double* S, double* sq, double* ell, const double* beta, uint64_t seed,
                                uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count,
                                uint32_t* status, cudaStream_t s) {
  if (p.N <= 0) return cudaSuccess;
  if (!vec_ok(p)) return cudaErrorInvalidValue;
  return accept_vec<true>(phi, nullptr, (const __half*)delta_f16, p, keep_reference, S, sq, ell, beta,
                          philox_key(seed, stream_id), counter_word0(RNG_ACCEPT, step), sweep, acc_count, status, s);
}

cudaError_t launch_accept(void* phi, const void* prop, int dtype, const ActionParams& p, int keep_reference,
                          double* S, double* sq, double* ell, const double* beta, uint64_t seed, uint64_t stream_id,
                          uint32_t step, uint32_t sweep, uint32_t* acc_count, uint32_t* status, cudaStream_t s,
                          const double* irmh_zz, double* irmh_r) {
  if (p.N <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(RNG_ACCEPT, step);
  if (irmh_zz) {
    if (dtype != 0) return cudaErrorInvalidValue;
    return accept_t<double>((double*)phi, (const double*)prop, p, keep_reference, S, sq, ell, beta, key, w0, sweep,
                            acc_count, status, s, irmh_zz, irmh_r);
  }
  if (dtype == 1 && vec_ok(p))
    return accept_vec<false>((float*)phi, (const float*)prop, nullptr, p, keep_reference, S, sq, ell, beta, key, w0,
                             sweep, acc_count, status, s);
  if (dtype == 0)
    return accept_t<double>((double*)phi, (const double*)prop, p, keep_reference, S, sq, ell, beta, key, w0, sweep,
                            acc_count, status, s);
  if (dtype == 1)
    return accept_t<float>((float*)phi, (const float*)prop, p, keep_reference, S, sq, ell, beta, key, w0, sweep,
                           acc_count, status, s);
  return cudaErrorInvalidValue;
}

__global__ void apply_delta_kernel(const float* __restrict__ phi, const __half* __restrict__ delta,
                                   float* __restrict__ prop, long long n) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    prop[k] = phi[k] + __half2float(delta[k]);
}

cudaError_t launch_apply_delta(const float* phi, const void* delta_f16, float* prop, long long n, cudaStream_t s) {
  apply_delta_kernel<<<sm_count() * 8, 256, 0, s>>>(phi, (const __half*)delta_f16, prop, n);
  return cudaGetLastError();
}

cudaError_t launch_magnetisation(const void* phi, int dtype, int N, int D, double* M, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((N + 7) / 8);
  if (dtype == 0) magnetisation_kernel<double><<<grid, 256, 0, s>>>((const double*)phi, N, D, M);
  else if (dtype == 1) magnetisation_kernel<float><<<grid, 256, 0, s>>>((const float*)phi, N, D, M);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace phi4
