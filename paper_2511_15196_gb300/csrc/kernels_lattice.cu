// Periodic 4-neighbour stencil of Eq. (1): action, squared norm, Metropolis
// accept step and magnetisation. A particle's row is staged in shared memory
// (coalesced loads), each thread evaluates a strided set of sites, and the
// per-particle sums are reduced in a fixed order (deterministic).
//   D >= 1024: one particle per 256-thread CTA;  D < 1024: one particle per warp.
#include <math.h>
#include "internal.h"
#include "philox.cuh"

namespace phi4 {

template <typename T>
struct SiteCoef {
  T ck, cm, lm;
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
    KahanF s, q;
    for (int x = t; x < D; x += TPP) {
      const int cl = c == 0 ? L - 1 : c - 1, cr = c == L - 1 ? 0 : c + 1;
      const int ru = r == 0 ? L - 1 : r - 1, rd = r == L - 1 ? 0 : r + 1;
      const float f = row[x];
      const float nb = row[r * L + cl] + row[r * L + cr] + row[ru * L + c] + row[rd * L + c];
      const float f2 = f * f;
      s.add(k.ck * (f * (4.0f * f - nb)) + k.cm * f2 + k.lm * (f2 * f2));
      q.add(f2);
      c += dc; r += dr;
      if (c >= L) { c -= L; ++r; }
    }
    s_out = s.value(); q_out = q.value();
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
  return SiteCoef<T>{(T)p.c_kin, (T)(p.c_mass * p.m2), (T)p.lam};
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
                                                          uint32_t* __restrict__ status) {
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
    const double log_alpha = keep_ref ? (-beta * dS - 0.5 * dq) : (-beta * dS - (1.0 - beta) * 0.5 * dq);
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
      atomicAdd(acc_count, 1u);
    }
  }
  __syncthreads();
  if (i < p.N && accept_flag[g])
    for (int x = t; x < p.D; x += TPP) phi[(size_t)i * p.D + x] = row[x];
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
                            uint32_t* acc, uint32_t* status, cudaStream_t s) {
  if (p.D >= kBigD) {
    const size_t sm = (size_t)p.D * sizeof(T);
    cudaError_t e = set_smem(accept_kernel<T, 1, 256>, sm);
    if (e != cudaSuccess) return e;
    accept_kernel<T, 1, 256><<<p.N, 256, sm, s>>>(phi, prop, p, keep_ref, S, sq, ell, beta, key, w0, sweep, acc,
                                                  status);
  } else {
    const size_t sm = (size_t)8 * p.D * sizeof(T);
    cudaError_t e = set_smem(accept_kernel<T, 8, 32>, sm);
    if (e != cudaSuccess) return e;
    accept_kernel<T, 8, 32><<<(p.N + 7) / 8, 256, sm, s>>>(phi, prop, p, keep_ref, S, sq, ell, beta, key, w0,
                                                           sweep, acc, status);
  }
  return cudaGetLastError();
}

cudaError_t launch_accept(void* phi, const void* prop, int dtype, const ActionParams& p, int keep_reference,
                          double* S, double* sq, double* ell, const double* beta, uint64_t seed, uint64_t stream_id,
                          uint32_t step, uint32_t sweep, uint32_t* acc_count, uint32_t* status, cudaStream_t s) {
  if (p.N <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(RNG_ACCEPT, step);
  if (dtype == 0)
    return accept_t<double>((double*)phi, (const double*)prop, p, keep_reference, S, sq, ell, beta, key, w0, sweep,
                            acc_count, status, s);
  if (dtype == 1)
    return accept_t<float>((float*)phi, (const float*)prop, p, keep_reference, S, sq, ell, beta, key, w0, sweep,
                           acc_count, status, s);
  return cudaErrorInvalidValue;
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
