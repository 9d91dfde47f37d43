// Nested sampling with slice-sampling rejuvenation (Sec. 2 sampler (iv); App. A):
// deletion of the lowest-likelihood live points with the prior-volume
// bookkeeping, start points, the constrained slice chains, replacement, the
// stopping rule and the final evidence with its information-based error bar.
//
// Slice chains. Prior N(0, I), likelihood log L = -S + |phi|^2/2 + (D/2) log 2pi.
// Along a line y = x + t d the action of Eq. (1) is a polynomial of degree four in
// t, so one pass of eleven site reductions gives the five coefficients of
// log L(x + t d) and every shrinkage try costs O(1) instead of a stencil pass:
//   a0 = -(ck xAx + cm |x|^2 + lm sum x^4) + |x|^2/2 + (D/2) log 2pi
//   a1 = -(2 ck xAd + 2 cm x.d + 4 lm sum x^3 d) + x.d
//   a2 = -(ck dAd + cm |d|^2 + 6 lm sum x^2 d^2) + |d|^2/2
//   a3 = -4 lm sum x d^3,   a4 = -lm sum d^4
// with A = 4I - (4-neighbour adjacency), ck = c_kin, cm = c_mass m2, lm = lambda.
// The prior slice along the line is the exact interval |x + t d|^2 < |x|^2 + 2E.
#include <math.h>
#include "internal.h"
#include "philox.cuh"

namespace phi4 {

namespace {
constexpr int kSortThreads = 1024;
constexpr int kSliceThreads = 256;
constexpr int kNumRed = 11;

PHI4_DEV double logaddexp_d(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = fmax(a, b);
  return m + log(exp(a - m) + exp(b - m));
}
}  // namespace

// Stable ascending order of log L (ties by index) by a bitonic sort of (key, index)
// in shared memory (N <= 8192), then the deletion bookkeeping of the k lowest:
// log X_j = log X_{j-1} - 1/(N-j+1), log w_j = log X_{j-1} + log(-expm1(-1/(N-j+1))),
// log Z = logaddexp(log Z, log L_j + log w_j), appended to the dead list.
// ns[0] = log X, ns[1] = log Z, ns[2] = L*, ns[3] = dead count (as double).
__global__ void __launch_bounds__(kSortThreads) ns_select_kernel(const double* __restrict__ logl, int N, int k,
                                                                 int32_t* __restrict__ order, double* __restrict__ ns,
                                                                 double* __restrict__ dead, long long dead_cap,
                                                                 uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int P = 1;
  while (P < N) P <<= 1;
  double* key = reinterpret_cast<double*>(smem_raw);
  int* idx = reinterpret_cast<int*>(key + P);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    key[i] = i < N ? logl[i] : INFINITY;
    idx[i] = i;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const double ki = key[i], kj = key[j];
          const int ii = idx[i], ij = idx[j];
          const bool gt = (ki > kj) || (ki == kj && ii > ij);
          if (gt == up) {
            key[i] = kj; key[j] = ki;
            idx[i] = ij; idx[j] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) order[i] = idx[i];
  if (threadIdx.x == 0) {
    double logX = ns[0], logZ = ns[1];
    long long nd = (long long)ns[3];
    if (nd + k > dead_cap) {
      atomicOr(status, ST_TIMEOUT);
    } else {
      for (int j = 1; j <= k; ++j) {
        const double shrink = 1.0 / (double)(N - j + 1);
        const double logw = logX + log(-expm1(-shrink));
        logX = logX - shrink;
        const double lj = key[j - 1];
        if (!isfinite(lj)) atomicOr(status, ST_NONFINITE);
        dead[2 * (nd + j - 1)] = lj;
        dead[2 * (nd + j - 1) + 1] = logw;
        logZ = logaddexp_d(logZ, lj + logw);
      }
      nd += k;
    }
    ns[0] = logX;
    ns[1] = logZ;
    ns[2] = key[k - 1];
    ns[3] = (double)nd;
  }
}

// Start point of every slot: survivors are order[k..N-1]; slot j starts from
// survivor floor(u (N-k)), u = word 0 of (NS_START, it, 0, j, 0) times 2^-32.
template <typename T>
__global__ void ns_start_kernel(const T* __restrict__ live, const int32_t* __restrict__ order, int N, int k, int D,
                                PhiloxKey key, uint32_t w0, T* __restrict__ X) {
  const int j = blockIdx.x;
  __shared__ int start;
  if (threadIdx.x == 0) {
    const uint4 w = philox4x32_10(make_uint4(w0, 0u, (uint32_t)j, 0u), key);
    const double u = (double)w.x * 0x1p-32;
    const int pick = (int)floor(u * (double)(N - k));
    start = order[k + pick];
  }
  __syncthreads();
  for (int x = threadIdx.x; x < D; x += blockDim.x) X[(size_t)j * D + x] = live[(size_t)start * D + x];
}

struct NsSliceParams {
  int L, D, steps, max_shrink;
  double ck, cm, lm, hc;  // c_kin, c_mass m2, lambda, (D/2) log 2pi
  const double* lstar;  // device: largest deleted log L of this iteration
};

// Per-site contributions to the eleven line reductions.
template <typename T>
PHI4_DEV void line_terms(const T* x, const T* d, int L, int site, T (&v)[kNumRed]) {
  const int r = site / L, c = site - r * L;
  const int cl = c == 0 ? L - 1 : c - 1, cr = c == L - 1 ? 0 : c + 1;
  const int ru = r == 0 ? L - 1 : r - 1, rd = r == L - 1 ? 0 : r + 1;
  const int a = r * L + cl, b = r * L + cr, u = ru * L + c, w = rd * L + c;
  const T xi = x[site], di = d[site];
  const T Ax = (T)4 * xi - (x[a] + x[b] + x[u] + x[w]);
  const T Ad = (T)4 * di - (d[a] + d[b] + d[u] + d[w]);
  const T x2 = xi * xi, d2 = di * di;
  v[0] = xi * Ax;       // xAx
  v[1] = xi * Ad;       // xAd
  v[2] = di * Ad;       // dAd
  v[3] = x2;            // |x|^2
  v[4] = xi * di;       // x.d
  v[5] = d2;            // |d|^2
  v[6] = x2 * x2;       // x^4
  v[7] = x2 * xi * di;  // x^3 d
  v[8] = x2 * d2;       // x^2 d^2
  v[9] = xi * di * d2;  // x d^3
  v[10] = d2 * d2;      // d^4
}

template <typename T>
PHI4_DEV T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Eleven reductions over the lattice; the result (double) lands in out[] for all threads.
template <typename T>
PHI4_DEV void line_reduce(const T* x, const T* d, int L, int D, double* warp_part, double* out) {
  T acc[kNumRed];
#pragma unroll
  for (int q = 0; q < kNumRed; ++q) acc[q] = (T)0;
  for (int site = threadIdx.x; site < D; site += blockDim.x) {
    T v[kNumRed];
    line_terms<T>(x, d, L, site, v);
#pragma unroll
    for (int q = 0; q < kNumRed; ++q) acc[q] += v[q];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < kNumRed; ++q) {
    const T s = warp_sum_t<T>(acc[q]);
    if (lane == 0) warp_part[wid * kNumRed + q] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < kNumRed) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += warp_part[w * kNumRed + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// One CTA per slot: `steps` slice steps from X[slot] under log L > L*; writes the
// final point back to X[slot] and its log L (exact quartic value a0) to logl_out[slot].
template <typename T>
__global__ void __launch_bounds__(kSliceThreads) ns_slice_kernel(T* __restrict__ X, double* __restrict__ logl_out,
                                                                 const T* __restrict__ Lf, NsSliceParams p,
                                                                 PhiloxKey key, uint32_t w0_dir, uint32_t w0_slice,
                                                                 uint32_t* __restrict__ capped) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* x = reinterpret_cast<T*>(smem_raw);
  T* z = x + p.D;
  T* d = z + ((p.D + 3) & ~3);
  __shared__ double warp_part[(kSliceThreads / 32) * kNumRed];
  __shared__ double red[kNumRed];
  __shared__ double t_move;
  __shared__ int moved;
  const int j = blockIdx.x, D = p.D;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < D; i += blockDim.x) x[i] = X[(size_t)j * D + i];
  __syncthreads();
  unsigned n_capped = 0;
  for (int s = 0; s < p.steps; ++s) {
    // direction normals z ~ N(0, I): block b of (NS_DIRECTION, it, s, slot, b)
    const int nblk = (D + 3) >> 2;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      const uint4 w = philox4x32_10(make_uint4(w0_dir, (uint32_t)s, (uint32_t)j, (uint32_t)b), key);
      T zz[4];
      if constexpr (sizeof(T) == 8) {
        const double2 a = box_muller_f64(w.x, w.y), c = box_muller_f64(w.z, w.w);
        zz[0] = a.x; zz[1] = a.y; zz[2] = c.x; zz[3] = c.y;
      } else {
        const float2 a = box_muller_f32(w.x, w.y), c = box_muller_f32(w.z, w.w);
        zz[0] = a.x; zz[1] = a.y; zz[2] = c.x; zz[3] = c.y;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * b + q < D) z[4 * b + q] = zz[q];
    }
    __syncthreads();
    // d = L z (L lower triangular): one warp per row, lanes split the dot product
    for (int i = wid; i < D; i += nw) {
      const T* row = Lf + (size_t)i * D;
      T acc = (T)0;
      for (int kk = lane; kk <= i; kk += 32) acc += row[kk] * z[kk];
      acc = warp_sum_t<T>(acc);
      if (lane == 0) d[i] = acc;
    }
    __syncthreads();
    line_reduce<T>(x, d, p.L, D, warp_part, red);
    if (threadIdx.x == 0) {
      const double xAx = red[0], xAd = red[1], dAd = red[2], xx = red[3], xd = red[4], dd = red[5];
      const double x4 = red[6], x3d = red[7], x2d2 = red[8], xd3 = red[9], d4 = red[10];
      const double a0 = -(p.ck * xAx + p.cm * xx + p.lm * x4) + 0.5 * xx + p.hc;
      const double a1 = -(2.0 * p.ck * xAd + 2.0 * p.cm * xd + 4.0 * p.lm * x3d) + xd;
      const double a2 = -(p.ck * dAd + p.cm * dd + 6.0 * p.lm * x2d2) + 0.5 * dd;
      const double a3 = -4.0 * p.lm * xd3;
      const double a4 = -p.lm * d4;
      const uint4 w = philox4x32_10(make_uint4(w0_slice, (uint32_t)s, (uint32_t)j, 0u), key);
      const double E = -log(uniform53(w.x, w.y));
      const double lstar = *p.lstar;
      int mv = 0;
      double tt = 0.0;
      if (dd > 0.0) {
        const double disc = sqrt(xd * xd + 2.0 * E * dd);
        double lo = (-xd - disc) / dd, hi = (-xd + disc) / dd;
        for (int r = 0; r < p.max_shrink; ++r) {
          const uint4 wr = philox4x32_10(make_uint4(w0_slice, (uint32_t)s, (uint32_t)j, (uint32_t)(1 + r)), key);
          const double u = uniform53(wr.x, wr.y);
          const double t = lo + u * (hi - lo);
          const double lt = a0 + t * (a1 + t * (a2 + t * (a3 + t * a4)));
          if (lt > lstar) {
            mv = 1;
            tt = t;
            break;
          }
          if (t < 0.0) lo = t; else hi = t;
        }
      }
      if (!mv) ++n_capped;
      moved = mv;
      t_move = tt;
    }
    __syncthreads();
    if (moved) {
      const T t = (T)t_move;
      for (int i = threadIdx.x; i < D; i += blockDim.x) x[i] = x[i] + t * d[i];
    }
    __syncthreads();
  }
  // exact log L of the final point (quartic coefficient a0 at t = 0)
  line_reduce<T>(x, x, p.L, D, warp_part, red);
  if (threadIdx.x == 0) {
    logl_out[j] = -(p.ck * red[0] + p.cm * red[3] + p.lm * red[6]) + 0.5 * red[3] + p.hc;
    if (n_capped) atomicAdd(capped, n_capped);
  }
  for (int i = threadIdx.x; i < D; i += blockDim.x) X[(size_t)j * D + i] = x[i];
}

// live[order[j]] = X[j], logl[order[j]] = xl[j] for the k deleted slots.
template <typename T>
__global__ void ns_replace_kernel(T* __restrict__ live, double* __restrict__ logl, const int32_t* __restrict__ order,
                                  const T* __restrict__ X, const double* __restrict__ xl, int D) {
  const int j = blockIdx.x;
  const int dst = order[j];
  for (int x = threadIdx.x; x < D; x += blockDim.x) live[(size_t)dst * D + x] = X[(size_t)j * D + x];
  if (threadIdx.x == 0) logl[dst] = xl[j];
}

// Remaining evidence log(X mean_live L) against log Z: ns[4] = 1 when below log(stop_frac).
// Also ns[5] = log(X mean_live L).
__global__ void ns_stop_kernel(const double* __restrict__ logl, int N, double log_stop, double* __restrict__ ns) {
  __shared__ double red[64];
  double m = -INFINITY;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, logl[i]);
  m = block_max(m, red);
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += exp(logl[i] - m);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double rem = ns[0] + m + log(s) - log((double)N);
    ns[5] = rem;
    ns[4] = (rem - ns[1] < log_stop) ? 1.0 : 0.0;
  }
}

// Final evidence with the live points (weight X/N each), the information
// H = sum_i p_i log L_i - log Z and the error sqrt(H / N): ns[6] = log Z, ns[7] = H.
__global__ void ns_final_kernel(const double* __restrict__ dead, long long n_dead, const double* __restrict__ logl,
                                int N, double* __restrict__ ns) {
  __shared__ double red[64];
  const double logw_live = ns[0] - log((double)N);
  double m = -INFINITY;
  for (long long i = threadIdx.x; i < n_dead; i += blockDim.x) m = fmax(m, dead[2 * i] + dead[2 * i + 1]);
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, logl[i] + logw_live);
  m = block_max(m, red);
  double s = 0.0;
  for (long long i = threadIdx.x; i < n_dead; i += blockDim.x) s += exp(dead[2 * i] + dead[2 * i + 1] - m);
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += exp(logl[i] + logw_live - m);
  s = block_sum(s, red);
  const double logZ = m + log(s);
  double h = 0.0;
  for (long long i = threadIdx.x; i < n_dead; i += blockDim.x)
    h += exp(dead[2 * i] + dead[2 * i + 1] - logZ) * dead[2 * i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) h += exp(logl[i] + logw_live - logZ) * logl[i];
  h = block_sum(h, red);
  if (threadIdx.x == 0) {
    ns[6] = logZ;
    ns[7] = h - logZ;
  }
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_ns_select(const double* logl, int N, int k, int32_t* order, double* ns, double* dead,
                             long long dead_cap, uint32_t* status, cudaStream_t s) {
  int P = 1;
  while (P < N) P <<= 1;
  const size_t sm = (size_t)P * (sizeof(double) + sizeof(int));
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(ns_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ns_select_kernel<<<1, kSortThreads, sm, s>>>(logl, N, k, order, ns, dead, dead_cap, status);
  return cudaGetLastError();
}

cudaError_t launch_ns_start(const void* live, int dtype, const int32_t* order, int N, int k, int D, uint64_t seed,
                            uint64_t stream_id, uint32_t it, void* X, cudaStream_t s) {
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(RNG_NS_START, it);
  if (dtype == 0) ns_start_kernel<double><<<k, 256, 0, s>>>((const double*)live, order, N, k, D, key, w0, (double*)X);
  else ns_start_kernel<float><<<k, 256, 0, s>>>((const float*)live, order, N, k, D, key, w0, (float*)X);
  return cudaGetLastError();
}

cudaError_t launch_ns_slice(void* X, int dtype, double* logl_out, const void* Lf, int k, int L, double c_kin,
                            double c_mass_m2, double lam, const double* lstar, int steps, int max_shrink, uint64_t seed,
                            uint64_t stream_id, uint32_t it, uint32_t* capped, cudaStream_t s) {
  NsSliceParams p;
  p.L = L;
  p.D = L * L;
  p.steps = steps;
  p.max_shrink = max_shrink;
  p.ck = c_kin;
  p.cm = c_mass_m2;
  p.lm = lam;
  p.hc = 0.5 * p.D * log(2.0 * M_PI);
  p.lstar = lstar;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t wd = counter_word0(RNG_NS_DIRECTION, it), ws = counter_word0(RNG_NS_SLICE, it);
  const size_t elems = (size_t)2 * p.D + ((p.D + 3) & ~3);
  cudaError_t e;
  if (dtype == 0) {
    const size_t sm = elems * sizeof(double);
    if ((e = cudaFuncSetAttribute(ns_slice_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
      return e;
    ns_slice_kernel<double><<<k, kSliceThreads, sm, s>>>((double*)X, logl_out, (const double*)Lf, p, key, wd, ws,
                                                         capped);
  } else {
    const size_t sm = elems * sizeof(float);
    if ((e = cudaFuncSetAttribute(ns_slice_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
      return e;
    ns_slice_kernel<float><<<k, kSliceThreads, sm, s>>>((float*)X, logl_out, (const float*)Lf, p, key, wd, ws,
                                                        capped);
  }
  return cudaGetLastError();
}

cudaError_t launch_ns_replace(void* live, int dtype, double* logl, const int32_t* order, const void* X,
                              const double* xl, int k, int D, cudaStream_t s) {
  if (dtype == 0)
    ns_replace_kernel<double><<<k, 256, 0, s>>>((double*)live, logl, order, (const double*)X, xl, D);
  else
    ns_replace_kernel<float><<<k, 256, 0, s>>>((float*)live, logl, order, (const float*)X, xl, D);
  return cudaGetLastError();
}

cudaError_t launch_ns_stop(const double* logl, int N, double log_stop, double* ns, cudaStream_t s) {
  ns_stop_kernel<<<1, 1024, 0, s>>>(logl, N, log_stop, ns);
  return cudaGetLastError();
}

cudaError_t launch_ns_final(const double* dead, long long n_dead, const double* logl, int N, double* ns,
                            cudaStream_t s) {
  ns_final_kernel<<<1, 1024, 0, s>>>(dead, n_dead, logl, N, ns);
  return cudaGetLastError();
}

}  // namespace phi4
