// Particle covariance (App. A: a single covariance re-estimated from the
// population at every outer step): column means, centred and transposed copy
// Xc^T, Sigma = Xc^T Xc / (N - 1) on the lower triangle, and the ridge
// delta = jitter_rel * trace(Sigma) / D.
// FP64 and FP32 forms: Xc^T in the state type and a SIMT SYRK. Mixed form: Xc^T as
// two planes of fixed-point digits per site and an exact Gram matrix on the tensor
// cores (launch_gram_tc): the computed Sigma is the covariance of the rounded fields,
// positive semi-definite by construction, where bf16 operands with fp32 sums over N
// terms perturb it by ~sqrt(N) 2^-24 of sum |x||y| and make a nearly singular
// covariance indefinite.
#include <algorithm>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int kColTile = 32, kRowLanes = 16;
}

// mean[j] = (1/N) sum_n phi[n][j]; float fields accumulate with compensated float
// sums per thread, combined in double in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kColTile* kRowLanes) colmean_kernel(const T* __restrict__ phi, int N, int D,
                                                                      double* __restrict__ mean) {
  __shared__ double part[kRowLanes][kColTile];
  const int tx = threadIdx.x % kColTile, ty = threadIdx.x / kColTile;
  const int j = blockIdx.x * kColTile + tx;
  double s = 0.0;
  if (j < D) {
    if constexpr (sizeof(T) == 8) {
      for (int n = ty; n < N; n += kRowLanes) s += phi[(size_t)n * D + j];
    } else {
      KahanF k;
      for (int n = ty; n < N; n += kRowLanes) k.add(phi[(size_t)n * D + j]);
      s = k.value();
    }
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && j < D) {
    double t = 0.0;
    for (int r = 0; r < kRowLanes; ++r) t += part[r][tx];
    mean[j] = t / N;
  }
}

// XcT[j][n] = To(phi[n][j] - mean[j]) through a 32 x 32 shared tile.
template <typename T, typename To>
__global__ void center_transpose_kernel(const T* __restrict__ phi, int N, int D, const double* __restrict__ mean,
                                        To* __restrict__ XcT, int ldx) {
  __shared__ float tile32[32][33];
  __shared__ double tile64[sizeof(T) == 8 ? 32 : 1][33];
  const int n0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, j = j0 + threadIdx.x;
    if (n < N && j < D) {
      if constexpr (sizeof(T) == 8) tile64[r][threadIdx.x] = phi[(size_t)n * D + j] - mean[j];
      else tile32[r][threadIdx.x] = (float)((double)phi[(size_t)n * D + j] - mean[j]);
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, n = n0 + threadIdx.x;
    if (n < N && j < D) {
      if constexpr (sizeof(T) == 8) XcT[(size_t)j * ldx + n] = (To)tile64[threadIdx.x][r];
      else XcT[(size_t)j * ldx + n] = to_t<To>(tile32[threadIdx.x][r]);
    }
  }
}

// Mixed form: per site j the mean (as colmean) and the shift s_j = B - e_j, where
// 2^(e_j - 1) <= max_n |phi_nj - mean_j| < 2^e_j (from the column's extrema), so that
// every centred field scaled by 2^s_j lies within 2^B.
__global__ void __launch_bounds__(kColTile* kRowLanes) colstats_kernel(const float* __restrict__ phi, int N, int D,
                                                                       int B, double* __restrict__ mean,
                                                                       int* __restrict__ shift) {
  __shared__ double part[kRowLanes][kColTile];
  __shared__ float pmin[kRowLanes][kColTile], pmax[kRowLanes][kColTile];
  const int tx = threadIdx.x % kColTile, ty = threadIdx.x / kColTile;
  const int j = blockIdx.x * kColTile + tx;
  KahanF k;
  float lo = INFINITY, hi = -INFINITY;
  if (j < D) {
    for (int n = ty; n < N; n += kRowLanes) {
      const float v = phi[(size_t)n * D + j];
      k.add(v);
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
  }
  part[ty][tx] = k.value();
  pmin[ty][tx] = lo;
  pmax[ty][tx] = hi;
  __syncthreads();
  if (ty == 0 && j < D) {
    double t = 0.0;
    for (int r = 0; r < kRowLanes; ++r) {
      t += part[r][tx];
      lo = fminf(lo, pmin[r][tx]);
      hi = fmaxf(hi, pmax[r][tx]);
    }
    const double mu = t / N;
    mean[j] = mu;
    const double dev = fmax((double)hi - mu, mu - (double)lo);
    int e = 0;
    if (dev > 0.0) frexp(dev, &e);
    shift[j] = dev > 0.0 ? B - e : 0;
  }
}

// Digit planes of the mixed form: x = phi_nj - mean_j (in float, the mean as a
// float pair), v = rint(x 2^s_j) with |v| <= 2^B, h = rint(v 2^-a), l = v - 2^a h
// (|l| <= 2^(a-1), |h| <= 2^(B-a)); H[j][n] = h, Lo[j][n] = l as exact bf16 integers,
// transposed through a 32 x 32 shared tile.
__global__ void center_digits_kernel(const float* __restrict__ phi, int N, int D, const double* __restrict__ mean,
                                     const int* __restrict__ shift, int a, __nv_bfloat16* __restrict__ H,
                                     __nv_bfloat16* __restrict__ Lo, int ldx) {
  __shared__ float th[32][33], tl[32][33];
  __shared__ float mhi[32], mlo[32];
  __shared__ int sh[32];
  const int n0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < 32) {
    const int j = j0 + tid;
    const double mu = j < D ? mean[j] : 0.0;
    const float m1 = (float)mu;
    mhi[tid] = m1;
    mlo[tid] = (float)(mu - (double)m1);
    sh[tid] = j < D ? shift[j] : 0;
  }
  __syncthreads();
  const float pa = ldexpf(1.f, a), ra = ldexpf(1.f, -a);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, j = j0 + threadIdx.x;
    float h = 0.f, l = 0.f;
    if (n < N && j < D) {
      const float x = (phi[(size_t)n * D + j] - mhi[threadIdx.x]) - mlo[threadIdx.x];
      const float v = rintf(ldexpf(x, sh[threadIdx.x]));
      h = rintf(v * ra);
      l = fmaf(-h, pa, v);
    }
    th[r][threadIdx.x] = h;
    tl[r][threadIdx.x] = l;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, n = n0 + threadIdx.x;
    if (n < N && j < D) {
      H[(size_t)j * ldx + n] = __float2bfloat16_rn(th[threadIdx.x][r]);
      Lo[(size_t)j * ldx + n] = __float2bfloat16_rn(tl[threadIdx.x][r]);
    }
  }
}

__global__ void ridge_kernel(const double* __restrict__ sigma, int D, double jitter_rel, double* __restrict__ ridge) {
  __shared__ double red[64];
  double s = 0.0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) s += sigma[(size_t)i * D + i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *ridge = jitter_rel * s / D;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t covariance_scratch_bytes(int N, int D, int precision) {
  const size_t mean = align256((size_t)D * sizeof(double));
  if (precision == 0) return mean + align256((size_t)D * N * sizeof(double));
  if (precision == 1) return mean + align256((size_t)D * N * sizeof(float));
  const size_t ldx = ((size_t)N + 7) & ~(size_t)7;
  return mean + align256((size_t)D * sizeof(int)) + 2 * align256((size_t)D * ldx * 2);
}

cudaError_t launch_covariance(const void* phi, int precision, int N, int D, double* sigma, void* scratch,
                              uint32_t* status, cudaStream_t s) {
  if (N < 2 || D < 1) return cudaErrorInvalidValue;
  unsigned char* base = (unsigned char*)scratch;
  double* mean = (double*)base;
  void* xct = base + align256((size_t)D * sizeof(double));
  const dim3 tgrid((N + 31) / 32, (D + 31) / 32), tblock(32, 8);
  const unsigned mgrid = (unsigned)((D + kColTile - 1) / kColTile);
  const double inv = 1.0 / (double)(N - 1);
  cudaError_t e;
  if (precision == 0) {
    colmean_kernel<double><<<mgrid, kColTile * kRowLanes, 0, s>>>((const double*)phi, N, D, mean);
    center_transpose_kernel<double, double><<<tgrid, tblock, 0, s>>>((const double*)phi, N, D, mean, (double*)xct, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_syrk_simt(xct, 0, D, N, N, inv, sigma, s);
  }
  if (precision == 1) {
    colmean_kernel<float><<<mgrid, kColTile * kRowLanes, 0, s>>>((const float*)phi, N, D, mean);
    center_transpose_kernel<float, float><<<tgrid, tblock, 0, s>>>((const float*)phi, N, D, mean, (float*)xct, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_syrk_simt(xct, 1, D, N, N, inv, sigma, s);
  }
  // mixed: B = 23 - ceil(log2 N) (at most 14) keeps every digit-product sum within 2^23
  int c = 0;
  while ((1 << c) < N) ++c;
  const int B = std::min(14, 23 - c), a = (B + 1) / 2;
  const int ldx = (N + 7) & ~7;
  int* shift = (int*)(base + align256((size_t)D * sizeof(double)));
  __nv_bfloat16* H = (__nv_bfloat16*)((unsigned char*)shift + align256((size_t)D * sizeof(int)));
  __nv_bfloat16* Lo = H + align256((size_t)D * ldx * 2) / 2;
  colstats_kernel<<<mgrid, kColTile * kRowLanes, 0, s>>>((const float*)phi, N, D, B, mean, shift);
  center_digits_kernel<<<tgrid, tblock, 0, s>>>((const float*)phi, N, D, mean, shift, a, H, Lo, ldx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_gram_tc(H, Lo, ldx, D, N, shift, a, inv, sigma, status, s);
}

// ---------------------------------------------------------------------------
// Particle-independent kernel covariance (PHI4_FLAG_FREE_KERNEL_COV): the exact
// covariance of the Gaussian part of the tempered target gamma_beta, whose log density
// has the quadratic part -(1/2) phi^T P phi with
//   P = a I + 2 beta (c_kin K + c_mass m2 I),  K = sum_mu (2 - T_mu - T_mu^{-1}),
// a = 1 - beta (reference dropped at beta = 1) or 1 (reference kept). For lambda = 0 it
// is the target's covariance. P is diagonal in the lattice Fourier basis with
//   p_k = a + 2 beta (c_kin sum_mu 4 sin^2(pi k_mu / L) + c_mass m2),
// so Sigma_xy = (1/D) sum_k cos(2 pi k.(x - y) / L) / p_k depends only on the
// displacement (dr, dc) = (x - y) mod L; the sine parts cancel under k -> -k (p_k is
// even), leaving the product of the two cosines. Three kernels: 1/p_k, the displacement
// table (one CTA per displacement, FP64 sums in a fixed order), the D x D fill.
__global__ void free_inv_spectrum_kernel(int L, const double* __restrict__ beta_p, double m2c, double c_kin,
                                         int keep, double* __restrict__ invp) {
  const int D = L * L;
  const double beta = *beta_p, a = keep ? 1.0 : 1.0 - beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < D; k += gridDim.x * blockDim.x) {
    const int k1 = k / L, k2 = k - (k / L) * L;
    const double s1 = sinpi((double)k1 / L), s2 = sinpi((double)k2 / L);
    invp[k] = 1.0 / (a + 2.0 * beta * (c_kin * 4.0 * (s1 * s1 + s2 * s2) + m2c));
  }
}

constexpr int kFreeThreads = 256;
__global__ void __launch_bounds__(kFreeThreads) free_table_kernel(int L, const double* __restrict__ invp,
                                                                  double* __restrict__ table) {
  __shared__ double cs[128];
  __shared__ double red[64];
  const int D = L * L, e = blockIdx.x, dr = e / L, dc = e - (e / L) * L;
  for (int j = threadIdx.x; j < L; j += kFreeThreads) cs[j] = cospi(2.0 * (double)j / L);
  __syncthreads();
  double acc = 0.0;
  for (int k = threadIdx.x; k < D; k += kFreeThreads) {
    const int k1 = k / L, k2 = k - (k / L) * L;
    acc += cs[(k1 * dr) % L] * cs[(k2 * dc) % L] * invp[k];
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) table[e] = acc / D;
}

__global__ void free_fill_kernel(int L, const double* __restrict__ table, double* __restrict__ sigma) {
  const int D = L * L;
  const long long total = (long long)D * D;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / D), j = (int)(q - (long long)i * D);
    const int ri = i / L, ci = i - ri * L, rj = j / L, cj = j - rj * L;
    const int dr = (ri - rj + L) % L, dc = (ci - cj + L) % L;
    sigma[q] = table[dr * L + dc];
  }
}

size_t free_covariance_scratch_bytes(int L) { return 2 * align256((size_t)L * L * sizeof(double)); }

cudaError_t launch_free_covariance(int L, const double* beta, double m2c, double c_kin, int keep, double* sigma,
                                   void* scratch, cudaStream_t s) {
  if (L < 1 || L > 128) return cudaErrorInvalidValue;
  const int D = L * L;
  double* invp = (double*)scratch;
  double* table = (double*)((unsigned char*)scratch + align256((size_t)D * sizeof(double)));
  free_inv_spectrum_kernel<<<(D + 255) / 256, 256, 0, s>>>(L, beta, m2c, c_kin, keep, invp);
  free_table_kernel<<<D, kFreeThreads, 0, s>>>(L, invp, table);
  free_fill_kernel<<<sm_count() * 8, 256, 0, s>>>(L, table, sigma);
  return cudaGetLastError();
}

cudaError_t launch_ridge(const double* sigma, int D, double jitter_rel, double* ridge, cudaStream_t s) {
  ridge_kernel<<<1, 256, 0, s>>>(sigma, D, jitter_rel, ridge);
  return cudaGetLastError();
}

}  // namespace phi4
