// FP64 Cholesky of the particle covariance (App. A), blocked right-looking with
// 64 x 64 blocks: per block column, (1) factor the diagonal block in one CTA,
// (2) triangular solve of the panel below it, (3) symmetric update of the
// trailing lower blocks. All arithmetic is double. A non-positive pivot sets
// ST_NOT_PD in the status word; later kernels see the bit and return.
#include <math.h>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int NB = 64;
}

// dst = lower triangle of src, zeros strictly above the diagonal (src may equal dst).
__global__ void copy_lower_kernel(const double* __restrict__ src, double* __restrict__ dst, int D) {
  const long long total = (long long)D * D;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / D), j = (int)(k - (long long)i * D);
    dst[k] = j <= i ? src[k] : 0.0;
  }
}

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* __restrict__ a, int D, int k0,
                                                         const double* __restrict__ ridge,
                                                         uint32_t* __restrict__ status) {
  __shared__ double blk[NB][NB + 1];
  __shared__ int fail;
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const double r = ridge ? *ridge : 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double v = (j <= i) ? a[(size_t)(k0 + i) * D + k0 + j] : 0.0;
    if (i == j) v += r;
    blk[i][j] = v;
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = blk[j][j];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      else blk[j][j] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double piv = blk[j][j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) blk[i][j] /= piv;
    __syncthreads();
    const int m = n - j - 1;  // trailing size
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, l = j + 1 + e % m;
      if (l <= i) blk[i][l] -= blk[i][j] * blk[l][j];
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) atomicOr(status, ST_NOT_PD);
    return;
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    a[(size_t)(k0 + i) * D + k0 + j] = (j <= i) ? blk[i][j] : 0.0;
  }
}

// Rows r0.. of the panel below diagonal block k0: X L_kk^T = A  ->  A := X.
__global__ void __launch_bounds__(NB) trsm_panel_kernel(double* __restrict__ a, int D, int k0,
                                                        const uint32_t* __restrict__ status) {
  extern __shared__ double trsm_smem[];
  double(*Lkk)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(trsm_smem);
  double(*X)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(trsm_smem + NB * (NB + 1));
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const int r0 = k0 + n + blockIdx.x * NB;
  const int rows = min(NB, D - r0);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    Lkk[i][j] = a[(size_t)(k0 + i) * D + k0 + j];
  }
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    X[i][j] = a[(size_t)(r0 + i) * D + k0 + j];
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < rows) {
    for (int j = 0; j < n; ++j) {
      double v = X[t][j];
      for (int m = 0; m < j; ++m) v -= X[t][m] * Lkk[j][m];
      X[t][j] = v / Lkk[j][j];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    a[(size_t)(r0 + i) * D + k0 + j] = X[i][j];
  }
}

// Trailing update of lower block (bi, bj), bj <= bi, both below block column k0:
// A_ij -= L_ik L_jk^T (K = width of the block column). 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) syrk_update_kernel(double* __restrict__ a, int D, int k0,
                                                          const uint32_t* __restrict__ status) {
  __shared__ double As[16][NB + 2];
  __shared__ double Bs[16][NB + 2];
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  // decode the lower-triangular tile index
  const long long t = blockIdx.x;
  int bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while ((long long)bi * (bi + 1) / 2 > t) --bi;
  const int bj = (int)(t - (long long)bi * (bi + 1) / 2);
  const int base = k0 + n;
  const int i0 = base + bi * NB, j0 = base + bj * NB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int kk = 0; kk < n; kk += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      const int r = e / 16, k = e % 16;
      const int gk = k0 + kk + k;
      const bool kin = (kk + k) < n;
      As[k][r] = (kin && i0 + r < D) ? a[(size_t)(i0 + r) * D + gk] : 0.0;
      Bs[k][r] = (kin && j0 + r < D) ? a[(size_t)(j0 + r) * D + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) y[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + ty + 16 * i;
    if (gi >= D) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj >= D || gj > gi) continue;
      a[(size_t)gi * D + gj] -= acc[i][j];
    }
  }
}

template <typename To>
__global__ void convert_factor_kernel(const double* __restrict__ Lc, int D, To* __restrict__ out, int ld) {
  const long long total = (long long)D * ld;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / ld), j = (int)(k - (long long)i * ld);
    const double v = (j < D && j <= i) ? Lc[(size_t)i * D + j] : 0.0;
    if constexpr (sizeof(To) == 2) out[k] = __float2bfloat16_rn((float)v);
    else out[k] = (To)v;
  }
}

cudaError_t launch_copy_lower(const double* src, double* dst, int D, cudaStream_t s) {
  copy_lower_kernel<<<sm_count() * 4, 256, 0, s>>>(src, dst, D);
  return cudaGetLastError();
}

cudaError_t launch_cholesky(double* a, int D, const double* ridge, uint32_t* status, cudaStream_t s) {
  const int nblk = (D + NB - 1) / NB;
  const size_t trsm_smem = 2 * sizeof(double) * NB * (NB + 1);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(trsm_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB;
    potrf_diag_kernel<<<1, 256, 0, s>>>(a, D, k0, ridge, status);
    const int below = nblk - kb - 1;
    if (below > 0) {
      trsm_panel_kernel<<<below, NB, trsm_smem, s>>>(a, D, k0, status);
      const long long tiles = (long long)below * (below + 1) / 2;
      syrk_update_kernel<<<(unsigned)tiles, 256, 0, s>>>(a, D, k0, status);
    }
  }
  return cudaGetLastError();
}

int cholesky_launches(int D) {
  const int nblk = (D + NB - 1) / NB;
  return nblk + 2 * (nblk - 1);
}

cudaError_t launch_factor_convert(const double* Lc, int D, int dtype, void* out, int ld, cudaStream_t s) {
  const int grid = sm_count() * 4;
  if (dtype == 0) convert_factor_kernel<double><<<grid, 256, 0, s>>>(Lc, D, (double*)out, ld);
  else if (dtype == 1) convert_factor_kernel<float><<<grid, 256, 0, s>>>(Lc, D, (float*)out, ld);
  else if (dtype == 2) convert_factor_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(Lc, D, (__nv_bfloat16*)out, ld);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace phi4
