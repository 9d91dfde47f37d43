// Particle covariance (App. A: a single covariance re-estimated from the
// population at every outer step): column means, centred and transposed copy
// Xc^T (in the GEMM operand type), Sigma = Xc^T Xc / (N - 1) on the lower
// triangle, and the ridge delta = jitter_rel * trace(Sigma) / D.
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
  return mean + align256((size_t)D * ldx * 2);
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
  colmean_kernel<float><<<mgrid, kColTile * kRowLanes, 0, s>>>((const float*)phi, N, D, mean);
  if (precision == 1) {
    center_transpose_kernel<float, float><<<tgrid, tblock, 0, s>>>((const float*)phi, N, D, mean, (float*)xct, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_syrk_simt(xct, 1, D, N, N, inv, sigma, s);
  }
  const int ldx = (N + 7) & ~7;
  center_transpose_kernel<float, __nv_bfloat16>
      <<<tgrid, tblock, 0, s>>>((const float*)phi, N, D, mean, (__nv_bfloat16*)xct, ldx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_syrk_tc(xct, ldx, D, N, inv, sigma, status, s);
}

cudaError_t launch_ridge(const double* sigma, int D, double jitter_rel, double* ridge, cudaStream_t s) {
  ridge_kernel<<<1, 256, 0, s>>>(sigma, D, jitter_rel, ridge);
  return cudaGetLastError();
}

}  // namespace phi4
