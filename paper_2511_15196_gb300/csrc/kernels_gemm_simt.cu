// SIMT register-blocked GEMM, C = A B^T with both operands K-contiguous
// (A: M x K rows, B: Nn x K rows), for the FP32 and FP64 forms of the sampler:
//   EPI_PROPOSE: prop[m][n] = phi[m][n] + scale * sum_{k <= n} Z[m][k] L[n][k] (phi's row
//                pitch phi_ld; 0 adds one row, the SMC-IRMH mean, to every row)
//                (L lower triangular; a tile of columns [n0, n0+BN) stops at k = n0+BN);
//   EPI_SYRK:    sigma[m][n] = inv * sum_k XcT[m][k] XcT[n][k] for n <= m only
//                (tiles strictly above the diagonal are skipped).
#include "internal.h"
#include "common.cuh"

namespace phi4 {

enum { EPI_PROPOSE = 0, EPI_SYRK = 1 };

template <typename T, int BM, int BN, int BK, int TM, int TN, int EPI>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    simt_gemm_kernel(const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb, int M, int Nn, int K,
                     const T* __restrict__ phi, int phi_ld, T* __restrict__ out, double* __restrict__ sigma,
                     double scale) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (EPI == EPI_SYRK && n0 > m0 + BM - 1) return;
  int kend = K;
  if (EPI == EPI_PROPOSE) kend = min(K, n0 + BN);
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  // thread's rows/cols: two halves so neighbouring threads read neighbouring smem words
  int rr[TM], cc[TN];
#pragma unroll
  for (int i = 0; i < TM; ++i) rr[i] = (i < TM / 2) ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + (i - TM / 2);
#pragma unroll
  for (int j = 0; j < TN; ++j) cc[j] = (j < TN / 2) ? tx * (TN / 2) + j : BN / 2 + tx * (TN / 2) + (j - TN / 2);

  for (int k0 = 0; k0 < kend; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int m = idx / BK, k = idx % BK;
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < M && gk < kend) ? A[(size_t)gm * lda + gk] : T(0);
    }
    for (int idx = tid; idx < BN * BK; idx += NT) {
      const int n = idx / BK, k = idx % BK;
      const int gn = n0 + n, gk = k0 + k;
      Bs[k][n] = (gn < Nn && gk < kend) ? B[(size_t)gn * ldb + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][rr[i]];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][cc[j]];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + rr[i];
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + cc[j];
      if (gn >= Nn) continue;
      if (EPI == EPI_PROPOSE) {
        out[(size_t)gm * Nn + gn] = phi[(size_t)gm * phi_ld + gn] + (T)scale * acc[i][j];
      } else {
        if (gn <= gm) sigma[(size_t)gm * Nn + gn] = (double)acc[i][j] * scale;
      }
    }
  }
}

template <typename T, int BM, int BN, int TM, int TN, int EPI>
static cudaError_t run_gemm(const T* A, int lda, const T* B, int ldb, int M, int Nn, int K, const T* phi, int phi_ld,
                            T* out, double* sigma, double scale, cudaStream_t s) {
  dim3 grid((Nn + BN - 1) / BN, (M + BM - 1) / BM);
  simt_gemm_kernel<T, BM, BN, 16, TM, TN, EPI>
      <<<grid, (BM / TM) * (BN / TN), 0, s>>>(A, lda, B, ldb, M, Nn, K, phi, phi_ld, out, sigma, scale);
  return cudaGetLastError();
}

cudaError_t launch_propose_simt(const void* phi, void* prop, const void* Z, const void* Lf, int dtype, int N, int D,
                                double scale, cudaStream_t s, int phi_ld) {
  if (phi_ld < 0) phi_ld = D;
  if (dtype == 0)
    return run_gemm<double, 64, 64, 4, 4, EPI_PROPOSE>((const double*)Z, D, (const double*)Lf, D, N, D, D,
                                                       (const double*)phi, phi_ld, (double*)prop, nullptr, scale, s);
  if (dtype == 1)
    return run_gemm<float, 128, 128, 8, 8, EPI_PROPOSE>((const float*)Z, D, (const float*)Lf, D, N, D, D,
                                                        (const float*)phi, phi_ld, (float*)prop, nullptr, scale, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_syrk_simt(const void* XcT, int dtype, int D, int N, int ldx, double inv_nm1, double* sigma,
                             cudaStream_t s) {
  if (dtype == 0)
    return run_gemm<double, 64, 64, 4, 4, EPI_SYRK>((const double*)XcT, ldx, (const double*)XcT, ldx, D, D, N,
                                                    nullptr, 0, nullptr, sigma, inv_nm1, s);
  if (dtype == 1)
    return run_gemm<float, 128, 128, 8, 8, EPI_SYRK>((const float*)XcT, ldx, (const float*)XcT, ldx, D, D, N,
                                                     nullptr, 0, nullptr, sigma, inv_nm1, s);
  return cudaErrorInvalidValue;
}

}  // namespace phi4
