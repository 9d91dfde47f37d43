// Systematic resampling in exact fixed point (resample.cuh) and the particle gather.
#include <math.h>
#include <algorithm>
#include "internal.h"
#include "resample.cuh"

namespace phi4 {

__global__ void __launch_bounds__(kResampleThreads) resample_kernel(const double* __restrict__ w, int N,
                                                                    uint32_t U_host,
                                                                    const uint32_t* __restrict__ U_dev,
                                                                    int32_t* __restrict__ anc,
                                                                    unsigned long long* __restrict__ C) {
  resample_body(w, N, U_dev ? *U_dev : U_host, anc, C);
}

// Row gather dst[r] = src[anc[r]]: CTA y-index walks rows, so each CTA reads its row's
// ancestor once and copies the row with consecutive threads on consecutive 16-byte
// words (kUnroll loads in flight per thread before the stores).
constexpr int kGatherThreads = 256, kUnroll = 4;
template <typename V>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const V* __restrict__ src, V* __restrict__ dst,
                                                                long long per_row, int N,
                                                                const int32_t* __restrict__ anc) {
  const long long step = (long long)gridDim.x * kGatherThreads;
  for (int r = blockIdx.y; r < N; r += gridDim.y) {
    const V* __restrict__ s = src + (long long)__ldg(anc + r) * per_row;
    V* __restrict__ d = dst + (long long)r * per_row;
    long long c = (long long)blockIdx.x * kGatherThreads + threadIdx.x;
    for (; c + (kUnroll - 1) * step < per_row; c += kUnroll * step) {
      V t[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) t[k] = s[c + k * step];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) d[c + k * step] = t[k];
    }
    for (; c < per_row; c += step) d[c] = s[c];
  }
}

template <typename V>
static void gather_go(const V* src, V* dst, long long per_row, int N, const int32_t* anc, cudaStream_t s) {
  // x: CTAs per row (each thread moves kUnroll words per pass), y: rows in flight
  long long gx = (per_row + (long long)kGatherThreads * kUnroll - 1) / ((long long)kGatherThreads * kUnroll);
  if (gx > 65535) gx = 65535;
  if (gx < 1) gx = 1;
  const long long want = (long long)sm_count() * 16 / gx;
  const int gy = (int)std::min<long long>(std::max<long long>(want, 1), std::min<long long>(N, 65535));
  gather_kernel<V><<<dim3((unsigned)gx, (unsigned)gy), kGatherThreads, 0, s>>>(src, dst, per_row, N, anc);
}

size_t resample_scratch_bytes(int N) { return (size_t)N * sizeof(unsigned long long); }

cudaError_t launch_resample(const double* w, int N, uint32_t U, const uint32_t* U_dev, int32_t* anc, void* scratch,
                            cudaStream_t s) {
  if (N <= 0) return cudaErrorInvalidValue;
  resample_kernel<<<1, kResampleThreads, 0, s>>>(w, N, U, U_dev, anc, (unsigned long long*)scratch);
  return cudaGetLastError();
}

cudaError_t launch_gather(const void* src, void* dst, size_t row_bytes, int N, const int32_t* anc,
                          cudaStream_t s) {
  if (N <= 0 || row_bytes == 0) return cudaSuccess;
  const uintptr_t al = (uintptr_t)src | (uintptr_t)dst;
  if (row_bytes % 16 == 0 && al % 16 == 0)
    gather_go<uint4>((const uint4*)src, (uint4*)dst, (long long)(row_bytes / 16), N, anc, s);
  else if (row_bytes % 8 == 0 && al % 8 == 0)
    gather_go<uint2>((const uint2*)src, (uint2*)dst, (long long)(row_bytes / 8), N, anc, s);
  else if (row_bytes % 4 == 0 && al % 4 == 0)
    gather_go<uint32_t>((const uint32_t*)src, (uint32_t*)dst, (long long)(row_bytes / 4), N, anc, s);
  else
    gather_go<unsigned char>((const unsigned char*)src, (unsigned char*)dst, (long long)row_bytes, N, anc, s);
  return cudaGetLastError();
}

// dst_k[r] = src_k[anc[r]] for the per-particle doubles (up to three arrays, one launch)
__global__ void gather3_f64_kernel(const double* __restrict__ s0, double* __restrict__ d0,
                                   const double* __restrict__ s1, double* __restrict__ d1,
                                   const double* __restrict__ s2, double* __restrict__ d2, int N,
                                   const int32_t* __restrict__ anc) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
    const int a = anc[r];
    d0[r] = s0[a];
    if (d1) d1[r] = s1[a];
    if (d2) d2[r] = s2[a];
  }
}

cudaError_t launch_gather_f64(const double* src, double* dst, int N, const int32_t* anc, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  gather3_f64_kernel<<<(N + 255) / 256, 256, 0, s>>>(src, dst, nullptr, nullptr, nullptr, nullptr, N, anc);
  return cudaGetLastError();
}

cudaError_t launch_gather3_f64(const double* s0, double* d0, const double* s1, double* d1, const double* s2,
                               double* d2, int N, const int32_t* anc, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  gather3_f64_kernel<<<(N + 255) / 256, 256, 0, s>>>(s0, d0, s1, d1, s2, d2, N, anc);
  return cudaGetLastError();
}

}  // namespace phi4
