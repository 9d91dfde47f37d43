// Systematic resampling in exact fixed point and the particle gather.
//   q_i = floor(ldexp(w_i / max w, 46)),  C = inclusive prefix sum of q (uint64),
//   p_i = floor((i 2^32 + U) Q / (N 2^32)),  anc_i = min{ j : C_j > p_i }.
// One 1024-thread CTA: per-thread serial scans of contiguous chunks, a warp-
// shuffle scan of the chunk totals, then a binary search per position. Integer
// arithmetic only after the (correctly rounded) division, so any implementation
// of this definition returns the same ancestors.
#include <math.h>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int kResampleThreads = 1024;
}

__global__ void __launch_bounds__(kResampleThreads) resample_kernel(const double* __restrict__ w, int N,
                                                                    uint32_t U_host,
                                                                    const uint32_t* __restrict__ U_dev,
                                                                    int32_t* __restrict__ anc,
                                                                    unsigned long long* __restrict__ C) {
  __shared__ double red[64];
  __shared__ unsigned long long tot[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  double m = 0.0;
  for (int i = t; i < N; i += kResampleThreads) m = fmax(m, w[i]);
  m = block_max(m, red);
  const int chunk = (N + kResampleThreads - 1) / kResampleThreads;
  const int i0 = min(N, t * chunk), i1 = min(N, i0 + chunk);
  unsigned long long run = 0;
  for (int i = i0; i < i1; ++i) {
    const unsigned long long q = (unsigned long long)floor(ldexp(w[i] / m, 46));
    run += q;
    C[i] = run;
  }
  const unsigned long long incl = warp_incl_scan(run, lane);
  if (lane == 31) tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const unsigned long long v = tot[lane];
    tot[lane] = warp_incl_scan(v, lane);
  }
  __syncthreads();
  const unsigned long long offset = (incl - run) + (wid > 0 ? tot[wid - 1] : 0ull);
  for (int i = i0; i < i1; ++i) C[i] += offset;
  const unsigned long long Q = tot[31];
  __syncthreads();
  const unsigned long long U = U_dev ? (unsigned long long)*U_dev : (unsigned long long)U_host;
  for (int i = t; i < N; i += kResampleThreads) {
    const unsigned long long T = ((unsigned long long)i << 32) | U;
    const unsigned __int128 prod = (unsigned __int128)T * Q;
    const unsigned long long p = (unsigned long long)((prod >> 32) / (unsigned)N);
    int lo = 0, hi = N - 1;  // first j with C[j] > p (exists: p < Q = C[N-1])
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (C[mid] > p) hi = mid; else lo = mid + 1;
    }
    anc[i] = lo;
  }
}

template <typename V>
__global__ void gather_kernel(const V* __restrict__ src, V* __restrict__ dst, long long per_row, int N,
                              const int32_t* __restrict__ anc) {
  const long long total = per_row * N;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / per_row, c = k - r * per_row;
    dst[k] = src[(long long)anc[r] * per_row + c];
  }
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
  const int threads = 256;
  const int grid = sm_count() * 8;
  const uintptr_t al = (uintptr_t)src | (uintptr_t)dst;
  if (row_bytes % 16 == 0 && al % 16 == 0)
    gather_kernel<uint4><<<grid, threads, 0, s>>>((const uint4*)src, (uint4*)dst, (long long)(row_bytes / 16), N, anc);
  else if (row_bytes % 8 == 0 && al % 8 == 0)
    gather_kernel<uint2><<<grid, threads, 0, s>>>((const uint2*)src, (uint2*)dst, (long long)(row_bytes / 8), N, anc);
  else if (row_bytes % 4 == 0 && al % 4 == 0)
    gather_kernel<uint32_t><<<grid, threads, 0, s>>>((const uint32_t*)src, (uint32_t*)dst,
                                                      (long long)(row_bytes / 4), N, anc);
  else
    gather_kernel<unsigned char><<<grid, threads, 0, s>>>((const unsigned char*)src, (unsigned char*)dst,
                                                           (long long)row_bytes, N, anc);
  return cudaGetLastError();
}

cudaError_t launch_gather_f64(const double* src, double* dst, int N, const int32_t* anc, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  gather_kernel<double><<<(N + 255) / 256, 256, 0, s>>>(src, dst, 1, N, anc);
  return cudaGetLastError();
}

}  // namespace phi4
