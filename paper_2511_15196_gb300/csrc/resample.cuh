// Systematic resampling of one population in exact fixed point (a reading of Sec. 2
// sampler (i); the paper does not fix the arithmetic):
//   q_i = floor(ldexp(w_i / max w, 46)),  C = inclusive prefix sum of q (uint64),
//   p_i = floor((i 2^32 + U) Q / (N 2^32)),  anc_i = min{ j : C_j > p_i }.
// One 1024-thread CTA: per-thread serial scans of contiguous chunks, a warp-shuffle scan
// of the chunk totals, then a binary search per position. Integer arithmetic only after
// the (correctly rounded) division, so any implementation of this definition returns the
// same ancestors; every ancestor lies in [0, N) whatever the weights.
#pragma once
#include <math.h>
#include "common.cuh"

namespace phi4 {

constexpr int kResampleThreads = 1024;

PHI4_DEV void resample_body(const double* __restrict__ w, int N, uint32_t U32, int32_t* __restrict__ anc,
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
  const unsigned long long U = (unsigned long long)U32;
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
  __syncthreads();  // the CTA may run the next population's scan over the same shared arrays
}

}  // namespace phi4
