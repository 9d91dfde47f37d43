// Cholesky of the particle covariance (App. A), blocked right-looking with 64 x 64
// blocks: per block column, (1) factor the diagonal block in one CTA, (2) triangular
// solve of the panel below it, (3) symmetric update of the trailing lower blocks.
// Templated on the element type: double for the FP64 and mixed forms, float for the
// plain FP32 form. A non-positive pivot sets ST_NOT_PD in the status word; later
// kernels see the bit and return.
#include <math.h>
#include <algorithm>
#include <cstdlib>
#include "internal.h"
#include "common.cuh"

namespace phi4 {

namespace {
constexpr int NB = 64;
size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
int mpad_of(int D) { return ((D + 127) / 128) * 128; }
}  // namespace

// dst = lower triangle of src, zeros strictly above the diagonal (src may equal dst).
template <typename T>
__global__ void copy_lower_kernel(const double* src, T* dst, int D) {
  const long long total = (long long)D * D;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / D), j = (int)(k - (long long)i * D);
    const double v = j <= i ? src[k] : 0.0;
    dst[k] = (T)v;
  }
}

// x > 0 and finite (not NaN), from the bit pattern (keeps the test off the FP64 pipe)
__device__ __forceinline__ bool positive_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}
__device__ __forceinline__ bool positive_finite(float x) {
  const int b = __float_as_int(x);
  return b > 0 && b < 0x7F800000;
}

// Factor the diagonal block A_kk = L_kk L_kk^T (+ ridge) in one CTA, right-looking by
// columns with one column of look-ahead. On this part an FP64 instruction occupies
// its SM sub-partition's FP64 unit for 64 cycles whatever its lane mask (rsqrt is
// about six of them), so the roles follow the FP64 instruction count:
//   warp 0, alone on its sub-partition, runs only the scalar pivot chain: d_j ->
//     rsqrt -> L_{j+1,j} -> d_{j+1} (nine FP64 instructions per column);
//   warp 1 (the column warp) scales column j once rsqrt(d_j) is known and publishes
//     L_:j in a ring of four shared vectors (and writes it out);
//   warps 2, 3, 5, 6, 7, 9 hold the trailing elements packed column by column from
//     the last column down, so the live set (columns >= k+2 at step k) is a prefix
//     and every FP64 instruction has full lanes; at step k they update column k+2
//     first, signal, then the rest. Warps 4 and 8 share warp 0's sub-partition and idle.
// Hand-offs are mbarrier pairs (phase k on object k & 1, bounded parity waits):
//   C(j): pivot -> column warp, rsqrt(d_j) and d_j are ready;
//   B(k): column warp -> update warps, L_:k is published;
//   A(k): update warps -> pivot, column k+2 has every update of columns <= k (and,
//   since the update warps passed B(k) first, column k is published).
// A barrier's next phase on the same object needs every waiter past the current one,
// so no wait can skip a phase. (Polling shared-memory flags instead measured slower:
// the spinning warps cost more than the mbarrier round trips.) rsqrt(d_j) goes to
// `rdiag` for the inverse.
constexpr int kPotrfThreads = 320;
constexpr int kUpdWarps = 6;
constexpr int kUpdThreads = 32 * kUpdWarps;
constexpr int kUpdSlots = ((NB - 2) * (NB - 1) / 2 + kUpdThreads - 1) / kUpdThreads;  // 11
__device__ __forceinline__ int upd_warp_index(int warp) {  // -1: not an update warp
  switch (warp) {
    case 2: return 0;
    case 3: return 1;
    case 5: return 2;
    case 6: return 3;
    case 7: return 4;
    case 9: return 5;
    default: return -1;
  }
}
// The diagonal block's factorisation. With col_flag, column j of L and rsqrt(d_j) are
// published behind a release store of j + 1 (the streamed inverse consumes them); -1
// tells the consumers that the factorisation stopped.
template <typename T>
__device__ __forceinline__ void potrf_body(T* __restrict__ a, int D, int k0, const double* __restrict__ ridge,
                                           T* __restrict__ rdiag, uint32_t* __restrict__ status, int* col_flag,
                                           int pub_every) {
  __shared__ T S[NB][NB + 1];
  __shared__ T lcol[4][NB];
  __shared__ T rds[NB];
  __shared__ T dpiv[2];
  // update element e = slot * kUpdThreads + t of update thread t, packed (row << 8) | column:
  // columns from n-1 down to 2, rows >= column (column c = n-1-r for the triangular
  // root r of e, row = c + e - r(r+1)/2), so the live set of every step is a prefix
  __shared__ uint32_t eidx[kUpdSlots][kUpdThreads];
  __shared__ __align__(8) uint64_t barA[2], barB[2], barC[2];
  __shared__ int fail;
  __shared__ volatile int abort_flag;
  if (*status & ST_NOT_PD) {
    if (col_flag && threadIdx.x == 0) gpu_flag_release(col_flag, -1);
    return;
  }
  const int n = min(NB, D - k0);
  const T r = ridge ? (T)*ridge : (T)0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < n * n; e += kPotrfThreads) {
    const int i = e / n, c = e - (e / n) * n;
    if (c <= i) S[i][c] = a[(size_t)(k0 + i) * D + k0 + c] + (c == i ? r : (T)0);
  }
  const int Eb = (n - 2) * (n - 1) / 2;
  for (int e = tid; e < kUpdSlots * kUpdThreads; e += kPotrfThreads) {
    uint32_t v = 0;
    if (e < Eb) {
      int t = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (t * (t + 1) / 2 > e) --t;
      while ((t + 1) * (t + 2) / 2 <= e) ++t;
      const int c = n - 1 - t;
      v = ((uint32_t)(c + e - t * (t + 1) / 2) << 8) | (uint32_t)c;
    }
    eidx[e / kUpdThreads][e % kUpdThreads] = v;
  }
  if (tid == 0) {
    fail = 0;
    abort_flag = 0;
    for (int q = 0; q < 2; ++q) {
      cta_mbar_init(&barA[q], kUpdWarps);
      cta_mbar_init(&barB[q], 1);
      cta_mbar_init(&barC[q], 1);
    }
  }
  __syncthreads();
  const int uw = upd_warp_index(warp);
  if (warp == 0) {
    // ---- pivot chain (every lane computes the same scalars). Iteration j: rsqrt(d_j)
    // and publish it at once (the column warp and the update warps then have the
    // iteration's remaining time to deliver what iteration j+1 waits for), then
    // L_{j+1,j} and d_{j+1}. (Waiting first and publishing later measured slower: it
    // lengthens the pivot -> column -> update -> pivot cycle.)
    bool ok = true;
    T d = S[0][0];
    T lprev = (T)0;  // L_{j,j-1}
    for (int j = 0; j < n; ++j) {
      const bool good = positive_finite(d);
      ok = ok && good;
      const T rd = good ? rsqrt(d) : (T)0;
      if (lane == 0) {
        rds[j] = rd;
        dpiv[j & 1] = d;
        cta_mbar_arrive(&barC[j & 1]);
      }
      if (j + 1 >= n) break;
      // L_{j+1,j} = (A_{j+1,j} - L_{j+1,j-1} L_{j,j-1}) rd_j needs column j's entry with
      // every update of columns <= j-2 and column j-1 published; d_{j+1} needs
      // A_{j+1,j+1} with the updates of columns <= j-1: all given by A(j-1)
      T l1 = (T)0;
      if (j >= 1) {
        if (!cta_mbar_wait(&barA[(j - 1) & 1], ((j - 1) >> 1) & 1, &abort_flag)) {
          abort_flag = 1;
          break;
        }
        l1 = lcol[(j - 1) & 3][j + 1];
      }
      const T lnext = fma(-l1, lprev, S[j + 1][j]) * rd;
      d = fma(-lnext, lnext, S[j + 1][j + 1]);
      lprev = lnext;
    }
    if (!ok && lane == 0) fail = 1;
  } else if (warp == 1) {
    // ---- column warp: L_:j = (A_:j - L_:j-1 L_{j,j-1}) rd_j, L_jj = d_j rd_j
    const int i0 = lane, i1 = lane + 32;
    for (int j = 0; j < n; ++j) {
      if (!cta_mbar_wait(&barC[j & 1], (j >> 1) & 1, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      const T rd = rds[j], dj = dpiv[j & 1];
      const T* lp = lcol[(j - 1) & 3];
      const T lj = j >= 1 ? lp[j] : (T)0;  // column 0 has no previous column (its ring slot is unwritten)
      T* lo = lcol[j & 3];
      if (j < 32 && i0 >= j && i0 < n) {
        const T c0 = i0 == j ? dj : (j >= 1 ? fma(-lp[i0], lj, S[i0][j]) : S[i0][j]);
        const T l0 = c0 * rd;
        lo[i0] = l0;
        a[(size_t)(k0 + i0) * D + k0 + j] = l0;
      }
      if (i1 >= j && i1 < n) {
        const T c1 = i1 == j ? dj : (j >= 1 ? fma(-lp[i1], lj, S[i1][j]) : S[i1][j]);
        const T l1 = c1 * rd;
        lo[i1] = l1;
        a[(size_t)(k0 + i1) * D + k0 + j] = l1;
      }
      __syncwarp();
      if (lane == 0) cta_mbar_arrive(&barB[j & 1]);
      if (col_flag && (j % pub_every == pub_every - 1 || j == n - 1)) {
        // columns up to j and their rsqrt(d) for the streamed inverse, pub_every at a time
        // (a fence per column would sit on this warp's part of the pivot cycle)
        const int j0 = j - j % pub_every;
        if (lane <= j - j0) rdiag[j0 + lane] = rds[j0 + lane];
        __threadfence();
        __syncwarp();
        if (lane == 0) gpu_flag_release(col_flag, j + 1);
      }
    }
  } else if (uw >= 0) {
    // ---- trailing update
    const int bt = uw * 32 + lane;
    const int wbase = bt - lane;
    // The passes loop over live slots only, with warp-uniform bounds: a predicated-off
    // FP64 instruction would still hold the FP64 unit for its full 64 cycles.
    for (int k = 0; k + 2 < n; ++k) {
      if (!cta_mbar_wait(&barB[k & 1], (k >> 1) & 1, &abort_flag)) {  // L_:k is published
        abort_flag = 1;
        break;
      }
      const T* lp = lcol[k & 3];
      const int live = (n - k - 2) * (n - k - 1) / 2;  // elements of columns >= k+2
      const int rest = (n - k - 3) * (n - k - 2) / 2;  // elements of columns >= k+3
      // column k+2 (elements rest .. live-1) first
      const int first = rest - wbase - 31;  // first slot whose warp range reaches e >= rest
#pragma unroll 1
      for (int sl = first > 0 ? (first + kUpdThreads - 1) / kUpdThreads : 0; sl * kUpdThreads + wbase < live; ++sl) {
        const int e = sl * kUpdThreads + bt;
        if (e >= rest && e < live) {
          const uint32_t v = eidx[sl][bt];
          const int i = (int)(v >> 8), c = (int)(v & 255u);
          S[i][c] = fma(-lp[i], lp[c], S[i][c]);
        }
      }
      __syncwarp();
      if (lane == 0) cta_mbar_arrive(&barA[k & 1]);
      // slots whose warp range starts below `rest`; all but the last are fully live.
      // Pairs: both loads, then both FMAs, then both stores (independent chains).
      const int nsl = rest > wbase ? (rest - wbase + kUpdThreads - 1) / kUpdThreads : 0;
      int sl = 0;
#pragma unroll 1
      for (; sl + 1 < nsl; sl += 2) {
        const uint32_t v0 = eidx[sl][bt], v1 = eidx[sl + 1][bt];
        const int i0 = (int)(v0 >> 8), c0 = (int)(v0 & 255u), i1 = (int)(v1 >> 8), c1 = (int)(v1 & 255u);
        const bool on1 = (sl + 1) * kUpdThreads + bt < rest;
        const T s0 = S[i0][c0], s1 = S[i1][c1];
        const T x0 = fma(-lp[i0], lp[c0], s0), x1 = fma(-lp[i1], lp[c1], s1);
        S[i0][c0] = x0;
        if (on1) S[i1][c1] = x1;
      }
      if (sl < nsl && sl * kUpdThreads + bt < rest) {
        const uint32_t v = eidx[sl][bt];
        const int i = (int)(v >> 8), c = (int)(v & 255u);
        S[i][c] = fma(-lp[i], lp[c], S[i][c]);
      }
    }
  }
  __syncthreads();
  pdl_trigger();  // the next kernel may launch: only the zero fill and rdiag remain
  if (abort_flag || fail) {
    if (tid == 0) {
      atomicOr(status, abort_flag ? ST_TIMEOUT : ST_NOT_PD);
      if (col_flag) gpu_flag_release(col_flag, -1);
    }
    return;
  }
  // L itself was written by the column warp; zeros above the diagonal
  for (int e = tid; e < n * n; e += kPotrfThreads) {
    const int i = e / n, c = e - (e / n) * n;
    if (c > i) a[(size_t)(k0 + i) * D + k0 + c] = (T)0;
  }
  if (tid < n) rdiag[tid] = rds[tid];
}

template <typename T>
__global__ void __launch_bounds__(kPotrfThreads) potrf_kernel(T* __restrict__ a, int D, int k0,
                                                              const double* __restrict__ ridge,
                                                              T* __restrict__ rdiag, uint32_t* __restrict__ status) {
  pdl_wait();
  potrf_body<T>(a, D, k0, ridge, rdiag, status, nullptr, 1);
}

// Column c of W = L_kk^{-1} (lower; it turns the panel solve into a product) while the
// diagonal block is being factored: right-looking forward substitution of L w = e_c with
// rows lane and lane + 32 in warp 0's registers, w_m = (accumulated value) rsqrt(d_m),
// then rows below subtract L_im w_m; step m is taken as soon as column m of L and
// rsqrt(d_m) are published (loads from L2). One CTA per column spreads the FP64 work
// over many SMs. Bounded waits; a published -1 ends it.
template <typename T>
__device__ __forceinline__ void inv_streamed(const T* __restrict__ a, int D, int k0, const T* __restrict__ rdiag,
                                             T* __restrict__ W, uint32_t* __restrict__ status,
                                             const int* col_flag, int c) {
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  if (c >= n) return;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < c; i += blockDim.x) W[i * NB + c] = (T)0;
  if (tid >= 32) return;
  const int i0 = lane, i1 = lane + 32;
  T acc0 = (i0 == c) ? (T)1 : (T)0, acc1 = (i1 == c) ? (T)1 : (T)0;
  int have = 0;  // columns every lane has seen published (warp-uniform)
  for (int m = c; m < n; ++m) {
    if (have < m + 1) {
      // every lane acquires the flag itself; the decisions are taken warp-wide so that
      // no lane leaves while another still waits in a shuffle
      const long long t0 = clock64(), lim = spin_limit();
      for (;;) {
        const int f = gpu_flag_acquire(col_flag);
        if (__any_sync(0xffffffffu, f < 0)) return;
        if (__all_sync(0xffffffffu, f >= m + 1)) {
          have = __reduce_min_sync(0xffffffffu, (unsigned)f);
          break;
        }
        const int late = lane == 0 ? (clock64() - t0 > lim) : 0;
        if (__shfl_sync(0xffffffffu, late, 0)) {
          if (lane == 0) atomicOr(status, ST_TIMEOUT);
          return;
        }
        __nanosleep(64);
      }
    }
    const T l0 = (m < 31 && i0 > m) ? a[(size_t)(k0 + i0) * D + k0 + m] : (T)0;
    const T l1 = (i1 > m && i1 < n) ? a[(size_t)(k0 + i1) * D + k0 + m] : (T)0;
    const T w = __shfl_sync(0xffffffffu, m < 32 ? acc0 : acc1, m & 31) * rdiag[m];
    if (lane == (m & 31)) W[m * NB + c] = w;
    if (m < 31) acc0 = fma(-l0, w, acc0);
    acc1 = fma(-l1, w, acc1);
  }
}

// Diagonal block (CTA 0) and the 64 columns of its inverse (CTAs 1..64) in one grid,
// launched cooperatively so that all CTAs are resident: the inverse trails the
// factorisation by about one column instead of starting after it.
template <typename T>
__global__ void __launch_bounds__(kPotrfThreads) potrf_inv_kernel(T* __restrict__ a, int D, int k0,
                                                                  const double* __restrict__ ridge,
                                                                  T* __restrict__ rdiag, T* __restrict__ W,
                                                                  uint32_t* __restrict__ status, int* col_flag,
                                                                  int pub_every) {
  pdl_wait();
  if (blockIdx.x == 0) potrf_body<T>(a, D, k0, ridge, rdiag, status, col_flag, pub_every);
  else inv_streamed<T>(a, D, k0, rdiag, W, status, col_flag, (int)blockIdx.x - 1);
}

// Exact digit split of one panel row for the tensor-core trailing update. The warp
// holds the row's 64 values (x0 in column lane, x1 in column lane + 32). The row gets
// the exponent e = ilogb(max |x|) + 1 (so |x| < 2^e) and every element the integer
// N = floor(|x| 2^(56 - e)) < 2^56, cut into eight base-128 digits
// d_k = (N >> (56 - 7k)) & 127 carrying x's sign: x = sum_k d_k 2^(e - 7k) up to
// 2^(e - 56). The digits are integers below 128 in magnitude, exact in bf16; plane k
// (0..7) holds rows [k m_pad, (k+1) m_pad) of a [8 m_pad][64] array.
__device__ __forceinline__ void split_row_digits(double x0, int c0, double x1, int c1, int row, int m_pad,
                                                 __nv_bfloat16* __restrict__ planes, int* __restrict__ rexp) {
  // integer operations on the bit patterns only (the FP64 unit is the scarce one):
  // |x| as an unsigned integer orders like |x|, so the row maximum is an integer max
  const unsigned long long b0 = (unsigned long long)__double_as_longlong(x0),
                           b1 = (unsigned long long)__double_as_longlong(x1);
  const unsigned long long mag = 0x7FFFFFFFFFFFFFFFull;
  unsigned long long amax = (b0 & mag) > (b1 & mag) ? (b0 & mag) : (b1 & mag);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, amax, o);
    amax = t > amax ? t : amax;
  }
  // e = ilogb(max |x|) + 1, or 0 for a zero row
  int e = 0;
  if (amax != 0ull) {
    const int ex = (int)(amax >> 52);
    e = ex > 0 ? ex - 1022 : (63 - __clzll((long long)amax)) - 1074 + 1;
  }
  const int lane = threadIdx.x & 31;
  if (lane == 0) rexp[row] = e;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const unsigned long long bits = h ? b1 : b0;
    const int col = h ? c1 : c0;
    // N = floor(|x| 2^(56-e)) with |x| = M 2^(E-1075): shift the 53-bit significand
    const int E = (int)((bits >> 52) & 0x7FF);
    const unsigned long long M = (bits & 0x000FFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    const int sh = (E ? E : 1) - 1019 - e;
    const unsigned long long N = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> -sh) : 0ull);
    const bool neg = (bits >> 63) != 0ull;
#pragma unroll
    for (int k = 1; k <= 8; ++k) {
      const int d = (int)((N >> (56 - 7 * k)) & 127ull);
      planes[((size_t)(k - 1) * m_pad + row) * 64 + col] = __float2bfloat16_rn((float)(neg ? -d : d));
    }
  }
}

// Panel below diagonal block k0: X = A W^T with W = L_kk^{-1} (solves X L_kk^T = A),
// kTrsmRows rows per CTA (many small CTAs keep the panel solve short on the critical
// path of the factorisation), written in place. Only full 64-wide panels come here
// (the last diagonal block has no panel below it).
constexpr int kTrsmRows = 8;
template <typename T>
__global__ void __launch_bounds__(kTrsmRows * 32) trsm_gemm_kernel(T* __restrict__ a, int D, int k0, const T* __restrict__ W,
                                                        const uint32_t* __restrict__ status,
                                                        __nv_bfloat16* __restrict__ planes, int* __restrict__ rexp,
                                                        int m_pad) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T(*Ws)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem);
  T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem + sizeof(T) * NB * (NB + 1));
  pdl_wait();
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const int r0 = k0 + n + blockIdx.x * kTrsmRows;
  const int rows = min(kTrsmRows, D - r0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int i = e >> 6, c = e & 63;
    Ws[i][c] = (i < n && c < n) ? W[i * NB + c] : (T)0;
  }
  for (int e = threadIdx.x; e < kTrsmRows * NB; e += blockDim.x) {
    const int i = e >> 6, c = e & 63;
    As[i][c] = (i < rows && c < n) ? a[(size_t)(r0 + i) * D + k0 + c] : (T)0;
  }
  __syncthreads();
  // W is lower triangular (W[c][m] = 0 for m > c): lane l forms columns l and 63 - l,
  // l + 1 and 64 - l terms, one 65-step loop with the same trip count in every lane
  // (a predicated-off FP64 instruction would cost as much as a live one)
  const int rr = threadIdx.x >> 5, l = threadIdx.x & 31;
  T acc = (T)0, acc_a = (T)0;
#pragma unroll 5
  for (int t = 0; t <= NB; ++t) {
    if (t == l + 1) {
      acc_a = acc;
      acc = (T)0;
    }
    const bool first = t <= l;
    const int m = first ? t : t - l - 1;
    const int col = first ? l : NB - 1 - l;
    acc = fma(As[rr][m], Ws[col][m], acc);
  }
  const T acc_b = acc;
  if (rr < rows) {
    a[(size_t)(r0 + rr) * D + k0 + l] = acc_a;
    a[(size_t)(r0 + rr) * D + k0 + NB - 1 - l] = acc_b;
  }
  if constexpr (sizeof(T) == 8) {
    // the warp holds one whole panel row: split it into the digit planes of the
    // tensor-core trailing update (rows past the panel get zero digits)
    if (planes != nullptr)
      split_row_digits(acc_a, l, acc_b, NB - 1 - l, blockIdx.x * kTrsmRows + rr, m_pad, planes, rexp);
  }
}

// Trailing update after block column k0: A_ij -= L_ik L_jk^T on 64 x 64 lower tiles
// (bi >= bj, block indices relative to the trailing matrix) with bj in [blk_lo, blk_hi),
// column by column.
template <typename T>
__global__ void __launch_bounds__(256) syrk_update_kernel(T* __restrict__ a, int D, int k0, int blk_lo, int blk_hi,
                                                          const uint32_t* __restrict__ status) {
  __shared__ T As[16][NB + 2];
  __shared__ T Bs[16][NB + 2];
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const int below = (D - k0 - n + NB - 1) / NB;
  int t = blockIdx.x, bj = blk_lo;
  while (bj < blk_hi && t >= below - bj) {
    t -= below - bj;
    ++bj;
  }
  if (bj >= blk_hi || bj >= below) return;
  const int bi = bj + t;
  const int base = k0 + n;
  const int i0 = base + bi * NB, j0 = base + bj * NB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int kk = 0; kk < n; kk += 16) {
    for (int e = threadIdx.x; e < NB * 16; e += 256) {
      const int r = e / 16, k = e % 16;
      const int gk = k0 + kk + k;
      const bool kin = (kk + k) < n;
      As[k][r] = (kin && i0 + r < D) ? a[(size_t)(i0 + r) * D + gk] : (T)0;
      Bs[k][r] = (kin && j0 + r < D) ? a[(size_t)(j0 + r) * D + gk] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T x[4], y[4];
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

template <typename Ti, typename To>
__global__ void convert_factor_kernel(const Ti* __restrict__ Lc, int D, To* __restrict__ out, int ld) {
  const long long total = (long long)D * ld;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / ld), j = (int)(k - (long long)i * ld);
    const double v = (j < D && j <= i) ? (double)Lc[(size_t)i * D + j] : 0.0;
    if constexpr (sizeof(To) == 2) out[k] = __float2bfloat16_rn((float)v);
    else out[k] = (To)v;
  }
}

cudaError_t launch_copy_lower(const double* src, double* dst, int D, cudaStream_t s) {
  copy_lower_kernel<double><<<sm_count() * 4, 256, 0, s>>>(src, dst, D);
  return cudaGetLastError();
}

// Blocked right-looking factorisation. With a second stream `side` (and two events),
// the next block column's update and its diagonal/panel factorisation run on `side`
// while `s` applies the rest of the trailing update (look-ahead); the arithmetic of
// every tile is the same either way, so both schedules give identical results.
// Cooperative launch: every CTA of the grid resident at once (the streamed inverse's
// CTAs wait on the factorising CTA).
template <typename... KArgs, typename... Args>
static cudaError_t launch_coop(void (*kern)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Launch with programmatic stream serialisation (the kernel calls pdl_wait first).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename T>
static cudaError_t cholesky_t(T* a, int D, const double* ridge, void* aux, uint32_t* status, cudaStream_t s,
                              cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB, bool tensor_update,
                              LaunchTimer* timer = nullptr) {
  const int nblk = (D + NB - 1) / NB;
  const bool ahead = side != nullptr && nblk > 2;
  T* W = (T*)aux;
  T* rdiag = (T*)((unsigned char*)aux + round256((size_t)nblk * NB * NB * sizeof(double)));
  const int m_pad = mpad_of(D);
  unsigned char* dig0 = (unsigned char*)rdiag + round256((size_t)nblk * NB * sizeof(double));
  // digit-plane buffers by panel mod 3 (two suffice for one column of look-ahead: the
  // bulk update of panel kb ends before panel kb+2 is solved)
  const size_t plane_bytes = round256(8 * (size_t)m_pad * 64 * 2), rexp_bytes = round256((size_t)m_pad * sizeof(int));
  __nv_bfloat16* planes[3];
  int* rexp[3];
  for (int q = 0; q < 3; ++q) {
    planes[q] = (__nv_bfloat16*)(dig0 + q * plane_bytes);
    rexp[q] = (int*)(dig0 + 3 * plane_bytes + q * rexp_bytes);
  }
  // columns the diagonal block publishes at a time to its streamed inverse (1..32)
  static const int kPublishEvery = [] {
    const char* v = getenv("PHI4_PUBLISH_EVERY");
    return v ? std::min(32, std::max(1, atoi(v))) : 8;
  }();
  // per diagonal block, the count of its published columns (streamed inverse)
  int* col_flags = (int*)(dig0 + 3 * plane_bytes + 3 * rexp_bytes);
  {
    const cudaError_t e = cudaMemsetAsync(col_flags, 0, (size_t)nblk * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  const bool tcu = tensor_update && sizeof(T) == 8;
  // trailing update by panel kb of the 64-column blocks [lo, hi) of its trailing matrix
  auto update = [&](int kb, int lo, int hi, cudaStream_t st) -> cudaError_t {
    const int k0 = kb * NB, b0 = k0 + NB;
    const int below = nblk - kb - 1;
    hi = std::min(hi, below);
    if (lo >= hi) return cudaSuccess;
    if (tcu) {
      // timed: the bulk of each update (an event between the next block column's update
      // and the diagonal block would stop the latter's programmatic early launch)
      cudaEvent_t t0 = timer && lo >= 1 ? timer->begin(st) : nullptr;
      const cudaError_t e = launch_chol_update_tc((double*)a, D, b0, D - b0, planes[kb % 3], m_pad, rexp[kb % 3], lo,
                                                  hi >= below ? (1 << 20) : hi, ahead && lo >= 1, status, st);
      if (t0) timer->end(st, t0);
      return e;
    }
    long long g = 0;
    for (int bj = lo; bj < hi; ++bj) g += below - bj;
    if (g > 0) syrk_update_kernel<T><<<(unsigned)g, 256, 0, st>>>(a, D, k0, lo, hi, status);
    return cudaGetLastError();
  };
  const size_t sm_trsm = sizeof(T) * (NB + kTrsmRows) * (NB + 1);
  cudaError_t e0 = cudaFuncSetAttribute(trsm_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_trsm);
  if (e0 != cudaSuccess) return e0;
  // the chain's kernels are launched as programmatic dependents of their predecessors
  // (each waits for it at entry), so their launch latency overlaps the predecessor
  auto panel = [&](int kb, cudaStream_t st) {
    const int k0 = kb * NB;
    const int rows = D - k0 - min(NB, D - k0);
    if (rows <= 0) {  // the last diagonal block: no panel, no inverse
      launch_pdl(potrf_kernel<T>, 1, kPotrfThreads, 0, st, a, D, k0, ridge, rdiag + (size_t)kb * NB, status);
    } else {
      // the diagonal block with its inverse streamed beside it (the inverse only feeds
      // the panel solve)
      launch_coop(potrf_inv_kernel<T>, 1 + min(NB, D - k0), kPotrfThreads, st, a, D, k0, ridge,
                  rdiag + (size_t)kb * NB, W + (size_t)kb * NB * NB, status, col_flags + kb, kPublishEvery);
      // with the tensor-core update the solve also writes the digit planes, for every
      // row of the update's 128-row tiles (rows >= `rows` get zeros)
      const int grid_rows = tcu ? (rows + 127) / 128 * 128 : rows;
      launch_pdl(trsm_gemm_kernel<T>, (grid_rows + kTrsmRows - 1) / kTrsmRows, kTrsmRows * 32, sm_trsm, st, a, D, k0,
                 (const T*)(W + (size_t)kb * NB * NB), (const uint32_t*)status,
                 tcu ? planes[kb % 3] : (__nv_bfloat16*)nullptr, rexp[kb % 3], m_pad);
    }
  };
  panel(0, s);
  cudaError_t e;
  if (!ahead) {
    for (int kb = 0; kb < nblk - 1; ++kb) {
      if ((e = update(kb, 0, nblk, s)) != cudaSuccess) return e;
      panel(kb + 1, s);
    }
    return cudaGetLastError();
  }
  // One block column of look-ahead: per panel kb, `side` (high priority) updates block
  // column kb+1 and factors/solves panel kb+1 while `s` applies the rest of the update.
  // Block column kb+1 gets panel kb-1's update from `s` at the previous step, hence the
  // wait on evA. (Looking two columns ahead measured slower: the extra one-column
  // update launch per panel cost more than the waits it removed.)
  for (int kb = 0; kb < nblk - 1; ++kb) {
    if ((e = cudaEventRecord(evA, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, evA, 0)) != cudaSuccess) return e;
    if ((e = update(kb, 0, 1, side)) != cudaSuccess) return e;
    panel(kb + 1, side);
    if ((e = cudaEventRecord(evB, side)) != cudaSuccess) return e;
    if ((e = update(kb, 1, nblk, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, evB, 0)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

PHI4_SPIN_LIMIT_SETTER(set_spin_limit_chol)

size_t cholesky_aux_bytes(int D) {
  const size_t nblk = (size_t)(D + NB - 1) / NB;
  const size_t mp = (size_t)mpad_of(D);
  return round256(nblk * NB * NB * sizeof(double)) + round256(nblk * NB * sizeof(double)) +
         3 * round256(8 * mp * 64 * 2) + 3 * round256(mp * sizeof(int)) + round256(nblk * sizeof(int));
}

// Which trailing update the double factorisation uses (mode 0 = automatic).
static bool use_tensor_update(int D, int mode) {
  if (mode == 1) return false;
  if (mode == 2) return tc_available();
  return D >= 256 && tc_available();
}

cudaError_t launch_cholesky(double* a, int D, const double* ridge, uint32_t* status, void* aux, cudaStream_t s,
                            cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB, int mode, LaunchTimer* timer) {
  return cholesky_t<double>(a, D, ridge, aux, status, s, side, evA, evB, use_tensor_update(D, mode), timer);
}

cudaError_t launch_cholesky_f32(const double* sigma, float* a, int D, const double* ridge, uint32_t* status,
                                void* aux, cudaStream_t s, cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB) {
  copy_lower_kernel<float><<<sm_count() * 4, 256, 0, s>>>(sigma, a, D);
  return cholesky_t<float>(a, D, ridge, aux, status, s, side, evA, evB, false);
}

int cholesky_launches(int D) {
  const int nblk = (D + NB - 1) / NB;
  return nblk + 3 * (nblk - 1);  // diagonal blocks (with their inverses); per panel: solve, two update parts
}

cudaError_t launch_factor_convert(const double* Lc, int D, int dtype, void* out, int ld, cudaStream_t s) {
  const int grid = sm_count() * 4;
  if (dtype == 0) convert_factor_kernel<double, double><<<grid, 256, 0, s>>>(Lc, D, (double*)out, ld);
  else if (dtype == 1) convert_factor_kernel<double, float><<<grid, 256, 0, s>>>(Lc, D, (float*)out, ld);
  else if (dtype == 2)
    convert_factor_kernel<double, __nv_bfloat16><<<grid, 256, 0, s>>>(Lc, D, (__nv_bfloat16*)out, ld);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_factor_convert_f32(const float* Lc, int D, float* out, cudaStream_t s) {
  convert_factor_kernel<float, float><<<sm_count() * 4, 256, 0, s>>>(Lc, D, out, D);
  return cudaGetLastError();
}

}  // namespace phi4
