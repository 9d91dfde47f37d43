// Cholesky of the particle covariance (App. A), blocked right-looking with 64 x 64
// blocks: per block column, (1) factor the diagonal block in one CTA, (2) triangular
// solve of the panel below it, (3) symmetric update of the trailing lower blocks.
// Templated on the element type: double for the FP64 and mixed forms, float for the
// plain FP32 form. A non-positive pivot sets ST_NOT_PD in the status word; later
// kernels see the bit and return.
#include <math.h>
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

// Factor the diagonal block in one CTA and form its inverse W = L_kk^{-1} (lower),
// which turns the panel's triangular solve into a dependency-free product.
// Per column: one thread forms the pivot with a single rsqrt (FP64 square roots and
// divisions are long sequences on the FP64 pipe, so they are done once per column),
// the column is scaled by multiplication, then the trailing block gets a rank-1 update.
template <typename T>
__global__ void __launch_bounds__(256) potrf_inv_kernel(T* __restrict__ a, int D, int k0,
                                                        const double* __restrict__ ridge, T* __restrict__ W,
                                                        uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T(*blk)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem);
  T(*inv)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem + sizeof(T) * NB * (NB + 1));
  __shared__ T rdiag[NB];
  __shared__ int fail;
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const T r = ridge ? (T)*ridge : (T)0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    T v = (j <= i) ? a[(size_t)(k0 + i) * D + k0 + j] : (T)0;
    if (i == j) v += r;
    blk[i][j] = v;
  }
  if (threadIdx.x == 0) fail = 0;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const T d = blk[j][j];
      if (!(d > (T)0) || !isfinite(d)) {
        fail = 1;
      } else {
        const T ip = rsqrt(d);
        rdiag[j] = ip;
        blk[j][j] = d * ip;
      }
    }
    __syncthreads();
    if (fail) break;
    const T ip = rdiag[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) blk[i][j] *= ip;
    __syncthreads();
    // rank-1 update of the trailing block: thread (ty, tx) of a 16 x 16 layout owns
    // rows ty + 16a and columns tx + 16b
#pragma unroll
    for (int a4 = 0; a4 < 4; ++a4) {
      const int i = ty + 16 * a4;
      if (i > j && i < n) {
        const T lij = blk[i][j];
#pragma unroll
        for (int b4 = 0; b4 < 4; ++b4) {
          const int l = tx + 16 * b4;
          if (l > j && l <= i) blk[i][l] -= lij * blk[l][j];
        }
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) atomicOr(status, ST_NOT_PD);
    return;
  }
  T(*Lo)[NB + 1] = blk;
  // W column j by forward substitution of L w = e_j, four lanes per column splitting each
  // dot product. Every lane runs the same trip count (the shuffles and warp barriers need
  // all 32 lanes); lanes whose column has not started yet contribute zero.
  const int j = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const bool col = j < n;
  if (col && sub == 0) inv[j][j] = rdiag[j];
  __syncwarp();
  for (int i = 1; i < n; ++i) {
    const bool act = col && i > j;
    T part = (T)0;
    if (act)
      for (int m = j + sub; m < i; m += 4) part += Lo[i][m] * inv[m][j];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    if (act && sub == 0) inv[i][j] = -part * rdiag[i];
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e % n;
    a[(size_t)(k0 + i) * D + k0 + c] = (c <= i) ? Lo[i][c] : (T)0;
    W[i * NB + c] = (c <= i) ? inv[i][c] : (T)0;
  }
}

// Panel below diagonal block k0: X = A W^T with W = L_kk^{-1} (solves X L_kk^T = A),
// kTrsmRows rows per CTA (many small CTAs keep the panel solve short on the critical
// path of the factorisation), written in place.
constexpr int kTrsmRows = 8;
template <typename T>
__global__ void __launch_bounds__(256) trsm_gemm_kernel(T* __restrict__ a, int D, int k0, const T* __restrict__ W,
                                                        const uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T(*Ws)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem);
  T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(chol_smem + sizeof(T) * NB * (NB + 1));
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
  // thread -> (row = tid / 32, output columns lane and lane + 32); W[c][m] = 0 for m > c
  const int rr = threadIdx.x >> 5, c0 = threadIdx.x & 31;
  T acc0 = (T)0, acc1 = (T)0;
  for (int m = 0; m < n; ++m) {
    const T x = As[rr][m];
    acc0 = fma(x, Ws[c0][m], acc0);
    acc1 = fma(x, Ws[c0 + 32][m], acc1);
  }
  if (rr < rows) {
    if (c0 < n) a[(size_t)(r0 + rr) * D + k0 + c0] = acc0;
    if (c0 + 32 < n) a[(size_t)(r0 + rr) * D + k0 + c0 + 32] = acc1;
  }
}

// Trailing update after block column k0: A_ij -= L_ik L_jk^T on 64 x 64 lower tiles.
// part 0: every tile; part 1: only the next block column (bj = 0); part 2: the rest.
template <typename T>
__global__ void __launch_bounds__(256) syrk_update_kernel(T* __restrict__ a, int D, int k0, int part,
                                                          const uint32_t* __restrict__ status) {
  __shared__ T As[16][NB + 2];
  __shared__ T Bs[16][NB + 2];
  if (*status & ST_NOT_PD) return;
  const int n = min(NB, D - k0);
  const long long t = blockIdx.x;
  int bi, bj;
  if (part == 1) {
    bi = (int)t;
    bj = 0;
  } else {
    bi = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while ((long long)bi * (bi + 1) / 2 > t) --bi;
    bj = (int)(t - (long long)bi * (bi + 1) / 2);
    if (part == 2) { ++bi; ++bj; }
  }
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

// Exact digit splitting of a Cholesky panel for the tensor-core trailing update.
// Row i of the panel (64 doubles below the diagonal block) gets the exponent
// e_i = ilogb(max |x|) + 1 (so |x| < 2^e_i) and every element the integer
// N = floor(|x| 2^(56 - e_i)) < 2^56, cut into eight base-128 digits
// d_k = (N >> (56 - 7k)) & 127 carrying x's sign: x = sum_k d_k 2^(e_i - 7k) up to
// 2^(e_i - 56). Digits are integers below 128 in magnitude, exact in bf16.
// Planes: plane k (0..7) holds rows [k m_pad, (k+1) m_pad) of a [8 m_pad][64] array.
__global__ void digit_split_kernel(const double* __restrict__ a, int D, int row0, int col0, int m, int m_pad,
                                   __nv_bfloat16* __restrict__ planes, int* __restrict__ rexp) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= m_pad) return;
  double x0 = 0.0, x1 = 0.0;
  if (row < m) {
    const double* src = a + (size_t)(row0 + row) * D + col0;
    x0 = src[lane];
    x1 = src[lane + 32];
  }
  const double amax = warp_max(fmax(fabs(x0), fabs(x1)));
  const int e = amax > 0.0 ? ilogb(amax) + 1 : 0;
  if (lane == 0) rexp[row] = e;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double x = h ? x1 : x0;
    const unsigned long long N = (unsigned long long)ldexp(fabs(x), 56 - e);
    const bool neg = x < 0.0;
#pragma unroll
    for (int k = 1; k <= 8; ++k) {
      const int d = (int)((N >> (56 - 7 * k)) & 127ull);
      planes[((size_t)(k - 1) * m_pad + row) * 64 + lane + 32 * h] = __float2bfloat16_rn((float)(neg ? -d : d));
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
template <typename T>
static cudaError_t cholesky_t(T* a, int D, const double* ridge, void* aux, uint32_t* status, cudaStream_t s,
                              cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB, bool tensor_update) {
  const int nblk = (D + NB - 1) / NB;
  const bool ahead = side != nullptr && nblk > 2;
  T* W = (T*)aux;
  const int m_pad = mpad_of(D);
  unsigned char* dig0 = (unsigned char*)aux + round256((size_t)nblk * NB * NB * sizeof(double));
  __nv_bfloat16* planes[2] = {(__nv_bfloat16*)dig0, (__nv_bfloat16*)(dig0 + round256(8 * (size_t)m_pad * 64 * 2))};
  int* rexp0 = (int*)(dig0 + 2 * round256(8 * (size_t)m_pad * 64 * 2));
  int* rexp[2] = {rexp0, (int*)((unsigned char*)rexp0 + round256((size_t)m_pad * sizeof(int)))};
  const bool tcu = tensor_update && sizeof(T) == 8;
  // trailing update after block column kb (part: 0 all, 1 next block column, 2 the rest)
  auto update = [&](int kb, int part, unsigned grid_all, unsigned grid_col, unsigned grid_rest,
                    cudaStream_t st) -> cudaError_t {
    const int k0 = kb * NB, b0 = k0 + NB;
    if (tcu)
      return launch_chol_update_tc((double*)a, D, b0, D - b0, planes[kb & 1], m_pad, rexp[kb & 1], part, status, st);
    const unsigned g = part == 0 ? grid_all : (part == 1 ? grid_col : grid_rest);
    if (g > 0) syrk_update_kernel<T><<<g, 256, 0, st>>>(a, D, k0, part, status);
    return cudaGetLastError();
  };
  const size_t sm_potrf = 2 * sizeof(T) * NB * (NB + 1), sm_trsm = sizeof(T) * (NB + kTrsmRows) * (NB + 1);
  cudaError_t e0 = cudaFuncSetAttribute(potrf_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_potrf);
  if (e0 != cudaSuccess) return e0;
  e0 = cudaFuncSetAttribute(trsm_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_trsm);
  if (e0 != cudaSuccess) return e0;
  auto panel = [&](int kb, cudaStream_t st) {
    const int k0 = kb * NB;
    potrf_inv_kernel<T><<<1, 256, sm_potrf, st>>>(a, D, k0, ridge, W + (size_t)kb * NB * NB, status);
    const int rows = D - k0 - min(NB, D - k0);
    if (rows > 0) {
      trsm_gemm_kernel<T><<<(rows + kTrsmRows - 1) / kTrsmRows, 256, sm_trsm, st>>>(a, D, k0, W + (size_t)kb * NB * NB, status);
      if (tcu)  // planes use the stride m_pad of the update kernel's tensor maps; rows >= `rows` get zeros
        digit_split_kernel<<<(m_pad * 32 + 255) / 256, 256, 0, st>>>((const double*)a, D, k0 + NB, k0, rows, m_pad,
                                                                     planes[kb & 1], rexp[kb & 1]);
    }
  };
  panel(0, s);
  for (int kb = 0; kb < nblk - 1; ++kb) {
    const int k0 = kb * NB;
    const int below = nblk - kb - 1;
    const long long all = (long long)below * (below + 1) / 2;
    const long long rest = all - below;
    cudaError_t e;
    if (!ahead) {
      if ((e = update(kb, 0, (unsigned)all, (unsigned)below, (unsigned)rest, s)) != cudaSuccess) return e;
      panel(kb + 1, s);
      continue;
    }
    if ((e = cudaEventRecord(evA, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, evA, 0)) != cudaSuccess) return e;
    if ((e = update(kb, 1, (unsigned)all, (unsigned)below, (unsigned)rest, side)) != cudaSuccess) return e;
    panel(kb + 1, side);
    if ((e = cudaEventRecord(evB, side)) != cudaSuccess) return e;
    if ((e = update(kb, 2, (unsigned)all, (unsigned)below, (unsigned)rest, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, evB, 0)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

size_t cholesky_aux_bytes(int D) {
  const size_t nblk = (size_t)(D + NB - 1) / NB;
  const size_t mp = (size_t)mpad_of(D);
  return round256(nblk * NB * NB * sizeof(double)) + 2 * round256(8 * mp * 64 * 2) + 2 * round256(mp * sizeof(int));
}

// Which trailing update the double factorisation uses (mode 0 = automatic).
static bool use_tensor_update(int D, int mode) {
  if (mode == 1) return false;
  if (mode == 2) return tc_available();
  return D >= 256 && tc_available();
}

cudaError_t launch_cholesky(double* a, int D, const double* ridge, uint32_t* status, void* aux, cudaStream_t s,
                            cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB, int mode) {
  return cholesky_t<double>(a, D, ridge, aux, status, s, side, evA, evB, use_tensor_update(D, mode));
}

cudaError_t launch_cholesky_f32(const double* sigma, float* a, int D, const double* ridge, uint32_t* status,
                                void* aux, cudaStream_t s, cudaStream_t side, cudaEvent_t evA, cudaEvent_t evB) {
  copy_lower_kernel<float><<<sm_count() * 4, 256, 0, s>>>(sigma, a, D);
  return cholesky_t<float>(a, D, ridge, aux, status, s, side, evA, evB, false);
}

int cholesky_launches(int D) {
  const int nblk = (D + NB - 1) / NB;
  return nblk + 2 * (nblk - 1) + (nblk - 1);
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
