// Philox normals written to a row-major buffer (one thread per two blocks of 4 outputs).
#include <algorithm>
#include "internal.h"
#include "philox.cuh"
#include "batch.h"

namespace phi4 {

// Each thread makes two consecutive blocks of four normals (counter words 2 and 3 =
// particle, block) of one row; rows come from the grid's y dimension (no 64-bit index
// division), and the eight values of a thread are stored together.
template <typename T>
__global__ void normals_kernel(PhiloxKey key, uint32_t w0, uint32_t sub, int row0, int n_rows, int n_cols, int ld,
                               T* __restrict__ out) {
  const int nblk = (n_cols + 3) >> 2;
  const int b0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (b0 >= nblk) return;
  for (int r = blockIdx.y; r < n_rows; r += gridDim.y) {
    T z[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint4 w = philox4x32_10(make_uint4(w0, sub, (uint32_t)(row0 + r), (uint32_t)(b0 + h)), key);
      if constexpr (sizeof(T) == 8) {
        const double2 z01 = box_muller_f64(w.x, w.y), z23 = box_muller_f64(w.z, w.w);
        z[4 * h] = z01.x; z[4 * h + 1] = z01.y; z[4 * h + 2] = z23.x; z[4 * h + 3] = z23.y;
      } else {
        const float2 z01 = box_muller_f32(w.x, w.y), z23 = box_muller_f32(w.z, w.w);
        z[4 * h] = to_t<T>(z01.x); z[4 * h + 1] = to_t<T>(z01.y);
        z[4 * h + 2] = to_t<T>(z23.x); z[4 * h + 3] = to_t<T>(z23.y);
      }
    }
    T* o = out + (size_t)r * ld + 4 * b0;
    const int left = n_cols - 4 * b0;
    if (left >= 8 && (((uintptr_t)o) & (8 * sizeof(T) - 1)) == 0) {
      if constexpr (sizeof(T) == 2) {
        *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(z);
      } else if constexpr (sizeof(T) == 4) {
        reinterpret_cast<uint4*>(o)[0] = reinterpret_cast<const uint4*>(z)[0];
        reinterpret_cast<uint4*>(o)[1] = reinterpret_cast<const uint4*>(z)[1];
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = z[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < left) o[j] = z[j];
    }
  }
}

// Global Z2 move: row n of phi is negated when bit 0 of the first Philox word of
// counter (w0, 0, n, 0) is set. Grid (column chunks, rows); the row's bit is drawn once
// per block.
template <typename T>
__global__ void z2_flip_kernel(PhiloxKey key, uint32_t w0, int N, int D, T* __restrict__ phi) {
  __shared__ int flip;
  const int n = blockIdx.y;
  if (threadIdx.x == 0) flip = (int)(philox4x32_10(make_uint4(w0, 0u, (uint32_t)n, 0u), key).x & 1u);
  __syncthreads();
  if (!flip) return;
  T* row = phi + (size_t)n * D;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) row[j] = -row[j];
}

cudaError_t launch_z2_flip(uint64_t seed, uint64_t stream_id, uint32_t step, void* phi, int dtype, int N, int D,
                           cudaStream_t s) {
  if (N <= 0 || D <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(RNG_FLIP, step);
  const dim3 grid((unsigned)std::min((D + 255) / 256, 16), (unsigned)std::min(N, 65535));
  if (N > 65535) return cudaErrorInvalidValue;
  if (dtype == 0) z2_flip_kernel<double><<<grid, 256, 0, s>>>(key, w0, N, D, (double*)phi);
  else if (dtype == 1) z2_flip_kernel<float><<<grid, 256, 0, s>>>(key, w0, N, D, (float*)phi);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Batched form: the proposal normals of every member run in one launch. Global row gr
// (grid y) belongs to run r with row0[r] <= gr < row0[r + 1]; each thread makes the same
// eight values of its row as normals_kernel (counter (PROPOSE << 24 | t, sweep, row,
// block), t the run's temperature counter) in the run's element type. Runs that are done
// or have fewer sweeps are skipped.
__global__ void batch_normals_kernel(const BatchRun* __restrict__ runs, int R, const int* __restrict__ row0,
                                     int total_rows, uint32_t sweep) {
  for (int gr = blockIdx.y; gr < total_rows; gr += gridDim.y) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (row0[mid] <= gr) lo = mid; else hi = mid - 1;
    }
    const BatchRun& b = runs[lo];
    if (b.scal[SC_ACTIVE] == 0.0 || (int)sweep >= b.n_mcmc) continue;
    const int r = gr - row0[lo], n_cols = b.ap.D;
    const int nblk = (n_cols + 3) >> 2;
    const uint32_t w0 = counter_word0(RNG_PROPOSE, (uint32_t)b.scal[SC_T]);
    for (int b0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x); b0 < nblk; b0 += 2 * (int)(gridDim.x * blockDim.x)) {
      float z[8];
      double zd[8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 w = philox4x32_10(make_uint4(w0, sweep, (uint32_t)r, (uint32_t)(b0 + h)), b.key);
        if (b.zdtype == 0) {  // double
          const double2 z01 = box_muller_f64(w.x, w.y), z23 = box_muller_f64(w.z, w.w);
          zd[4 * h] = z01.x; zd[4 * h + 1] = z01.y; zd[4 * h + 2] = z23.x; zd[4 * h + 3] = z23.y;
        } else {
          const float2 z01 = box_muller_f32(w.x, w.y), z23 = box_muller_f32(w.z, w.w);
          z[4 * h] = z01.x; z[4 * h + 1] = z01.y; z[4 * h + 2] = z23.x; z[4 * h + 3] = z23.y;
        }
      }
      const int left = n_cols - 4 * b0;
      if (b.zdtype == 0) {  // double
        double* o = (double*)b.Z + (size_t)r * b.ldz + 4 * b0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < left) o[j] = zd[j];
      } else if (b.zdtype == 1) {  // float
        float* o = (float*)b.Z + (size_t)r * b.ldz + 4 * b0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < left) o[j] = z[j];
      } else {
        __nv_bfloat16* o = (__nv_bfloat16*)b.Z + (size_t)r * b.ldz + 4 * b0;
        if (left >= 8 && (((uintptr_t)o) & 15) == 0) {
          __nv_bfloat16 zb[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) zb[j] = __float2bfloat16_rn(z[j]);
          *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(zb);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < left) o[j] = __float2bfloat16_rn(z[j]);
        }
      }
    }
  }
}

cudaError_t launch_batch_normals(const BatchRun* runs, int R, const int* row0, int total_rows, int max_d,
                                 uint32_t sweep, int threads, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  const int nblk = (max_d + 3) / 4;
  const dim3 grid((unsigned)((nblk + 2 * threads - 1) / (2 * threads)), (unsigned)std::min(total_rows, 65535));
  batch_normals_kernel<<<grid, threads, 0, s>>>(runs, R, row0, total_rows, sweep);
  return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint64_t stream_id, uint32_t kind, uint32_t step, uint32_t sub,
                           int row0, int n_rows, int n_cols, int ld, int dtype, void* out, cudaStream_t s) {
  if (n_rows <= 0 || n_cols <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(kind, step);
  const int nblk = (n_cols + 3) / 4;
  const int threads = 256;
  const dim3 grid((unsigned)((nblk + 2 * threads - 1) / (2 * threads)), (unsigned)std::min(n_rows, 65535));
  switch (dtype) {
    case 0: normals_kernel<double><<<grid, threads, 0, s>>>(key, w0, sub, row0, n_rows, n_cols, ld, (double*)out); break;
    case 1: normals_kernel<float><<<grid, threads, 0, s>>>(key, w0, sub, row0, n_rows, n_cols, ld, (float*)out); break;
    case 2: normals_kernel<__nv_bfloat16><<<grid, threads, 0, s>>>(key, w0, sub, row0, n_rows, n_cols, ld,
                                                                    (__nv_bfloat16*)out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace phi4
