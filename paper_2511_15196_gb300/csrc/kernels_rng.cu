// Philox normals written to a row-major buffer (one thread per block of 4 outputs).
#include "internal.h"
#include "philox.cuh"

namespace phi4 {

template <typename T>
__global__ void normals_kernel(PhiloxKey key, uint32_t w0, uint32_t sub, int row0, int n_rows, int n_cols, int ld,
                               T* __restrict__ out) {
  const int nblk = (n_cols + 3) >> 2;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)n_rows * nblk) return;
  const int r = (int)(gid / nblk), b = (int)(gid % nblk);
  const uint4 w = philox4x32_10(make_uint4(w0, sub, (uint32_t)(row0 + r), (uint32_t)b), key);
  T* o = out + (size_t)r * ld + 4 * b;
  const int left = n_cols - 4 * b;
  if constexpr (sizeof(T) == 8) {
    const double2 z01 = box_muller_f64(w.x, w.y), z23 = box_muller_f64(w.z, w.w);
    const double z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < left) o[j] = z[j];
  } else {
    const float2 z01 = box_muller_f32(w.x, w.y), z23 = box_muller_f32(w.z, w.w);
    const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < left) o[j] = to_t<T>(z[j]);
  }
}

cudaError_t launch_normals(uint64_t seed, uint64_t stream_id, uint32_t kind, uint32_t step, uint32_t sub,
                           int row0, int n_rows, int n_cols, int ld, int dtype, void* out, cudaStream_t s) {
  if (n_rows <= 0 || n_cols <= 0) return cudaSuccess;
  const PhiloxKey key = philox_key(seed, stream_id);
  const uint32_t w0 = counter_word0(kind, step);
  const long long work = (long long)n_rows * ((n_cols + 3) / 4);
  const int threads = 256;
  const unsigned grid = (unsigned)((work + threads - 1) / threads);
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
