// Device descriptor of one member run of a batch (the batched form: many independent SMC
// runs advanced together, one launch per stage over all of them). One array of these per
// parity of the particle buffers: at a step of parity q the gather reads the `src`
// buffers and writes the `dst` buffers, and every later stage of the step works on `dst`.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>
#include "internal.h"
#include "philox.cuh"

namespace phi4 {

// The batched stages read a run's temperature counter (the Philox step of the current
// temperature) and its participation in the current step (beta was below 1 when the step
// began) from its scalar block: SC_T and SC_ACTIVE.
struct BatchRun {
  ActionParams ap;
  PhiloxKey key;
  double rho;
  int iters, keep_ref, n_mcmc;
  int dtype;   // element type of the fields (0 double, 1 float)
  int zdtype;  // element type of the proposal normals Z (0 double, 1 float, 2 bf16)
  int ldz;
  int ppb, tpp;  // block shape of the fused accept (the single-run launcher's)
  const void* phi_src;
  void* phi_dst;
  const double *S_src, *sq_src, *ell_src;
  double *S_dst, *sq_dst, *ell_dst;
  double *w, *scal;
  int32_t* anc;
  unsigned long long* csum;  // resampling prefix sums
  unsigned* bar;             // bisection barrier words (one CTA: its own arrival)
  double* part;              // bisection partials
  uint32_t *status, *acc;
  void* Z;                   // proposal normals (dtype of the proposal GEMM's operand)
  const __half* delta;       // mixed form: the fp16 increment of the tensor-core proposal
};

cudaError_t set_smem_bytes(const void* kernel, size_t bytes);
void accept_vec_shape(int D, int* ppb, int* tpp);
// one launch over the accept blocks of every run: blk0[r] = first block of run r (R + 1 entries);
// batch_accept_prepare(smem) once before (outside any stream capture)
cudaError_t batch_accept_prepare(size_t smem);
cudaError_t launch_batch_accept(const BatchRun* runs, int R, const int* blk0, int n_blocks, size_t smem,
                                uint32_t sweep, cudaStream_t s);
// one launch over the normal rows of every run: row0[r] = first row of run r (R + 1 entries)
cudaError_t launch_batch_normals(const BatchRun* runs, int R, const int* row0, int total_rows, int max_d,
                                 uint32_t sweep, int threads, cudaStream_t s);

// Grouped proposal GEMM (kernels_tc.cu): the tiles of every run in one persistent launch.
// Per run, 64-byte aligned in device memory: its two tensor maps and its sizes.
struct __align__(64) GemmRun {
  unsigned char mapA[128], mapB[128];  // CUtensorMap of Z (bf16 [N][ldz]) and of L (bf16 [D][ldl])
  __half* delta;
  const double* scal;                  // the run's scalar block (SC_ACTIVE)
  float scale;
  int M, Nn, K, tiles_m, tiles_n, tile0, n_mcmc;
};
bool make_gemm_run(GemmRun* g, const void* Zb, int ldz, const void* Lb, int ldl, int N, int D, float scale,
                   __half* delta, const double* scal, int n_mcmc);
// grouped_propose_prepare() once before launching (outside any stream capture)
cudaError_t grouped_propose_prepare();
cudaError_t launch_grouped_propose(const GemmRun* runs, int R, int total_tiles, int grid, uint32_t sweep,
                                   uint32_t* status, cudaStream_t s);

}  // namespace phi4
