// Nested-sampling driver (Sec. 2 sampler (iv); App. A): one deletion iteration per
// call. Order of work follows the sampler: delete the k lowest live points and
// update log X / log Z, refit the covariance of the survivors, run the k slice
// chains from random survivors, then put the new points in the deleted slots.
#include "run.h"

namespace phi4 {

namespace {
enum { NS_LOGX = 0, NS_LOGZ = 1, NS_LSTAR = 2, NS_NDEAD = 3, NS_STOP = 4, NS_REM = 5, NS_FZ = 6, NS_H = 7 };
}

phi4_status ns_replace(phi4_run* r, int32_t* done_out) {
  const phi4_config& c = r->cfg;
  const int N = c.N, D = r->D, k = c.ns_n_delete;
  cudaStream_t s = r->stream;
  double* ns = r->scal + SC_NS;
  const uint32_t it = (uint32_t)(++r->t);
  const int steps = c.ns_slice_steps > 0 ? c.ns_slice_steps : 3 * D;
  {
    StageScope sc(r, STG_NS_SELECT);
    CUDA_TRY(launch_ns_select(r->ell, N, k, r->ns_order, ns, r->ns_dead, r->ns_dead_cap, r->status, s));
    r->kernel_launches += 1;
  }
  {
    StageScope sc(r, STG_GATHER);
    CUDA_TRY(launch_gather(r->phi, r->phi_alt, (size_t)D * r->elem, N - k, r->ns_order + k, s));
    r->kernel_launches += 1;
  }
  phi4_status ps = refit_factor(r, r->phi_alt, N - k);
  if (ps != PHI4_OK) return ps;
  CUDA_TRY(cudaMemsetAsync(r->acc_count, 0, 4, s));
  {
    StageScope sc(r, STG_NS_SLICE);
    CUDA_TRY(launch_ns_start(r->phi, r->dtype, r->ns_order, N, k, D, c.seed, c.stream_id, it, r->prop, s));
    CUDA_TRY(launch_ns_slice(r->prop, r->dtype, r->w, r->Lg, k, c.L, c.c_kin, c.c_mass * c.m2, c.lambda,
                             ns + NS_LSTAR, steps, c.slice_max_shrink, c.seed, c.stream_id, it, r->acc_count, s));
    CUDA_TRY(launch_ns_replace(r->phi, r->dtype, r->ell, r->ns_order, r->prop, r->w, k, D, s));
    CUDA_TRY(launch_ns_stop(r->ell, N, log(c.ns_stop_frac), ns, s));
    r->kernel_launches += 4;
  }
  r->n_evals += (int64_t)k * (steps + 1);
  double h[8];
  uint32_t st[2];
  CUDA_TRY(cudaMemcpyAsync(h, ns, sizeof(h), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(st, r->status, 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (r->timing) collect_stage_times(r);
  ps = status_to_error(st[0]);
  if (ps != PHI4_OK) return ps;
  r->logX = h[NS_LOGX];
  r->logz_ns = h[NS_LOGZ];
  r->ns_dead_n = (int64_t)h[NS_NDEAD];
  r->slice_capped += st[1];
  if (h[NS_STOP] != 0.0) r->done = true;
  if (done_out) *done_out = r->done ? 1 : 0;
  return PHI4_OK;
}

phi4_status ns_evidence(phi4_run* r, double* logz, double* logz_err) {
  double* ns = r->scal + SC_NS;
  CUDA_TRY(launch_ns_final(r->ns_dead, r->ns_dead_n, r->ell, r->cfg.N, ns, r->stream));
  double h[8];
  CUDA_TRY(cudaMemcpyAsync(h, ns, sizeof(h), cudaMemcpyDeviceToHost, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  if (logz) *logz = h[NS_FZ];
  if (logz_err) *logz_err = sqrt(fmax(h[NS_H], 0.0) / r->cfg.N);
  return PHI4_OK;
}

}  // namespace phi4
