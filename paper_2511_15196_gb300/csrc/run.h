// Run state shared by the drivers in capi.cu (SMC) and ns.cu (nested sampling).
#pragma once
#include <math.h>
#include <vector>
#include "../../include/phi4smc.h"
#include "internal.h"

static const char* const kStageNames[PHI4_N_STAGES] = {"bisect_reweight", "resample", "gather", "covariance",
                                                 "cholesky",        "normals",  "propose", "accept",
                                                 "observables",     "ns_select", "ns_slice", "other",
                                                 "chol_update",     "mutation"};
enum { STG_BISECT, STG_RESAMPLE, STG_GATHER, STG_COV, STG_CHOL, STG_NORMALS, STG_PROPOSE, STG_ACCEPT, STG_OBS,
       STG_NS_SELECT, STG_NS_SLICE, STG_OTHER, STG_CHOL_UPDATE /* kernel-level, inside STG_CHOL */,
       STG_MUTATION /* wall time of the n_mcmc sweeps (their stages overlap on three streams) */ };

namespace phi4 {
struct BatchHost;  // host state of a batch handle (batch.cu)
}

struct phi4_run {
  phi4_config cfg;
  int D = 0, dtype = 0;
  size_t elem = 0;
  cudaStream_t stream = nullptr;
  // device buffers (inside the caller's workspace)
  void *phi = nullptr, *phi_alt = nullptr, *prop = nullptr, *Z = nullptr, *Lg = nullptr;
  int ldz = 0, ldl = 0, zdtype = 0;
  double *S = nullptr, *sq = nullptr, *ell = nullptr, *S_alt = nullptr, *sq_alt = nullptr, *ell_alt = nullptr;
  double *w = nullptr, *M = nullptr, *sigma = nullptr, *chol = nullptr, *scal = nullptr;
  int32_t* anc = nullptr;
  double *irmh_r = nullptr, *irmh_zz = nullptr;  // SMC-IRMH: whitened |L^-1 (phi - mu)|^2, |z|^2
  double* hmc_e = nullptr;                        // SMC-HMC: leapfrog scales eps sqrt(Sigma_ss + ridge)
  uint32_t *status = nullptr, *acc_count = nullptr;
  void *cov_scratch = nullptr, *bisect_scratch = nullptr, *resample_scratch = nullptr;
  size_t cov_scratch_bytes = 0;
  // NS state (device)
  double *ns_dead = nullptr;  // [capacity][2]: (log L, log w)
  int64_t ns_dead_cap = 0, ns_dead_n = 0;
  int32_t *ns_order = nullptr, *ns_start = nullptr;
  // host mirrors
  double beta = 0.0, last_ess = NAN, last_acc = NAN, logz_ns = -INFINITY, logX = 0.0;
  int64_t t = 0, n_evals = 0, slice_capped = 0;
  bool done = false;
  double scale = 0.0;
  // stage timing
  bool timing = false;
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double stage_ms[PHI4_N_STAGES] = {0};
  phi4::LaunchTimer upd_timer;  // the tensor-core trailing-update launches (STG_CHOL_UPDATE)
  // pipelined sweeps of the mixed form: normals and proposal GEMM of sweep t+1 run on
  // their own streams while sweep t's accept runs on `stream`
  void* Z2 = nullptr;                 // second normals buffer (ring slot 1)
  // ring of normals buffers of the pipelined sweeps: slot s % n_zslots holds sweep s's
  // normals (slot 0 is Z, slot 1 is Z2); up to kZRing sweeps are drawn ahead, during the
  // temperature's refit; ev_nz[slot] marks a slot's normals drawn, ev_gz[slot] its GEMM done
  int n_zslots = 0;
  std::vector<cudaEvent_t> ev_nz, ev_gz;
  // accept (the fields' chain, highest priority), GEMM, normals (lowest priority)
  cudaStream_t s_norm = nullptr, s_gemm = nullptr, s_acc = nullptr;
  cudaEvent_t ev_done = nullptr;
  phi4::LaunchTimer acc_timer;  // STG_ACCEPT on s_acc
  cudaEvent_t ev_n[2] = {nullptr, nullptr}, ev_g[2] = {nullptr, nullptr}, ev_a[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;
  phi4::LaunchTimer norm_timer, gemm_timer;  // STG_NORMALS / STG_PROPOSE on those streams
  int64_t kernel_launches = 0;  // kernels this run has launched
  int ridge_level = 0;          // decades above chol_jitter_rel that made the last Cholesky succeed
  void* chol_aux = nullptr;     // diagonal-block inverses of the blocked Cholesky
  cudaStream_t side = nullptr;  // high-priority look-ahead stream of the Cholesky
  cudaEvent_t evA = nullptr, evB = nullptr;
  // batched form: a batch handle owns its member runs (each with its own stream);
  // a member's `owner` points back to the batch
  bool batch = false;
  phi4_run* owner = nullptr;
  std::vector<phi4_run*> members;
  bool owns_stream = false;
  phi4::BatchHost* bh = nullptr;      // batch handle: streams, descriptors, graphs, tuning
  double* batch_scalars = nullptr;    // device [R][12] gathered per-run results
  void** batch_ptrs = nullptr;        // device [R][2]: each member's scal and status
  cudaEvent_t join = nullptr;
  int64_t stage_launches[PHI4_N_STAGES] = {0};
};


namespace phi4 {
struct StageScope {
  phi4_run* r;
  int stage;
  cudaEvent_t a = nullptr, b = nullptr;
  StageScope(phi4_run* run, int st) : r(run), stage(st) {
    if (!r->timing) return;
    a = take();
    b = take();
    cudaEventRecord(a, r->stream);
  }
  ~StageScope() {
    if (!r->timing) return;
    cudaEventRecord(b, r->stream);
    r->pending.push_back({stage, a, b});
  }
  cudaEvent_t take() {
    if (!r->pool.empty()) {
      cudaEvent_t e = r->pool.back();
      r->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

inline void collect_stage_times(phi4_run* r) {
  for (auto& rec : r->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, rec.a, rec.b) == cudaSuccess) {
      r->stage_ms[rec.stage] += ms;
      r->stage_launches[rec.stage] += 1;
    }
    r->pool.push_back(rec.a);
    r->pool.push_back(rec.b);
  }
  r->pending.clear();
  auto take = [&](phi4::LaunchTimer& tm, int stage) {
    const double before = tm.ms;
    const int64_t nb = tm.launches;
    tm.collect();
    r->stage_ms[stage] += tm.ms - before;
    r->stage_launches[stage] += tm.launches - nb;
  };
  take(r->upd_timer, STG_CHOL_UPDATE);
  take(r->norm_timer, STG_NORMALS);
  take(r->gemm_timer, STG_PROPOSE);
  take(r->acc_timer, STG_ACCEPT);
}


ActionParams action_params(const phi4_run* r);
phi4_status read_status(phi4_run* r, uint32_t* st);
phi4_status status_to_error(uint32_t st);
phi4_status refit_factor(phi4_run* r, const void* pts, int n_pts);
phi4_status refit_enqueue(phi4_run* r, const void* pts, int n_pts);
phi4_status factor_attempt(phi4_run* r);
phi4_status refit_check(phi4_run* r, uint32_t st);
phi4_status step_front(phi4_run* r, bool single_cta_bisect);
phi4_status step_back(phi4_run* r);
phi4_status step_finish(phi4_run* r, const double* h, const uint32_t* sw, double* beta_out);
phi4_status ns_replace(phi4_run* r, int32_t* done_out);
phi4_status ns_evidence(phi4_run* r, double* logz, double* logz_err);
void batch_release(phi4_run* b);

}  // namespace phi4

#define CUDA_TRY(expr)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      phi4::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return PHI4_ERR_CUDA;                                                                    \
    }                                                                                          \
  } while (0)

#define ARG_CHECK(cond, ...)        \
  do {                              \
    if (!(cond)) {                  \
      phi4::set_error(__VA_ARGS__); \
      return PHI4_ERR_ARG;          \
    }                               \
  } while (0)
