// C ABI of libphi4smc (include/phi4smc.h): argument checking, workspace layout,
// the SMC temperature pipeline, the nested-sampling iteration and the
// kernel-level entry points. All device memory comes from the caller.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "philox.cuh"
#include "run.h"
#include <cstdlib>

namespace phi4 {

static thread_local char g_err[512] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  return n;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sweeps whose proposal normals are drawn ahead, during the temperature's refit.
constexpr int kZRing = 32;

}  // namespace phi4

using namespace phi4;

namespace {

phi4_status check_config(const phi4_config* c) {
  ARG_CHECK(c != nullptr, "config is NULL");
  ARG_CHECK(c->L >= 1 && c->L <= 128, "L = %d outside [1, 128]", c->L);
  ARG_CHECK(c->N >= 2 && c->N <= 131072, "N = %d outside [2, 131072]", c->N);
  ARG_CHECK(c->kind == PHI4_SMC_RW || c->kind == PHI4_NS_SLICE || c->kind == PHI4_SMC_IRMH ||
                c->kind == PHI4_SMC_HMC,
            "kind = %d unknown", c->kind);
  ARG_CHECK(c->kind != PHI4_SMC_IRMH || (c->precision == PHI4_FP64 && c->L * c->L <= 1024),
            "SMC-IRMH runs in the FP64 form with D <= 1024");
  ARG_CHECK(c->kind != PHI4_SMC_HMC || (c->precision != PHI4_MIXED_BF16 && c->L * c->L <= 4096),
            "SMC-HMC runs in the FP64 or FP32 form with D <= 4096");
  ARG_CHECK(c->precision >= PHI4_FP64 && c->precision <= PHI4_MIXED_BF16, "precision = %d unknown", c->precision);
  ARG_CHECK(isfinite(c->m2) && isfinite(c->lambda) && c->lambda >= 0.0, "m2/lambda invalid");
  ARG_CHECK(isfinite(c->c_kin) && isfinite(c->c_mass) && c->c_kin >= 0.0, "c_kin/c_mass invalid");
  if (c->kind != PHI4_NS_SLICE) {
    ARG_CHECK(c->ess_target > 0.0 && c->ess_target < 1.0, "ess_target = %g outside (0, 1)", c->ess_target);
    ARG_CHECK(c->n_mcmc >= 0 && c->n_mcmc <= 100000, "n_mcmc = %d invalid", c->n_mcmc);
    ARG_CHECK(c->bisect_iters >= 1 && c->bisect_iters <= 200, "bisect_iters = %d invalid", c->bisect_iters);
  } else {
    ARG_CHECK(c->ns_n_delete >= 1 && c->ns_n_delete < c->N, "ns_n_delete = %d outside [1, N)", c->ns_n_delete);
    ARG_CHECK(c->ns_stop_frac > 0.0 && c->ns_stop_frac < 1.0, "ns_stop_frac invalid");
    ARG_CHECK(c->slice_max_shrink >= 1 && c->slice_max_shrink <= 1024, "slice_max_shrink invalid");
    ARG_CHECK(c->N <= 8192, "nested sampling supports N <= 8192 live points (N = %d)", c->N);
  }
  ARG_CHECK(c->chol_jitter_rel >= 0.0 && isfinite(c->chol_jitter_rel), "chol_jitter_rel invalid");
  ARG_CHECK(c->chol_mode >= 0 && c->chol_mode <= 2, "chol_mode = %d unknown", c->chol_mode);
  ARG_CHECK((c->flags & ~(PHI4_FLAG_Z2_FLIP | PHI4_FLAG_FREE_KERNEL_COV)) == 0, "flags 0x%x: unknown bits",
            c->flags);
  ARG_CHECK(!(c->flags & PHI4_FLAG_FREE_KERNEL_COV) ||
                ((c->kind == PHI4_SMC_RW || c->kind == PHI4_SMC_HMC) && c->c_mass * c->m2 > 0.0),
            "the free-field kernel covariance needs an SMC_RW or SMC_HMC run with c_mass * m2 > 0");
  ARG_CHECK(!(c->flags & PHI4_FLAG_Z2_FLIP) || c->kind != PHI4_NS_SLICE, "the Z2 flip move is an SMC move");
  return PHI4_OK;
}

// The run's own streams and events (the caller's stream is not touched).
void release_streams(phi4_run* r) {
  for (cudaStream_t* st : {&r->side, &r->s_norm, &r->s_gemm, &r->s_acc})
    if (*st) {
      cudaStreamSynchronize(*st);
      cudaStreamDestroy(*st);
      *st = nullptr;
    }
  for (cudaEvent_t* ev : {&r->evA, &r->evB, &r->ev_n[0], &r->ev_n[1], &r->ev_g[0], &r->ev_g[1], &r->ev_a[0],
                          &r->ev_a[1], &r->ev_start, &r->ev_done})
    if (*ev) {
      cudaEventDestroy(*ev);
      *ev = nullptr;
    }
  for (auto* v : {&r->ev_nz, &r->ev_gz}) {
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
    v->clear();
  }
}

// Workspace layout; with base == nullptr only the total size is computed.
struct Layout {
  size_t off = 0;
  unsigned char* base = nullptr;
  void* take(size_t bytes) {
    void* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  }
};

// The address `bytes` past `p` inside the workspace (nullptr while only sizing it).
void* base_or_null(const Layout& L, void* p, size_t bytes) {
  return L.base ? (void*)((unsigned char*)p + bytes) : (void*)1;
}

void lay_out(phi4_run* r, Layout& L) {
  const phi4_config& c = r->cfg;
  const int N = c.N, D = c.L * c.L;
  const size_t e = (c.precision == PHI4_FP64) ? 8 : 4;
  r->phi = L.take((size_t)N * D * e);
  r->phi_alt = L.take((size_t)N * D * e);
  r->prop = L.take((size_t)N * D * e);
  if (c.precision == PHI4_MIXED_BF16 && c.kind == PHI4_SMC_RW) {
    r->ldz = (D + 7) & ~7;
    r->ldl = (D + 7) & ~7;
    r->zdtype = PHI4_DT_BF16;
    // pipelined sweeps draw up to kZRing sweeps' normals ahead into a ring of slots
    r->n_zslots = std::max(2, std::min(c.n_mcmc, kZRing));
    r->Z = L.take((size_t)N * r->ldz * 2 * r->n_zslots);
    r->Z2 = base_or_null(L, r->Z, (size_t)N * r->ldz * 2);
    r->Lg = L.take((size_t)D * r->ldl * 2);
  } else {
    r->ldz = D;
    r->ldl = D;
    r->zdtype = (c.precision == PHI4_FP64) ? PHI4_DT_F64 : PHI4_DT_F32;
    r->Z = L.take((size_t)N * D * e);
    r->Lg = L.take((size_t)D * D * e);
  }
  r->S = (double*)L.take(N * 8);
  r->sq = (double*)L.take(N * 8);
  r->ell = (double*)L.take(N * 8);
  r->S_alt = (double*)L.take(N * 8);
  r->sq_alt = (double*)L.take(N * 8);
  r->ell_alt = (double*)L.take(N * 8);
  r->w = (double*)L.take(N * 8);
  r->M = (double*)L.take(N * 8);
  r->anc = (int32_t*)L.take(N * 4);
  r->sigma = (double*)L.take((size_t)D * D * 8);
  r->chol = (double*)L.take((size_t)D * D * 8);
  r->chol_aux = L.take(cholesky_aux_bytes(D));
  r->scal = (double*)L.take(SC_COUNT * 8);
  r->status = (uint32_t*)L.take(16);
  r->acc_count = r->status + 1;
  r->cov_scratch_bytes = std::max(covariance_scratch_bytes(N, D, c.precision), free_covariance_scratch_bytes(c.L));
  r->ns_dead_n = 0;
  r->cov_scratch = L.take(r->cov_scratch_bytes);
  r->bisect_scratch = L.take(bisect_scratch_bytes(N));
  r->resample_scratch = L.take(resample_scratch_bytes(N));
  if (c.kind == PHI4_SMC_HMC) r->hmc_e = (double*)L.take((size_t)D * 8);
  if (c.kind == PHI4_SMC_IRMH) {
    r->irmh_r = (double*)L.take(N * 8);
    r->irmh_zz = (double*)L.take(N * 8);
  }
  if (c.kind == PHI4_NS_SLICE) {
    r->ns_dead_cap = std::min<int64_t>((int64_t)4 * 1024 * 1024, (int64_t)512 * N);
    r->ns_dead = (double*)L.take((size_t)r->ns_dead_cap * 2 * 8);
    r->ns_order = (int32_t*)L.take(N * 4);
    r->ns_start = (int32_t*)L.take(N * 4);
  }
}

}  // namespace

namespace phi4 {
ActionParams action_params(const phi4_run* r) {
  ActionParams p;
  p.L = r->cfg.L;
  p.D = r->D;
  p.N = r->cfg.N;
  p.m2 = r->cfg.m2;
  p.lam = r->cfg.lambda;
  p.c_kin = r->cfg.c_kin;
  p.c_mass = r->cfg.c_mass;
  p.half_d_log2pi = 0.5 * r->D * log(2.0 * M_PI);
  return p;
}

phi4_status read_status(phi4_run* r, uint32_t* st) {
  CUDA_TRY(cudaMemcpyAsync(st, r->status, 4, cudaMemcpyDeviceToHost, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  return PHI4_OK;
}

phi4_status status_to_error(uint32_t st) {
  if (st & ST_TIMEOUT) { set_error("a bounded device wait gave up (status 0x%x)", st); return PHI4_ERR_TIMEOUT; }
  if (st & ST_NONFINITE) { set_error("non-finite action or log-weight (status 0x%x)", st); return PHI4_ERR_NONFINITE; }
  if (st & ST_NOT_PD) { set_error("covariance not positive definite (status 0x%x)", st); return PHI4_ERR_NOT_PD; }
  return PHI4_OK;
}

// Covariance, regularised FP64 Cholesky and the GEMM copy of the factor. The ridge
// starts at chol_jitter_rel * 10^level * trace / D with the level that succeeded at
// the previous outer step, and grows x10 per failed try (up to 6 tries).
// refit_enqueue: covariance, ridge and the first factorisation attempt (no host sync).
// The proposal normals of a temperature's first sweeps do not depend on the fields: the
// pipelined mixed form draws them on its lowest-priority stream at the start of the
// temperature, beside the bisection, resampling, gather and covariance, off the sweeps'
// critical path. (Drawn after the covariance, beside the Cholesky, they slowed the
// factorisation by 0.48 ms per step, against 0.28 ms for the covariance and bisection here.)
// The previous temperature's GEMMs, which read the ring's slots, finished before this
// stream's point.
static phi4_status draw_normals_ahead(phi4_run* r) {
  const phi4_config& c = r->cfg;
  if (!(c.kind == PHI4_SMC_RW && c.precision == PHI4_MIXED_BF16 && c.L % 4 == 0 && r->Z2 && r->s_norm) ||
      r->owner)
    return PHI4_OK;  // batch members draw their normals in the batch's own sweeps
  CUDA_TRY(cudaEventRecord(r->ev_start, r->stream));
  CUDA_TRY(cudaStreamWaitEvent(r->s_norm, r->ev_start, 0));
  const size_t zslot = (size_t)c.N * r->ldz * 2;
  LaunchTimer* tn = r->timing ? &r->norm_timer : nullptr;
  for (int sweep = 0; sweep < std::min(c.n_mcmc, r->n_zslots); ++sweep) {
    cudaEvent_t a0 = tn ? tn->begin(r->s_norm) : nullptr;
    CUDA_TRY(launch_normals(c.seed, c.stream_id, RNG_PROPOSE, (uint32_t)r->t, (uint32_t)sweep, 0, c.N, r->D, r->ldz,
                            r->zdtype, (unsigned char*)r->Z + (size_t)sweep * zslot, r->s_norm));
    if (tn) tn->end(r->s_norm, a0);
    CUDA_TRY(cudaEventRecord(r->ev_nz[sweep], r->s_norm));
    r->kernel_launches += 1;
  }
  return PHI4_OK;
}

phi4_status refit_enqueue(phi4_run* r, const void* pts, int n_pts) {
  const int D = r->D;
  cudaStream_t s = r->stream;
  {
    StageScope sc(r, STG_COV);
    if (r->cfg.flags & PHI4_FLAG_FREE_KERNEL_COV)  // at the new beta, written by the reweighting
      CUDA_TRY(launch_free_covariance(r->cfg.L, r->scal + SC_BETA, r->cfg.c_mass * r->cfg.m2, r->cfg.c_kin,
                                      r->cfg.keep_reference, r->sigma, r->cov_scratch, s));
    else
      CUDA_TRY(launch_covariance(pts, r->cfg.precision, n_pts, D, r->sigma, r->cov_scratch, r->status, s));
    CUDA_TRY(launch_ridge(r->sigma, D, r->cfg.chol_jitter_rel * pow(10.0, r->ridge_level), r->scal + SC_RIDGE, s));
    r->kernel_launches += 4;
  }
  return factor_attempt(r);
}

phi4_status factor_attempt(phi4_run* r) {
  const int D = r->D;
  cudaStream_t s = r->stream;
  const bool f32 = r->cfg.precision == PHI4_FP32;  // the plain float form factors in float
  StageScope sc(r, STG_CHOL);
  if (f32) {
    CUDA_TRY(launch_cholesky_f32(r->sigma, (float*)r->chol, D, r->scal + SC_RIDGE, r->status, r->chol_aux, s,
                                 r->side, r->evA, r->evB));
  } else {
    CUDA_TRY(launch_copy_lower(r->sigma, r->chol, D, s));
    CUDA_TRY(launch_cholesky(r->chol, D, r->scal + SC_RIDGE, r->status, r->chol_aux, s, r->side, r->evA, r->evB,
                             r->cfg.chol_mode, r->timing ? &r->upd_timer : nullptr));
  }
  r->kernel_launches += 1 + cholesky_launches(D);
  return PHI4_OK;
}

// refit_check: with the attempt's status word `st` already read, retry with larger
// ridges until the factorisation succeeds (synchronous), then enqueue the conversion.
phi4_status refit_check(phi4_run* r, uint32_t st) {
  const int D = r->D;
  cudaStream_t s = r->stream;
  for (int tries = 1;; ++tries) {
    if (st & (ST_TIMEOUT | ST_NONFINITE)) return status_to_error(st);
    if (!(st & ST_NOT_PD)) {
      r->ridge_level += tries - 1;  // the next outer step starts from the level that worked
      StageScope sc(r, STG_OTHER);
      if (r->cfg.precision == PHI4_FP32)
        CUDA_TRY(launch_factor_convert_f32((const float*)r->chol, D, (float*)r->Lg, s));
      else
        CUDA_TRY(launch_factor_convert(r->chol, D, r->zdtype, r->Lg, r->ldl, s));
      r->kernel_launches += 1;
      return PHI4_OK;
    }
    if (tries >= 6) break;
    double ridge = 0.0;
    CUDA_TRY(cudaMemcpy(&ridge, r->scal + SC_RIDGE, 8, cudaMemcpyDeviceToHost));
    ridge = ridge > 0.0 ? ridge * 10.0 : 1e-12;
    const uint32_t clear = st & ~ST_NOT_PD;
    CUDA_TRY(cudaMemcpy(r->scal + SC_RIDGE, &ridge, 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(r->status, &clear, 4, cudaMemcpyHostToDevice));
    phi4_status ps = factor_attempt(r);
    if (ps != PHI4_OK) return ps;
    ps = read_status(r, &st);
    if (ps != PHI4_OK) return ps;
  }
  set_error("covariance not positive definite after 6 ridge increases");
  return PHI4_ERR_NOT_PD;
}

phi4_status refit_factor(phi4_run* r, const void* pts, int n_pts) {
  phi4_status ps = refit_enqueue(r, pts, n_pts);
  if (ps != PHI4_OK) return ps;
  uint32_t st = 0;
  ps = read_status(r, &st);
  if (ps != PHI4_OK) return ps;
  return refit_check(r, st);
}

}  // namespace phi4

namespace {
phi4_status propose(phi4_run* r, uint32_t step, uint32_t sweep) {
  const int N = r->cfg.N, D = r->D;
  cudaStream_t s = r->stream;
  {
    StageScope sc(r, STG_NORMALS);
    CUDA_TRY(launch_normals(r->cfg.seed, r->cfg.stream_id, RNG_PROPOSE, step, sweep, 0, N, D, r->ldz, r->zdtype,
                            r->Z, s));
  }
  r->kernel_launches += 2;
  StageScope sc(r, STG_PROPOSE);
  if (r->cfg.precision == PHI4_MIXED_BF16)  // fp16 increment into the proposal buffer
    CUDA_TRY(launch_propose_tc(r->prop, r->Z, r->ldz, r->Lg, r->ldl, N, D, (float)r->scale, r->status, s));
  else
    CUDA_TRY(launch_propose_simt(r->phi, r->prop, r->Z, r->Lg, r->dtype, N, D, r->scale, s));
  return PHI4_OK;
}

}  // namespace

namespace phi4 {

// Front of a temperature: bisection + reweighting, resampling, gather, covariance and
// the first factorisation attempt, all enqueued on the run's stream.
phi4_status step_front(phi4_run* r, bool single_cta_bisect) {
  const phi4_config& c = r->cfg;
  const int N = c.N, D = r->D;
  cudaStream_t s = r->stream;
  const uint32_t t = (uint32_t)(++r->t);
  double* out = r->scal + SC_OUT;
  phi4_status pn = draw_normals_ahead(r);
  if (pn != PHI4_OK) return pn;
  {
    StageScope sc(r, STG_BISECT);
    CUDA_TRY(launch_bisect(r->ell, N, r->scal + SC_BETA, c.ess_target, c.bisect_iters, r->w, out, r->bisect_scratch,
                           r->status, s, single_cta_bisect));
    CUDA_TRY(launch_logz_accumulate(out, r->scal + SC_KAHAN, r->scal + SC_BETA, s));
    r->kernel_launches += 2;
  }
  {
    StageScope sc(r, STG_RESAMPLE);
    const uint4 wd = philox4x32_10_host(make_uint4(counter_word0(RNG_RESAMPLE, t), 0u, 0u, 0u),
                                        philox_key(c.seed, c.stream_id));
    CUDA_TRY(launch_resample(r->w, N, wd.x, nullptr, r->anc, r->resample_scratch, s));
    r->kernel_launches += 1;
  }
  {
    StageScope sc(r, STG_GATHER);
    CUDA_TRY(launch_gather(r->phi, r->phi_alt, (size_t)D * r->elem, N, r->anc, s));
    CUDA_TRY(launch_gather3_f64(r->S, r->S_alt, r->sq, r->sq_alt, r->ell, r->ell_alt, N, r->anc, s));
    r->kernel_launches += 2;
    std::swap(r->phi, r->phi_alt);
    std::swap(r->S, r->S_alt);
    std::swap(r->sq, r->sq_alt);
    std::swap(r->ell, r->ell_alt);
  }
  return refit_enqueue(r, r->phi, N);
}

// The n_mcmc random-walk sweeps of a temperature (normals, proposal, accept).
// In the mixed form on L % 4 == 0 lattices the increment Delta = s Z L^T does not
// depend on the fields, so sweep t+1's normals (stream s_norm, ALU-bound, lowest
// priority) and proposal GEMM (stream s_gemm, tensor cores) run while sweep t's
// accept (stream s_acc, HBM-bound, highest priority: it carries the fields' chain)
// runs: Z and Delta are double-buffered (Delta in the two halves of the proposal
// buffer) and events order each buffer's writer after its last reader. The
// arithmetic of every sweep is unchanged.
static phi4_status step_sweeps(phi4_run* r) {
  const phi4_config& c = r->cfg;
  const int N = c.N, D = r->D;
  cudaStream_t s = r->stream;
  const uint32_t t = (uint32_t)r->t;
  CUDA_TRY(cudaMemsetAsync(r->acc_count, 0, 4, s));
  const ActionParams ap = action_params(r);
  StageScope wall(r, STG_MUTATION);
  if (c.precision == PHI4_MIXED_BF16 && c.L % 4 == 0 && r->Z2) {
    const int R = r->n_zslots;
    const size_t zslot = (size_t)N * r->ldz * 2;
    auto Zs = [&](int sweep) { return (void*)((unsigned char*)r->Z + (size_t)(sweep % R) * zslot); };
    void* Db[2] = {r->prop, (unsigned char*)r->prop + (size_t)N * D * 2};
    CUDA_TRY(cudaEventRecord(r->ev_start, s));  // the factor and the fields are ready
    CUDA_TRY(cudaStreamWaitEvent(r->s_gemm, r->ev_start, 0));
    CUDA_TRY(cudaStreamWaitEvent(r->s_acc, r->ev_start, 0));
    cudaStream_t sa = r->s_acc;
    LaunchTimer* tn = r->timing ? &r->norm_timer : nullptr;
    LaunchTimer* tg = r->timing ? &r->gemm_timer : nullptr;
    LaunchTimer* ta = r->timing ? &r->acc_timer : nullptr;
    cudaStream_t sn = r->s_norm;
    for (int sweep = 0; sweep < c.n_mcmc; ++sweep) {
      const int q = sweep & 1, slot = sweep % R;
      if (sweep >= R) {
        // normals of this sweep into its slot once the GEMM of sweep - R has read it (the
        // first R sweeps' normals were drawn during the refit, step_front)
        CUDA_TRY(cudaStreamWaitEvent(sn, r->ev_gz[slot], 0));
        cudaEvent_t a0 = tn ? tn->begin(sn) : nullptr;
        CUDA_TRY(launch_normals(c.seed, c.stream_id, RNG_PROPOSE, t, (uint32_t)sweep, 0, N, D, r->ldz, r->zdtype,
                                Zs(sweep), sn));
        if (tn) tn->end(sn, a0);
        CUDA_TRY(cudaEventRecord(r->ev_nz[slot], sn));
        r->kernel_launches += 1;
      }
      // Delta[q] = s Z[slot] L^T once the normals are there and the accept of sweep-2 read Delta[q]
      CUDA_TRY(cudaStreamWaitEvent(r->s_gemm, r->ev_nz[slot], 0));
      if (sweep >= 2) CUDA_TRY(cudaStreamWaitEvent(r->s_gemm, r->ev_a[q], 0));
      cudaEvent_t a1 = tg ? tg->begin(r->s_gemm) : nullptr;
      CUDA_TRY(launch_propose_tc(Db[q], Zs(sweep), r->ldz, r->Lg, r->ldl, N, D, (float)r->scale, r->status,
                                 r->s_gemm));
      if (tg) tg->end(r->s_gemm, a1);
      CUDA_TRY(cudaEventRecord(r->ev_g[q], r->s_gemm));
      CUDA_TRY(cudaEventRecord(r->ev_gz[slot], r->s_gemm));
      // the accept chain
      CUDA_TRY(cudaStreamWaitEvent(sa, r->ev_g[q], 0));
      cudaEvent_t a2 = ta ? ta->begin(sa) : nullptr;
      CUDA_TRY(launch_accept_delta((float*)r->phi, Db[q], ap, c.keep_reference, r->S, r->sq, r->ell,
                                   r->scal + SC_BETA, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count,
                                   r->status, sa));
      if (ta) ta->end(sa, a2);
      CUDA_TRY(cudaEventRecord(r->ev_a[q], sa));
      r->kernel_launches += 2;
    }
    CUDA_TRY(cudaEventRecord(r->ev_done, sa));  // the last accept follows every GEMM and normals draw
    CUDA_TRY(cudaStreamWaitEvent(s, r->ev_done, 0));
    r->n_evals += (int64_t)N * c.n_mcmc;
    return PHI4_OK;
  }
  if (c.kind == PHI4_SMC_HMC) {
    // HMC transitions with the refit's covariance diagonal (plus the ridge) as inverse mass
    const double eps = c.rw_scale > 0.0 ? c.rw_scale : 0.8 * pow((double)D, -0.25);
    {
      StageScope sc(r, STG_OTHER);
      CUDA_TRY(launch_hmc_scale(r->sigma, D, r->scal + SC_RIDGE, eps, r->hmc_e, s));
      r->kernel_launches += 1;
    }
    for (int sweep = 0; sweep < c.n_mcmc; ++sweep) {
      {
        StageScope sc(r, STG_NORMALS);
        CUDA_TRY(launch_normals(c.seed, c.stream_id, RNG_PROPOSE, t, (uint32_t)sweep, 0, N, D, D, r->zdtype, r->Z,
                                s));
      }
      StageScope sc(r, STG_ACCEPT);
      CUDA_TRY(launch_hmc(r->phi, r->Z, r->zdtype, r->hmc_e, ap, c.keep_reference, r->S, r->sq, r->ell,
                          r->scal + SC_BETA, kHmcLeapfrog, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count,
                          r->status, s));
      r->kernel_launches += 2;
    }
    r->n_evals += (int64_t)N * c.n_mcmc * (kHmcLeapfrog + 1);
    return PHI4_OK;
  }
  if (c.kind == PHI4_SMC_IRMH) {
    // independent proposals mu + L z of the refit's mean (the covariance scratch's first
    // D doubles) and factor; the Hastings factor from the whitened norms
    const double* mu = (const double*)r->cov_scratch;
    {
      StageScope sc(r, STG_OTHER);
      CUDA_TRY(launch_whitened_sq_norm((const double*)r->phi, mu, (const double*)r->Lg, r->ldl, N, D, r->irmh_r, s));
      r->kernel_launches += 1;
    }
    for (int sweep = 0; sweep < c.n_mcmc; ++sweep) {
      {
        StageScope sc(r, STG_NORMALS);
        CUDA_TRY(launch_normals(c.seed, c.stream_id, RNG_PROPOSE, t, (uint32_t)sweep, 0, N, D, D, PHI4_DT_F64, r->Z,
                                s));
      }
      {
        StageScope sc(r, STG_PROPOSE);
        CUDA_TRY(launch_propose_simt(mu, r->prop, r->Z, r->Lg, PHI4_DT_F64, N, D, 1.0, s, 0));
        CUDA_TRY(launch_row_sq_norm((const double*)r->Z, N, D, r->irmh_zz, s));
      }
      StageScope sc(r, STG_ACCEPT);
      CUDA_TRY(launch_accept(r->phi, r->prop, PHI4_DT_F64, ap, c.keep_reference, r->S, r->sq, r->ell,
                             r->scal + SC_BETA, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count, r->status, s,
                             r->irmh_zz, r->irmh_r));
      r->kernel_launches += 4;
    }
    r->n_evals += (int64_t)N * c.n_mcmc;
    return PHI4_OK;
  }
  for (int sweep = 0; sweep < c.n_mcmc; ++sweep) {
    phi4_status ps = propose(r, t, (uint32_t)sweep);
    if (ps != PHI4_OK) return ps;
    StageScope sc(r, STG_ACCEPT);
    if (c.precision == PHI4_MIXED_BF16) {
      if (c.L % 4 == 0) {
        CUDA_TRY(launch_accept_delta((float*)r->phi, r->prop, ap, c.keep_reference, r->S, r->sq, r->ell,
                                     r->scal + SC_BETA, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count,
                                     r->status, s));
      } else {  // generic lattices: materialise phi + delta next to it, then the generic accept
        float* prop = (float*)r->phi_alt;
        CUDA_TRY(launch_apply_delta((const float*)r->phi, r->prop, prop, (long long)N * D, s));
        CUDA_TRY(launch_accept(r->phi, prop, r->dtype, ap, c.keep_reference, r->S, r->sq, r->ell,
                               r->scal + SC_BETA, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count, r->status,
                               s));
        r->kernel_launches += 1;
      }
    } else {
      CUDA_TRY(launch_accept(r->phi, r->prop, r->dtype, ap, c.keep_reference, r->S, r->sq, r->ell,
                             r->scal + SC_BETA, c.seed, c.stream_id, t, (uint32_t)sweep, r->acc_count, r->status,
                             s));
    }
    r->kernel_launches += 1;
  }
  r->n_evals += (int64_t)N * c.n_mcmc;
  return PHI4_OK;
}

// Back of a temperature: the sweeps, then (PHI4_FLAG_Z2_FLIP) the global Z2 move.
phi4_status step_back(phi4_run* r) {
  phi4_status ps = step_sweeps(r);
  if (ps != PHI4_OK) return ps;
  if (r->cfg.flags & PHI4_FLAG_Z2_FLIP) {
    const int dt = r->cfg.precision == PHI4_FP64 ? PHI4_DT_F64 : PHI4_DT_F32;
    CUDA_TRY(launch_z2_flip(r->cfg.seed, r->cfg.stream_id, (uint32_t)r->t, r->phi, dt, r->cfg.N, r->D, r->stream));
    r->kernel_launches += 1;
  }
  return PHI4_OK;
}

// After the stream has drained: bisection results h[0..7] and status words sw[0..1].
phi4_status step_finish(phi4_run* r, const double* h, const uint32_t* sw, double* beta_out) {
  if (r->timing) collect_stage_times(r);
  phi4_status ps = status_to_error(sw[0]);
  if (ps != PHI4_OK) return ps;
  r->beta = h[1];
  r->last_ess = h[2];
  r->last_acc = r->cfg.n_mcmc > 0 ? (double)sw[1] / ((double)r->cfg.N * r->cfg.n_mcmc) : NAN;
  if (r->beta >= 1.0) r->done = true;
  if (beta_out) *beta_out = r->beta;
  return PHI4_OK;
}

}  // namespace phi4

extern "C" {

const char* phi4_last_error(void) { return g_err; }

phi4_status phi4_device_sm_count(int32_t* out) {
  ARG_CHECK(out, "out is NULL");
  *out = sm_count();
  return PHI4_OK;
}

const char* phi4_stage_name(int32_t stage) {
  return (stage >= 0 && stage < PHI4_N_STAGES) ? kStageNames[stage] : "unknown";
}

phi4_status phi4_workspace_bytes(const phi4_config* cfg, size_t* bytes) {
  phi4_status st = check_config(cfg);
  if (st != PHI4_OK) return st;
  ARG_CHECK(bytes, "bytes is NULL");
  phi4_run tmp;
  tmp.cfg = *cfg;
  Layout L;
  lay_out(&tmp, L);
  *bytes = L.off;
  return PHI4_OK;
}

phi4_status smc_init(const phi4_config* cfg, void* d_workspace, size_t workspace_bytes, void* stream,
                     phi4_run** out) {
  phi4_status st = check_config(cfg);
  if (st != PHI4_OK) return st;
  ARG_CHECK(out, "out is NULL");
  ARG_CHECK(d_workspace && ((uintptr_t)d_workspace & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  size_t need = 0;
  phi4_workspace_bytes(cfg, &need);
  if (workspace_bytes < need) {
    set_error("workspace of %zu bytes, need %zu", workspace_bytes, need);
    return PHI4_ERR_WORKSPACE;
  }
  if (cfg->precision == PHI4_MIXED_BF16 && !tc_available()) {
    set_error("tensor-map encoder unavailable from the CUDA driver");
    return PHI4_ERR_UNSUPPORTED;
  }
  phi4_run* r = new phi4_run();
  r->cfg = *cfg;
  r->D = cfg->L * cfg->L;
  r->dtype = cfg->precision == PHI4_FP64 ? PHI4_DT_F64 : PHI4_DT_F32;
  r->elem = cfg->precision == PHI4_FP64 ? 8 : 4;
  r->stream = (cudaStream_t)stream;
  r->scale = cfg->rw_scale > 0.0 ? cfg->rw_scale : 2.38 / sqrt((double)r->D);
  Layout L;
  L.base = (unsigned char*)d_workspace;
  lay_out(r, L);
  cudaStream_t s = r->stream;
  auto fail = [&](cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    release_streams(r);
    delete r;
    return PHI4_ERR_CUDA;
  };
  cudaError_t e;
  int lo_prio = 0, hi_prio = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio)) != cudaSuccess) return fail(e, "priority range");
  if ((e = cudaStreamCreateWithPriority(&r->side, cudaStreamNonBlocking, hi_prio)) != cudaSuccess)
    return fail(e, "look-ahead stream");
  if ((e = cudaEventCreateWithFlags(&r->evA, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  if ((e = cudaEventCreateWithFlags(&r->evB, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
  if (r->Z2) {
    // block scheduling favours the accept chain, then the GEMM, then the normals
    const int mid_prio = (lo_prio + hi_prio) / 2;
    if ((e = cudaStreamCreateWithPriority(&r->s_norm, cudaStreamNonBlocking, lo_prio)) != cudaSuccess)
      return fail(e, "stream");
    if ((e = cudaStreamCreateWithPriority(&r->s_gemm, cudaStreamNonBlocking, mid_prio)) != cudaSuccess)
      return fail(e, "stream");
    if ((e = cudaStreamCreateWithPriority(&r->s_acc, cudaStreamNonBlocking, hi_prio)) != cudaSuccess)
      return fail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&r->ev_done, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    for (int q = 0; q < 2; ++q) {
      if ((e = cudaEventCreateWithFlags(&r->ev_n[q], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
      if ((e = cudaEventCreateWithFlags(&r->ev_g[q], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
      if ((e = cudaEventCreateWithFlags(&r->ev_a[q], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    }
    if ((e = cudaEventCreateWithFlags(&r->ev_start, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    r->ev_nz.assign(r->n_zslots, nullptr);
    r->ev_gz.assign(r->n_zslots, nullptr);
    for (int q = 0; q < r->n_zslots; ++q) {
      if ((e = cudaEventCreateWithFlags(&r->ev_nz[q], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
      if ((e = cudaEventCreateWithFlags(&r->ev_gz[q], cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    }
  }
  if ((e = cudaMemsetAsync(r->scal, 0, SC_COUNT * 8, s)) != cudaSuccess) return fail(e, "memset");
  if ((e = cudaMemsetAsync(r->status, 0, 16, s)) != cudaSuccess) return fail(e, "memset");
  if ((e = launch_normals(cfg->seed, cfg->stream_id, RNG_INIT, 0, 0, 0, cfg->N, r->D, r->D, r->dtype, r->phi, s)) !=
      cudaSuccess)
    return fail(e, "initial draw");
  const ActionParams ap = action_params(r);
  if ((e = launch_action(r->phi, r->dtype, ap, r->S, r->sq, r->ell, cfg->keep_reference, s)) != cudaSuccess)
    return fail(e, "initial action");
  r->n_evals = cfg->N;
  if (cfg->kind == PHI4_NS_SLICE) {
    const double init_ns[4] = {0.0, -INFINITY, -INFINITY, 0.0};
    if ((e = cudaMemcpyAsync(r->scal + SC_NS, init_ns, sizeof(init_ns), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return fail(e, "NS init");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "NS init");
  }
  *out = r;
  return PHI4_OK;
}

phi4_status smc_temper_step(phi4_run* r, double* beta_out) {
  ARG_CHECK(r, "run is NULL");
  ARG_CHECK(r->cfg.kind != PHI4_NS_SLICE, "smc_temper_step on a nested-sampling run");
  ARG_CHECK(!r->batch, "smc_temper_step on a batch handle (use smc_temper_step_batch)");
  if (r->done) {
    set_error("beta already 1");
    return PHI4_ERR_DONE;
  }
  phi4_status ps = step_front(r, false);
  if (ps != PHI4_OK) return ps;
  uint32_t st = 0;
  if ((ps = read_status(r, &st)) != PHI4_OK) return ps;
  if ((ps = refit_check(r, st)) != PHI4_OK) return ps;
  if ((ps = step_back(r)) != PHI4_OK) return ps;
  double h[8];
  uint32_t sw[2];
  CUDA_TRY(cudaMemcpyAsync(h, r->scal + SC_OUT, 8 * sizeof(double), cudaMemcpyDeviceToHost, r->stream));
  CUDA_TRY(cudaMemcpyAsync(sw, r->status, 8, cudaMemcpyDeviceToHost, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  return step_finish(r, h, sw, beta_out);
}

phi4_status ns_replace_step(phi4_run* r, int32_t* done_out) {
  ARG_CHECK(r, "run is NULL");
  ARG_CHECK(!r->batch, "ns_replace_step on a batch handle");
  ARG_CHECK(r->cfg.kind == PHI4_NS_SLICE, "ns_replace_step on an SMC run");
  if (r->done) {
    set_error("nested sampling already stopped");
    return PHI4_ERR_DONE;
  }
  return ns_replace(r, done_out);
}

phi4_status smc_log_evidence(const phi4_run* rc, double* logz, double* logz_err) {
  ARG_CHECK(rc, "run is NULL");
  phi4_run* r = const_cast<phi4_run*>(rc);
  if (r->cfg.kind != PHI4_NS_SLICE) {
    double k[2];
    CUDA_TRY(cudaMemcpyAsync(k, r->scal + SC_KAHAN, 16, cudaMemcpyDeviceToHost, r->stream));
    CUDA_TRY(cudaStreamSynchronize(r->stream));
    if (logz) *logz = k[0];
    if (logz_err) *logz_err = NAN;
    return PHI4_OK;
  }
  return ns_evidence(r, logz, logz_err);
}

phi4_status smc_observables(const phi4_run* rc, phi4_obs* o) {
  ARG_CHECK(rc && o, "NULL argument");
  phi4_run* r = const_cast<phi4_run*>(rc);
  const int N = r->cfg.N;
  {
    StageScope sc(r, STG_OBS);
    CUDA_TRY(launch_observables(r->phi, r->dtype, N, r->D, nullptr, r->M, r->scal + SC_OBS, r->stream));
    r->kernel_launches += 2;
  }
  double h[6];
  CUDA_TRY(cudaMemcpyAsync(h, r->scal + SC_OBS, sizeof(h), cudaMemcpyDeviceToHost, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  if (r->timing) collect_stage_times(r);
  memset(o, 0, sizeof(*o));
  o->beta = r->beta;
  double lz = NAN, le = NAN;
  phi4_status ps = smc_log_evidence(r, &lz, &le);
  if (ps != PHI4_OK) return ps;
  o->logz = lz;
  o->logz_err = le;
  o->mean_M = h[0];
  o->mean_absM = h[1];
  o->mean_M2 = h[2];
  o->chi = h[3];
  o->mode_balance = h[4];
  o->ess = r->last_ess;
  o->acc_rate = r->last_acc;
  o->n_steps = r->t;
  o->n_likelihood_evals = r->n_evals;
  o->slice_capped = r->slice_capped;
  return PHI4_OK;
}

phi4_status smc_copy_particles(const phi4_run* rc, void* dst, size_t bytes) {
  ARG_CHECK(rc && dst, "NULL argument");
  phi4_run* r = const_cast<phi4_run*>(rc);
  const size_t need = (size_t)r->cfg.N * r->D * r->elem;
  ARG_CHECK(bytes >= need, "destination of %zu bytes, need %zu", bytes, need);
  CUDA_TRY(cudaMemcpyAsync(dst, r->phi, need, cudaMemcpyDefault, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  return PHI4_OK;
}

phi4_status smc_load_particles(phi4_run* r, const void* src, size_t bytes) {
  ARG_CHECK(r && src, "NULL argument");
  const size_t need = (size_t)r->cfg.N * r->D * r->elem;
  ARG_CHECK(bytes >= need, "source of %zu bytes, need %zu", bytes, need);
  CUDA_TRY(cudaMemcpyAsync(r->phi, src, need, cudaMemcpyDefault, r->stream));
  const ActionParams ap = action_params(r);
  CUDA_TRY(launch_action(r->phi, r->dtype, ap, r->S, r->sq, r->ell, r->cfg.keep_reference, r->stream));
  return PHI4_OK;
}

/* ---------------------------- checkpoint / resume ---------------------------- */

namespace {
constexpr uint64_t kStateMagic = 0x3154415453344950ull;  // "PHI4STAT1" (first 8 bytes)

// Host part of a run's state: everything besides the device arrays that feeds later steps.
struct StateHeader {
  uint64_t magic;
  uint64_t bytes;            // whole state, header included
  phi4_config cfg;
  int64_t t, n_evals, slice_capped, ns_dead_n;
  int32_t ridge_level, done;
  double beta, last_ess, last_acc, logz_ns, logX;
};

// Device arrays of the state, in order: the fields, S, |phi|^2, ell, the scalar block,
// and for nested sampling the dead points' (log L, log w) pairs.
struct StatePart { void* dev; size_t bytes; };
std::vector<StatePart> state_parts(const phi4_run* r) {
  const size_t N = (size_t)r->cfg.N;
  std::vector<StatePart> v = {{r->phi, N * r->D * r->elem}, {r->S, N * 8}, {r->sq, N * 8}, {r->ell, N * 8},
                              {r->scal, SC_COUNT * 8}};
  if (r->cfg.kind == PHI4_NS_SLICE) v.push_back({r->ns_dead, (size_t)r->ns_dead_n * 2 * 8});
  return v;
}
bool same_config(const phi4_config& a, const phi4_config& b) {
  return a.L == b.L && a.N == b.N && a.kind == b.kind && a.precision == b.precision && a.m2 == b.m2 &&
         a.lambda == b.lambda && a.c_kin == b.c_kin && a.c_mass == b.c_mass && a.keep_reference == b.keep_reference &&
         a.n_mcmc == b.n_mcmc && a.ess_target == b.ess_target && a.rw_scale == b.rw_scale &&
         a.ns_n_delete == b.ns_n_delete && a.ns_slice_steps == b.ns_slice_steps && a.ns_stop_frac == b.ns_stop_frac &&
         a.chol_jitter_rel == b.chol_jitter_rel && a.bisect_iters == b.bisect_iters &&
         a.slice_max_shrink == b.slice_max_shrink && a.seed == b.seed && a.stream_id == b.stream_id &&
         a.chol_mode == b.chol_mode && a.flags == b.flags;
}
size_t state_total(const phi4_run* r) {
  size_t b = sizeof(StateHeader);
  for (const StatePart& q : state_parts(r)) b += q.bytes;
  return b;
}
}  // namespace

phi4_status phi4_state_bytes(const phi4_run* r, size_t* bytes) {
  ARG_CHECK(r && bytes, "NULL argument");
  ARG_CHECK(!r->batch, "a batch handle has no single state (save its members)");
  *bytes = state_total(r);
  return PHI4_OK;
}

phi4_status smc_save_state(const phi4_run* rc, void* host_dst, size_t bytes) {
  ARG_CHECK(rc && host_dst, "NULL argument");
  ARG_CHECK(!rc->batch, "a batch handle has no single state (save its members)");
  phi4_run* r = const_cast<phi4_run*>(rc);
  const size_t need = state_total(r);
  ARG_CHECK(bytes >= need, "state buffer of %zu bytes, need %zu", bytes, need);
  StateHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.bytes = need;
  h.cfg = r->cfg;
  h.t = r->t;
  h.n_evals = r->n_evals;
  h.slice_capped = r->slice_capped;
  h.ns_dead_n = r->ns_dead_n;
  h.ridge_level = r->ridge_level;
  h.done = r->done ? 1 : 0;
  h.beta = r->beta;
  h.last_ess = r->last_ess;
  h.last_acc = r->last_acc;
  h.logz_ns = r->logz_ns;
  h.logX = r->logX;
  unsigned char* dst = (unsigned char*)host_dst;
  memcpy(dst, &h, sizeof(h));
  size_t off = sizeof(h);
  for (const StatePart& q : state_parts(r)) {
    if (q.bytes) CUDA_TRY(cudaMemcpyAsync(dst + off, q.dev, q.bytes, cudaMemcpyDeviceToHost, r->stream));
    off += q.bytes;
  }
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  return PHI4_OK;
}

phi4_status smc_restore_state(phi4_run* r, const void* host_src, size_t bytes) {
  ARG_CHECK(r && host_src, "NULL argument");
  ARG_CHECK(!r->batch, "a batch handle has no single state");
  ARG_CHECK(!r->owner, "a batch member's buffers follow the batch's steps: it cannot be restored");
  ARG_CHECK(bytes >= sizeof(StateHeader), "state buffer of %zu bytes is too small", bytes);
  StateHeader h;
  memcpy(&h, host_src, sizeof(h));
  ARG_CHECK(h.magic == kStateMagic, "not a phi4smc state (bad magic)");
  ARG_CHECK(h.bytes <= bytes, "state of %llu bytes truncated to %zu", (unsigned long long)h.bytes, bytes);
  ARG_CHECK(same_config(h.cfg, r->cfg),
            "the state was saved from a run with another configuration");
  ARG_CHECK(h.ns_dead_n >= 0 && h.ns_dead_n <= r->ns_dead_cap, "dead-point count %lld out of range",
            (long long)h.ns_dead_n);
  r->ns_dead_n = h.ns_dead_n;  // sizes the NS dead list part
  ARG_CHECK(state_total(r) == h.bytes, "state size %llu does not match this run's %zu",
            (unsigned long long)h.bytes, state_total(r));
  const unsigned char* src = (const unsigned char*)host_src;
  size_t off = sizeof(h);
  for (const StatePart& q : state_parts(r)) {
    if (q.bytes) CUDA_TRY(cudaMemcpyAsync(q.dev, src + off, q.bytes, cudaMemcpyHostToDevice, r->stream));
    off += q.bytes;
  }
  CUDA_TRY(cudaMemsetAsync(r->status, 0, 16, r->stream));
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  r->t = h.t;
  r->n_evals = h.n_evals;
  r->slice_capped = h.slice_capped;
  r->ridge_level = h.ridge_level;
  r->done = h.done != 0;
  r->beta = h.beta;
  r->last_ess = h.last_ess;
  r->last_acc = h.last_acc;
  r->logz_ns = h.logz_ns;
  r->logX = h.logX;
  return PHI4_OK;
}

phi4_status smc_free(phi4_run* r) {
  if (!r) return PHI4_OK;
  ARG_CHECK(!r->owner, "this run belongs to a batch: free the batch handle");
  if (r->batch) {
    batch_release(r);
    for (phi4_run* m : r->members) {
      m->owner = nullptr;
      cudaStream_t ms = m->stream;
      if (m->join) cudaEventDestroy(m->join);
      smc_free(m);
      if (ms) cudaStreamDestroy(ms);
    }
    if (r->join) cudaEventDestroy(r->join);
    delete r;
    return PHI4_OK;
  }
  cudaStreamSynchronize(r->stream);
  for (auto& rec : r->pending) {
    cudaEventDestroy(rec.a);
    cudaEventDestroy(rec.b);
  }
  for (auto e : r->pool) cudaEventDestroy(e);
  r->upd_timer.release();
  r->norm_timer.release();
  r->gemm_timer.release();
  r->acc_timer.release();
  release_streams(r);
  delete r;
  return PHI4_OK;
}

phi4_status phi4_set_spin_limit(int64_t cycles) {
  const long long c = cycles > 0 ? (long long)cycles : kSpinLimitCyclesDefault;
  CUDA_TRY(set_spin_limit_temper(c));
  CUDA_TRY(set_spin_limit_chol(c));
  return PHI4_OK;
}

phi4_status phi4_kernel_launches(const phi4_run* r, int64_t* out) {
  ARG_CHECK(r && out, "NULL argument");
  *out = r->kernel_launches;
  return PHI4_OK;
}

phi4_status phi4_set_stage_timing(phi4_run* r, int32_t enable) {
  ARG_CHECK(r, "run is NULL");
  r->timing = enable != 0;
  return PHI4_OK;
}

phi4_status phi4_stage_times(phi4_run* r, double* ms_out, int64_t* launches_out, int32_t reset) {
  ARG_CHECK(r, "run is NULL");
  CUDA_TRY(cudaStreamSynchronize(r->stream));
  collect_stage_times(r);
  for (int i = 0; i < PHI4_N_STAGES; ++i) {
    if (ms_out) ms_out[i] = r->stage_ms[i];
    if (launches_out) launches_out[i] = r->stage_launches[i];
    if (reset) {
      r->stage_ms[i] = 0;
      r->stage_launches[i] = 0;
    }
  }
  return PHI4_OK;
}

/* -------------------------- kernel-level API -------------------------- */

size_t phi4_free_covariance_scratch_bytes(int32_t L) {
  return (L >= 1 && L <= 128) ? free_covariance_scratch_bytes(L) : 0;
}

phi4_status phi4_free_field_covariance(int32_t L, const double* d_beta, double m2, double c_kin, double c_mass,
                                       int32_t keep_reference, double* sigma, void* scratch, size_t scratch_bytes,
                                       void* stream) {
  ARG_CHECK(d_beta && sigma && scratch, "NULL argument");
  ARG_CHECK(L >= 1 && L <= 128, "L = %d outside [1, 128]", L);
  ARG_CHECK(c_mass * m2 > 0.0 && c_kin >= 0.0, "needs c_mass * m2 > 0 and c_kin >= 0");
  ARG_CHECK(scratch_bytes >= free_covariance_scratch_bytes(L), "scratch of %zu bytes, need %zu", scratch_bytes,
            free_covariance_scratch_bytes(L));
  CUDA_TRY(launch_free_covariance(L, d_beta, c_mass * m2, c_kin, keep_reference, sigma, scratch,
                                  (cudaStream_t)stream));
  return PHI4_OK;
}

phi4_status phi4_observables(const void* phi, int32_t dtype, int32_t N, int32_t L, const double* w, double* M,
                             double* out, void* stream) {
  ARG_CHECK(phi && M && out, "NULL argument");
  ARG_CHECK(dtype == PHI4_DT_F64 || dtype == PHI4_DT_F32, "dtype %d: fields are F64 or F32", dtype);
  ARG_CHECK(N >= 1 && L >= 1 && (int64_t)L * L <= (1 << 20), "bad sizes N = %d, L = %d", N, L);
  CUDA_TRY(launch_observables(phi, dtype, N, L * L, w, M, out, (cudaStream_t)stream));
  return PHI4_OK;
}

phi4_status phi4_philox_normals(uint64_t seed, uint64_t stream_id, int32_t kind, uint32_t step, uint32_t sub,
                                int32_t row0, int32_t n_rows, int32_t n_cols, int32_t ld, int32_t dtype, void* out,
                                void* stream) {
  ARG_CHECK(out, "out is NULL");
  ARG_CHECK(n_rows >= 0 && n_cols >= 0 && ld >= n_cols && row0 >= 0, "bad sizes");
  ARG_CHECK(dtype >= 0 && dtype <= 2, "dtype %d unknown", dtype);
  ARG_CHECK(kind >= 0 && kind < 256, "kind %d outside [0, 256)", kind);
  CUDA_TRY(launch_normals(seed, stream_id, (uint32_t)kind, step, sub, row0, n_rows, n_cols, ld, dtype, out,
                          (cudaStream_t)stream));
  return PHI4_OK;
}

phi4_status phi4_action(const void* phi, int32_t dtype, int32_t N, int32_t L, double m2, double lambda,
                        double c_kin, double c_mass, double* S, double* sq, void* stream) {
  ARG_CHECK(phi && S && sq, "NULL argument");
  ARG_CHECK(N >= 0 && L >= 1 && L <= 128, "bad sizes");
  ARG_CHECK(dtype == PHI4_DT_F64 || dtype == PHI4_DT_F32, "dtype must be F64 or F32");
  ActionParams p{L, L * L, N, m2, lambda, c_kin, c_mass, 0.5 * L * L * log(2.0 * M_PI)};
  CUDA_TRY(launch_action(phi, dtype, p, S, sq, nullptr, 0, (cudaStream_t)stream));
  return PHI4_OK;
}

size_t phi4_bisect_scratch_bytes(int32_t N) { return bisect_scratch_bytes(N) + 256; }

phi4_status phi4_ess_bisect(const double* ell, int32_t N, const double* beta_in, double rho, int32_t iters,
                            double* w, double* out, void* scratch, size_t scratch_bytes, void* stream) {
  ARG_CHECK(ell && beta_in && w && out && scratch, "NULL argument");
  ARG_CHECK(N >= 1 && N <= 131072, "N = %d outside [1, 131072]", N);
  ARG_CHECK(rho > 0 && rho < 1 && iters >= 0 && iters <= 200, "rho/iters invalid");
  ARG_CHECK(scratch_bytes >= phi4_bisect_scratch_bytes(N), "scratch too small");
  uint32_t* status = (uint32_t*)((unsigned char*)scratch + bisect_scratch_bytes(N));
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemsetAsync(status, 0, 4, s));
  CUDA_TRY(launch_bisect(ell, N, beta_in, rho, iters, w, out, scratch, status, s));
  uint32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return status_to_error(st & ~ST_BISECT_FLOOR);
}

size_t phi4_resample_scratch_bytes(int32_t N) { return resample_scratch_bytes(N); }

phi4_status phi4_resample_systematic(const double* w, int32_t N, uint32_t U, int32_t* anc, void* scratch,
                                     size_t scratch_bytes, void* stream) {
  ARG_CHECK(w && anc && scratch, "NULL argument");
  ARG_CHECK(N >= 1 && N <= 131072, "N = %d outside [1, 131072]", N);
  ARG_CHECK(scratch_bytes >= resample_scratch_bytes(N), "scratch too small");
  CUDA_TRY(launch_resample(w, N, U, nullptr, anc, scratch, (cudaStream_t)stream));
  return PHI4_OK;
}

phi4_status phi4_gather_rows(const void* src, void* dst, size_t row_bytes, int32_t N, const int32_t* anc,
                             void* stream) {
  ARG_CHECK(src && dst && anc, "NULL argument");
  ARG_CHECK(N >= 0, "N < 0");
  CUDA_TRY(launch_gather(src, dst, row_bytes, N, anc, (cudaStream_t)stream));
  return PHI4_OK;
}

size_t phi4_covariance_scratch_bytes(int32_t N, int32_t D, int32_t precision) {
  return covariance_scratch_bytes(N, D, precision) + 256;
}

phi4_status phi4_covariance(const void* phi, int32_t precision, int32_t N, int32_t D, double* sigma, void* scratch,
                            size_t scratch_bytes, void* stream) {
  ARG_CHECK(phi && sigma && scratch, "NULL argument");
  ARG_CHECK(N >= 2 && D >= 1 && D <= 16384, "bad sizes");
  ARG_CHECK(precision >= 0 && precision <= 2, "precision %d unknown", precision);
  ARG_CHECK(scratch_bytes >= phi4_covariance_scratch_bytes(N, D, precision), "scratch too small");
  if (precision == PHI4_MIXED_BF16 && !tc_available()) {
    set_error("tensor-map encoder unavailable");
    return PHI4_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* status = (uint32_t*)((unsigned char*)scratch + covariance_scratch_bytes(N, D, precision));
  CUDA_TRY(cudaMemsetAsync(status, 0, 4, s));
  CUDA_TRY(launch_covariance(phi, precision, N, D, sigma, scratch, status, s));
  uint32_t st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return status_to_error(st);
}

size_t phi4_cholesky_scratch_bytes(int32_t D) { return D > 0 ? cholesky_aux_bytes(D) : 0; }

phi4_status phi4_cholesky(double* a, int32_t D, const double* d_ridge, uint32_t* d_status, void* scratch,
                          size_t scratch_bytes, int32_t mode, void* stream) {
  ARG_CHECK(a && d_status && scratch, "NULL argument");
  ARG_CHECK(D >= 1 && D <= 16384, "D = %d outside [1, 16384]", D);
  ARG_CHECK(mode >= 0 && mode <= 2, "mode %d unknown", mode);
  ARG_CHECK(scratch_bytes >= cholesky_aux_bytes(D), "scratch too small");
  ARG_CHECK(((uintptr_t)scratch & 255) == 0, "scratch must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_copy_lower(a, a, D, s));
  CUDA_TRY(launch_cholesky(a, D, d_ridge, d_status, scratch, s, nullptr, nullptr, nullptr, mode));
  return PHI4_OK;
}

phi4_status phi4_cholesky_f32(const double* sigma, float* a, int32_t D, const double* d_ridge, uint32_t* d_status,
                              void* scratch, size_t scratch_bytes, void* stream) {
  ARG_CHECK(sigma && a && d_status && scratch, "NULL argument");
  ARG_CHECK(D >= 1 && D <= 16384, "D = %d outside [1, 16384]", D);
  ARG_CHECK(scratch_bytes >= cholesky_aux_bytes(D), "scratch too small");
  CUDA_TRY(launch_cholesky_f32(sigma, a, D, d_ridge, d_status, scratch, (cudaStream_t)stream));
  return PHI4_OK;
}

size_t phi4_propose_scratch_bytes(int32_t N, int32_t D, int32_t precision) {
  if (precision == PHI4_MIXED_BF16)
    return align256((size_t)N * (((size_t)D + 7) & ~(size_t)7) * 2) + align256((size_t)N * D * 2) + 256;
  return align256((size_t)N * D * (precision == PHI4_FP64 ? 8 : 4)) + 256;
}

phi4_status phi4_rw_propose(const void* phi, void* prop, const void* Lfac, int32_t ldl, int32_t precision, int32_t N,
                            int32_t D, double scale, uint64_t seed, uint64_t stream_id, uint32_t step, uint32_t sweep,
                            void* scratch, size_t scratch_bytes, void* stream) {
  ARG_CHECK(phi && prop && Lfac && scratch, "NULL argument");
  ARG_CHECK(N >= 1 && D >= 1 && D <= 16384, "bad sizes");
  ARG_CHECK(precision >= 0 && precision <= 2, "precision %d unknown", precision);
  ARG_CHECK(scratch_bytes >= phi4_propose_scratch_bytes(N, D, precision), "scratch too small");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == PHI4_MIXED_BF16) {
    ARG_CHECK(ldl >= D && ldl % 8 == 0, "ldl must be >= D and a multiple of 8");
    ARG_CHECK(((uintptr_t)Lfac & 15) == 0 && ((uintptr_t)scratch & 15) == 0, "operands must be 16-byte aligned");
    if (!tc_available()) {
      set_error("tensor-map encoder unavailable");
      return PHI4_ERR_UNSUPPORTED;
    }
    const int ldz = (D + 7) & ~7;
    unsigned char* delta = (unsigned char*)scratch + align256((size_t)N * ldz * 2);
    uint32_t* status = (uint32_t*)(delta + align256((size_t)N * D * 2));
    CUDA_TRY(cudaMemsetAsync(status, 0, 4, s));
    CUDA_TRY(launch_normals(seed, stream_id, RNG_PROPOSE, step, sweep, 0, N, D, ldz, PHI4_DT_BF16, scratch, s));
    CUDA_TRY(launch_propose_tc(delta, scratch, ldz, Lfac, ldl, N, D, (float)scale, status, s));
    CUDA_TRY(launch_apply_delta((const float*)phi, delta, (float*)prop, (long long)N * D, s));
    uint32_t st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return status_to_error(st);
  }
  ARG_CHECK(ldl == D, "ldl must equal D for the FP64/FP32 forms");
  const int dt = precision == PHI4_FP64 ? PHI4_DT_F64 : PHI4_DT_F32;
  CUDA_TRY(launch_normals(seed, stream_id, RNG_PROPOSE, step, sweep, 0, N, D, D, dt, scratch, s));
  CUDA_TRY(launch_propose_simt(phi, prop, scratch, Lfac, dt, N, D, scale, s));
  return PHI4_OK;
}

phi4_status phi4_rw_accept(void* phi, const void* prop, int32_t dtype, int32_t N, int32_t L, double m2, double lambda,
                           double c_kin, double c_mass, int32_t keep_reference, double* S, double* sq, double* ell,
                           const double* beta, uint64_t seed, uint64_t stream_id, uint32_t step, uint32_t sweep,
                           uint32_t* acc_count, void* stream) {
  ARG_CHECK(phi && prop && S && sq && ell && beta && acc_count, "NULL argument");
  ARG_CHECK(N >= 0 && L >= 1 && L <= 128, "bad sizes");
  ARG_CHECK(dtype == PHI4_DT_F64 || dtype == PHI4_DT_F32, "dtype must be F64 or F32");
  ActionParams p{L, L * L, N, m2, lambda, c_kin, c_mass, 0.5 * L * L * log(2.0 * M_PI)};
  // the status word shares the counter's allocation: acc_count[1]
  CUDA_TRY(launch_accept(phi, prop, dtype, p, keep_reference, S, sq, ell, beta, seed, stream_id, step, sweep,
                         acc_count, acc_count + 1, (cudaStream_t)stream));
  return PHI4_OK;
}

phi4_status phi4_rw_accept_delta(float* phi, const void* delta_f16, int32_t N, int32_t L, double m2, double lambda,
                                 double c_kin, double c_mass, int32_t keep_reference, double* S, double* sq,
                                 double* ell, const double* beta, uint64_t seed, uint64_t stream_id, uint32_t step,
                                 uint32_t sweep, uint32_t* acc_count, void* stream) {
  ARG_CHECK(phi && delta_f16 && S && sq && ell && beta && acc_count, "NULL argument");
  ARG_CHECK(N >= 0 && L >= 4 && L <= 128 && L % 4 == 0 && L * L <= 8192, "L = %d: need L %% 4 == 0, L*L <= 8192", L);
  ActionParams p{L, L * L, N, m2, lambda, c_kin, c_mass, 0.5 * L * L * log(2.0 * M_PI)};
  CUDA_TRY(launch_accept_delta(phi, delta_f16, p, keep_reference, S, sq, ell, beta, seed, stream_id, step, sweep,
                               acc_count, acc_count + 1, (cudaStream_t)stream));
  return PHI4_OK;
}


}  // extern "C"
