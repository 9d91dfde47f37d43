// Host-side launchers shared by the translation units of libphi4smc (not part of the ABI).
#pragma once
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace phi4 {

// About one second of SM clock: the default limit of every spin-wait in this library.
constexpr long long kSpinLimitCyclesDefault = 2000000000LL;

// Device scalars of a run (one 256-byte block): bisection results, the Kahan pair of
// log Z, beta, the ridge, nested-sampling bookkeeping, observables, and for the batched
// form the temperature counter and the run's participation in the current step.
enum { SC_OUT = 0 /* 8 doubles: bisection results */, SC_KAHAN = 8 /* 2 */, SC_BETA = 10, SC_RIDGE = 11,
       SC_NS = 12 /* NS bookkeeping, 8 doubles */, SC_OBS = 20 /* observables, 6 doubles */, SC_T = 26,
       SC_ACTIVE = 27, SC_COUNT = 32 };

struct ActionParams {
  int L, D, N;
  double m2, lam, c_kin, c_mass;
  double half_d_log2pi;  // (D/2) log(2 pi): minus the log-normaliser of N(0, I_D)
};

// Per-thread error message of the last failed call (capi.cu).
void set_error(const char* fmt, ...);

// kernels_rng.cu
cudaError_t launch_normals(uint64_t seed, uint64_t stream_id, uint32_t kind, uint32_t step, uint32_t sub,
                           int row0, int n_rows, int n_cols, int ld, int dtype, void* out, cudaStream_t s);

// kernels_lattice.cu
cudaError_t launch_action(const void* phi, int dtype, const ActionParams& p, double* S, double* sq,
                          double* ell, int keep_reference, cudaStream_t s);
// irmh_zz / irmh_r (optional, SMC-IRMH): log alpha gains (zz - r) / 2 and an accepted
// particle's r becomes its zz
cudaError_t launch_accept(void* phi, const void* prop, int dtype, const ActionParams& p, int keep_reference,
                          double* S, double* sq, double* ell, const double* beta, uint64_t seed,
                          uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count,
                          uint32_t* status, cudaStream_t s, const double* irmh_zz = nullptr,
                          double* irmh_r = nullptr);
// SMC-IRMH (kernels_irmh.cu): r_n = |L^{-1}(phi_n - mu)|^2 (L: D x D lower, row pitch ld;
// D <= 1024) and zz_n = |Z_n|^2, FP64
cudaError_t launch_whitened_sq_norm(const double* phi, const double* mu, const double* Lf, int ld, int N, int D,
                                    double* r, cudaStream_t s);
cudaError_t launch_row_sq_norm(const double* Z, int N, int D, double* zz, cudaStream_t s);
// SMC-HMC (kernels_lattice.cu): escale_s = eps sqrt(sigma_ss + *ridge) (D doubles), once per
// temperature; then one HMC transition per particle, D <= 4096, fields and Z of `dtype`
// (F64 or F32; the energies in double): momenta Z / sqrt(v) with inverse mass
// v_s = sigma_ss + ridge, n_leap leapfrog steps of size eps on the tempered target at
// *beta, accept on the Philox RNG_ACCEPT uniform of (step, sweep)
constexpr int kHmcLeapfrog = 20;  // App. A
cudaError_t launch_hmc_scale(const double* sigma, int D, const double* ridge, double eps, double* escale,
                             cudaStream_t s);
cudaError_t launch_hmc(void* phi, const void* Z, int dtype, const double* escale, const ActionParams& p,
                       int keep_reference, double* S, double* sq, double* ell, const double* beta, int n_leap,
                       uint64_t seed, uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count,
                       uint32_t* status, cudaStream_t s);
// float fields, proposal = phi + delta (fp16 increment), L % 4 == 0
cudaError_t launch_accept_delta(float* phi, const void* delta_f16, const ActionParams& p, int keep_reference,
                                double* S, double* sq, double* ell, const double* beta, uint64_t seed,
                                uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count,
                                uint32_t* status, cudaStream_t s);
// Z2 move: negate row n of phi (dtype 0 double, 1 float) when the Philox flip bit of
// (RNG_FLIP, step, particle n) is set.
cudaError_t launch_z2_flip(uint64_t seed, uint64_t stream_id, uint32_t step, void* phi, int dtype, int N, int D,
                           cudaStream_t s);
cudaError_t launch_magnetisation(const void* phi, int dtype, int N, int D, double* M, cudaStream_t s);
// kernels_obs.cu: M per particle into M[N], then the weighted moments (w NULL: uniform)
// out[0..5] = <M>, <|M|>, <M^2>, chi, mode balance, total weight (FP64, one CTA)
cudaError_t launch_observables(const void* phi, int dtype, int N, int D, const double* w, double* M, double* out,
                               cudaStream_t s);

// kernels_temper.cu
size_t bisect_scratch_bytes(int N);
cudaError_t launch_bisect(const double* ell, int N, const double* beta_in, double rho, int iters, double* w,
                          double* out, void* scratch, uint32_t* status, cudaStream_t s, bool single_cta = false);
cudaError_t launch_logz_accumulate(const double* out, double* logz_kahan, double* beta, cudaStream_t s);

// kernels_resample.cu
size_t resample_scratch_bytes(int N);
cudaError_t launch_resample(const double* w, int N, uint32_t U, const uint32_t* U_dev, int32_t* anc,
                            void* scratch, cudaStream_t s);
cudaError_t launch_gather(const void* src, void* dst, size_t row_bytes, int N, const int32_t* anc,
                          cudaStream_t s);
cudaError_t launch_gather_f64(const double* src, double* dst, int N, const int32_t* anc, cudaStream_t s);
cudaError_t launch_gather3_f64(const double* s0, double* d0, const double* s1, double* d1, const double* s2,
                               double* d2, int N, const int32_t* anc, cudaStream_t s);

// kernels_cov.cu
size_t covariance_scratch_bytes(int N, int D, int precision);
cudaError_t launch_covariance(const void* phi, int precision, int N, int D, double* sigma, void* scratch,
                              uint32_t* status, cudaStream_t s);
cudaError_t launch_ridge(const double* sigma, int D, double jitter_rel, double* ridge, cudaStream_t s);
// exact covariance of the Gaussian part of the tempered target at *beta (device), the
// whole D x D matrix into sigma; scratch: free_covariance_scratch_bytes(L)
size_t free_covariance_scratch_bytes(int L);
cudaError_t launch_free_covariance(int L, const double* beta, double m2c, double c_kin, int keep, double* sigma,
                                   void* scratch, cudaStream_t s);

// CUDA-event pairs around selected kernel launches, each pair on the launch's own
// stream (kernel-level timing inside a stage that spans two streams).
struct LaunchTimer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> pool;
  double ms = 0.0;
  int64_t launches = 0;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t begin(cudaStream_t s) {
    cudaEvent_t a = take();
    cudaEventRecord(a, s);
    return a;
  }
  void end(cudaStream_t s, cudaEvent_t a) {
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    pending.push_back({a, b});
  }
  // after the streams are synchronised
  void collect() {
    for (auto& pr : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) {
        ms += t;
        launches += 1;
      } else {
        (void)cudaGetLastError();  // a failed query must not surface at an unrelated call
      }
      pool.push_back(pr.first);
      pool.push_back(pr.second);
    }
    pending.clear();
  }
  void release() {
    for (auto& pr : pending) {
      pool.push_back(pr.first);
      pool.push_back(pr.second);
    }
    pending.clear();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// kernels_chol.cu
cudaError_t launch_copy_lower(const double* src, double* dst, int D, cudaStream_t s);
// In-place blocked Cholesky; aux: cholesky_aux_bytes(D) device scratch for the diagonal-block
// inverses. With side != nullptr the look-ahead schedule uses `side` and the two events.
size_t cholesky_aux_bytes(int D);
// mode: 0 automatic (tensor-core trailing update for D >= 256), 1 FP64 SIMT update, 2 tensor-core update
// `timer` (optional) brackets every tensor-core launch of the bulk of a trailing update.
cudaError_t launch_cholesky(double* a, int D, const double* ridge, uint32_t* status, void* aux, cudaStream_t s,
                            cudaStream_t side = nullptr, cudaEvent_t evA = nullptr, cudaEvent_t evB = nullptr,
                            int mode = 0, LaunchTimer* timer = nullptr);
// A22 -= P P^T from the digit planes of the panel P (kernels_tc.cu), on the 64-column
// blocks [blk_lo, blk_hi) of the trailing matrix (blk_hi >= 2^20: to the end);
// leave_sms: the bulk update beside the look-ahead chain keeps a few SMs free for it
cudaError_t launch_chol_update_tc(double* a, int D, int b0, int m, const void* planes, int m_pad, const int* rexp,
                                  int blk_lo, int blk_hi, bool leave_sms, uint32_t* status, cudaStream_t s);
int cholesky_launches(int D);  // kernels one launch_cholesky enqueues
// float factorisation of the lower triangle of sigma (copied into a) for the plain FP32 form
cudaError_t launch_cholesky_f32(const double* sigma, float* a, int D, const double* ridge, uint32_t* status,
                                void* aux, cudaStream_t s, cudaStream_t side = nullptr, cudaEvent_t evA = nullptr,
                                cudaEvent_t evB = nullptr);
cudaError_t launch_factor_convert_f32(const float* Lc, int D, float* out, cudaStream_t s);
cudaError_t launch_factor_convert(const double* Lc, int D, int dtype, void* out, int ld, cudaStream_t s);

// kernels_gemm_simt.cu
// prop = phi + scale Z L^T; phi_ld = 0 adds the one row `phi` to every row (SMC-IRMH: mu)
cudaError_t launch_propose_simt(const void* phi, void* prop, const void* Z, const void* Lf, int dtype, int N,
                                int D, double scale, cudaStream_t s, int phi_ld = -1);
cudaError_t launch_syrk_simt(const void* XcT, int dtype, int D, int N, int ldx, double inv_nm1, double* sigma,
                             cudaStream_t s);

// kernels_tc.cu (tcgen05 / TMA)
bool tc_available();
// increment Delta = scale * Z L^T as fp16 [N][D] (tensor cores, bf16 operands)
cudaError_t launch_propose_tc(void* delta_f16, const void* Zb, int ldz, const void* Lb, int ldl, int N, int D,
                              float scale, uint32_t* status, cudaStream_t s);
// prop = phi + float(delta) elementwise (float fields)
cudaError_t launch_apply_delta(const float* phi, const void* delta_f16, float* prop, long long n, cudaStream_t s);
// Sigma = 2^(-s_i - s_j) (2^(2a) H H^T + 2^a (H L^T + L H^T) + L L^T) / (N - 1) on the
// lower triangle, exact digit products on the tensor cores (H, L: D x N bf16 digit planes).
cudaError_t launch_gram_tc(const void* H, const void* Lo, int ldx, int D, int N, const int* shift, int a,
                           double inv_nm1, double* sigma, uint32_t* status, cudaStream_t s);

// kernels_ns.cu
cudaError_t launch_ns_select(const double* logl, int N, int k, int32_t* order, double* ns, double* dead,
                             long long dead_cap, uint32_t* status, cudaStream_t s);
cudaError_t launch_ns_start(const void* live, int dtype, const int32_t* order, int N, int k, int D, uint64_t seed,
                            uint64_t stream_id, uint32_t it, void* X, cudaStream_t s);
cudaError_t launch_ns_slice(void* X, int dtype, double* logl_out, const void* Lf, int k, int L, double c_kin,
                            double c_mass_m2, double lam, const double* lstar, int steps, int max_shrink,
                            uint64_t seed, uint64_t stream_id, uint32_t it, uint32_t* capped, cudaStream_t s);
cudaError_t launch_ns_replace(void* live, int dtype, double* logl, const int32_t* order, const void* X,
                              const double* xl, int k, int D, cudaStream_t s);
cudaError_t launch_ns_stop(const double* logl, int N, double log_stop, double* ns, cudaStream_t s);
cudaError_t launch_ns_final(const double* dead, long long n_dead, const double* logl, int N, double* ns,
                            cudaStream_t s);

// device properties (capi.cu)
int sm_count();

// limit of the software waits of each translation unit that has them (common.cuh)
cudaError_t set_spin_limit_temper(long long cycles);
cudaError_t set_spin_limit_chol(long long cycles);

}  // namespace phi4
