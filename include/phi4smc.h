/*
 * phi4smc -- GB300 (sm_103a) particle Monte Carlo for lattice phi^4 theory.
 *
 * C ABI of the library libphi4smc.so. It implements the data-parallel hot path
 * of the particle samplers of arXiv 2511.15196, "Particle Monte Carlo methods
 * for Lattice Field Theory":
 *   - adaptive tempered SMC with covariance-preconditioned random-walk
 *     Metropolis moves (Sec. 2, sampler (i); App. A), and
 *   - nested sampling with slice-sampling rejuvenation (Sec. 2, sampler (iv);
 *     App. A),
 * on the Euclidean action of Eq. (1) on a periodic L x L lattice.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Fields.  A population of N fields is a row-major [N][D] array, D = L*L,
 *          site x = r*L + c. Element type follows phi4_dtype.
 * Action.  S = sum_x [ c_kin * sum_mu phi_x(2 phi_x - phi_{x+mu} - phi_{x-mu})
 *                      + c_mass * m2 * phi_x^2 + lambda * phi_x^4 ]
 *          (Eq. (1) with its 1/2 factors made coefficients: c_kin = c_mass = 1/2
 *          is Eq. (1) verbatim, c_kin = c_mass = 1 the unhalved form).
 * Memory.  The caller owns all memory. Pointers documented "device" must be
 *          device (or managed) memory on the current CUDA device; "host" means
 *          host memory. The library never calls cudaMalloc/cudaFree: state
 *          lives in a caller-provided workspace.
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *          stream). Entry points that only enqueue work return before it runs.
 * Errors.  Every function returns phi4_status. A message for the last error on
 *          the calling thread is available from phi4_last_error(). Device-side
 *          anomalies (non-finite values, a non positive-definite covariance, a
 *          bounded device wait that gave up) are written to a device status
 *          word and reported by the next synchronising call.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *          key = (seed mod 2^32, (seed >> 32) xor stream_id) and
 *          counter = (kind << 24 | step, sub, particle, block), see phi4_rng_kind.
 */
#ifndef PHI4SMC_H
#define PHI4SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PHI4_OK = 0,
  PHI4_ERR_ARG = 1,          /* invalid argument (message says which) */
  PHI4_ERR_CUDA = 2,         /* a CUDA runtime/driver call failed */
  PHI4_ERR_NOT_PD = 3,       /* covariance not positive definite after all ridge increases */
  PHI4_ERR_NONFINITE = 4,    /* NaN/Inf met in log-weights or the action */
  PHI4_ERR_DONE = 5,         /* SMC already at beta = 1, or nested sampling stopped */
  PHI4_ERR_WORKSPACE = 6,    /* workspace too small or misaligned */
  PHI4_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
  PHI4_ERR_UNSUPPORTED = 8   /* configuration outside what this build supports */
} phi4_status;

/* Samplers. SMC_RW: adaptive tempered SMC with covariance-preconditioned random-walk
 * sweeps (Sec. 2 sampler (i)). NS_SLICE: nested sampling with slice rejuvenation
 * (sampler (iv)). SMC_IRMH: the same tempered SMC with independent Metropolis-Hastings
 * sweeps (sampler (ii)): each particle proposes mu + L z from the Gaussian of the
 * population's mean mu and covariance L L^T, accepted with the tempered-target ratio
 * times q(phi) / q(phi'); FP64 form, D <= 1024. SMC_HMC: the same tempered SMC with
 * Hamiltonian Monte Carlo transitions (sampler (iii)): 20 leapfrog steps (App. A) per
 * transition with the refit's covariance diagonal plus the ridge as inverse mass and
 * step size rw_scale (<= 0 selects 0.8 D^(-1/4)); n_mcmc transitions per temperature;
 * FP64 or FP32 form (float trajectories, energies summed in double), D <= 4096. */
typedef enum { PHI4_SMC_RW = 0, PHI4_NS_SLICE = 1, PHI4_SMC_IRMH = 2, PHI4_SMC_HMC = 3 } phi4_kind;

/* Arithmetic forms of a run.
 * FP64:      fields, proposal GEMM, covariance and everything else in double.
 * FP32:      the plain float form: float fields, SIMT float proposal GEMM,
 *            covariance and Cholesky; float per-site action terms with compensated
 *            float partial sums; the per-particle sums, log-weights and log Z stay
 *            double (a few operations per particle).
 * MIXED_BF16: float fields; proposal GEMM on the tcgen05 tensor cores with bf16
 *            operands and fp32 accumulation; covariance as the exact Gram matrix of
 *            fixed-point digits of the centred fields, also on the tensor cores (see
 *            phi4_covariance); double Cholesky, acceptance test, log-weights and
 *            compensated log Z. */
typedef enum { PHI4_FP64 = 0, PHI4_FP32 = 1, PHI4_MIXED_BF16 = 2 } phi4_precision;

/* Element types of the kernel-level entry points. */
typedef enum { PHI4_DT_F64 = 0, PHI4_DT_F32 = 1, PHI4_DT_BF16 = 2 } phi4_dtype;

/* Stream kinds of the Philox counter word 0 (bits 24..31). */
typedef enum {
  PHI4_RNG_INIT = 1, PHI4_RNG_RESAMPLE = 2, PHI4_RNG_PROPOSE = 3, PHI4_RNG_ACCEPT = 4,
  PHI4_RNG_NS_START = 5, PHI4_RNG_NS_DIRECTION = 6, PHI4_RNG_NS_SLICE = 7, PHI4_RNG_FLIP = 8
} phi4_rng_kind;

typedef struct {
  int32_t L;                 /* lattice side, D = L*L sites (1 <= L <= 128) */
  int32_t N;                 /* particles (SMC) or live points (NS), 2 <= N <= 131072 (NS: N <= 8192) */
  int32_t kind;              /* phi4_kind */
  int32_t precision;         /* phi4_precision */
  double m2, lambda;         /* bare mass^2 and quartic coupling */
  double c_kin, c_mass;      /* action coefficients, 1.0 / 1.0 = unhalved form, 0.5 / 0.5 = Eq. (1) */
  int32_t keep_reference;    /* 0: tempering path N(0,I)^(1-beta) e^{-beta S}, target e^{-S} at beta=1;
                                1: path N(0,I) e^{-beta S}, i.e. exp(-[U0 + beta S]) of Sec. 2 */
  int32_t n_mcmc;            /* inner-kernel sweeps (SMC_HMC: transitions) per temperature (SMC) */
  double ess_target;         /* rho in (0,1): next beta keeps ESS = rho N (SMC) */
  double rw_scale;           /* proposal scale on the Cholesky factor; <= 0 selects 2.38/sqrt(D) (App. A);
                                SMC_HMC: the leapfrog step size, <= 0 selects 0.8 D^(-1/4) */
  int32_t ns_n_delete;       /* live points deleted per nested-sampling iteration (1 <= k < N) */
  int32_t ns_slice_steps;    /* slice steps per new point; <= 0 selects 3*D */
  double ns_stop_frac;       /* stop when remaining evidence < ns_stop_frac * Z */
  double chol_jitter_rel;    /* ridge delta = chol_jitter_rel * trace(Sigma) / D, x10 per failed try */
  int32_t bisect_iters;      /* maximum bisection steps for the next beta (64) */
  int32_t slice_max_shrink;  /* slice shrinkage tries before a step is abandoned (64) */
  uint64_t seed, stream_id;  /* Philox key material */
  int32_t chol_mode;         /* double Cholesky trailing update: 0 automatic (tensor cores for D >= 256),
                                1 FP64 SIMT, 2 FP64-accurate exact-digit emulation on the tensor cores */
  int32_t flags;             /* PHI4_FLAG_* bits, 0 for the sampler as the paper runs it */
} phi4_config;

/* phi4_config.flags. Z2_FLIP (SMC): after each temperature's sweeps every particle is
 * negated with probability 1/2 (one Philox bit per particle, stream kind
 * PHI4_RNG_FLIP, counter (kind << 24 | temperature, 0, particle, 0), bit 0 of the first
 * word). Every tempered target is even in phi (S is even and the reference N(0, I) is
 * symmetric), so the global flip phi -> -phi is a Metropolis move accepted with
 * probability 1; S, |phi|^2 and the log-weights are unchanged. The paper leaves such
 * symmetry moves out of its black-box samplers (Sec. 2) and gives them to its AHMC
 * control. */
#define PHI4_FLAG_Z2_FLIP 1
/* phi4_config.flags. FREE_KERNEL_COV (SMC_RW, SMC_HMC; needs c_mass * m2 > 0): the
 * covariance that scales the proposals (the random-walk factor, HMC's inverse mass) is
 * not estimated from the population but is, at each new beta, the exact covariance of
 * the Gaussian part of the tempered target (phi4_free_field_covariance); for lambda = 0
 * that is the target's own covariance. It does not depend on the particles it moves, so
 * with it the sampler's evidence estimate is unbiased in Z. A control for comparisons
 * with the free field's closed form: the paper's sampler estimates the covariance from
 * the population (flag off). */
#define PHI4_FLAG_FREE_KERNEL_COV 2

typedef struct {
  double beta;               /* current inverse temperature (SMC) */
  double logz, logz_err;     /* running log-evidence; error bar (NS: sqrt(H/N); SMC: NaN) */
  double mean_M, mean_absM, mean_M2, chi, mode_balance; /* uniform-weight population moments of
                                M = (1/D) sum_x phi_x; chi = D(<M^2> - <M>^2); mode balance of App. F */
  double ess;                /* ESS of the last reweighting (SMC) */
  double acc_rate;           /* acceptance rate of the last temperature's sweeps (SMC) */
  int64_t n_steps;           /* temperatures (SMC) or deletion iterations (NS) done */
  int64_t n_likelihood_evals;/* action evaluations so far */
  int64_t slice_capped;      /* NS slice steps abandoned after slice_max_shrink tries */
} phi4_obs;

typedef struct phi4_run phi4_run; /* opaque, host memory owned by the library until smc_free */

/* ------------------------------------------------------------------------ */
/* Library                                                                   */
/* ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread (static storage, never NULL). */
const char* phi4_last_error(void);

/* Number of streaming multiprocessors of the current device (host query). */
phi4_status phi4_device_sm_count(int32_t* out);

/* Limit, in SM clock cycles, of the library's software waits on the current device:
 * the grid barrier of the ESS bisection, the flags between the diagonal-block CTA and
 * the CTAs of its streamed inverse, and the hand-offs between the diagonal block's
 * warps. A wait that reaches the limit gives up: its kernel sets the timeout bit of
 * the run's device status word and returns, and the next synchronising call of the
 * run returns PHI4_ERR_TIMEOUT. cycles <= 0 restores the default (2e9, about one
 * second). Waits on TMA copies and tensor-core commits keep the default: they wait for
 * hardware that completes by itself. Synchronous; affects every later launch on the
 * device, so set it while no run is in flight. Failure detection (no counterpart in the
 * paper): a short limit lets a test see a wait give up without hanging anything. */
phi4_status phi4_set_spin_limit(int64_t cycles);

/* ------------------------------------------------------------------------ */
/* Run-level API: a population advanced one outer step per call.             */
/* ------------------------------------------------------------------------ */

/* Workspace bytes smc_init needs for `cfg` (host only; validates cfg). */
phi4_status phi4_workspace_bytes(const phi4_config* cfg, size_t* bytes);

/* Creates a run in the caller's device workspace `d_workspace` (>= phi4_workspace_bytes,
 * 256-byte aligned), enqueues on `stream` the initial draw phi ~ N(0, I_D)
 * (PHI4_RNG_INIT, step 0) and its action, and returns the host handle.
 * SMC (Sec. 2 (i)): beta = 0, log Z = 0. NS (Sec. 2 (iv)): N live points, log X = 0.
 * The workspace must stay valid until smc_free. */
phi4_status smc_init(const phi4_config* cfg, void* d_workspace, size_t workspace_bytes,
                     void* stream, phi4_run** out);

/* One SMC temperature (Sec. 2 (i); App. A): ESS bisection for the next beta,
 * reweighting with Kahan-compensated log Z, systematic resampling and particle
 * gather, covariance and Cholesky refit (double; float in the FP32 form), n_mcmc
 * sweeps of the run's inner kernel at the new beta (random-walk Metropolis,
 * independent Metropolis-Hastings or HMC transitions, by phi4_config.kind), then
 * the global flip move when PHI4_FLAG_Z2_FLIP is set. Synchronises the run's stream and writes the new beta
 * to *beta_out (may be NULL). PHI4_ERR_DONE once beta == 1; PHI4_ERR_ARG on an NS run. */
phi4_status smc_temper_step(phi4_run* run, double* beta_out);

/* One nested-sampling iteration (Sec. 2 (iv); App. A): delete the ns_n_delete
 * lowest-likelihood live points, update log X and log Z, refit the live-point
 * covariance, and replace each deleted point by ns_slice_steps constrained slice
 * steps from a random survivor. Synchronises; *done_out = 1 when the stopping
 * rule holds. PHI4_ERR_DONE if already stopped; PHI4_ERR_ARG on an SMC run. */
phi4_status ns_replace_step(phi4_run* run, int32_t* done_out);

/* Running log-evidence (Sec. 2: SMC accumulates the log mean incremental weight of
 * each temperature; NS sums dead and live points' prior-volume weights, App. A) and its
 * error bar (NS: sqrt(H/N) including the live points; SMC: NaN). Synchronises the
 * run's stream. */
phi4_status smc_log_evidence(const phi4_run* run, double* logz, double* logz_err);

/* Population observables (uniform weights over the current population): moments of
 * the magnetisation M (Sec. 2), susceptibility, mode balance (App. F).
 * Synchronises the run's stream. */
phi4_status smc_observables(const phi4_run* run, phi4_obs* out);

/* Copies the current fields ([N][D], element type of the run's precision:
 * f64 for PHI4_FP64, f32 otherwise) to `dst` (host or device), `bytes` >= N*D*elem.
 * Synchronises the run's stream. */
phi4_status smc_copy_particles(const phi4_run* run, void* dst, size_t bytes);

/* Replaces the current fields by `src` (host or device, same layout as
 * smc_copy_particles) and recomputes their action and log-weights on the run's
 * stream (enqueued; returns after the copy is enqueued). */
phi4_status smc_load_particles(phi4_run* run, const void* src, size_t bytes);

/* Checkpoint and resume (no counterpart in the paper): the state that determines every
 * later step of a run, copied to or from a caller's host buffer of phi4_state_bytes:
 * a header (the configuration, the temperature or iteration counter that fixes the
 * Philox counters of the next step, beta, the ridge level, the counters and, for nested
 * sampling, log X and the running log Z), then the fields, S, |phi|^2 and ell of every
 * particle, the run's scalar block (Kahan pair of log Z, beta, NS bookkeeping) and the
 * nested-sampling dead points. smc_restore_state into a run created with the identical
 * configuration (checked) continues bit for bit as the saved run would have; the
 * counters are restored too. Both synchronise the run's stream. A batch handle has no single
 * state; a batch member can be saved but not restored (its buffers follow the batch's
 * steps). */
phi4_status phi4_state_bytes(const phi4_run* run, size_t* bytes);
phi4_status smc_save_state(const phi4_run* run, void* host_dst, size_t bytes);
phi4_status smc_restore_state(phi4_run* run, const void* host_src, size_t bytes);

/* Releases the handle (not the workspace); for a batch handle, every member.
 * Synchronises the run's stream. */
phi4_status smc_free(phi4_run* run);

/* Number of kernels the run has launched since smc_init (host counter). */
phi4_status phi4_kernel_launches(const phi4_run* run, int64_t* out);

/* Per-stage device timing of a run. When enabled, CUDA events bracket each
 * stage on the run's stream; phi4_stage_times returns accumulated milliseconds
 * and launch counts since the last reset, for stage ids 0..PHI4_N_STAGES-1
 * (names from phi4_stage_name). Synchronises the run's stream. Stage 12
 * ("chol_update") is kernel-level: event pairs around the launch of the bulk of each
 * tensor-core trailing update of the Cholesky (all but the next block column), on
 * the stream it runs on; its time is part of stage 4 ("cholesky"). In the mixed form
 * the sweeps run on three streams (normals and proposal GEMM of the next sweep
 * beside the current accept): stages 5, 6 and 7 are then kernel-level event pairs on
 * their own streams and stage 13 ("mutation") is the wall time of all n_mcmc sweeps
 * on the run's stream. */
#define PHI4_N_STAGES 14
phi4_status phi4_set_stage_timing(phi4_run* run, int32_t enable);
phi4_status phi4_stage_times(phi4_run* run, double* ms_out, int64_t* launches_out, int32_t reset);
const char* phi4_stage_name(int32_t stage);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent SMC runs advanced together.                */
/* ------------------------------------------------------------------------ */

/* Workspace bytes for `n_runs` SMC runs with configurations cfgs[0..n_runs-1]
 * (different L, N, couplings, precisions and seeds allowed; N <= 4096 each). */
phi4_status phi4_batch_workspace_bytes(const phi4_config* cfgs, int32_t n_runs, size_t* bytes);

/* Creates the runs in one caller workspace (>= phi4_batch_workspace_bytes, 256-byte
 * aligned) and returns a batch handle. Each member gets its own CUDA stream so the
 * members' kernels overlap on the GPU; `stream` is the caller's stream, which every
 * batch call orders itself after and joins before returning. */
phi4_status smc_init_batch(const phi4_config* cfgs, int32_t n_runs, void* d_workspace, size_t workspace_bytes,
                           void* stream, phi4_run** out);

/* One temperature for every member still below beta = 1: the same steps as
 * smc_temper_step, each stage one launch over all members. The ESS bisection with the
 * reweighting and log Z (one CTA per member), the resampling and the particle gather
 * run on the batch's own stream; the covariance and Cholesky of each member on the
 * member's stream; the sweeps of the mixed-form members with L % 4 == 0 as one CUDA
 * graph per buffer parity (per sweep: the normals of all members, one grouped tcgen05
 * proposal GEMM over all members' tiles, one fused accept over all members' particles),
 * captured at the first temperature and replayed; other members' sweeps on their own
 * streams. Each member's arithmetic is that of the run advanced alone, except that its
 * bisection sums in one CTA. Launch shapes come from the autotuner (phi4_batch_tuning;
 * environment PHI4_TUNE=0 keeps the defaults, PHI4_TUNE_CACHE names the JSON cache file,
 * default $HOME/.cache/phi4smc_tune.json). *n_active_out = members still below beta = 1
 * afterwards. Synchronises. PHI4_ERR_DONE when no member is active. Members must have
 * flags == 0. */
phi4_status smc_temper_step_batch(phi4_run* batch, int32_t* n_active_out);

/* The launch shapes the batch's autotuner chose at its first temperature, as a JSON
 * object (each with its source: "measured", "cache" or "default"; the cache file; whether
 * the sweeps run as a captured CUDA graph), into `out` (host, `cap` bytes). "{}" before
 * the first smc_temper_step_batch. The tuned shapes (CTAs of the grouped proposal GEMM,
 * threads of the batched normals and gather) change no result. */
phi4_status phi4_batch_tuning(const phi4_run* batch, char* out, size_t cap);

/* Borrowed handle of member r for smc_log_evidence / smc_observables /
 * smc_copy_particles (owned by the batch; smc_free on it is rejected). */
phi4_status phi4_batch_member(phi4_run* batch, int32_t r, phi4_run** member_out);

/* ------------------------------------------------------------------------ */
/* Kernel-level API: each step of the path on caller buffers.                */
/* All enqueue on `stream` and return immediately unless stated.             */
/* ------------------------------------------------------------------------ */

/* Standard normals out[r*ld + j] for r < n_rows, j < n_cols, from Philox with
 * counter (kind << 24 | step, sub, row0 + r, j / 4): outputs (0,1) and (2,3) of
 * each block are Box-Muller pairs. dtype F64: uniforms from 32-bit words,
 * u1 = (w+1) 2^-32, u2 = w 2^-32, evaluated in double. F32/BF16: uniforms from
 * the top 24 bits, evaluated in float (BF16: rounded to nearest). `out` device. */
phi4_status phi4_philox_normals(uint64_t seed, uint64_t stream_id, int32_t kind, uint32_t step, uint32_t sub,
                                int32_t row0, int32_t n_rows, int32_t n_cols, int32_t ld, int32_t dtype,
                                void* out, void* stream);

/* Action (Eq. (1), coefficient form) and squared norm of N fields:
 * S[i], sq[i] (device double) from phi (device, [N][D], dtype F64 or F32).
 * F32 fields: per-site terms in float, compensated float partial sums, double total. */
phi4_status phi4_action(const void* phi, int32_t dtype, int32_t N, int32_t L, double m2, double lambda,
                        double c_kin, double c_mass, double* S, double* sq, void* stream);

/* Scratch bytes for phi4_ess_bisect with N weights. */
size_t phi4_bisect_scratch_bytes(int32_t N);

/* Next temperature and reweighting (Sec. 2 (i)): with a_i = ell_i - max ell,
 * ESS(d) = (sum e^{d a})^2 / sum e^{2 d a}; if ESS(1-beta) >= rho N then
 * dbeta = 1-beta, else bisection on [0, 1-beta] (at most `iters` halvings, stops
 * when the bracket cannot shrink) returns the lower end. Then writes
 * w[i] = exp(dbeta a_i) (device, max weight 1) and
 * out[0] = dbeta, out[1] = beta + dbeta (exactly 1 when the last step),
 * out[2] = ESS(dbeta), out[3] = log Z increment = dbeta max ell + log sum w - log N,
 * out[4] = number of bisection halvings. ell, beta_in, w, out: device.
 * One cooperative launch over several CTAs with a bounded grid barrier;
 * `scratch` (device, phi4_bisect_scratch_bytes) is zeroed by the call. */
phi4_status phi4_ess_bisect(const double* ell, int32_t N, const double* beta_in, double rho, int32_t iters,
                            double* w, double* out, void* scratch, size_t scratch_bytes, void* stream);

/* Scratch bytes for phi4_resample_systematic with N weights. */
size_t phi4_resample_scratch_bytes(int32_t N);

/* Systematic resampling in fixed point (a reading of Sec. 2 (i); bit-exact):
 * q_i = floor(ldexp(w_i / max w, 46)), C_j = sum_{k<=j} q_k, Q = C_{N-1},
 * p_i = floor((i 2^32 + U) Q / (N 2^32)), anc[i] = min{ j : C_j > p_i }.
 * w (device double, >= 0, max > 0), anc (device int32, nondecreasing), N <= 131072.
 * `scratch` (device, phi4_resample_scratch_bytes). */
phi4_status phi4_resample_systematic(const double* w, int32_t N, uint32_t U, int32_t* anc,
                                     void* scratch, size_t scratch_bytes, void* stream);

/* Same systematic resampling as phi4_resample_systematic, for callers that cannot
 * allocate device memory and have no scratch buffer to pass: for example code that
 * only receives the weight and ancestor buffers from a host framework whose allocator
 * owns the device memory, or a latency-critical loop that must not enter any
 * allocator. The paper has no counterpart; this entry point only changes where the
 * scratch lives. It allocates nothing: its N 64-bit prefix sums use an array of
 * PHI4_RESAMPLE_STATIC_MAX_N words (512 KiB) built into the library, which every GPU
 * that loads the library keeps until the process exits.
 * w: device double[N] (>= 0, max > 0); anc: device int32[N]; stream as elsewhere.
 * N > PHI4_RESAMPLE_STATIC_MAX_N returns PHI4_ERR_ARG (use phi4_resample_systematic).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress
 * with that device current) and caches it; make that first call before any stream
 * capture. A cudaDeviceReset of that device discards the array and with it the cached
 * address: do not call this entry point on the device after such a reset. All calls share the one array and it keeps the last call's contents (each
 * launch writes every entry it reads, so nothing needs clearing): calls that overlap
 * on the GPU, e.g. on two streams, race and must be serialised by the caller. */
#define PHI4_RESAMPLE_STATIC_MAX_N 65536
phi4_status phi4_resample_systematic_static(const double* w, int32_t N, uint32_t U, int32_t* anc, void* stream);

/* Exact covariance of the Gaussian part of the tempered target at beta = *d_beta (device
 * double): the log density -beta S - (1-beta) |phi|^2 / 2 (keep_reference: -|phi|^2 / 2 -
 * beta S) has the quadratic part -(1/2) phi^T P phi with P = a I + 2 beta (c_kin K +
 * c_mass m2 I), K the lattice Laplacian form of Eq. (1)'s kinetic term, a = 1 - beta (1
 * with the reference kept); sigma (device double [D][D], D = L*L, every element written)
 * = P^{-1}, formed from P's Fourier eigenvalues a + 2 beta (c_kin sum_mu 4 sin^2(pi k_mu /
 * L) + c_mass m2) as a function of the site displacement, in FP64. Needs c_mass m2 > 0
 * (P is then positive definite for every beta in [0, 1]). `scratch` (device,
 * phi4_free_covariance_scratch_bytes(L)). The free field's covariance (lambda = 0) along
 * the tempering path of Sec. 2; used by PHI4_FLAG_FREE_KERNEL_COV. */
size_t phi4_free_covariance_scratch_bytes(int32_t L);
phi4_status phi4_free_field_covariance(int32_t L, const double* d_beta, double m2, double c_kin, double c_mass,
                                       int32_t keep_reference, double* sigma, void* scratch, size_t scratch_bytes,
                                       void* stream);

/* Population observables on the device (Sec. 2: magnetisation M = (1/D) sum_x phi_x;
 * App. F: mode balance): M[i] (device double[N]) of each field of phi (device [N][D],
 * D = L*L, dtype F64 or F32), then, with weights w (device double[N], >= 0, positive
 * sum; NULL for uniform weights) normalised by their sum, out (device double[6]):
 * out[0] = <M>, out[1] = <|M|>, out[2] = <M^2>, out[3] = chi = D (<M^2> - <M>^2),
 * out[4] = mode balance = weight of M > 0 over weight of M < 0 (zeros ignored; +inf
 * when no M < 0, NaN when neither side has weight), out[5] = the sum of the weights.
 * FP64 sums in a fixed order (deterministic). smc_observables uses this reduction. */
phi4_status phi4_observables(const void* phi, int32_t dtype, int32_t N, int32_t L, const double* w, double* M,
                             double* out, void* stream);

/* Particle gather after resampling (Sec. 2 (i)):
 * dst row i = src row anc[i] for i < N, rows of `row_bytes` (device buffers;
 * dst and src must not overlap). */
phi4_status phi4_gather_rows(const void* src, void* dst, size_t row_bytes, int32_t N, const int32_t* anc,
                             void* stream);

/* Scratch bytes for phi4_covariance. */
size_t phi4_covariance_scratch_bytes(int32_t N, int32_t D, int32_t precision);

/* Particle covariance (App. A): Sigma = Xc^T Xc / (N-1), Xc = phi - mean, lower
 * triangle (j <= i) of the row-major D x D double matrix `sigma` (device); the
 * strictly upper part is left untouched. precision FP64 / FP32: SIMT GEMM in that
 * type (phi dtype F64 / F32). MIXED_BF16 (phi F32): site j's centred fields are
 * rounded to integers v = rint(x 2^s_j) with s_j set by the site's largest deviation
 * so that |v| <= 2^B, B = min(14, 23 - ceil(log2 N)); each v is split into two
 * digits held exactly in bf16, and the digit planes' Gram matrices are formed on the
 * tcgen05 tensor cores, whose fp32 sums of integer digit products stay within the
 * integers fp32 holds exactly, then combined and scaled in double: sigma is the covariance of the
 * rounded fields, positive semi-definite by construction. A device-side anomaly is
 * returned as a status code; the call synchronises `stream`. */
phi4_status phi4_covariance(const void* phi, int32_t precision, int32_t N, int32_t D, double* sigma,
                            void* scratch, size_t scratch_bytes, void* stream);

/* Cholesky factor of the particle covariance, which scales the random-walk proposal
 * (App. A). In-place A = L L^T (+ ridge): on entry the lower triangle of the
 * row-major D x D double matrix `a` (device) holds Sigma; `*d_ridge` (device
 * double) is added to its diagonal; on exit the lower triangle holds L and the
 * strictly upper triangle is zeroed. A non-positive pivot sets bit 2 of
 * `*d_status` (device uint32) and stops the factorisation. Blocked right-looking
 * with 64 x 64 blocks; the inverses of the diagonal blocks (used for the panel
 * solves) and the digit planes of the tensor-core update live in `scratch` (device,
 * phi4_cholesky_scratch_bytes). `mode` as phi4_config.chol_mode: the trailing update
 * A22 -= P P^T either in FP64 on the SIMT pipes, or exactly emulated on the tcgen05
 * tensor cores (each panel row split into eight 7-bit integer digits under a per-row
 * power of two, digit products summed exactly in fp32 by weight, recombined in
 * double-float and subtracted in FP64; error comparable to a length-64 FP64 dot
 * product). Diagonal blocks and panel solves are always FP64. */
size_t phi4_cholesky_scratch_bytes(int32_t D);
phi4_status phi4_cholesky(double* a, int32_t D, const double* d_ridge, uint32_t* d_status, void* scratch,
                          size_t scratch_bytes, int32_t mode, void* stream);

/* The same factorisation in float for the plain FP32 form: `sigma` (device double,
 * lower triangle read) is rounded to float into `a` (device float[D*D], row-major),
 * *d_ridge is added to the diagonal and `a` is factorised in place (lower L, zeros
 * above). Non-positive pivot: bit 2 of *d_status. */
phi4_status phi4_cholesky_f32(const double* sigma, float* a, int32_t D, const double* d_ridge, uint32_t* d_status,
                              void* scratch, size_t scratch_bytes, void* stream);

/* Random-walk proposal (App. A): prop = phi + scale * Z L^T with Z the normals of
 * (PHI4_RNG_PROPOSE, step, sweep, particle, block) drawn for this call.
 * precision FP64/FP32: L double/float [D][D] lower (device), SIMT GEMM.
 * MIXED_BF16: L bf16 [D][ldl] (ldl >= D, multiple of 8); the tcgen05 GEMM (bf16
 * operands, fp32 accumulation) writes the increment scale * Z L^T rounded to fp16,
 * and prop = phi + that increment (the run pipeline instead hands the increment to
 * phi4_rw_accept_delta). phi, prop: device [N][D] (F64 for FP64, else F32).
 * `scratch` holds Z (and the fp16 increment) (phi4_propose_scratch_bytes). */
size_t phi4_propose_scratch_bytes(int32_t N, int32_t D, int32_t precision);
phi4_status phi4_rw_propose(const void* phi, void* prop, const void* Lfac, int32_t ldl, int32_t precision,
                            int32_t N, int32_t D, double scale, uint64_t seed, uint64_t stream_id,
                            uint32_t step, uint32_t sweep, void* scratch, size_t scratch_bytes, void* stream);

/* Metropolis accept step (Sec. 2 tempering; App. A): for every particle,
 * S', |phi'|^2 of prop; log alpha = -beta (S' - S) - (1-beta)(|phi'|^2 - |phi|^2)/2
 * (keep_reference: -beta (S'-S) - (|phi'|^2-|phi|^2)/2) in double; u from
 * (PHI4_RNG_ACCEPT, step, sweep, particle, 0), words 0 and 1 as a 53-bit uniform
 * in (0,1]; accept iff log u < log alpha, then phi row := prop row, S, sq and
 * ell (tempering log-weight) updated. *beta (device double) is read on the device.
 * acc_count: device uint32[2]; [0] is incremented by the number of accepted
 * moves, bit 0 of [1] is set when an action is not finite (that move is rejected). */
phi4_status phi4_rw_accept(void* phi, const void* prop, int32_t dtype, int32_t N, int32_t L, double m2,
                           double lambda, double c_kin, double c_mass, int32_t keep_reference,
                           double* S, double* sq, double* ell, const double* beta, uint64_t seed,
                           uint64_t stream_id, uint32_t step, uint32_t sweep, uint32_t* acc_count, void* stream);

/* The accept step of the mixed form: as phi4_rw_accept with float fields and the
 * proposal phi' = phi + delta, delta the fp16 increment (device __half [N][D]) of the
 * tensor-core proposal; phi' is formed while phi is loaded, so neither phi' nor the
 * full-precision increment is stored. Requires L % 4 == 0 (float4 site groups within
 * a lattice row) and D <= 8192. acc_count: device uint32[2] as for phi4_rw_accept. */
phi4_status phi4_rw_accept_delta(float* phi, const void* delta_f16, int32_t N, int32_t L, double m2, double lambda,
                                 double c_kin, double c_mass, int32_t keep_reference, double* S, double* sq,
                                 double* ell, const double* beta, uint64_t seed, uint64_t stream_id, uint32_t step,
                                 uint32_t sweep, uint32_t* acc_count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PHI4SMC_H */
