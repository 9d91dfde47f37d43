// Batched form: many independent SMC runs (different lattice sizes, particle counts,
// couplings, arithmetic forms) advanced one temperature at a time together. Each stage of
// a temperature is one launch over all member runs:
//   front (batch stream): ESS bisection + reweighting + Kahan log Z (one CTA per run),
//     systematic resampling (one CTA per run), particle gather (all runs' rows);
//   refit (each run's own stream, overlapping): covariance, ridge, FP64 Cholesky;
//   back (batch stream): per sweep, proposal normals of all runs, the grouped tcgen05
//     proposal GEMM over all runs' tiles, the fused accept over all runs' particle blocks,
//     for the mixed-form members with L % 4 == 0 (their sweeps are captured once per
//     buffer parity in a CUDA graph and replayed at every temperature; each kernel reads
//     the run's temperature counter and participation from the run's device scalars);
//     the other members' sweeps are enqueued per run on their own streams.
// Launch shapes that do not change any result (CTAs of the grouped GEMM, threads of the
// normals and gather kernels) are chosen by a small autotuner that times each candidate on
// the batch's own buffers at its first temperature and remembers the choice in a JSON
// file (PHI4_TUNE_CACHE, else $HOME/.cache/phi4smc_tune.json; PHI4_TUNE=0 keeps the
// defaults). Every member follows the same arithmetic as the run advanced alone, except
// that its ESS bisection sums in one CTA.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "batch.h"
#include "bisect.cuh"
#include "resample.cuh"
#include "run.h"

namespace phi4 {

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// ----------------------------------------------------------------- front kernels

// Per run: whether it takes part (beta below 1), the temperature counter, the bisection
// for the next beta with the weights and the log-evidence increment, then Kahan log Z.
__global__ void __launch_bounds__(kBisectThreads) batch_bisect_kernel(const BatchRun* __restrict__ runs) {
  const BatchRun& b = runs[blockIdx.x];
  double* sc = b.scal;
  __shared__ int active;
  if (threadIdx.x == 0) {
    active = sc[SC_BETA] < 1.0;
    sc[SC_ACTIVE] = active ? 1.0 : 0.0;
    if (active) {
      sc[SC_T] += 1.0;
      b.acc[0] = 0u;
      b.bar[0] = 0u;
      b.bar[1] = 0u;
    }
  }
  __syncthreads();
  if (!active) return;
  GridSync gs{b.bar, b.bar + 1, b.part, b.status};
  bisect_body<32>(b.ell_src, b.ap.N, sc + SC_BETA, b.rho, b.iters, b.w, sc + SC_OUT, gs, 1, 0);
  __syncthreads();
  if (threadIdx.x == 0) logz_accumulate(sc + SC_OUT, sc + SC_KAHAN, sc + SC_BETA);
}

// Per run: the resampling offset word (PHI4_RNG_RESAMPLE, t) and the ancestors.
__global__ void __launch_bounds__(kResampleThreads) batch_resample_kernel(const BatchRun* __restrict__ runs) {
  const BatchRun& b = runs[blockIdx.x];
  if (b.scal[SC_ACTIVE] == 0.0) return;
  const uint32_t t = (uint32_t)b.scal[SC_T];
  const uint32_t U = philox4x32_10(make_uint4(counter_word0(RNG_RESAMPLE, t), 0u, 0u, 0u), b.key).x;
  resample_body(b.w, b.ap.N, U, b.anc, b.csum);
}

// Row gr of all runs (grid y) -> run r by its row offset; dst row = src row anc[row], in
// 16-byte words when the row allows, and the per-particle S, |phi|^2, ell alike.
__global__ void batch_gather_kernel(const BatchRun* __restrict__ runs, int R, const int* __restrict__ row0,
                                    int total_rows) {
  for (int gr = blockIdx.y; gr < total_rows; gr += gridDim.y) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (row0[mid] <= gr) lo = mid; else hi = mid - 1;
    }
    const BatchRun& b = runs[lo];
    if (b.scal[SC_ACTIVE] == 0.0) continue;
    const int r = gr - row0[lo];
    const int a = b.anc[r];
    const size_t row_bytes = (size_t)b.ap.D * (b.dtype == 0 ? 8 : 4);
    const unsigned char* s = (const unsigned char*)b.phi_src + (size_t)a * row_bytes;
    unsigned char* d = (unsigned char*)b.phi_dst + (size_t)r * row_bytes;
    if (row_bytes % 16 == 0) {
      for (size_t c = threadIdx.x; c < row_bytes / 16; c += blockDim.x)
        reinterpret_cast<uint4*>(d)[c] = reinterpret_cast<const uint4*>(s)[c];
    } else {
      for (size_t c = threadIdx.x; c < row_bytes / 4; c += blockDim.x)
        reinterpret_cast<uint32_t*>(d)[c] = reinterpret_cast<const uint32_t*>(s)[c];
    }
    if (threadIdx.x == 0) {
      b.S_dst[r] = b.S_src[a];
      b.sq_dst[r] = b.sq_src[a];
      b.ell_dst[r] = b.ell_src[a];
    }
  }
}

// Per-member results into one array: [0..7] bisection results, [8] log Z, [9] beta,
// [10] status word, [11] accepted moves of the last sweeps; the batch's own status word
// (grouped GEMM) is folded into every member's.
__global__ void batch_results_kernel(void* const* __restrict__ ptrs, int R, const uint32_t* __restrict__ bstatus,
                                     double* __restrict__ out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const double* scal = (const double*)ptrs[2 * r];
    const uint32_t* st = (const uint32_t*)ptrs[2 * r + 1];
    double* o = out + (size_t)r * 12;
    for (int k = 0; k < 8; ++k) o[k] = scal[SC_OUT + k];
    o[8] = scal[SC_KAHAN];
    o[9] = scal[SC_BETA];
    o[10] = (double)(st[0] | *bstatus);
    o[11] = (double)st[1];
  }
}

// ----------------------------------------------------------------- autotuner cache

std::string cache_path() {
  const char* p = getenv("PHI4_TUNE_CACHE");
  if (p && *p) return p;
  const char* h = getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/phi4smc_tune.json";
}

// The cache is a flat JSON object of "key": integer pairs.
std::map<std::string, long> cache_read(const std::string& path) {
  std::map<std::string, long> m;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return m;
  std::string s;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
  fclose(f);
  size_t i = 0;
  while ((i = s.find('"', i)) != std::string::npos) {
    const size_t j = s.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = s.substr(i + 1, j - i - 1);
    const size_t c = s.find(':', j);
    if (c == std::string::npos) break;
    m[key] = strtol(s.c_str() + c + 1, nullptr, 10);
    i = s.find_first_of(",}", c);
    if (i == std::string::npos) break;
  }
  return m;
}

void cache_write(const std::string& path, const std::map<std::string, long>& m) {
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // may exist already
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;  // the cache is an optimisation: an unwritable path only loses it
  fprintf(f, "{\n");
  size_t k = 0;
  for (const auto& kv : m) fprintf(f, "  \"%s\": %ld%s\n", kv.first.c_str(), kv.second, ++k < m.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

}  // namespace

// Host state of a batch handle.
struct BatchHost {
  int R = 0;
  cudaStream_t bs = nullptr;      // the batch's own stream (capturable; the caller's may be the legacy one)
  cudaEvent_t ev = nullptr, ev_front = nullptr;
  BatchRun* runs[2] = {nullptr, nullptr};  // device descriptors per buffer parity
  GemmRun* gemm = nullptr;        // device, the vec members' proposal GEMMs
  int* grow0 = nullptr;           // device [R + 1]: gather row offsets (all members)
  int* nrow0 = nullptr;           // device [R + 1]: normals row offsets (vec members)
  int* blk0 = nullptr;            // device [R + 1]: accept block offsets (vec members)
  uint32_t* bstatus = nullptr;    // device: status word of the batched kernels
  std::vector<char> vec;          // member r takes the batched sweeps
  int n_vec = 0, total_rows = 0, vec_rows = 0, vec_blocks = 0, gemm_tiles = 0, max_d = 0, max_mcmc = 0;
  size_t accept_smem = 0;
  int64_t steps = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // tuned launch shapes
  bool tuned = false;
  int gemm_grid = 0, normal_threads = 256, gather_threads = 256;
  std::string tune_json;
};

size_t batch_header_bytes(const phi4_config* cfgs, int32_t n) {
  (void)cfgs;
  return al256((size_t)n * 12 * 8) + al256((size_t)n * 2 * 8) + 2 * al256((size_t)n * sizeof(BatchRun)) +
         al256((size_t)n * sizeof(GemmRun)) + 3 * al256((size_t)(n + 1) * sizeof(int)) + 256;
}

namespace {

phi4_status results(phi4_run* b, std::vector<double>& host) {
  BatchHost* h = b->bh;
  for (phi4_run* m : b->members) {
    CUDA_TRY(cudaEventRecord(m->join, m->stream));
    CUDA_TRY(cudaStreamWaitEvent(h->bs, m->join, 0));
  }
  batch_results_kernel<<<(h->R + 127) / 128, 128, 0, h->bs>>>(b->batch_ptrs, h->R, h->bstatus, b->batch_scalars);
  CUDA_TRY(cudaGetLastError());
  host.resize((size_t)h->R * 12);
  CUDA_TRY(cudaMemcpyAsync(host.data(), b->batch_scalars, host.size() * 8, cudaMemcpyDeviceToHost, h->bs));
  CUDA_TRY(cudaStreamSynchronize(h->bs));
  return PHI4_OK;
}

// The sweeps of the vec members, sweep by sweep: normals of every run, the grouped GEMM,
// the fused accept.
phi4_status enqueue_sweeps(BatchHost* h, int q, cudaStream_t s) {
  for (int sw = 0; sw < h->max_mcmc; ++sw) {
    CUDA_TRY(launch_batch_normals(h->runs[q], h->R, h->nrow0, h->vec_rows, h->max_d, (uint32_t)sw,
                                  h->normal_threads, s));
    CUDA_TRY(launch_grouped_propose(h->gemm, h->n_vec, h->gemm_tiles, h->gemm_grid, (uint32_t)sw, h->bstatus, s));
    CUDA_TRY(launch_batch_accept(h->runs[q], h->R, h->blk0, h->vec_blocks, h->accept_smem, (uint32_t)sw, s));
  }
  return PHI4_OK;
}

// Times `launch` (idempotent on the batch's current buffers) three times per candidate and
// returns the fastest candidate.
template <class F>
int pick(cudaStream_t s, const std::vector<int>& cands, F launch) {
  cudaEvent_t a, z;
  cudaEventCreate(&a);
  cudaEventCreate(&z);
  int best = cands[0];
  float best_ms = 1e30f;
  for (int c : cands) {
    launch(c);  // warm-up
    cudaEventRecord(a, s);
    for (int k = 0; k < 3; ++k) launch(c);
    cudaEventRecord(z, s);
    cudaEventSynchronize(z);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, z) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  (void)cudaGetLastError();
  return best;
}

// Launch shapes for this batch: from the cache, else measured now (at the first
// temperature's sweeps, on the batch's buffers; every candidate computes the same values).
phi4_status tune(phi4_run* b, int q) {
  BatchHost* h = b->bh;
  h->tuned = true;
  h->gemm_grid = sm_count();
  const char* env = getenv("PHI4_TUNE");
  const bool on = !(env && env[0] == '0');
  int dev = 0;
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  std::string sig;
  {
    std::vector<std::string> parts;
    for (phi4_run* m : b->members) {
      char t[64];
      snprintf(t, sizeof(t), "%dx%dp%d", m->cfg.L, m->cfg.N, m->cfg.precision);
      parts.push_back(t);
    }
    std::sort(parts.begin(), parts.end());
    for (auto& t : parts) sig += t + ",";
  }
  const std::string key0 = std::string(prop.name) + "|";
  const std::string path = cache_path();
  std::map<std::string, long> cache = on ? cache_read(path) : std::map<std::string, long>();
  bool measured = false;
  auto get = [&](const char* stage, const std::vector<int>& cands, auto launch, int& out) {
    const std::string key = key0 + stage + "|" + sig;
    auto it = cache.find(key);
    if (it != cache.end() && std::find(cands.begin(), cands.end(), (int)it->second) != cands.end()) {
      out = (int)it->second;
      return std::string("cache");
    }
    if (!on) return std::string("default");
    out = pick(h->bs, cands, launch);
    cache[key] = out;
    measured = true;
    return std::string("measured");
  };
  const int S = sm_count();
  std::string src_g = "none", src_n = "none", src_a = "none";
  if (h->n_vec > 0) {
    src_g = get("gemm_ctas", {S, S * 3 / 4, S / 2}, [&](int c) {
      launch_grouped_propose(h->gemm, h->n_vec, h->gemm_tiles, c, 0u, h->bstatus, h->bs);
    }, h->gemm_grid);
    src_n = get("normals_threads", {64, 128, 256}, [&](int c) {
      launch_batch_normals(h->runs[q], h->R, h->nrow0, h->vec_rows, h->max_d, 0u, c, h->bs);
    }, h->normal_threads);
  }
  src_a = get("gather_threads", {128, 256, 512}, [&](int c) {
    const int gy = std::min(h->total_rows, 65535);
    // the gather of the current parity reads src and writes dst: rerunning it is harmless
    batch_gather_kernel<<<dim3(1, (unsigned)std::max(gy, 1)), c, 0, h->bs>>>(h->runs[q], h->R, h->grow0,
                                                                             h->total_rows);
  }, h->gather_threads);
  CUDA_TRY(cudaStreamSynchronize(h->bs));
  if (measured) cache_write(path, cache);
  char js[512];
  snprintf(js, sizeof(js),
           "{\"gemm_ctas\": %d, \"gemm_ctas_source\": \"%s\", \"normals_threads\": %d, "
           "\"normals_threads_source\": \"%s\", \"gather_threads\": %d, \"gather_threads_source\": \"%s\", "
           "\"cache\": \"%s\", \"graph\": %s}",
           h->gemm_grid, src_g.c_str(), h->normal_threads, src_n.c_str(), h->gather_threads, src_a.c_str(),
           path.c_str(), h->n_vec > 0 ? "true" : "false");
  h->tune_json = js;
  return PHI4_OK;
}

}  // namespace

void batch_release(phi4_run* b) {
  BatchHost* h = b->bh;
  if (!h) return;
  if (h->bs) cudaStreamSynchronize(h->bs);
  for (auto& g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->ev_front) cudaEventDestroy(h->ev_front);
  if (h->bs) cudaStreamDestroy(h->bs);
  delete h;
  b->bh = nullptr;
}

}  // namespace phi4

using namespace phi4;

extern "C" {

phi4_status phi4_batch_workspace_bytes(const phi4_config* cfgs, int32_t n_runs, size_t* bytes) {
  ARG_CHECK(cfgs && bytes, "NULL argument");
  ARG_CHECK(n_runs >= 1 && n_runs <= 4096, "n_runs = %d outside [1, 4096]", n_runs);
  size_t tot = batch_header_bytes(cfgs, n_runs);
  for (int r = 0; r < n_runs; ++r) {
    size_t b = 0;
    phi4_status st = phi4_workspace_bytes(&cfgs[r], &b);
    if (st != PHI4_OK) return st;
    ARG_CHECK(cfgs[r].kind == PHI4_SMC_RW, "batch member %d: only SMC runs are batched", r);
    ARG_CHECK(cfgs[r].N <= 4096, "batch member %d: N = %d above the 4096 of a one-CTA bisection", r, cfgs[r].N);
    ARG_CHECK(cfgs[r].flags == 0, "batch member %d: flags are not supported in a batch", r);
    tot += al256(b);
  }
  *bytes = tot;
  return PHI4_OK;
}

phi4_status smc_init_batch(const phi4_config* cfgs, int32_t n_runs, void* d_ws, size_t ws_bytes, void* stream,
                           phi4_run** out) {
  ARG_CHECK(out, "out is NULL");
  size_t need = 0;
  phi4_status ps = phi4_batch_workspace_bytes(cfgs, n_runs, &need);
  if (ps != PHI4_OK) return ps;
  ARG_CHECK(d_ws && ((uintptr_t)d_ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) {
    set_error("workspace of %zu bytes, need %zu", ws_bytes, need);
    return PHI4_ERR_WORKSPACE;
  }
  phi4_run* b = new phi4_run();
  b->batch = true;
  b->cfg = cfgs[0];
  b->stream = (cudaStream_t)stream;
  BatchHost* h = new BatchHost();
  b->bh = h;
  h->R = n_runs;
  const int R = n_runs;
  unsigned char* base = (unsigned char*)d_ws;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += al256(bytes);
    return p;
  };
  b->batch_scalars = (double*)take((size_t)R * 12 * 8);
  b->batch_ptrs = (void**)take((size_t)R * 2 * 8);
  h->runs[0] = (BatchRun*)take((size_t)R * sizeof(BatchRun));
  h->runs[1] = (BatchRun*)take((size_t)R * sizeof(BatchRun));
  h->gemm = (GemmRun*)take((size_t)R * sizeof(GemmRun));
  h->grow0 = (int*)take((size_t)(R + 1) * sizeof(int));
  h->nrow0 = (int*)take((size_t)(R + 1) * sizeof(int));
  h->blk0 = (int*)take((size_t)(R + 1) * sizeof(int));
  h->bstatus = (uint32_t*)take(16);
  off = batch_header_bytes(cfgs, R);
  auto fail = [&](phi4_status st) {
    smc_free(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&h->bs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_front, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
    set_error("batch stream or events: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(PHI4_ERR_CUDA);
  }
  std::vector<void*> ptrs((size_t)R * 2);
  for (int r = 0; r < R; ++r) {
    size_t bytes = 0;
    phi4_workspace_bytes(&cfgs[r], &bytes);
    cudaStream_t ms = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking);
    phi4_run* m = nullptr;
    if (e == cudaSuccess) ps = smc_init(&cfgs[r], base + off, bytes, ms, &m);
    if (e != cudaSuccess || ps != PHI4_OK) {
      if (e != cudaSuccess) set_error("member stream: %s", cudaGetErrorString(e));
      if (ms) cudaStreamDestroy(ms);
      return fail(e != cudaSuccess ? PHI4_ERR_CUDA : ps);
    }
    m->owner = b;
    m->owns_stream = true;
    cudaEventCreateWithFlags(&m->join, cudaEventDisableTiming);
    b->members.push_back(m);
    ptrs[2 * r] = m->scal;
    ptrs[2 * r + 1] = m->status;
    off += al256(bytes);
  }
  // descriptors of both buffer parities, the row / block / tile offsets and the GEMM maps
  std::vector<BatchRun> d0(R), d1(R);
  std::vector<int> grow(R + 1, 0), nrow(R + 1, 0), blk(R + 1, 0);
  std::vector<GemmRun> gm;
  h->vec.assign(R, 0);
  for (int r = 0; r < R; ++r) {
    phi4_run* m = b->members[r];
    const phi4_config& c = m->cfg;
    BatchRun d;
    memset(&d, 0, sizeof(d));
    d.ap = action_params(m);
    d.key = philox_key(c.seed, c.stream_id);
    d.rho = c.ess_target;
    d.iters = c.bisect_iters;
    d.keep_ref = c.keep_reference;
    d.dtype = m->dtype;
    d.zdtype = m->zdtype;
    d.ldz = m->ldz;
    d.w = m->w;
    d.scal = m->scal;
    d.anc = m->anc;
    d.csum = (unsigned long long*)m->resample_scratch;
    d.bar = (unsigned*)m->bisect_scratch;
    d.part = (double*)((unsigned char*)m->bisect_scratch + 256);
    d.status = m->status;
    d.acc = m->acc_count;
    d.Z = m->Z;
    d.delta = (const __half*)m->prop;
    const bool vec = c.precision == PHI4_MIXED_BF16 && c.L % 4 == 0 && m->D <= 8192 && m->Z2;
    h->vec[r] = vec;
    d.n_mcmc = vec ? c.n_mcmc : 0;
    accept_vec_shape(m->D, &d.ppb, &d.tpp);
    // parity 0 gathers from the initial buffers into the alternates, parity 1 back
    BatchRun a = d, z = d;
    a.phi_src = m->phi; a.phi_dst = m->phi_alt;
    a.S_src = m->S; a.S_dst = m->S_alt; a.sq_src = m->sq; a.sq_dst = m->sq_alt; a.ell_src = m->ell; a.ell_dst = m->ell_alt;
    z.phi_src = m->phi_alt; z.phi_dst = m->phi;
    z.S_src = m->S_alt; z.S_dst = m->S; z.sq_src = m->sq_alt; z.sq_dst = m->sq; z.ell_src = m->ell_alt; z.ell_dst = m->ell;
    d0[r] = a;
    d1[r] = z;
    grow[r + 1] = grow[r] + c.N;
    nrow[r + 1] = nrow[r] + (vec ? c.N : 0);
    blk[r + 1] = blk[r] + (vec ? (c.N + d.ppb - 1) / d.ppb : 0);
    if (vec) {
      GemmRun g;
      memset(&g, 0, sizeof(g));
      if (!make_gemm_run(&g, m->Z, m->ldz, m->Lg, m->ldl, c.N, m->D, (float)m->scale, (__half*)m->prop, m->scal,
                         c.n_mcmc)) {
        set_error("batch member %d: tensor map of the proposal operands", r);
        return fail(PHI4_ERR_CUDA);
      }
      g.tile0 = h->gemm_tiles;
      h->gemm_tiles += g.tiles_m * g.tiles_n;
      gm.push_back(g);
      h->n_vec += 1;
      h->max_d = std::max(h->max_d, m->D);
      h->max_mcmc = std::max(h->max_mcmc, c.n_mcmc);
      h->accept_smem = std::max(h->accept_smem, (size_t)d.ppb * m->D * sizeof(float));
    }
  }
  h->total_rows = grow[R];
  h->vec_rows = nrow[R];
  h->vec_blocks = blk[R];
  if (h->n_vec > 0) {
    // kernel attributes are set here, outside the sweeps' stream capture
    cudaError_t e = batch_accept_prepare(h->accept_smem);
    if (e == cudaSuccess) e = grouped_propose_prepare();
    if (e != cudaSuccess) {
      set_error("batched kernels: %s", cudaGetErrorString(e));
      return fail(PHI4_ERR_CUDA);
    }
  }
  cudaStream_t s = h->bs;
  bool ok = cudaMemcpyAsync(b->batch_ptrs, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice, s) ==
                cudaSuccess &&
            cudaMemcpyAsync(h->runs[0], d0.data(), R * sizeof(BatchRun), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(h->runs[1], d1.data(), R * sizeof(BatchRun), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(h->grow0, grow.data(), (R + 1) * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(h->nrow0, nrow.data(), (R + 1) * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(h->blk0, blk.data(), (R + 1) * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemsetAsync(h->bstatus, 0, 16, s) == cudaSuccess &&
            (gm.empty() || cudaMemcpyAsync(h->gemm, gm.data(), gm.size() * sizeof(GemmRun), cudaMemcpyHostToDevice,
                                           s) == cudaSuccess);
  // the host vectors must outlive the copies
  if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
  for (phi4_run* m : b->members) ok = ok && cudaStreamSynchronize(m->stream) == cudaSuccess;
  if (!ok) {
    set_error("batch descriptors: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(PHI4_ERR_CUDA);
  }
  *out = b;
  return PHI4_OK;
}

phi4_status smc_temper_step_batch(phi4_run* b, int32_t* n_active_out) {
  ARG_CHECK(b && b->batch && b->bh, "not a batch handle");
  BatchHost* h = b->bh;
  std::vector<phi4_run*> act;
  for (phi4_run* m : b->members)
    if (!m->done) act.push_back(m);
  if (act.empty()) {
    if (n_active_out) *n_active_out = 0;
    set_error("every run of the batch is at beta = 1");
    return PHI4_ERR_DONE;
  }
  const int q = (int)(h->steps & 1);
  cudaStream_t s = h->bs;
  // the batch starts after the caller's earlier work
  CUDA_TRY(cudaEventRecord(h->ev, b->stream));
  CUDA_TRY(cudaStreamWaitEvent(s, h->ev, 0));
  // front: bisection + reweighting + log Z, resampling, gather (every active run)
  batch_bisect_kernel<<<h->R, kBisectThreads, 0, s>>>(h->runs[q]);
  CUDA_TRY(cudaGetLastError());
  batch_resample_kernel<<<h->R, kResampleThreads, 0, s>>>(h->runs[q]);
  CUDA_TRY(cudaGetLastError());
  batch_gather_kernel<<<dim3(1, (unsigned)std::max(1, std::min(h->total_rows, 65535))), h->gather_threads, 0, s>>>(
      h->runs[q], h->R, h->grow0, h->total_rows);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(h->ev_front, s));
  for (phi4_run* m : act) {
    m->t += 1;
    m->kernel_launches += 3;
    std::swap(m->phi, m->phi_alt);
    std::swap(m->S, m->S_alt);
    std::swap(m->sq, m->sq_alt);
    std::swap(m->ell, m->ell_alt);
  }
  b->kernel_launches += 3;
  // refit on each run's stream: covariance, ridge, the first factorisation attempt
  phi4_status ps;
  for (phi4_run* m : act) {
    CUDA_TRY(cudaStreamWaitEvent(m->stream, h->ev_front, 0));
    if ((ps = refit_enqueue(m, m->phi, m->cfg.N)) != PHI4_OK) return ps;
  }
  std::vector<double> res;
  if ((ps = results(b, res)) != PHI4_OK) return ps;
  for (phi4_run* m : act) {
    const size_t i = (size_t)(std::find(b->members.begin(), b->members.end(), m) - b->members.begin());
    if ((ps = refit_check(m, (uint32_t)res[i * 12 + 10])) != PHI4_OK) return ps;
  }
  // back: the vec members' sweeps on the batch stream, the others' on their own streams
  for (size_t i = 0; i < b->members.size(); ++i) {
    phi4_run* m = b->members[i];
    if (m->done || !h->vec[i]) continue;
    CUDA_TRY(cudaEventRecord(m->join, m->stream));
    CUDA_TRY(cudaStreamWaitEvent(s, m->join, 0));
    m->n_evals += (int64_t)m->cfg.N * m->cfg.n_mcmc;
    m->kernel_launches += 3 * m->cfg.n_mcmc;
  }
  // the autotuner reruns this step's gather (into buffers nothing else touches until the
  // sweeps below) and the vec members' normals and GEMM (both recomputed by the sweeps)
  if (!h->tuned && (ps = tune(b, q)) != PHI4_OK) return ps;
  for (size_t i = 0; i < b->members.size(); ++i) {
    phi4_run* m = b->members[i];
    if (m->done || h->vec[i]) continue;
    if ((ps = step_back(m)) != PHI4_OK) return ps;
  }
  if (h->n_vec > 0) {
    if (!h->graph[q]) {
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      ps = enqueue_sweeps(h, q, s);
      const cudaError_t e = cudaStreamEndCapture(s, &g);
      if (ps != PHI4_OK) {
        if (g) cudaGraphDestroy(g);
        return ps;
      }
      CUDA_TRY(e);
      const cudaError_t ei = cudaGraphInstantiate(&h->graph[q], g, 0);
      cudaGraphDestroy(g);
      CUDA_TRY(ei);
    }
    CUDA_TRY(cudaGraphLaunch(h->graph[q], s));
    b->kernel_launches += 3 * h->max_mcmc;
  }
  h->steps += 1;
  if ((ps = results(b, res)) != PHI4_OK) return ps;
  int n_active = 0;
  for (size_t i = 0; i < b->members.size(); ++i) {
    phi4_run* m = b->members[i];
    if (std::find(act.begin(), act.end(), m) != act.end()) {
      const uint32_t sw[2] = {(uint32_t)res[i * 12 + 10], (uint32_t)res[i * 12 + 11]};
      if ((ps = step_finish(m, &res[i * 12], sw, nullptr)) != PHI4_OK) return ps;
    }
    if (!m->done) ++n_active;
  }
  // the caller's stream continues after the batch
  CUDA_TRY(cudaEventRecord(h->ev, s));
  CUDA_TRY(cudaStreamWaitEvent(b->stream, h->ev, 0));
  if (n_active_out) *n_active_out = n_active;
  return PHI4_OK;
}

phi4_status phi4_batch_member(phi4_run* b, int32_t r, phi4_run** member_out) {
  ARG_CHECK(b && b->batch && member_out, "not a batch handle");
  ARG_CHECK(r >= 0 && r < (int32_t)b->members.size(), "member %d outside [0, %d)", r, (int)b->members.size());
  *member_out = b->members[r];
  return PHI4_OK;
}

phi4_status phi4_batch_tuning(const phi4_run* b, char* out, size_t cap) {
  ARG_CHECK(b && b->batch && b->bh && out && cap > 0, "not a batch handle or no buffer");
  const std::string& j = b->bh->tuned ? b->bh->tune_json : std::string("{}");
  ARG_CHECK(j.size() + 1 <= cap, "buffer of %zu bytes, need %zu", cap, j.size() + 1);
  memcpy(out, j.c_str(), j.size() + 1);
  return PHI4_OK;
}

}  // extern "C"
