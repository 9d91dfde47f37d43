// tcgen05 tensor-core kernels with TMA operand staging (sm_103a):
//   proposal   increment Delta = s Z L^T stored as fp16 (Z: N x D normals, L: D x D
//              lower Cholesky factor; a 256-column tile [n0, n0+256) only needs
//              k < n0+256); the accept kernel forms Phi + Delta while it loads Phi;
//   covariance the mixed form's Sigma as the exact Gram matrix of fixed-point digits
//              (namespace gram);
//   Cholesky   the FP64 trailing update, exactly emulated with bf16 digits (namespace emu).
// Operands are bf16, K-contiguous, loaded by TMA into 128B-swizzled shared tiles; one
// elected thread issues tcgen05.mma (fp32 accumulate) into TMEM while epilogue warps
// drain the accumulators with tcgen05.ld and apply the epilogue to global memory.
// Persistent CTAs (one per SM) walk a static tile list; warp 0 = TMA producer,
// warp 1 = MMA issuer (and TMEM owner), the other warps = epilogue.
// Every mbarrier wait is bounded (about one second); a wait that gives up sets
// ST_TIMEOUT and an abort flag that stops the other roles.
#include <cuda.h>
#include <cuda_fp16.h>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include "internal.h"
#include "common.cuh"
#include "batch.h"

namespace phi4 {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;  // the grouped (batched) kernel's ring
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;
constexpr int NUM_THREADS = 192;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
// shared memory of a ring of S stages
__host__ __device__ constexpr int smem_bytes(int S) { return S * STAGE_BYTES + 1024 + 256; }

// kind::f16 instruction descriptor: D fp32 (bits 4-5 = 1), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct Params {
  int M, Nn, K;
  int tiles_m, tiles_n, num_tiles;
  __half* delta;
  float scale;
  uint32_t* status;
};

PHI4_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

PHI4_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
PHI4_DEV void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
PHI4_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
PHI4_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for completion of the phase with the given parity.
PHI4_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kSpinLimitCycles) return false;
  }
}

PHI4_DEV void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address >> 4
// (bits 0-13), leading byte offset 16 >> 4 (unused for this layout), stride byte
// offset 1024 >> 4 (8 rows x 128 B, bits 32-45), version 1 (bit 46), layout
// SWIZZLE_128B = 2 (bits 61-63). Tile bases are 1024-byte aligned.
PHI4_DEV uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

PHI4_DEV void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}
PHI4_DEV void umma_idesc(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
PHI4_DEV void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
PHI4_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
PHI4_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

PHI4_DEV void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld of 32 columns, no wait::ld (the caller waits before use)
PHI4_DEV void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
}

// One tile of the proposal GEMM as the three roles see it: the two tensor maps, the row
// and column tile, the K blocks it needs, and where and how its epilogue writes.
struct Tile {
  const CUtensorMap* ma;
  const CUtensorMap* mb_map;
  int mb, nb, kblocks, M, Nn;
  __half* delta;
  float scale;
  bool skip;  // a unit of a run that sits out this launch (all roles skip it alike)
};

// Tiles of one run. Column tiles are walked in decreasing K extent (heaviest first); the
// row tiles of one column tile are consecutive units, so CTAs working at the same time
// share the factor tile in L2. A column tile [n0, n0 + BN) needs only k < n0 + BN.
struct SingleTiles {
  const CUtensorMap* ma;
  const CUtensorMap* mb_map;
  const Params* p;
  PHI4_DEV Tile get(int u) const {
    Tile t;
    t.ma = ma;
    t.mb_map = mb_map;
    t.nb = p->tiles_n - 1 - u / p->tiles_m;
    t.mb = u % p->tiles_m;
    t.kblocks = (min(p->K, (t.nb + 1) * BN) + BK - 1) / BK;
    t.M = p->M;
    t.Nn = p->Nn;
    t.delta = p->delta;
    t.scale = p->scale;
    t.skip = false;
    return t;
  }
};

// Tiles of every run of a batch: unit u belongs to the run r with tile0[r] <= u <
// tile0[r + 1] (binary search), then the run's own order as above. A run that is done
// (SC_ACTIVE == 0) or has fewer sweeps than this launch's sweep index sits out.
struct GroupedTiles {
  const GemmRun* runs;
  int R;
  uint32_t sweep;
  PHI4_DEV Tile get(int u) const {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (runs[mid].tile0 <= u) lo = mid; else hi = mid - 1;
    }
    const GemmRun& g = runs[lo];
    const int v = u - g.tile0;
    Tile t;
    t.ma = reinterpret_cast<const CUtensorMap*>(g.mapA);
    t.mb_map = reinterpret_cast<const CUtensorMap*>(g.mapB);
    t.nb = g.tiles_n - 1 - v / g.tiles_m;
    t.mb = v % g.tiles_m;
    t.kblocks = (min(g.K, (t.nb + 1) * BN) + BK - 1) / BK;
    t.M = g.M;
    t.Nn = g.Nn;
    t.delta = g.delta;
    t.scale = g.scale;
    t.skip = g.scal[SC_ACTIVE] == 0.0 || (int)sweep >= g.n_mcmc;
    return t;
  }
};

// Persistent CTAs (one per SM) walk units cid, cid + grid, ...; warp 0 = TMA producer,
// warp 1 = MMA issuer and TMEM owner, warps 2..5 = epilogue (s * acc -> fp16 Delta).
template <int S, class Tiles>
PHI4_DEV void gemm_body(const Tiles& tiles, int num_units, uint32_t* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int cid = blockIdx.x, ncl = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(status, ST_TIMEOUT);
  };

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      const CUtensorMap* last = nullptr;
      for (int u = cid; u < num_units && !*abort_flag; u += ncl) {
        const Tile t = tiles.get(u);
        if (t.skip) continue;
        if (t.ma != last) {
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)t.ma) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)t.mb_map) : "memory");
          last = t.ma;
        }
        for (int kb = 0; kb < t.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) { give_up(); break; }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          tma_load_2d(t.ma, &full[stage], sa, kb * BK, t.mb * BM);
          tma_load_2d(t.mb_map, &full[stage], sa + A_BYTES, kb * BK, t.nb * BN);
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      for (int u = cid; u < num_units && !*abort_flag; u += ncl) {
        const Tile t = tiles.get(u);
        if (t.skip) continue;
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, abort_flag)) { give_up(); break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        bool ok = true;
        for (int kb = 0; kb < t.kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) { give_up(); ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + stage * STAGE_BYTES), b0 = a0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma_bf16(d_tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), (kb | kk) != 0);
          umma_commit(&empty[stage]);
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        umma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1u;
      }
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int u = cid; u < num_units; u += ncl) {
      const Tile t = tiles.get(u);
      if (t.skip) continue;
      if (!mbar_wait(&tfull[acc], acc_phase, abort_flag)) { give_up(); break; }
      tc_fence_after();
      const int gm = t.mb * BM + r;
      const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(trow + (uint32_t)(c * 32), v);
        const int gn0 = t.nb * BN + c * 32;
        if (gm < t.M && gn0 < t.Nn) {
          const size_t o = (size_t)gm * t.Nn + gn0;
          if (gn0 + 32 <= t.Nn && (t.Nn & 7) == 0) {
            uint4* dst = reinterpret_cast<uint4*>(t.delta + o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint4 pk;
              __half2 h0 = __floats2half2_rn(t.scale * v[8 * j], t.scale * v[8 * j + 1]);
              __half2 h1 = __floats2half2_rn(t.scale * v[8 * j + 2], t.scale * v[8 * j + 3]);
              __half2 h2 = __floats2half2_rn(t.scale * v[8 * j + 4], t.scale * v[8 * j + 5]);
              __half2 h3 = __floats2half2_rn(t.scale * v[8 * j + 6], t.scale * v[8 * j + 7]);
              pk.x = *reinterpret_cast<uint32_t*>(&h0);
              pk.y = *reinterpret_cast<uint32_t*>(&h1);
              pk.z = *reinterpret_cast<uint32_t*>(&h2);
              pk.w = *reinterpret_cast<uint32_t*>(&h3);
              dst[j] = pk;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (gn0 + j < t.Nn) t.delta[o + j] = __float2half_rn(t.scale * v[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

template <int S>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Params p) {
  SingleTiles tiles{&tmA, &tmB, &p};
  gemm_body<S>(tiles, p.num_tiles, p.status);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_grouped_kernel(const GemmRun* __restrict__ runs, int R, int num_units, uint32_t sweep,
                           uint32_t* status) {
  GroupedTiles tiles{runs, R, sweep};
  gemm_body<STAGES>(tiles, num_units, status);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
  }
  return fn;
}

// 2-D bf16 tensor map over rows x inner (row pitch `ld` elements), box 64 x box_rows, 128B swizzle.
static bool make_map(CUtensorMap* map, const void* ptr, int inner, int rows, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)ptr & 15) || (ld % 8)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Ring depth of the single-run proposal GEMM: 4 stages (192 KB of shared memory);
// PHI4_PROPOSE_STAGES=3 selects a 144 KB ring, which leaves room on each SM for more of the
// fused accept running beside it on another stream (measured slower in the step: the sweeps
// of a temperature took 3.97 ms against 3.76 ms with 4 stages).
static cudaError_t launch(const CUtensorMap& a, const CUtensorMap& b, const Params& p, cudaStream_t s) {
  static const int stages = [] {
    const char* v = getenv("PHI4_PROPOSE_STAGES");
    return (v && atoi(v) == 3) ? 3 : 4;
  }();
  // persistent CTAs: one per SM, or PHI4_PROPOSE_CTAS of them (the SMs left over then run
  // the accept of the previous sweep, which overlaps the GEMM on another stream)
  static const int ctas = [] {
    const char* v = getenv("PHI4_PROPOSE_CTAS");
    return v ? std::max(1, atoi(v)) : 0;
  }();
  const int grid = std::min(ctas > 0 ? std::min(ctas, sm_count()) : sm_count(), p.num_tiles);
  if (grid < 1) return cudaSuccess;
  if (stages == 4) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(4));
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<4><<<grid, NUM_THREADS, smem_bytes(4), s>>>(a, b, p);
  } else {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(3));
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<3><<<grid, NUM_THREADS, smem_bytes(3), s>>>(a, b, p);
  }
  return cudaGetLastError();
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Mixed-form covariance as an exact Gram matrix on the tensor cores.
// The centred fields of site j are rounded to integers v = rint(x 2^s_j), |v| <= 2^B,
// and split into two digits v = 2^a h + l (small integers, exact in bf16); the digit
// planes H and L are D x N, K-contiguous. Three TMEM accumulators per 128 x 128 tile
// collect  G_hh = H H^T,  G_x = H L^T + L H^T  and  G_ll = L L^T  over the whole K = N:
// with N <= 2^c and B = 23 - c (a = ceil(B/2)) every partial sum is an integer of
// magnitude <= 2^23, so the fp32 accumulation is exact and
//   Sigma_ij = 2^(-s_i - s_j) (2^(2a) G_hh + 2^a G_x + G_ll) / (N - 1)
// is the covariance of the rounded fields up to one final FP64 rounding: positive
// semi-definite like the matrix it stands for, so the factorisation's ridge only has
// to absorb the Cholesky's own rounding. The combination is done in 64-bit integers
// and turned into a double with integer operations; one FP64 multiply per element.
// Persistent CTAs walk the lower tiles; warp 0 = TMA (four 16 KB digit tiles per
// stage), warp 1 = MMA (four MMAs per K step), warps 2..9 = epilogue (the tile's three
// accumulators use 384 of the 512 TMEM columns, so the next tile's MMAs wait for the
// epilogue to drain them).
namespace gram {
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // A_H, A_L, B_H, B_L
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int NUM_THREADS = 320;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct Params {
  int D, K, num_tiles, a;
  const int* shift;
  double inv;
  double* sigma;
  uint32_t* status;
};

// lower tile u (row block by row block: row block m holds tiles 0..m)
PHI4_DEV void get_tile(int u, int& mb, int& nb) {
  int m = 0;
  while (u > m) {
    u -= m + 1;
    ++m;
  }
  mb = m;
  nb = u;
}

// t 2^n as a double (exact for |t| < 2^53), built with integer operations.
PHI4_DEV double i64_pow2(long long t, int n) {
  if (t == 0) return 0.0;
  const unsigned long long sg = t < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  const int lz = __clzll(u);
  const int ex = 1023 + (63 - lz) + n;
  if (ex <= 0 || ex >= 2047) return ldexp((double)t, n);
  const unsigned long long man = (u << (lz - 11)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(sg | ((unsigned long long)ex << 52) | man));
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    gram_kernel(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmL, Params p) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 8);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmH) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmL) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int kblocks = (p.K + BK - 1) / BK;
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(p.status, ST_TIMEOUT);
  };
  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int u = blockIdx.x; u < p.num_tiles && !*abort_flag; u += gridDim.x) {
        int mb, nb;
        get_tile(u, mb, nb);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) { give_up(); break; }
          uint8_t* st = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          tma_load_2d(&tmH, &full[stage], st, kb * BK, mb * BM);
          tma_load_2d(&tmL, &full[stage], st + TILE_BYTES, kb * BK, mb * BM);
          tma_load_2d(&tmH, &full[stage], st + 2 * TILE_BYTES, kb * BK, nb * BN);
          tma_load_2d(&tmL, &full[stage], st + 3 * TILE_BYTES, kb * BK, nb * BN);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, tphase = 0;
      const uint32_t t_hh = tmem_base, t_x = tmem_base + BN, t_ll = tmem_base + 2 * BN;
      for (int u = blockIdx.x; u < p.num_tiles && !*abort_flag; u += gridDim.x) {
        // the epilogue has read the previous tile's accumulators
        if (!mbar_wait(tempty, tphase ^ 1u, abort_flag)) { give_up(); break; }
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) { give_up(); ok = false; break; }
          tc_fence_after();
          const uint32_t s0 = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t ah = sdesc(s0 + kk * 32), al = sdesc(s0 + TILE_BYTES + kk * 32);
            const uint64_t bh = sdesc(s0 + 2 * TILE_BYTES + kk * 32), bl = sdesc(s0 + 3 * TILE_BYTES + kk * 32);
            const uint32_t acc = (kb | kk) != 0;
            umma_idesc(t_hh, ah, bh, IDESC, acc);
            umma_idesc(t_x, ah, bl, IDESC, acc);
            umma_idesc(t_x, al, bh, IDESC, 1u);
            umma_idesc(t_ll, al, bl, IDESC, acc);
          }
          umma_commit(&empty[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        umma_commit(tfull);
        tphase ^= 1u;
      }
    }
  } else {
    // warps 2..9: lane quarter q of the accumulators, columns [grp * 64, grp * 64 + 64)
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const int a = p.a;
    uint32_t tphase = 0;
    for (int u = blockIdx.x; u < p.num_tiles; u += gridDim.x) {
      int mb, nb;
      get_tile(u, mb, nb);
      if (!mbar_wait(tfull, tphase, abort_flag)) { give_up(); break; }
      tphase ^= 1u;
      tc_fence_after();
      const int gm = mb * BM + r;
      const bool row_ok = gm < p.D;
      const int si = row_ok ? p.shift[gm] : 0;
      double* row = p.sigma + (size_t)(row_ok ? gm : 0) * p.D;
      const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        const int col = grp * 64 + c * 32;
        uint32_t hh[32], xx[32], ll[32];
        tmem_ld32_nw(trow + (uint32_t)col, hh);
        tmem_ld32_nw(trow + (uint32_t)(BN + col), xx);
        tmem_ld32_nw(trow + (uint32_t)(2 * BN + col), ll);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c == 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty);  // this warp's accumulators are in registers
        }
        const int gn0 = nb * BN + col;
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int gn = gn0 + j;
            if (gn <= gm) {
              const long long t = ((long long)__float2int_rn(__uint_as_float(hh[j])) << (2 * a)) +
                                  ((long long)__float2int_rn(__uint_as_float(xx[j])) << a) +
                                  (long long)__float2int_rn(__uint_as_float(ll[j]));
              row[gn] = i64_pow2(t, -(si + p.shift[gn])) * p.inv;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}
}  // namespace gram

// ---------------------------------------------------------------------------
// FP64 Cholesky trailing update on the tensor cores (exact digit emulation).
// A22 -= P P^T with P the 64-wide panel below the diagonal block, given as eight
// bf16 digit planes d_k (|d| < 128, exact) and row exponents e (written by the panel solve, split_row_digits):
//   (P P^T)_ij = 2^(e_i + e_j) sum_{k,l} 2^(-7(k+l)) T_kl,  T_kl = sum_n d_ik,n d_jl,n.
// Products are exact in fp32 and, grouped by c = k + l, each group sum is an integer
// below 2^23 in magnitude (at most 8 pairs x 64 terms x 2^14), so tcgen05 accumulates
// every U_c = sum_{k+l=c} T_kl exactly in TMEM. Groups c = 2..9 are kept (dropped
// groups weigh < 2^-47 of sum |x||y|, like the rounding of a length-64 FP64 dot
// product); U_9 .. U_2 are combined by a Horner pass in double-float (two fp32)
// and the result, scaled by 2^(e_i + e_j - 14), is subtracted in FP64.
// A launch covers the 64-column blocks [blk_lo, blk_hi) of the lower trailing matrix,
// each CTA a contiguous run of its tile list, so that the 128 KB of A digit planes are
// loaded once per 128-row band rather than once per tile. Two tile forms with the same
// arithmetic per element: 128 x 32 tiles (chol_update_kernel; two tiles' group
// accumulators fit in TMEM, so the MMAs of one tile overlap the epilogue of the
// previous one) for a single block column, and 128 x 64 tiles (chol_update_wide_kernel;
// N = 64 MMAs, half the shared-memory operand reads per product, the accumulators
// handed to the epilogue group by group) for the bulk of a panel's update.
namespace emu {
constexpr int BM = 128, BN = 32, KD = 64, ND = 8, NC = 8;
constexpr int A_PLANE = BM * KD * 2;
constexpr int B_PLANE = BN * KD * 2;
constexpr int SMEM_DATA = ND * (A_PLANE + B_PLANE);  // 160 KB
constexpr int EC = 8;                         // tile columns per epilogue warp
constexpr int RPP = 32 / EC;                  // rows per pass of the row-segment accesses
constexpr int NUM_EPI_WARPS = 4 * (BN / EC);  // four TMEM lane quarters x column groups
// per epilogue warp a 32 x EC FP64 patch that turns its row-per-lane products into
// row-contiguous accesses of EC lanes to the trailing matrix (coalesced loads and stores);
// element (row, col) at row EC + (col ^ swz(row)), free of bank conflicts both ways
constexpr int STAGE_BYTES = NUM_EPI_WARPS * 32 * EC * 8;
PHI4_DEV int swz(int row) { return (row >> 1) & 7; }
static_assert(EC == 8, "swz is laid out for eight columns per warp");
constexpr int SMEM_BYTES = SMEM_DATA + 256 + STAGE_BYTES + 1024;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
constexpr int ACC_COLS = NC * BN;  // one tile's eight group accumulators; two tiles fit in TMEM
constexpr int BLK_COLS = KD / BN;  // tile columns per 64-column block
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct Params {
  double* a;
  int D, b0, m, m_pad, tiles_m, tiles_n, num_tiles;
  int col_lo, col_hi;  // tile columns [col_lo, col_hi) of the lower trailing matrix
  const int* rexp;
  uint32_t* status;
};

// tcgen05.ld of 8 or 16 columns without the wait (the caller issues tmem_wait_ld before use)
PHI4_DEV void tmem_ld8_nw(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
PHI4_DEV void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
}
PHI4_DEV void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tile u of the launch's list: 128-row bands from the top, in each the lower tiles
// whose column lies in [col_lo, col_hi).
// Tile columns are TBN wide (p.tiles_n, p.col_lo and p.col_hi count them).
template <int TBN>
PHI4_DEV int band_tiles(const Params& p, int mb) {
  const int hi = min(min(p.col_hi, p.tiles_n), (mb * BM + BM - 1) / TBN + 1);
  return max(0, hi - p.col_lo);
}
template <int TBN>
PHI4_DEV void get_tile(const Params& p, int u, int& mb, int& bj) {
  int m = 0, base = 0;
  for (;;) {
    const int cnt = band_tiles<TBN>(p, m);
    if (u < base + cnt) break;
    base += cnt;
    ++m;
  }
  mb = m;
  bj = u - base + p.col_lo;
}

PHI4_DEV double pow2(int n) {
  if (n < -1022 || n > 1023) return ldexp(1.0, n);
  return __longlong_as_double((long long)(n + 1023) << 52);
}

// x 2^n as a double, built with integer operations (exact): x is zero or a normal
// float and the result a normal double. Keeps the conversions off the FP64 pipe.
PHI4_DEV double f2d_pow2(float x, int n) {
  const uint32_t b = __float_as_uint(x);
  if ((b << 1) == 0u) return 0.0;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ex = (unsigned long long)(((int)(b >> 23) & 0xff) + (1023 - 127) + n) << 52;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | ex | man));
}

constexpr int NUM_THREADS = 64 + 32 * NUM_EPI_WARPS;  // TMA warp, MMA warp, epilogue warps

__global__ void __launch_bounds__(NUM_THREADS, 1)
    chol_update_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Params p) {
  using namespace tc;
  pdl_trigger();  // the diagonal block's kernel (one CTA) may launch and wait for this one
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + ND * A_PLANE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SMEM_DATA);
  uint64_t* empty = full + 1;
  uint64_t* tfull = full + 2;   // [2]
  uint64_t* tempty = full + 4;  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* stage = reinterpret_cast<double*>(smem + SMEM_DATA + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, NUM_EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(p.status, ST_TIMEOUT);
  };
  // a contiguous run of the tile list per CTA: consecutive tiles mostly share a band
  const int chunk = (p.num_tiles + gridDim.x - 1) / gridDim.x;
  const int u_lo = min(p.num_tiles, (int)blockIdx.x * chunk), u_hi = min(p.num_tiles, u_lo + chunk);
  if (warp == 0) {
    if (lane == 0) {
      uint32_t phase = 0;
      int prev_mb = -1;
      for (int u = u_lo; u < u_hi && !*abort_flag; ++u) {
        int mb, bj;
        get_tile<BN>(p, u, mb, bj);
        if (!mbar_wait(empty, phase ^ 1u, abort_flag)) { give_up(); break; }
        // the band's A digit planes stay in shared memory while the band lasts
        const bool load_a = mb != prev_mb;
        mbar_expect_tx(full, load_a ? SMEM_DATA : ND * B_PLANE);
        for (int k = 0; k < ND; ++k) {
          if (load_a) tma_load_2d(&tmA, full, sA + k * A_PLANE, 0, k * p.m_pad + mb * BM);
          tma_load_2d(&tmB, full, sB + k * B_PLANE, 0, k * p.m_pad + bj * BN);
        }
        prev_mb = mb;
        phase ^= 1u;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t phase = 0, tph = 0;  // tph bit b: phase parity of accumulator set b
      int it = 0;
      for (int u = u_lo; u < u_hi && !*abort_flag; ++u, ++it) {
        const int buf = it & 1;
        // the epilogue must have drained this accumulator set (two tiles back)
        if (!mbar_wait(tempty + buf, ((tph >> buf) & 1u) ^ 1u, abort_flag)) { give_up(); break; }
        tc_fence_after();
        if (!mbar_wait(full, phase, abort_flag)) { give_up(); break; }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int c = 2; c <= NC + 1; ++c) {
          const uint32_t acc = tmem_base + (uint32_t)(buf * ACC_COLS + (c - 2) * BN);
          uint32_t accumulate = 0;
          for (int k = max(1, c - ND); k <= min(ND, c - 1); ++k) {
            const int l = c - k;
#pragma unroll
            for (int kk = 0; kk < KD / 16; ++kk) {
              umma_idesc(acc, sdesc(a0 + (k - 1) * A_PLANE + kk * 32), sdesc(b0 + (l - 1) * B_PLANE + kk * 32),
                         IDESC, accumulate);
              accumulate = 1;
            }
          }
        }
        umma_commit(empty);
        umma_commit(tfull + buf);
        phase ^= 1u;
        tph ^= 1u << buf;
      }
    }
  } else {
    // NUM_EPI_WARPS epilogue warps: warp w >= 2 reads TMEM lanes [32 (w % 4), 32 (w % 4) + 32)
    // (rows of the tile) in columns [grp EC, grp EC + EC), grp = (w - 2) / 4. A lane holds one
    // row's products (its TMEM lane); the trailing matrix is read and written through the
    // warp's staging patch in row segments: in pass k, lane (h, c) = (lane / EC, lane % EC)
    // takes row k RPP + h of the warp's 32 rows and column c, so EC lanes cover EC
    // consecutive doubles of one row.
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const int hl = lane / EC, cl = lane % EC;
    double* stg = stage + (warp - 2) * 32 * EC;
    uint32_t tph = 0;
    int it = 0;
    for (int u = u_lo; u < u_hi; ++u, ++it) {
      const int buf = it & 1;
      int mb, bj;
      get_tile<BN>(p, u, mb, bj);
      const int ir = mb * BM + r;  // this lane's row of products inside the trailing matrix
      const bool row_ok = ir < p.m;
      const int jc0 = bj * BN + grp * EC;
      const int jc = jc0 + cl;  // this lane's column in the row-segment passes
      const int ir0 = mb * BM + q * 32 + hl;  // its row in pass 0 (pass k: ir0 + k RPP)
      double* aseg = p.a + (size_t)(p.b0 + min(ir0, p.m - 1)) * p.D + p.b0 + jc;
      // load the FP64 targets and the exponents before waiting for the tile's products:
      // the loads run while the MMAs finish and the accumulators are combined (no other
      // tile of this launch, and no launch still running, writes these elements)
      const int ei = row_ok ? p.rexp[ir] : 0;
      const int ejl = jc < p.m ? p.rexp[jc] : 0;  // exponent of column jc0 + (lane % EC)
      double av[EC];
#pragma unroll
      for (int k = 0; k < EC; ++k) {
        const int irk = ir0 + k * RPP;
        const bool on = irk < p.m && jc < p.m && jc <= irk;
        av[k] = on ? aseg[(size_t)(k * RPP) * p.D] : 0.0;
      }

      if (!mbar_wait(tfull + buf, (tph >> buf) & 1u, abort_flag)) { give_up(); break; }
      tc_fence_after();
      const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * ACC_COLS + grp * EC);
      float hi[EC], lo[EC];
      // (hi, lo) <- (hi, lo) 2^-7 + U  in double-float (TwoSum, then renormalise)
      auto horner = [&](const uint32_t(&ur)[EC]) {
#pragma unroll
        for (int t = 0; t < EC; ++t) {
          const float uu = __uint_as_float(ur[t]);
          const float h = hi[t] * 0.0078125f, l = lo[t] * 0.0078125f;
          const float s = h + uu;
          const float bb = s - h;
          const float err = (h - (s - bb)) + (uu - bb);
          const float l2 = l + err;
          const float hs = s + l2;
          lo[t] = l2 - (hs - s);
          hi[t] = hs;
        }
      };
      {
        // the eight group accumulators U_9 .. U_2, two loads in flight per wait
        uint32_t r0[EC], r1[EC];
        tmem_ld8_nw(trow + (uint32_t)((NC - 1) * BN), r0);
        tmem_ld8_nw(trow + (uint32_t)((NC - 2) * BN), r1);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < EC; ++t) {
          hi[t] = __uint_as_float(r0[t]);
          lo[t] = 0.f;
        }
        horner(r1);
#pragma unroll 1
        for (int g = NC - 3; g >= 0; g -= 2) {
          tmem_ld8_nw(trow + (uint32_t)(g * BN), r0);
          tmem_ld8_nw(trow + (uint32_t)((g - 1) * BN), r1);
          tmem_wait_ld();
          horner(r0);
          horner(r1);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + buf);  // the accumulators are in registers now
      tph ^= 1u << buf;
      // The products (P P^T)_ij of this lane's row into the patch (values of rows and
      // columns outside the matrix are never stored). Every partial of (hi, lo) is a
      // multiple of 2^-49 below 2^24 in magnitude. While the row and column exponents
      // are moderate (the usual case, decided for the whole warp) the row's scale
      // 2^(e_i - 14) is applied here and the column's 2^(e_j) in the passes, as an
      // integer added to the exponent field: every value stays a normal double, so the
      // power-of-two scalings commute with the rounding of hi + lo and the result is the
      // one of scaling by 2^(e_i + e_j - 14) at once.
      const bool split = __all_sync(0xffffffffu, ei > -386 && ei < 414 && ejl > -400 && ejl < 400);
      if (split) {
        const int n = ei - 14;
#pragma unroll
        for (int t = 0; t < EC; ++t) stg[lane * EC + (t ^ swz(lane))] = f2d_pow2(hi[t], n) + f2d_pow2(lo[t], n);
      } else {
#pragma unroll
        for (int t = 0; t < EC; ++t) {
          const int n = ei + __shfl_sync(0xffffffffu, ejl, t) - 14;
          double v;
          if (n > -900 && n < 900) {
            v = f2d_pow2(hi[t], n) + f2d_pow2(lo[t], n);
          } else {
            v = ((double)hi[t] + (double)lo[t]) * pow2(n);
          }
          stg[lane * EC + (t ^ swz(lane))] = v;
        }
      }
      __syncwarp();
      const long long eadd = split ? (long long)ejl << 52 : 0ll;
      // the pass stride, opaque to the compiler so that the row addresses are recomputed
      // here rather than held in registers since the loads
      long long pstride;
      asm volatile("mov.b64 %0, %1;" : "=l"(pstride) : "l"((long long)RPP * p.D));
      double* dst = aseg;
#pragma unroll
      for (int k = 0; k < EC; ++k, dst += pstride) {
        const int rr = k * RPP + hl, irk = ir0 + k * RPP;
        if (irk < p.m && jc < p.m && jc <= irk) {
          const long long wb = __double_as_longlong(stg[rr * EC + (cl ^ swz(rr))]);
          *dst = av[k] - __longlong_as_double((wb << 1) ? wb + eadd : wb);
        }
      }
      __syncwarp();  // the patch is read before the next tile writes it
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}
// The bulk of a panel's update in 128 x 64 tiles. An N = 64 MMA reads its 4 KB A slice for
// 64 output columns, half the shared-memory operand traffic per product of the 128 x 32
// form (whose MMA issue is bound by those operand reads). A tile's eight group accumulators
// then take all 512 TMEM columns, so the MMA warp and the epilogue hand them over group by
// group: the MMAs produce U_9 (eight digit pairs) first and U_2 (one pair) last, the order
// in which the epilogue's Horner pass consumes them, and the next tile's group g waits only
// for every epilogue warp to have read this tile's group g.
namespace wide {
constexpr int TBN = 64;
constexpr int B_PLANE = TBN * KD * 2;                      // 8 KB
constexpr int SMEM_DATA = ND * (A_PLANE + B_PLANE);         // 192 KB
constexpr int EC = 16;                                      // tile columns per epilogue warp
constexpr int NUM_EPI_WARPS = 4 * (TBN / EC);               // four TMEM lane quarters x four column groups
constexpr int HALF = 8;                                     // columns per pass through the staging patch
constexpr int RPP = 32 / HALF;                              // rows per row-segment access
constexpr int STAGE_BYTES = NUM_EPI_WARPS * 32 * HALF * 8;  // 32 KB
constexpr int SMEM_BYTES = SMEM_DATA + 256 + STAGE_BYTES + 1024;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
static_assert(HALF == emu::EC, "the staging patch's swizzle is laid out for eight columns");
constexpr int NUM_THREADS = 64 + 32 * NUM_EPI_WARPS;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
}  // namespace wide

__global__ void __launch_bounds__(wide::NUM_THREADS, 1)
    chol_update_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                            Params p) {
  using namespace tc;
  pdl_trigger();  // the diagonal block's kernel (one CTA) may launch and wait for this one
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + ND * A_PLANE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + wide::SMEM_DATA);
  uint64_t* empty = full + 1;
  uint64_t* gfull = full + 2;     // [NC] group g of the tile is in TMEM
  uint64_t* gempty = gfull + NC;  // [NC] every epilogue warp has read group g
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gempty + NC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* stage = reinterpret_cast<double*>(smem + wide::SMEM_DATA + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(empty, 1);
    for (int g = 0; g < NC; ++g) {
      mbar_init(gfull + g, 1);
      mbar_init(gempty + g, wide::NUM_EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(p.status, ST_TIMEOUT);
  };
  const int chunk = (p.num_tiles + gridDim.x - 1) / gridDim.x;
  const int u_lo = min(p.num_tiles, (int)blockIdx.x * chunk), u_hi = min(p.num_tiles, u_lo + chunk);
  if (warp == 0) {
    if (lane == 0) {
      uint32_t phase = 0;
      int prev_mb = -1;
      for (int u = u_lo; u < u_hi && !*abort_flag; ++u) {
        int mb, bj;
        get_tile<wide::TBN>(p, u, mb, bj);
        if (!mbar_wait(empty, phase ^ 1u, abort_flag)) { give_up(); break; }
        const bool load_a = mb != prev_mb;  // the band's A digit planes stay while the band lasts
        mbar_expect_tx(full, load_a ? wide::SMEM_DATA : ND * wide::B_PLANE);
        for (int k = 0; k < ND; ++k) {
          if (load_a) tma_load_2d(&tmA, full, sA + k * A_PLANE, 0, k * p.m_pad + mb * BM);
          tma_load_2d(&tmB, full, sB + k * wide::B_PLANE, 0, k * p.m_pad + bj * wide::TBN);
        }
        prev_mb = mb;
        phase ^= 1u;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t phase = 0;
      int it = 0;
      for (int u = u_lo; u < u_hi && !*abort_flag; ++u, ++it) {
        if (!mbar_wait(full, phase, abort_flag)) { give_up(); break; }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        bool ok = true;
        for (int c = NC + 1; c >= 2; --c) {
          const int g = c - 2;
          // group g's accumulator of the previous tile has been read by the epilogue
          if (!mbar_wait(gempty + g, (uint32_t)(it & 1) ^ 1u, abort_flag)) { give_up(); ok = false; break; }
          tc_fence_after();
          const uint32_t acc = tmem_base + (uint32_t)(g * wide::TBN);
          uint32_t accumulate = 0;
          for (int k = max(1, c - ND); k <= min(ND, c - 1); ++k) {
            const int l = c - k;
#pragma unroll
            for (int kk = 0; kk < KD / 16; ++kk) {
              umma_idesc(acc, sdesc(a0 + (k - 1) * A_PLANE + kk * 32),
                         sdesc(b0 + (l - 1) * wide::B_PLANE + kk * 32), wide::IDESC, accumulate);
              accumulate = 1;
            }
          }
          umma_commit(gfull + g);
        }
        if (!ok) break;
        umma_commit(empty);
        phase ^= 1u;
      }
    }
  } else {
    // Epilogue warp w >= 2: TMEM lanes [32 (w % 4), 32 (w % 4) + 32) (rows of the tile),
    // columns [grp 16, grp 16 + 16), grp = (w - 2) / 4. The sixteen columns go through the
    // warp's 32 x 8 staging patch in two halves; in pass k of a half, lane (h, c) =
    // (lane / 8, lane % 8) takes row k RPP + h of the warp's 32 rows and column c.
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const int hl = lane / wide::HALF, cl = lane % wide::HALF;
    double* stg = stage + (warp - 2) * 32 * wide::HALF;
    int it = 0;
    for (int u = u_lo; u < u_hi; ++u, ++it) {
      int mb, bj;
      get_tile<wide::TBN>(p, u, mb, bj);
      const int ir = mb * BM + r;
      const bool row_ok = ir < p.m;
      const int jc0 = bj * wide::TBN + grp * wide::EC;
      const int ei = row_ok ? p.rexp[ir] : 0;
      const uint32_t par = (uint32_t)(it & 1);
      const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(grp * wide::EC);
      float hi[wide::EC], lo[wide::EC];
      bool ok = true;
      // U_9 .. U_2 as the MMAs deliver them; (hi, lo) <- (hi, lo) 2^-7 + U in double-float
#pragma unroll 1
      for (int g = NC - 1; g >= 0; --g) {
        if (!mbar_wait(gfull + g, par, abort_flag)) { give_up(); ok = false; break; }
        tc_fence_after();
        // the sixteen columns as two loads of eight (fewer registers in flight)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t ur[wide::HALF];
          tmem_ld8_nw(trow + (uint32_t)(g * wide::TBN + hh * wide::HALF), ur);
          tmem_wait_ld();
          if (hh == 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(gempty + g);
          }
#pragma unroll
          for (int tt = 0; tt < wide::HALF; ++tt) {
            const int t = hh * wide::HALF + tt;
            const float uu = __uint_as_float(ur[tt]);
            if (g == NC - 1) {
              hi[t] = uu;
              lo[t] = 0.f;
            } else {
              const float h = hi[t] * 0.0078125f, l = lo[t] * 0.0078125f;
              const float s = h + uu;
              const float bb = s - h;
              const float err = (h - (s - bb)) + (uu - bb);
              const float l2 = l + err;
              const float hs = s + l2;
              lo[t] = l2 - (hs - s);
              hi[t] = hs;
            }
          }
        }
      }
      if (!ok) break;
      const int ir0 = mb * BM + q * 32 + hl;  // this lane's row in pass 0 (pass k: ir0 + k RPP)
      const size_t row0 = (size_t)(p.b0 + min(ir0, p.m - 1)) * p.D + p.b0;
      // the targets of a half's passes (no other tile of this launch, and no launch still
      // running, writes them)
      auto load_half = [&](int h, double(&av)[wide::HALF]) {
        const int jc = jc0 + h * wide::HALF + cl;
        const double* src = p.a + row0 + jc;
#pragma unroll
        for (int k = 0; k < wide::HALF; ++k) {
          const int irk = ir0 + k * wide::RPP;
          av[k] = (irk < p.m && jc < p.m && jc <= irk) ? src[(size_t)(k * wide::RPP) * p.D] : 0.0;
        }
      };
      double av0[wide::HALF], av1[wide::HALF];
      // half h of the warp's sixteen columns into the patch; returns what the passes add
      // to the exponent field of each staged value
      auto stage_half = [&](const int h) -> long long {
        const int jc = jc0 + h * wide::HALF + cl;  // this lane's column in the passes
        const int ejl = jc < p.m ? p.rexp[jc] : 0;
        // Every partial of (hi, lo) is a multiple of 2^-49 below 2^24 in magnitude. With
        // moderate exponents (decided for the whole warp) the row's scale 2^(e_i - 14) is
        // applied here and the column's 2^(e_j) in the passes as an integer added to the
        // exponent field: every value stays a normal double, so the result equals scaling
        // by 2^(e_i + e_j - 14) at once.
        const bool split = __all_sync(0xffffffffu, ei > -386 && ei < 414 && ejl > -400 && ejl < 400);
        if (split) {
          const int n = ei - 14;
#pragma unroll
          for (int t = 0; t < wide::HALF; ++t)
            stg[lane * wide::HALF + (t ^ swz(lane))] =
                f2d_pow2(hi[h * wide::HALF + t], n) + f2d_pow2(lo[h * wide::HALF + t], n);
        } else {
#pragma unroll
          for (int t = 0; t < wide::HALF; ++t) {
            const int n = ei + __shfl_sync(0xffffffffu, ejl, t) - 14;
            const float x = hi[h * wide::HALF + t], y = lo[h * wide::HALF + t];
            const double v =
                (n > -900 && n < 900) ? f2d_pow2(x, n) + f2d_pow2(y, n) : ((double)x + (double)y) * pow2(n);
            stg[lane * wide::HALF + (t ^ swz(lane))] = v;
          }
        }
        __syncwarp();
        return split ? (long long)ejl << 52 : 0ll;
      };
      // row-segment passes of half h: target minus staged product
      auto pass_half = [&](const int h, const double(&av)[wide::HALF], long long eadd) {
        const int jc = jc0 + h * wide::HALF + cl;
        // the pass stride, opaque to the compiler so that the row addresses are recomputed
        // here rather than held in registers since the loads
        long long pstride;
        asm volatile("mov.b64 %0, %1;" : "=l"(pstride) : "l"((long long)wide::RPP * p.D));
        double* dst = p.a + row0 + jc;
#pragma unroll
        for (int k = 0; k < wide::HALF; ++k, dst += pstride) {
          const int rr = k * wide::RPP + hl, irk = ir0 + k * wide::RPP;
          if (irk < p.m && jc < p.m && jc <= irk) {
            const long long wb = __double_as_longlong(stg[rr * wide::HALF + (cl ^ swz(rr))]);
            *dst = av[k] - __longlong_as_double((wb << 1) ? wb + eadd : wb);
          }
        }
        __syncwarp();  // the patch is read before it is written again
      };
      // each half's targets load as one batch (eight loads in flight) while its products go
      // into the patch; the second half's loads wait for the first half's passes, which
      // keeps the live registers within the 96 of a 576-thread CTA
      load_half(0, av0);
      const long long e0 = stage_half(0);
      pass_half(0, av0, e0);
      load_half(1, av1);
      const long long e1 = stage_half(1);
      pass_half(1, av1, e1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}
}  // namespace emu

bool tc_available() { return tc::encode_fn() != nullptr; }

cudaError_t launch_propose_tc(void* delta_f16, const void* Zb, int ldz, const void* Lb, int ldl, int N, int D,
                              float scale, uint32_t* status, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (!tc::make_map(&ma, Zb, D, N, ldz, tc::BM) || !tc::make_map(&mb, Lb, D, D, ldl, tc::BN))
    return cudaErrorInvalidValue;
  tc::Params p{};
  p.M = N;
  p.Nn = D;
  p.K = D;
  p.tiles_m = (N + tc::BM - 1) / tc::BM;
  p.tiles_n = (D + tc::BN - 1) / tc::BN;
  p.num_tiles = p.tiles_m * p.tiles_n;
  p.delta = (__half*)delta_f16;
  p.scale = scale;
  p.status = status;
  return tc::launch(ma, mb, p, s);
}

bool make_gemm_run(GemmRun* g, const void* Zb, int ldz, const void* Lb, int ldl, int N, int D, float scale,
                   __half* delta, const double* scal, int n_mcmc) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  CUtensorMap ma, mb;
  if (!tc::make_map(&ma, Zb, D, N, ldz, tc::BM) || !tc::make_map(&mb, Lb, D, D, ldl, tc::BN)) return false;
  memcpy(g->mapA, &ma, sizeof(ma));
  memcpy(g->mapB, &mb, sizeof(mb));
  g->delta = delta;
  g->scal = scal;
  g->scale = scale;
  g->M = N;
  g->Nn = D;
  g->K = D;
  g->tiles_m = (N + tc::BM - 1) / tc::BM;
  g->tiles_n = (D + tc::BN - 1) / tc::BN;
  g->tile0 = 0;
  g->n_mcmc = n_mcmc;
  return true;
}

cudaError_t grouped_propose_prepare() {
  return cudaFuncSetAttribute(tc::tc_gemm_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
}

cudaError_t launch_grouped_propose(const GemmRun* runs, int R, int total_tiles, int grid, uint32_t sweep,
                                   uint32_t* status, cudaStream_t s) {
  if (total_tiles <= 0 || R <= 0) return cudaSuccess;
  grid = std::max(1, std::min(grid, total_tiles));
  tc::tc_gemm_grouped_kernel<<<grid, tc::NUM_THREADS, tc::SMEM_BYTES, s>>>(runs, R, total_tiles, sweep, status);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(const void* H, const void* Lo, int ldx, int D, int N, const int* shift, int a,
                           double inv_nm1, double* sigma, uint32_t* status, cudaStream_t s) {
  CUtensorMap mh, ml;
  if (!tc::make_map(&mh, H, N, D, ldx, gram::BM) || !tc::make_map(&ml, Lo, N, D, ldx, gram::BM))
    return cudaErrorInvalidValue;
  const int tiles = (D + gram::BM - 1) / gram::BM;
  gram::Params p{};
  p.D = D;
  p.K = N;
  p.num_tiles = tiles * (tiles + 1) / 2;
  p.a = a;
  p.shift = shift;
  p.inv = inv_nm1;
  p.sigma = sigma;
  p.status = status;
  cudaError_t e = cudaFuncSetAttribute(gram::gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gram::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int grid = std::min(sm_count(), p.num_tiles);
  gram::gram_kernel<<<grid, gram::NUM_THREADS, gram::SMEM_BYTES, s>>>(mh, ml, p);
  return cudaGetLastError();
}

cudaError_t launch_chol_update_tc(double* a, int D, int b0, int m, const void* planes, int m_pad, const int* rexp,
                                  int blk_lo, int blk_hi, bool leave_sms, uint32_t* status, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  // 128 x 64 tiles (N = 64 MMAs) for updates of two or more 64-column blocks, the
  // throughput-bound bulk; 128 x 32 tiles for one block column, the look-ahead chain's
  // latency-bound step, where twice the tiles run side by side. PHI4_CHOL_WIDE=0 keeps
  // every update in 128 x 32 tiles.
  static const bool wide_ok = [] {
    const char* v = getenv("PHI4_CHOL_WIDE");
    return !(v && atoi(v) == 0);
  }();
  const bool whole = blk_hi >= (1 << 20);
  const bool wide = wide_ok && (whole || blk_hi - blk_lo >= 2);
  const int tbn = wide ? emu::wide::TBN : emu::BN;
  const int per_blk = 64 / tbn;  // tile columns per 64-column block
  CUtensorMap ma, mb;
  if (!tc::make_map(&ma, planes, 64, 8 * m_pad, 64, emu::BM) || !tc::make_map(&mb, planes, 64, 8 * m_pad, 64, tbn))
    return cudaErrorInvalidValue;
  emu::Params p{};
  p.a = a;
  p.D = D;
  p.b0 = b0;
  p.m = m;
  p.m_pad = m_pad;
  p.tiles_m = (m + emu::BM - 1) / emu::BM;
  p.tiles_n = (m + tbn - 1) / tbn;
  p.col_lo = blk_lo * per_blk;
  p.col_hi = whole ? (1 << 30) : blk_hi * per_blk;
  int count = 0;
  for (int mm = 0; mm < p.tiles_m; ++mm) {
    const int hi = std::min(std::min(p.col_hi, p.tiles_n), (mm * emu::BM + emu::BM - 1) / tbn + 1);
    count += std::max(0, hi - p.col_lo);
  }
  p.num_tiles = count;
  p.rexp = rexp;
  p.status = status;
  if (p.num_tiles == 0) return cudaSuccess;
  cudaError_t e = wide ? cudaFuncSetAttribute(emu::chol_update_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              emu::wide::SMEM_BYTES)
                       : cudaFuncSetAttribute(emu::chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              emu::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  // the bulk of the update may leave a few SMs to the look-ahead chain (diagonal
  // block, inverse, panel solve, next block columns), which would otherwise wait for
  // whole update CTAs to retire
  static const int reserve = [] {
    const char* v = getenv("PHI4_CHOL_UPDATE_RESERVE");
    return v ? std::max(0, atoi(v)) : 32;
  }();
  const int avail = leave_sms ? std::max(1, sm_count() - reserve) : sm_count();
  const int grid = std::min(avail, p.num_tiles);
  if (wide)
    emu::chol_update_wide_kernel<<<grid, emu::wide::NUM_THREADS, emu::wide::SMEM_BYTES, s>>>(ma, mb, p);
  else
    emu::chol_update_kernel<<<grid, emu::NUM_THREADS, emu::SMEM_BYTES, s>>>(ma, mb, p);
  return cudaGetLastError();
}

}  // namespace phi4
