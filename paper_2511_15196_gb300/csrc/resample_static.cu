// Systematic resampling whose prefix-sum scratch is a fixed array compiled into
// the library, for callers that cannot allocate device memory or hand the library
// a scratch buffer. It runs the same kernel as phi4_resample_systematic.
//
// The array is a file-scope __device__ symbol: every GPU that loads the library
// holds it until the process exits. In host code its name is only a host-side
// stand-in, so its device address is looked up once per device (first call, with
// that device current) with cudaGetSymbolAddress and cached.
#include <mutex>

#include "run.h"

namespace {

constexpr int kStaticMaxN = PHI4_RESAMPLE_STATIC_MAX_N;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_resample_scratch[kStaticMaxN];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" phi4_status phi4_resample_systematic_static(const double* w, int32_t N, uint32_t U, int32_t* anc,
                                                       void* stream) {
  ARG_CHECK(w && anc, "NULL argument");
  ARG_CHECK(N >= 1, "N = %d must be at least 1", N);
  if (N > kStaticMaxN) {
    phi4::set_error("N = %d exceeds the %d weights the built-in scratch array holds; use "
                    "phi4_resample_systematic with a caller-provided scratch buffer",
                    N, kStaticMaxN);
    return PHI4_ERR_ARG;
  }
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  ARG_CHECK(dev >= 0 && dev < kMaxDevices, "device %d outside the %d devices this entry point tracks", dev,
            kMaxDevices);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_resample_scratch);
      if (e != cudaSuccess || addr == nullptr) {
        phi4::set_error("cudaGetSymbolAddress of the resampling scratch failed on device %d: %s", dev,
                        cudaGetErrorString(e));
        return PHI4_ERR_CUDA;
      }
      g_scratch_addr[dev] = addr;
    }
    scratch = g_scratch_addr[dev];
  }
  // Every entry the kernel reads it has written earlier in the same launch, so the
  // previous call's contents need no clearing.
  CUDA_TRY(phi4::launch_resample(w, N, U, nullptr, anc, scratch, (cudaStream_t)stream));
  return PHI4_OK;
}
