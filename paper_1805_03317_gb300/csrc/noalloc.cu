// Systematic resampling for callers that cannot allocate device memory.
//
// smc_resample computes its ancestors with scratch buffers that smc_init allocated. Some callers
// cannot call cudaMalloc at the point where they need ancestors: code running while a CUDA graph is
// being captured, engines whose memory plan is fixed before they run, or hosts that hand the GPU a
// fixed arena and forbid further allocations. smc_resample_noalloc serves them: the caller passes
// only the weights and the ancestor output, and the scratch (the integer prefix sums of the
// quantised weights plus two scalars) lives in one file-scope device array of fixed size. Every
// device that loads this library holds that array (SMC_NOALLOC_MAX_N + 2 eight-byte words, about
// 2 MiB) until the process exits.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "device.cuh"
#include "internal.h"
#include "subsmc.h"

namespace subsmc {
namespace {

constexpr int kScratchWords = SMC_NOALLOC_MAX_N + 2;  // prefix sums, then total and offset
constexpr int kMaxDevices = 64;
constexpr int kThreads = 1024;

static __device__ __align__(256) unsigned long long g_resample_scratch[kScratchWords];

// Integer weights w_i = floor(W_i 2^40), inclusive prefix sums into scratch[0..N), the total T
// and the offset floor(U T) (U from the stage's resampling stream) into the two trailing words.
// Every word read later is written here first, so nothing left by an earlier call is used.
__global__ void __launch_bounds__(kThreads)
    k_noalloc_scan(int N, const double *W, unsigned long long *scratch, uint64_t seed, int stage) {
  __shared__ unsigned long long tot[kThreads];
  const int tid = threadIdx.x;
  const int per = (N + kThreads - 1) / kThreads;
  const int i0 = tid * per, i1 = min(N, i0 + per);
  unsigned long long s = 0;
  for (int i = i0; i < i1; ++i) s += (unsigned long long)floor(W[i] * 0x1.0p40);
  tot[tid] = s;
  __syncthreads();
  for (int o = 1; o < kThreads; o <<= 1) {
    const unsigned long long v = tid >= o ? tot[tid - o] : 0ull;
    __syncthreads();
    tot[tid] += v;
    __syncthreads();
  }
  unsigned long long run = tid ? tot[tid - 1] : 0ull;
  for (int i = i0; i < i1; ++i) {
    run += (unsigned long long)floor(W[i] * 0x1.0p40);
    scratch[i] = run;
  }
  if (tid == kThreads - 1) {
    const unsigned long long T = tot[kThreads - 1];
    const Stream rs(seed, kResample, stage_move(stage, 0), 0u);
    const double U = draw_uniform(rs.draw(0));
    scratch[SMC_NOALLOC_MAX_N] = T;
    scratch[SMC_NOALLOC_MAX_N + 1] = (unsigned long long)floor(U * (double)T);
  }
}

__global__ void k_noalloc_ancestors(int N, const unsigned long long *scratch, int32_t *anc) {
  const unsigned long long T = scratch[SMC_NOALLOC_MAX_N], off = scratch[SMC_NOALLOC_MAX_N + 1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (T == 0) {
      anc[i] = i;
      continue;
    }
    const unsigned long long pos = ((unsigned long long)i * T + off) / (unsigned long long)N;
    int lo = 0, hi = N - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (scratch[mid] > pos)
        hi = mid;
      else
        lo = mid + 1;
    }
    anc[i] = lo;
  }
}

std::mutex g_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_on_current_device(unsigned long long **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    unsigned long long *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_resample_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace subsmc

extern "C" int smc_resample_noalloc(int32_t N, const double *W, uint64_t seed, int32_t stage,
                                    int32_t *ancestors, void *stream) {
  using namespace subsmc;
  if (N < 1 || N > SMC_NOALLOC_MAX_N) {
    set_global_error("smc_resample_noalloc: N must be in [1, SMC_NOALLOC_MAX_N = 262144]");
    return SMC_ERR_ARG;
  }
  if (!W || !ancestors || stage < 0) {
    set_global_error("smc_resample_noalloc: W and ancestors are required and stage must be >= 0");
    return SMC_ERR_ARG;
  }
  unsigned long long *scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) {
    set_global_error(std::string("smc_resample_noalloc: cudaGetSymbolAddress: ") +
                     cudaGetErrorString(e));
    return SMC_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_scan<<<1, kThreads, 0, s>>>(N, W, scratch, seed, stage);
  k_noalloc_ancestors<<<(N + 255) / 256, 256, 0, s>>>(N, scratch, ancestors);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("smc_resample_noalloc: launch: ") + cudaGetErrorString(e));
    return SMC_ERR_CUDA;
  }
  return SMC_OK;
}
