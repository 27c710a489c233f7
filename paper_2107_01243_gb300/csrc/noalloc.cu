// sem_dot_noalloc: the unique-dof inner product with no device allocation.
//
// Who needs it: callers that cannot call cudaMalloc where they need a dot
// product -- code that records work into a CUDA graph while a stream is being
// captured (an allocation there is not captured and breaks the capture), hosts
// that must not block on the allocator inside a latency-critical loop, and
// applications that hand the library a fixed device-memory budget up front
// and forbid allocations afterwards.  sem_dot keeps its partial sums in the
// handle's scratch; this variant keeps them in one file-scope device array
// that is part of the loaded library instead, so a call allocates nothing.
//
// Limits and sharing:
//  * The array holds kNoAllocMaxBlocks partial sums (128 KiB) plus one
//    completion ticket; every block sums kNoAllocPointsPerBlock points, so
//    n_L may be at most kNoAllocMaxPoints = 67,108,864 local points.
//  * Every GPU that loads the library holds the array until the process exits.
//  * All calls on a device share the array and it keeps the last call's
//    contents; each call clears the ticket before its kernel runs.  Calls
//    whose kernels overlap on the GPU (different streams, no ordering) race
//    on the array and give wrong results: order them on one stream.
//  * sem_setup looks up the array's device address once with
//    cudaGetSymbolAddress (noalloc_prepare, with the handle's device current);
//    a call then only clears the ticket and launches, so every call, the
//    first included, may run inside a stream capture.
#include <atomic>

#include "sem_internal.cuh"
#include "reduce.cuh"

namespace sem {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPointsPerBlock = 4096;                // 16 points per thread
constexpr int kNoAllocMaxBlocks = 16384;
constexpr int64_t kNoAllocMaxPoints = (int64_t)kNoAllocMaxBlocks * kNoAllocPointsPerBlock;
static_assert(kNoAllocMaxPoints == SEM_NOALLOC_MAX_POINTS, "limit stated in sem.h");

// [0, kNoAllocMaxBlocks): block partial sums; word kNoAllocMaxBlocks: ticket
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 32];

// One block per kNoAllocPointsPerBlock consecutive points (coalesced strides of
// the block size), then the shared grid reduction: fixed order, reproducible.
__global__ void __launch_bounds__(kNoAllocThreads)
k_wdot_static(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
              const float* __restrict__ imult, double* __restrict__ out,
              double* __restrict__ scratch) {
  const int64_t base = (int64_t)blockIdx.x * kNoAllocPointsPerBlock;
  double v[1] = {0.0};
#pragma unroll 4
  for (int m = threadIdx.x; m < kNoAllocPointsPerBlock; m += kNoAllocThreads) {
    const int64_t q = base + m;
    if (q < n) v[0] += a[q] * b[q] * (double)imult[q];
  }
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNoAllocMaxBlocks);
  double tot[1];
  if (grid_sum<1>(v, scratch, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

// Device address of the array, resolved once by sem_setup (the library drives
// one CUDA device per process, so one address serves every call).
static std::atomic<double*> g_noalloc_addr{nullptr};

// run by sem_setup with the handle's device current, so that every call, the
// first included, finds the address resolved (and may run inside a capture)
void noalloc_prepare() {
  if (g_noalloc_addr.load(std::memory_order_acquire)) return;
  void* p = nullptr;
  SEM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  g_noalloc_addr.store(static_cast<double*>(p), std::memory_order_release);
}

}  // namespace sem

using namespace sem;

extern "C" sem_status sem_dot_noalloc(sem_handle* h, const double* a, const double* b,
                                      double* out, void* stream) {
  return guarded("sem_dot_noalloc", [&] {
    SEM_REQUIRE(h && a && b && out, "sem_dot_noalloc: null argument");
    if (h->nL > kNoAllocMaxPoints)
      throw Error(SEM_ERR_ARG, "sem_dot_noalloc: n_L = " + std::to_string(h->nL) +
                                   " local points exceeds the maximum of " +
                                   std::to_string(kNoAllocMaxPoints) + "; use sem_dot");
    double* scratch = g_noalloc_addr.load(std::memory_order_acquire);
    if (!scratch) throw Error(SEM_ERR_STATE, "sem_dot_noalloc: no handle was set up");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((h->nL + kNoAllocPointsPerBlock - 1) / kNoAllocPointsPerBlock);
    SEM_CUDA(cudaMemsetAsync(scratch + kNoAllocMaxBlocks, 0, sizeof(double), s));
    k_wdot_static<<<blocks < 1 ? 1 : blocks, kNoAllocThreads, 0, s>>>(h->nL, a, b,
                                                                       h->imult.ptr, out, scratch);
    SEM_CHECK_LAUNCH();
  });
}
