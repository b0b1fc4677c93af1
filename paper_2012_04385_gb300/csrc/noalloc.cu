// Conservation sums over caller-provided blocks without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code running under an allocator
// that owns all device memory (a framework's caching allocator or a fixed
// arena handed out at start-up), or host code that must not take the driver's
// allocation lock while other work is in flight.  For them this entry point
// keeps its reduction scratch in a file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
//
// Limits and behaviour (also stated in include/mrb.h):
//  * at most MRB_NOALLOC_MAX_BLOCKS blocks per call (larger n is rejected with
//    MRB_ECAPACITY before anything is launched);
//  * the first call on a device looks up the array's device address with that
//    device current (cudaGetSymbolAddress) and caches it; make that first call
//    before any stream capture on the device;
//  * all calls share the one array, which keeps the last call's contents:
//    calls that overlap on the GPU (different streams, or different host
//    threads on one device) race on it;
//  * no cudaMalloc, cudaFree or allocating library routine is called.
#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "mrb.h"

namespace mrb {

constexpr int NOALLOC_MAX_BLOCKS = MRB_NOALLOC_MAX_BLOCKS;

// per-block partial sums [block][5]; every entry a call reads is written by the
// same call first, so nothing has to start at zero
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_BLOCKS * NV];

// Per block: sum of its internal cells (index order of [5][16^3]) times dx^3,
// reduced in the same fixed order as the pool-based kernel.
__global__ void __launch_bounds__(256) k_noalloc_partial(const double* __restrict__ blocks, int64_t n,
                                                          const int32_t* __restrict__ levels, double dx0,
                                                          double* __restrict__ partial) {
  __shared__ double sh[5][8];
  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    const double* U = blocks + (size_t)b * NV * NINT;
    double s[5] = {0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < NINT; e += blockDim.x) {
#pragma unroll
      for (int v = 0; v < 5; ++v) s[v] += U[v * NINT + e];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v)
      for (int o = 16; o > 0; o >>= 1) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    if ((threadIdx.x & 31) == 0)
      for (int v = 0; v < 5; ++v) sh[v][threadIdx.x >> 5] = s[v];
    __syncthreads();
    if (threadIdx.x < 5) {
      double x = 0.0;
      for (int q = 0; q < 8; ++q) x += sh[threadIdx.x][q];
      const double dx = ldexp(dx0, levels ? -levels[b] : 0);
      partial[(size_t)b * 5 + threadIdx.x] = x * (dx * dx * dx);
    }
    __syncthreads();
  }
}

__global__ void k_noalloc_finish(const double* __restrict__ partial, int64_t n, double* __restrict__ out) {
  const int v = threadIdx.x;
  if (v >= 5) return;
  double acc = 0.0;
  for (int64_t b = 0; b < n; ++b) acc += partial[(size_t)b * 5 + v];
  out[v] = acc;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

}  // namespace mrb

extern "C" int mrb_block_sums_noalloc(const double* blocks_dev, int64_t n_blocks, const int32_t* levels_dev,
                                      double dx0, void* stream, double* sums_dev) {
  using namespace mrb;
  if (n_blocks < 0 || !sums_dev || (n_blocks > 0 && !blocks_dev) || !(dx0 > 0)) return MRB_EINVAL;
  if (n_blocks > NOALLOC_MAX_BLOCKS) return MRB_ECAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MRB_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) return MRB_ECUDA;
      g_scratch_ptr[dev] = (double*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (n_blocks > 0) {
    const int grid = (int)std::min<int64_t>(n_blocks, (int64_t)sm_count() * 4);
    k_noalloc_partial<<<grid, 256, 0, st>>>(blocks_dev, n_blocks, levels_dev, dx0, scratch);
  }
  k_noalloc_finish<<<1, 32, 0, st>>>(scratch, n_blocks, sums_dev);
  return cudaGetLastError() == cudaSuccess ? MRB_OK : MRB_ECUDA;
}
