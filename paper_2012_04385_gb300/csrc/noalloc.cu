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
//  * the array's device address is looked up (cudaGetSymbolAddress) with the
//    calling device current on every call made outside a stream capture, and
//    cached per device; a call made while its stream is being captured uses
//    the cached address, so make one call on the device before any capture.
//    After a device reset the next uncaptured call looks the address up again;
//  * all calls share the one array, which keeps the last call's contents:
//    calls that overlap on the GPU (different streams, or different host
//    threads on one device) race on it;
//  * no cudaMalloc, cudaFree or allocating library routine is called;
//  * the status reports only this call's own launch errors: an error left
//    pending by an earlier, unrelated call stays pending for its owner.
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
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MRB_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
      if (cap != cudaStreamCaptureStatusNone) return MRB_ECUDA;   // no address known yet: call once uncaptured
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) return MRB_ECUDA;
      g_scratch_ptr[dev] = (double*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) return MRB_ECUDA;
  // each launch's own status (cudaLaunchKernel returns it), so that an error
  // pending from an unrelated earlier call is neither reported nor cleared here
  const cudaError_t pending = cudaPeekAtLastError();
  cudaError_t e = cudaSuccess;
  if (n_blocks > 0) {
    const int grid = (int)std::min<int64_t>(n_blocks, (int64_t)nsm * 4);
    void* a1[] = {(void*)&blocks_dev, (void*)&n_blocks, (void*)&levels_dev, (void*)&dx0, (void*)&scratch};
    e = cudaLaunchKernel((const void*)k_noalloc_partial, dim3(grid), dim3(256), a1, 0, st);
    if (e == cudaSuccess) ++g_kernel_launches;
  }
  if (e == cudaSuccess) {
    const double* partial = scratch;
    void* a2[] = {(void*)&partial, (void*)&n_blocks, (void*)&sums_dev};
    e = cudaLaunchKernel((const void*)k_noalloc_finish, dim3(1), dim3(32), a2, 0, st);
    if (e == cudaSuccess) ++g_kernel_launches;
  }
  if (e != cudaSuccess) {
    if (pending == cudaSuccess) cudaGetLastError();   // clear our own launch error
    return MRB_ECUDA;
  }
  return MRB_OK;
}
