// Throughput microbenchmarks for the roofline of the stage kernels: FP32 FMA,
// FP64 FMA, FP64<->FP32 conversion and special-function (MUFU) rates of the
// current GPU, each as independent dependent-chain loops on every SM.
#include <cstdio>

#include "kernels.cuh"
#include "mrb.h"

namespace mrb {

constexpr int PK_ITERS = 2048;
constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS) k_pk_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f, x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f,
        x7 = x0 + 7.f;
#pragma unroll 4
  for (int i = 0; i < PK_ITERS; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == 1234.5f) out[0] = x0;
}

// packed FP32 FMA (two lanes of FP32 per instruction, fma.rn.f32x2)
__device__ __forceinline__ unsigned long long ffma2(unsigned long long x, unsigned long long a,
                                                    unsigned long long b) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(a), "l"(b));
  return r;
}

__global__ void __launch_bounds__(PK_THREADS) k_pk_ffma2(float* out, float a, float b) {
  const unsigned long long A = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long Bv = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  unsigned long long x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    x[q] = ((unsigned long long)__float_as_uint(threadIdx.x + q + 0.5f) << 32) | __float_as_uint(threadIdx.x + q + 0.25f);
#pragma unroll 4
  for (int i = 0; i < PK_ITERS; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = ffma2(x[q], A, Bv);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += __uint_as_float((unsigned)x[q]) + __uint_as_float((unsigned)(x[q] >> 32));
  if (s == 1234.5f) out[0] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_pk_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
#pragma unroll 4
  for (int i = 0; i < PK_ITERS / 8; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == 1234.5) out[0] = x0;
}

// double -> float conversions (consumed by FP32 adds on the FMA pipe)
__global__ void __launch_bounds__(PK_THREADS) k_pk_d2f(float* out, double a) {
  double d0 = threadIdx.x * a, d1 = d0 + 1, d2 = d0 + 2, d3 = d0 + 3;
  float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 4
  for (int i = 0; i < PK_ITERS / 8; ++i) {
    s0 += __double2float_rn(d0);
    s1 += __double2float_rn(d1);
    s2 += __double2float_rn(d2);
    s3 += __double2float_rn(d3);
    d0 = __longlong_as_double(__double_as_longlong(d0) ^ 1);
    d1 = __longlong_as_double(__double_as_longlong(d1) ^ 1);
    d2 = __longlong_as_double(__double_as_longlong(d2) ^ 1);
    d3 = __longlong_as_double(__double_as_longlong(d3) ^ 1);
  }
  if (s0 + s1 + s2 + s3 == 1234.5f) out[0] = s0;
}

// float -> double conversions (consumed by integer xor on the ALU pipe)
__global__ void __launch_bounds__(PK_THREADS) k_pk_f2d(long long* out, float a) {
  float f0 = threadIdx.x * a, f1 = f0 + 1, f2 = f0 + 2, f3 = f0 + 3;
  long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 4
  for (int i = 0; i < PK_ITERS / 8; ++i) {
    s0 ^= __double_as_longlong((double)f0);
    s1 ^= __double_as_longlong((double)f1);
    s2 ^= __double_as_longlong((double)f2);
    s3 ^= __double_as_longlong((double)f3);
    f0 = __int_as_float(__float_as_int(f0) ^ 1);
    f1 = __int_as_float(__float_as_int(f1) ^ 1);
    f2 = __int_as_float(__float_as_int(f2) ^ 1);
    f3 = __int_as_float(__float_as_int(f3) ^ 1);
  }
  if ((s0 ^ s1 ^ s2 ^ s3) == 12345) out[0] = s0;
}

__global__ void __launch_bounds__(PK_THREADS) k_pk_mufu(float* out, float a) {
  float x0 = threadIdx.x + a, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
#pragma unroll 4
  for (int i = 0; i < PK_ITERS / 4; ++i) {
    x0 = __frsqrt_rn(x0) + 2.f;
    x1 = __frsqrt_rn(x1) + 2.f;
    x2 = __frsqrt_rn(x2) + 2.f;
    x3 = __frsqrt_rn(x3) + 2.f;
  }
  if (x0 + x1 + x2 + x3 == 1234.5f) out[0] = x0;
}

}  // namespace mrb

// out[0] FP32 FMA TFLOP/s (2 flops per FMA), out[1] FP64 FMA TFLOP/s,
// out[2] double->float conversions (10^12/s), out[3] float->double conversions
// (10^12/s), out[4] reciprocal square roots (10^12/s), out[5] SM count,
// out[6] SM clock (MHz) reported by the device, and with n >= 8 out[7] packed
// FP32 FMA (fma.rn.f32x2) TFLOP/s.  Synchronises the device.
extern "C" int mrb_measure_peaks(double* out, int32_t n) {
  using namespace mrb;
  if (!out || n < 7) return MRB_EINVAL;
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, 64) != cudaSuccess) return MRB_ENOMEM;
  const int sms = sm_count();
  const int grid = sms * 8;
  const double threads = (double)grid * PK_THREADS;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto launch) {
    launch();
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 5.0 * 1e-3;
  };
  double t;
  t = timed([&] { k_pk_ffma<<<grid, PK_THREADS>>>((float*)scratch, 0.999f, 0.001f); });
  out[0] = threads * PK_ITERS * 8 * 2 / t / 1e12;
  t = timed([&] { k_pk_dfma<<<grid, PK_THREADS>>>((double*)scratch, 0.999, 0.001); });
  out[1] = threads * (PK_ITERS / 8) * 8 * 2 / t / 1e12;
  t = timed([&] { k_pk_d2f<<<grid, PK_THREADS>>>((float*)scratch, 1.0001); });
  out[2] = threads * (PK_ITERS / 8) * 4 / t / 1e12;
  t = timed([&] { k_pk_f2d<<<grid, PK_THREADS>>>((long long*)scratch, 1.0001f); });
  out[3] = threads * (PK_ITERS / 8) * 4 / t / 1e12;
  t = timed([&] { k_pk_mufu<<<grid, PK_THREADS>>>((float*)scratch, 1.0f); });
  out[4] = threads * (PK_ITERS / 4) * 4 / t / 1e12;
  if (n >= 8) {
    t = timed([&] { k_pk_ffma2<<<grid, PK_THREADS>>>((float*)scratch, 0.999f, 0.001f); });
    out[7] = threads * PK_ITERS * 8 * 4 / t / 1e12;
  }
  int dev = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  out[5] = sms;
  out[6] = clk / 1000.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  return cudaGetLastError() == cudaSuccess ? MRB_OK : MRB_ECUDA;
}
