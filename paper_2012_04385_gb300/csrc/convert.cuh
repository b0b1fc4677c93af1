// FP64 <-> FP32 conversion on the integer pipe.
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate and the hardware
// double->float conversion (with its flush-to-zero range check) is issued
// there, so the mixed-precision kernels convert their FP64 inputs with integer
// instructions instead: the exponent is rebiased from 1023 to 127 and the
// mantissa rounded to 23 bits (round half away from zero).  Valid for values
// whose magnitude lies in the FP32 normal range, which holds for the
// conserved and primitive states of the solver; magnitudes below it (and
// zero) give a signed zero.
#pragma once

#include <cuda_runtime.h>

namespace mrb {

__device__ __forceinline__ float d2f_fast(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7FFFFFFFu;
  unsigned f = (((mag - (896u << 20)) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
  f = (mag < (897u << 20)) ? 0u : f;
  return __uint_as_float((hi & 0x80000000u) | f);
}

__device__ __forceinline__ double f2d_fast(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned mag = b & 0x7FFFFFFFu;
  const unsigned hi = (b & 0x80000000u) | (mag < 0x00800000u ? 0u : ((mag >> 3) + (896u << 20)));
  const unsigned lo = (mag < 0x00800000u) ? 0u : (mag << 29);
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace mrb
