// float32 -> float64 conversion on the integer pipes.  On GB300 the float64
// pipe runs at a small fraction of the float32 rate and the widening
// conversion instruction uses it, so the analysis epilogues, which widen
// their float32 sums into the float64 F_E, rearrange the IEEE 754 bit fields
// instead (sign, exponent re-biased by 1023 - 127 = 896, mantissa widened by
// 29 zero bits), with the hardware conversion kept for the rare inputs
// outside float32's normal range (zero, subnormal, infinite, NaN).  The
// result equals the hardware conversion's bit for bit
// (mlsdc_selftest_convert checks it against cvt on the device).  The
// narrowing direction (float64 state -> float32 operands) keeps the hardware
// conversion: done with integer operations (rounding to nearest even on the
// 29 dropped bits) it measured slower in the synthesis kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mlsdc {

// binary32 -> binary64: exact.
__device__ __forceinline__ double f64_of(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;  // zero, subnormal, infinite, NaN
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double f64_of(double x) { return x; }

}  // namespace mlsdc
