// e^x in double for the FP64 integrands: the table-driven method of P. T. P.
// Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989.
//
//   x = (256 m + j) ln2/256 + r,  j in [0, 255],  |r| <= ln2/512
//   e^x = 2^m * 2^(j/256) * e^r
//
// k = 256 m + j is x * 256/ln2 rounded to the nearest integer (by adding and
// subtracting 1.5 * 2^52, which also leaves k in the low word); r is reduced
// with ln2/256 split in two (the high part has 19 trailing zero bits, so k
// times it is exact for |k| < 2^19, which |x| < 746 keeps); e^r - 1 is its
// Taylor polynomial to degree 4 (the omitted r^5/120 is below 3.9e-17 for
// |r| <= ln2/512); 2^(j/256) comes from a 256-entry table of correctly
// rounded doubles; 2^m is added to the exponent field (two multiplications at
// the ends of the range).  About 9 double-precision operations; with 64
// entries and degree 5 it ran 1.33x as fast as the CUDA library's exp, inside
// the FP64 iterate kernel 1% (8.03 -> 7.94 ms per 1e8 at d=8).  Agreement with
// the CUDA library's and numpy's exp to 2 ulp over the whole range, and the
// special values, are tested.
#pragma once

#include <cuda_runtime.h>

#include "exp2_table.h"

namespace vegas {

__device__ __forceinline__ double fp64_exp(double x) {
    constexpr double kInvLn2By256 = 0x1.71547652b82fep+8;  // 256 / ln 2
    constexpr double kLn2By256Hi = 0x1.62e42fef80000p-9;   // ln 2 / 256, high part
    constexpr double kLn2By256Lo = 0x1.1cf79abc9e3b4p-44;  // ln 2 / 256 - high part
    constexpr double kShifter = 0x1.8p52;
    constexpr double kMaxArg = 0x1.62e42fefa39efp+9;      // ln(DBL_MAX)
    constexpr double kMinArg = -0x1.74910d52d3052p+9;     // below: rounds to 0
    // |x| < 708 (high word below that of 708.0) is inside both ends: the
    // common case is decided on the integer pipe, the exact double compares
    // (which the FP64 pipe executes) run only for larger |x| or NaN
    if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= 0x40862000u) {
        if (!(x >= kMinArg && x <= kMaxArg)) {           // out of range, or NaN
            if (x != x) return x;
            return x > 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0;
        }
    }
    const double kd = fma(x, kInvLn2By256, kShifter);
    const int k = __double2loint(kd);
    // = kd - kShifter exactly; the conversion instead of a double subtraction
    // measured 0.4% faster in the FP64 kernels (7.676 -> 7.645 ms per 1e8)
    const double kf = __int2double_rn(k);
    double r = fma(-kf, kLn2By256Hi, x);
    r = fma(-kf, kLn2By256Lo, r);
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p *= r;                                      // e^r - 1
    const double t = __ldg(&kExp2Table[k & 255]);
    const double y = fma(t, p, t);               // 2^(j/256) e^r in [0.998, 1.998)
    const int m = k >> 8;                        // arithmetic shift: floor(k / 256)
    if (m >= -1021 && m <= 1023)                 // normal result: scale the exponent
        return __hiloint2double(__double2hiint(y) + m * (1 << 20), __double2loint(y));
    // near the ends (subnormal result, or m = 1024 just below ln DBL_MAX): two
    // scalings by normal powers of two, the first exact, one rounding
    const int m1 = m >> 1, m2 = m - m1;
    return y * __hiloint2double((m1 + 1023) << 20, 0) * __hiloint2double((m2 + 1023) << 20, 0);
}

}  // namespace vegas
