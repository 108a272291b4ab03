// FP64 base-2 exponential of the symmetric FP64 pair kernels (and of the
// probe that tests it against the host's exp2).
#pragma once

#include <cuda_runtime.h>

#include "hk_exp2_table.h"

namespace hk {

// High word of -1076.0: for y <= 0, (unsigned)hi(y) <= kHiNeg1076 holds for
// every y >= -1076 (and a few below it); 2^y for y < -1076 rounds to zero.
constexpr unsigned kHiNeg1076 = 0xC090D000u;

// 2^y for y <= 0.  Tang's method in base 2: y = k + j/256 + f with
// |f| <= 2^-9, 2^y = 2^k T[j] (1 + q(f)), q the Taylor polynomial of 2^f - 1
// to degree 4 (truncation below 3.8e-17).  Arguments below -1100, -inf
// included, are clamped there; positive arguments (which the kernels only
// meet on pairs they discard) are taken as 0.  2^k is applied to the
// exponent field; for k < -1075 the result rounds to zero and is set so,
// and for -1075 <= k < -1021 one multiplication by a further power of two
// rounds it once into the subnormal range, done only when some lane of
// `mask` (the lanes making the call together) needs it.  Every add and
// multiply is written as a fused multiply-add with `one` = 1 or `mz` = -0
// (runtime values the compiler cannot fold), which leaves each result
// unchanged.  Measured against a 64-bit-mantissa exp2 on 2e7 arguments in
// [-1100, 0]: 1.32 ulp.
__device__ __forceinline__ double exp2_neg(double y, const double *__restrict__ tab, unsigned mask, double one,
                                           double mz)
{
    // clamps on the bit pattern (integer pipe): for y <= 0 a larger unsigned
    // high word means a larger magnitude
    const unsigned hy = (unsigned)__double2hiint(y);
    if ((int)hy >= 0)
        y = 0.0;
    else if (hy > 0xC0913000u)  // high word of -1100.0
        y = -1100.0;
    const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds 256 y to an integer
    const double m = fma(y, 256.0, magic);
    const int j = __double2loint(m);
    const double f = fma(fma(m, one, -magic), -0.00390625, y);  // exact
    double p = fma(f, kExp2C4, kExp2C3);
    p = fma(f, p, kExp2C2);
    p = fma(f, p, kExp2C1);
    const double T = tab[j & 255];
    const double r = fma(T, fma(f, p, mz), T);  // 2^(j mod 256 / 256 + f), in [0.99, 2)
    const int k = j >> 8;                       // floor(j / 256), >= -1100
    const int kk = max(k, -1021);               // 2^kk r is a normal double
    double res = __hiloint2double((int)((unsigned)__double2hiint(r) + ((unsigned)kk << 20)), __double2loint(r));
    if (__any_sync(mask, k < kk && k >= -1075))
        res = fma(res, __hiloint2double((k - kk + 1023) << 20, 0), mz);  // times 2^(k - kk) >= 2^-79
    return k < -1075 ? 0.0 : res;
}

}  // namespace hk
