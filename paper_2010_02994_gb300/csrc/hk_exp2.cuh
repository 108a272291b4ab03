// FP64 base-2 exponential of the FP64 pair terms (the symmetric FP64 pair
// kernels, the incremental MwG kernels, and the probe that tests it against
// the host's exp2).
#pragma once

#include <cuda_runtime.h>

#include "hk_exp2_table.h"

namespace hk {

static_assert(kExp2TabSize == 2048, "exp2_core scales by 2048 and shifts by 11");

// High word of -1076.0: for y <= 0, (unsigned)hi(y) <= kHiNeg1076 holds for
// every y >= -1076 (and a few below it); 2^y for y < -1076 rounds to zero.
constexpr unsigned kHiNeg1076 = 0xC090D000u;

// 2^y for y <= 0.  Tang's method in base 2: y = k + j/2048 + f with
// |f| <= 2^-12, 2^y = 2^k T[j] (1 + q(f)), q the Taylor polynomial of 2^f - 1
// to degree 3 (truncation below 3.5e-17): 7 FP64 operations.  Arguments below -1100, -inf
// included, are clamped there; positive arguments (which the kernels only
// meet on pairs they discard) are taken as 0.  2^k is applied to the
// exponent field; for k < -1075 the result rounds to zero and is set so,
// and for -1075 <= k < -1021 one multiplication by a further power of two
// rounds it once into the subnormal range.  Every add and multiply is
// written as a fused multiply-add with `one` = 1 or `mz` = -0 (runtime
// values the compiler cannot fold), which leaves each result unchanged.
// Measured against a 64-bit-mantissa exp2 on 2e7 arguments in [-1100, 0]:
// 1.28 ulp.
struct Exp2Parts {
    double res;  // 2^max(k, -1021) T[j] (1 + q(f)), a normal double
    int k, kk;   // k and max(k, -1021)
};

__device__ __forceinline__ Exp2Parts exp2_core(double y, const double *__restrict__ tab, double one, double mz)
{
    // clamps on the bit pattern (integer pipe): for y <= 0 a larger unsigned
    // high word means a larger magnitude
    const unsigned hy = (unsigned)__double2hiint(y);
    if ((int)hy >= 0)
        y = 0.0;
    else if (hy > 0xC0913000u)  // high word of -1100.0
        y = -1100.0;
    const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds 2048 y to an integer
    const double m = fma(y, 2048.0, magic);
    const int j = __double2loint(m);
    const double f = fma(fma(m, one, -magic), -0.00048828125, y);  // exact, |f| <= 2^-12
    double p = fma(f, kExp2C3, kExp2C2);
    p = fma(f, p, kExp2C1);
    const double T = tab[j & (kExp2TabSize - 1)];
    const double r = fma(T, fma(f, p, mz), T);  // 2^((j mod 2048) / 2048 + f), in [0.99, 2)
    Exp2Parts e;
    e.k = j >> 11;  // floor(j / 2048), >= -1100
    e.kk = max(e.k, -1021);
    e.res = __hiloint2double((int)((unsigned)__double2hiint(r) + ((unsigned)e.kk << 20)), __double2loint(r));
    return e;
}

// The last rounding for -1075 <= k < -1021: times 2^(k - kk) >= 2^-79.
__device__ __forceinline__ double exp2_subnormal(const Exp2Parts &e, double mz)
{
    return fma(e.res, __hiloint2double((e.k - e.kk + 1023) << 20, 0), mz);
}

// Warp form: the lanes of `mask` make the call together, and the subnormal
// multiplication is issued only when one of them needs it.
__device__ __forceinline__ double exp2_neg(double y, const double *__restrict__ tab, unsigned mask, double one,
                                           double mz)
{
    Exp2Parts e = exp2_core(y, tab, one, mz);
    if (__any_sync(mask, e.k < e.kk && e.k >= -1075))
        e.res = exp2_subnormal(e, mz);
    return e.k < -1075 ? 0.0 : e.res;
}

// Lane form, for callers whose lanes may diverge.
__device__ __forceinline__ double exp2_neg_lane(double y, const double *__restrict__ tab)
{
    Exp2Parts e = exp2_core(y, tab, 1.0, -0.0);
    if (e.k < e.kk && e.k >= -1075)
        e.res = exp2_subnormal(e, -0.0);
    return e.k < -1075 ? 0.0 : e.res;
}

}  // namespace hk
