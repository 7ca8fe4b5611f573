// detmath64.cuh -- deterministic FP64 elementary functions for the FP64 step.
//
// Paths that cross the wavy current sheet are chaotic at the level of one
// unit in the last place: two FP64 integrations that differ by one rounding
// in one step drift apart.  The FP64 step therefore uses its own
// exp / log / sin / cos / tanh / atan, each a classical algorithm in plain
// IEEE double +, -, *, / (Cody & Waite argument reduction, "Software Manual
// for the Elementary Functions", 1980, then a truncated Taylor series in
// Horner form).  Compiled without FMA contraction (-fmad=false), these give
// the same bits on any IEEE double machine, which is what lets the FP64 path
// be checked path by path.  sqrt and division are IEEE correctly rounded.
//
// Accuracy: a few ulp over the ranges the step uses; tanh to 4e-16 absolute.
//
// Include only from translation units built with -fmad=false.
#pragma once
#include <cstdint>

namespace cosmica {
namespace dm {

// ln 2 split so that k * kLn2Hi is exact for |k| < 2^21
constexpr double kLn2Hi = 0.6931471803691238;
constexpr double kLn2Lo = 1.9082149292705877e-10;
constexpr double kLog2e = 1.4426950408889634;
// pi/2 in three 33-bit pieces
constexpr double kPio2_1 = 1.5707963267341256;
constexpr double kPio2_2 = 6.077100506303966e-11;
constexpr double kPio2_3 = 2.0222662487959506e-21;
constexpr double k2OverPi = 0.6366197723675814;
constexpr double kPi_2 = 1.5707963267948966;
constexpr double kPi_4 = 0.7853981633974483;
constexpr double kPi_8 = 0.39269908169872414;
constexpr double kTanPi_8 = 0.41421356237309503;
constexpr double kSqrt2 = 1.4142135623730951;

__device__ __forceinline__ double exp(double x)
{
    if (!(x < 709.0)) return (x != x) ? x : __longlong_as_double(0x7FF0000000000000ll);
    if (x < -708.0) return 0.0;
    const double k = floor(x * kLog2e + 0.5);
    const double r = (x - k * kLn2Hi) - k * kLn2Lo;
    double p = 1.0 / 6227020800.0;
    p = p * r + 1.0 / 479001600.0;
    p = p * r + 1.0 / 39916800.0;
    p = p * r + 1.0 / 3628800.0;
    p = p * r + 1.0 / 362880.0;
    p = p * r + 1.0 / 40320.0;
    p = p * r + 1.0 / 5040.0;
    p = p * r + 1.0 / 720.0;
    p = p * r + 1.0 / 120.0;
    p = p * r + 1.0 / 24.0;
    p = p * r + 1.0 / 6.0;
    p = p * r + 0.5;
    p = p * r + 1.0;
    p = p * r + 1.0;
    const int ki = (int)k;
    return p * __longlong_as_double((long long)(ki + 1023) << 52);
}

__device__ __forceinline__ double log(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? __longlong_as_double(0xFFF0000000000000ll)
                                      : __longlong_as_double(0x7FF8000000000000ll);
    if (x == __longlong_as_double(0x7FF0000000000000ll)) return x;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    if (m > kSqrt2) { m = m * 0.5; e = e + 1; }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
    double q = 1.0 / 23.0;
    q = q * s2 + 1.0 / 21.0;
    q = q * s2 + 1.0 / 19.0;
    q = q * s2 + 1.0 / 17.0;
    q = q * s2 + 1.0 / 15.0;
    q = q * s2 + 1.0 / 13.0;
    q = q * s2 + 1.0 / 11.0;
    q = q * s2 + 1.0 / 9.0;
    q = q * s2 + 1.0 / 7.0;
    q = q * s2 + 1.0 / 5.0;
    q = q * s2 + 1.0 / 3.0;
    q = q * s2 + 1.0;
    const double lm = 2.0 * s * q;
    const double de = (double)e;
    return de * kLn2Hi + (de * kLn2Lo + lm);
}

__device__ __forceinline__ void sincos(double x, double *sn, double *cs)
{
    const double k = floor(x * k2OverPi + 0.5);
    const double r = ((x - k * kPio2_1) - k * kPio2_2) - k * kPio2_3;
    const double r2 = r * r;
    double ps = -1.0 / 121645100408832000.0;
    ps = ps * r2 + 1.0 / 355687428096000.0;
    ps = ps * r2 - 1.0 / 1307674368000.0;
    ps = ps * r2 + 1.0 / 6227020800.0;
    ps = ps * r2 - 1.0 / 39916800.0;
    ps = ps * r2 + 1.0 / 362880.0;
    ps = ps * r2 - 1.0 / 5040.0;
    ps = ps * r2 + 1.0 / 120.0;
    ps = ps * r2 - 1.0 / 6.0;
    ps = ps * r2 + 1.0;
    const double sr = r * ps;
    double pc = 1.0 / 2432902008176640000.0;
    pc = pc * r2 - 1.0 / 6402373705728000.0;
    pc = pc * r2 + 1.0 / 20922789888000.0;
    pc = pc * r2 - 1.0 / 87178291200.0;
    pc = pc * r2 + 1.0 / 479001600.0;
    pc = pc * r2 - 1.0 / 3628800.0;
    pc = pc * r2 + 1.0 / 40320.0;
    pc = pc * r2 - 1.0 / 720.0;
    pc = pc * r2 + 1.0 / 24.0;
    pc = pc * r2 - 0.5;
    pc = pc * r2 + 1.0;
    const double cr = pc;
    const int q = (int)((long long)k & 3);
    if (q == 0)      { *sn = sr;  *cs = cr;  }
    else if (q == 1) { *sn = cr;  *cs = -sr; }
    else if (q == 2) { *sn = -sr; *cs = -cr; }
    else             { *sn = -cr; *cs = sr;  }
}

__device__ __forceinline__ double tanh(double x)
{
    const double a = fabs(x);
    double t;
    if (a > 20.0) {
        t = 1.0;
    } else {
        const double e = dm::exp(2.0 * a);
        t = 1.0 - 2.0 / (e + 1.0);
    }
    return (x < 0.0) ? -t : t;
}

__device__ __forceinline__ double atan(double x)
{
    double a = fabs(x);
    int inv = 0;
    if (a > 1.0) { a = 1.0 / a; inv = 1; }
    double base = 0.0, y = a;
    if (a > 0.66817863791929891) {
        y = (a - 1.0) / (a + 1.0);
        base = kPi_4;
    } else if (a > 0.19891236737965800) {
        y = (a - kTanPi_8) / (1.0 + a * kTanPi_8);
        base = kPi_8;
    }
    const double y2 = y * y;
    double q = -1.0 / 23.0;
    q = q * y2 + 1.0 / 21.0;
    q = q * y2 - 1.0 / 19.0;
    q = q * y2 + 1.0 / 17.0;
    q = q * y2 - 1.0 / 15.0;
    q = q * y2 + 1.0 / 13.0;
    q = q * y2 - 1.0 / 11.0;
    q = q * y2 + 1.0 / 9.0;
    q = q * y2 - 1.0 / 7.0;
    q = q * y2 + 1.0 / 5.0;
    q = q * y2 - 1.0 / 3.0;
    q = q * y2 + 1.0;
    double res = base + y * q;
    if (inv) res = kPi_2 - res;
    return (x < 0.0) ? -res : res;
}

}  // namespace dm
}  // namespace cosmica
