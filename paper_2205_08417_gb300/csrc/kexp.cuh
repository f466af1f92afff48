// FP64 exponential for the quadrature sums, by the table-driven method of P. T. P. Tang
// ("Table-driven implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989), written from the mathematics with a 2048-entry table:
//   k = nearest integer to x * 2048 / ln2,  k = 2048 m + j (0 <= j < 2048),
//   r = x - k ln2/2048 (two-part constant, |r| <= ln2/4096),
//   exp(x) = 2^m * T_j * (1 + p(r)),  T_j = 2^(j/2048) (table, correctly rounded),
//   p(r) = r + r^2/2 + r^3/6 (truncation error below r^4/24 < 3.5e-17, a sixth of an ulp of 1,
//   for |r| <= ln2/4096).
// Eight FP64-pipe instructions on the common path (2 to round x to the table index, 2 for the
// two-part reduction, 3 for the polynomial, 1 for the table scaling); the scaling by 2^m is an
// integer add to the exponent field, and the range test reads the high word as an integer.
// Arguments below -707 return 0 (the true value is below 1e-307, a weight no sum here can see),
// above 709.78 return +inf, and NaN propagates.
#pragma once

namespace kitrt_dev {

constexpr int kExpTableBits = 11;  // 2^11 = 2048 table entries

__device__ __forceinline__ double kexp(double x, const double *__restrict__ tab)
{
    const double kInvL = 2954.639443740597;           // 2048 / ln2
    const double kL1 = 0.0003384507717577858;         // ln2/2048, leading part
    const double kL2 = 1.1323470770733885e-20;        // ln2/2048 - kL1
    const double kShift = 6755399441055744.0;         // 1.5 * 2^52: rounds to an integer
    // |x| < 512 is tested on the high word in integer arithmetic (the FP64 pipe is the narrow
    // resource); only the rare rest is compared in FP64
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40800000) {
        if (!(x > -707.0)) return x != x ? x : 0.0;
        if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    }
    const double t = fma(x, kInvL, kShift);
    const int k = __double2loint(t);
    const double kf = t - kShift;
    double r = fma(-kf, kL1, x);
    r = fma(-kf, kL2, r);
    // 1 + p(r) = exp(r) to degree 3: the truncation r^4/24 < 3.5e-17 for |r| <= ln2/4096
    const double q = fma(r, 1.0 / 6.0, 0.5);
    const double p = fma(r * r, q, r);
    const double Tj = __ldg(tab + (k & ((1 << kExpTableBits) - 1)));
    const double y = fma(Tj, p, Tj);
    const long long bits = __double_as_longlong(y) + ((long long)(k >> kExpTableBits) << 52);
    return __longlong_as_double(bits);
}

}  // namespace kitrt_dev
