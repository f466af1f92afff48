// Sum-factorised quadrature sums of the closure's dual on the folded product rule
// [Sec. 3.2, Eq. spherical-coordinatesProduct: Gauss-Legendre points in mu times equally spaced
// azimuths; Sec. 3.1: real spherical harmonics m_c = N_l^|k| P_l^|k|(mu) T_k(phi)].
//
// On a ring (one |mu|) every basis function is a Legendre factor times an azimuthal factor
// T_k(phi) (1, sqrt2 cos(k phi) or sqrt2 sin(|k| phi)), so
//   exponent   z(mu_r, phi) = alpha . m = sum_{k=-N..N} A_k(r) T_k(phi),
//              A_k(r) = sum_{c: k(c) = k} alpha_c P_c(mu_r)                 (once per ring),
//   moments    V_c = sum_r w_r P_c(mu_r) B_k(c)(r),  B_k(r) = sum_phi e(mu_r, phi) T_k(phi).
// The azimuths of a ring come in pairs (phi, 2 pi - phi) whose cosines agree and whose sines are
// opposite, so with C = sum_{k>=0} A_k T_k and S = sum_{k<0} A_k T_k at the pair's first point,
//   z = C + S and z' = C - S,   B_k += (e + e') T_k (k >= 0),   B_k += (e - e') T_k (k < 0).
// A pass over a cell's Q' points then costs about (2N+3)/2 FP64 operations per point for the
// exponent and (2L+3)/2 for moments up to degree L, instead of n and nmom(L) per point, plus n and
// nmom(L) per ring. The ring's remaining pair, (0, pi), has no sine terms and is summed directly.
//
// Tables (built by kitrt_mn_init in this point order): pair p covers folded points 2p and 2p+1;
// ring of pair p = p / P for p < npair (P pairs per ring), the all-zero row R for padding pairs;
// pair 0 of each ring is the (0, pi) pair. ptrig [npair_padded x (4N+1)]: T_0..T_2N at the pair's
// first point (cosines), then sqrt2 sin(k phi), k = 1..2N (for the (0, pi) pair: T_k(pi)).
// ringP, ringWP [(R+1) x n2]: P_c(mu_r) and w_r P_c(mu_r) over the degree-2N basis.
#pragma once

#include "kexp.cuh"
#include "kitrt_internal.cuh"

namespace kitrt_dev {

// Position of azimuthal index k in a coefficient vector of degree L: k >= 0 at k, k < 0 at L+|k|.
__host__ __device__ constexpr int kslot(int L, int k) { return k >= 0 ? k : L - k; }
// Index of basis function (l, k), l + |k| even, in the order l ascending, then k ascending.
__host__ __device__ constexpr int cindex(int l, int k) { return l * (l + 1) / 2 + (k + l) / 2; }

// Exponent coefficients A_k of one ring from the trial alpha (degree NN).
template <int NN>
__device__ __forceinline__ void ring_coeffs(const double (&at)[(NN + 1) * (NN + 2) / 2],
                                            const double *__restrict__ Pr, double (&A)[2 * NN + 1])
{
#pragma unroll
    for (int j = 0; j < 2 * NN + 1; ++j) A[j] = 0.0;
#pragma unroll
    for (int l = 0; l <= NN; ++l)
#pragma unroll
        for (int k = -l; k <= l; k += 2) {
            const int c = cindex(l, k);
            A[kslot(NN, k)] = fma(at[c], __ldg(Pr + c), A[kslot(NN, k)]);
        }
}

// Moments of the finished ring: V_c += w_r P_c(mu_r) B_k(c), c over the degree-LB basis; the
// azimuthal sums are cleared for the next ring.
template <int LB, typename Acc>
__device__ __forceinline__ void ring_flush(const double *__restrict__ wPr, double (&B)[2 * LB + 1],
                                           Acc &&V)
{
#pragma unroll
    for (int l = 0; l <= LB; ++l)
#pragma unroll
        for (int k = -l; k <= l; k += 2) {
            const int c = cindex(l, k);
            double &v = V(c);
            v = fma(__ldg(wPr + c), B[kslot(LB, k)], v);
        }
#pragma unroll
    for (int j = 0; j < 2 * LB + 1; ++j) B[j] = 0.0;
}

// An exponential (a non-negative double, or +inf) rounded to float in integer arithmetic, so that
// the narrow FP64 pipe does not convert it: the exponent is rebiased and the mantissa rounded
// half away from zero at bit 29 (a carry into the exponent is the correct result); values below
// the smallest normal float give 0, values beyond the float range give +inf.
__device__ __forceinline__ float exp_to_float(double e)
{
    const long long b = __double_as_longlong(e);
    const int ex = (int)(b >> 52);  // sign is 0
    if (ex < 1023 - 126) return 0.0f;
    const long long f = ((b + (1LL << 28)) >> 29) - ((long long)(1023 - 127) << 23);
    return f >= (255LL << 23) ? __int_as_float(0x7f800000) : __int_as_float((int)f);
}

// Conversions done in integer arithmetic, so that the narrow FP64 pipe does not execute them.
// Whether a double is finite (exponent field not all ones).
__device__ __forceinline__ bool finite_bits(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// A finite double rounded to float: the exponent rebiased and the mantissa rounded half away from
// zero at bit 29 (a carry into the exponent is the correct result); magnitudes below the smallest
// normal float give a signed zero, magnitudes beyond the float range a signed infinity.
__device__ __forceinline__ float d2f_bits(double x)
{
    const long long b = __double_as_longlong(x);
    const long long mag = b & 0x7fffffffffffffffLL;
    const int sign = (int)((unsigned long long)b >> 32) & (int)0x80000000u;
    if ((int)(mag >> 52) < 1023 - 126) return __int_as_float(sign);
    long long f = ((mag + (1LL << 28)) >> 29) - ((long long)(1023 - 127) << 23);
    if (f >= (255LL << 23)) f = 255LL << 23;
    return __int_as_float((int)f | sign);
}

// A float widened to double exactly; subnormal floats give a signed zero, infinities and NaNs
// stay infinities and NaNs.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned mag = b & 0x7fffffffu;
    if (mag < 0x00800000u) return __longlong_as_double((long long)sign);
    if (mag >= 0x7f800000u)
        return __longlong_as_double((long long)(sign | 0x7ff0000000000000ULL |
                                                ((unsigned long long)(mag & 0x7fffffu) << 29)));
    return __longlong_as_double(
        (long long)(sign | (((unsigned long long)mag << 29) + ((unsigned long long)(1023 - 127) << 52))));
}

// exp for an exponent already scaled by 2048 / ln2 (s = x * 2048/ln2, so exp(x) = 2^(s/2048)),
// with two FP64-pipe instructions on the common path instead of kexp's eight. Tang's table
// reduction as in kexp, rearranged for the scaled argument:
//   k = an integer within 0.5625 of s, k = 2048 m + j,   r = s - k (exact, |r| <= 0.5625),
//   2^(s/2048) = 2^m (T_j + T_j rho + T_j h),  rho = r ln2/2048 (|rho| <= 1.91e-4),
//   h = rho^2/2 + rho^3/6 + rho^4/24 (truncation below rho^5/120 < 3e-21),
// with T_j = 2^(j/2048) and C_j = T_j ln2/2048 from the two halves of the table.
// k comes from s rounded to float (|s| < 2^21 there, so within 1/16 of s) and rounded to an
// integer by the float shift 1.5 * 2^23; k as a double and the float of r are formed in integer
// arithmetic. T_j h (below 3.6e-8) is formed in FP32 and added to T_j in integer arithmetic as a
// fixed-point count of T_j's ulps (2^-52, as T_j is in [1, 2) and the sum stays below 2). Its
// FP32 rounding, about 5e-7 of T_j h, bounds the relative error of the result by about 1e-14.
// The two FP64 instructions are r = s - k and C_j r + (T_j + T_j h) (one rounding). The range
// handling is kexp's, in scaled units: arguments below -707 (scaled) return 0, above 709.78
// return +inf, NaN propagates.
__device__ __forceinline__ double kexp_scaled(double s, const double *__restrict__ tab)
{
    const float kC2 = 5.727446250602952e-08f;  // (ln2/2048)^2 / 2
    const float kC3 = 6.46152879466011e-12f;   // (ln2/2048)^3 / 6
    const float kC4 = 5.467273155028592e-16f;  // (ln2/2048)^4 / 24
    const float kShiftF = 12582912.0f;         // 1.5 * 2^23: rounds a float below 2^22 to an integer
    // |s| < 512 * 2048/ln2 is tested on the high word (0x41371547 is that bound's high word)
    if ((__double2hiint(s) & 0x7fffffff) >= 0x41371547) {
        if (!(s > -2088930.0867246022)) return s != s ? s : 0.0;  // -707 * 2048/ln2
        if (s > 2097143.984378201) return __longlong_as_double(0x7ff0000000000000LL);  // 709.78 * 2048/ln2
    }
    const float tf = __fadd_rn(d2f_bits(s), kShiftF);
    const int k = __float_as_int(tf) - 0x4B400000;  // the integer tf - 1.5 * 2^23
    const double r = s - f2d_bits(__fsub_rn(tf, kShiftF));
    const float rf = d2f_bits(r);
    const int j = k & ((1 << kExpTableBits) - 1);
    const long long tb = __double_as_longlong(__ldg(tab + j));
    const double Cj = __ldg(tab + (1 << kExpTableBits) + j);
    // T_j h in FP32, with T_j rounded to float from its bits (T_j in [1, 2): exponent field 0x3ff)
    const float tjf = __int_as_float(0x3f800000 | (int)(((tb + (1LL << 28)) >> 29) & 0x7fffff));
    const float hq = fmaf(rf, fmaf(rf, kC4, kC3), kC2);
    const float th = __fmul_rn(__fmul_rn(__fmul_rn(rf, rf), hq), tjf);
    // th in units of 2^-52, rounded: th = mant 2^(e - 150) with e its exponent field (th >= 0,
    // e <= 102), so th 2^52 = mant 2^(e - 98); a zero or subnormal th (e = 0) gives 0
    const int tbits = __float_as_int(th);
    const int e = tbits >> 23;
    const unsigned mant = (unsigned)(tbits & 0x7fffff) | 0x800000u;
    const int sh = e - 98;
    const unsigned fx = sh >= 0 ? mant << sh : ((mant >> min(-sh - 1, 31)) + 1u) >> 1;
    const double y0 = __longlong_as_double(tb + (long long)fx);  // T_j + T_j h
    const double y = fma(Cj, r, y0);
    const long long bits = __double_as_longlong(y) + ((long long)(k >> kExpTableBits) << 52);
    return __longlong_as_double(bits);
}

// One pair of points: both exponentials (e1 at the pair's first point, e2 at its mirror, or at
// phi = 0 and phi = pi for the ring's (0, pi) pair) and their azimuthal sums up to degree LB.
// t is the pair's row of ptrig (row width 4 NN + 1). SCALED: the coefficients A are those of the
// exponent times 2048/ln2, and the exponentials come from kexp_scaled.
template <int NN, int LB, bool SCALED = false>
__device__ __forceinline__ void pair_eval(const double (&A)[2 * NN + 1], const double *__restrict__ t,
                                          bool zero_pi, const double *__restrict__ exptab,
                                          double (&B)[2 * LB + 1], double &e1, double &e2)
{
    constexpr int L2 = 2 * NN;  // sines of the row start at t[L2 + 1]
    if (!zero_pi) {
        double c = A[0];  // T_0 = 1
#pragma unroll
        for (int k = 1; k <= NN; ++k) c = fma(A[k], __ldg(t + k), c);
        double s = A[NN + 1] * __ldg(t + L2 + 1);
#pragma unroll
        for (int k = 2; k <= NN; ++k) s = fma(A[NN + k], __ldg(t + L2 + k), s);
        e1 = SCALED ? kexp_scaled(c + s, exptab) : kexp(c + s, exptab);
        e2 = SCALED ? kexp_scaled(c - s, exptab) : kexp(c - s, exptab);
        const double ep = e1 + e2, em = e1 - e2;
        B[0] += ep;
#pragma unroll
        for (int k = 1; k <= LB; ++k) B[k] = fma(ep, __ldg(t + k), B[k]);
#pragma unroll
        for (int k = 1; k <= LB; ++k) B[LB + k] = fma(em, __ldg(t + L2 + k), B[LB + k]);
    } else {
        double z1 = A[0], z2 = A[0];
#pragma unroll
        for (int k = 1; k <= NN; ++k) {
            z1 = fma(A[k], __ldg(t + k), z1);
            z2 = fma(A[k], __ldg(t + L2 + k), z2);
        }
        e1 = SCALED ? kexp_scaled(z1, exptab) : kexp(z1, exptab);
        e2 = SCALED ? kexp_scaled(z2, exptab) : kexp(z2, exptab);
        B[0] += e1 + e2;
#pragma unroll
        for (int k = 1; k <= LB; ++k) B[k] = fma(e1, __ldg(t + k), fma(e2, __ldg(t + L2 + k), B[k]));
    }
}

// Split of a sweep's work: tiles of 128 listed cells times parts of the quadrature (units of 16
// pairs). When few cells are listed each tile's quadrature is split over up to `nunits` parts so
// that every SM gets work; part j of list slot i lands in column j * cnt + i of the accumulator,
// and the Newton kernel adds the parts in order (deterministic). The same function sizes the
// split in the sweep and in its consumer.
struct SweepSplit {
    int tiles, parts, units_per_part;
};
__host__ __device__ inline SweepSplit sweep_split(int cnt, int target_items, int nunits)
{
    SweepSplit sp;
    sp.tiles = (cnt + 127) / 128;
    int ks = sp.tiles > 0 && target_items > 0 ? (target_items + sp.tiles - 1) / sp.tiles : 1;
    ks = ks < 1 ? 1 : (ks > nunits ? nunits : ks);
    sp.units_per_part = (nunits + ks - 1) / ks;
    sp.parts = (nunits + sp.units_per_part - 1) / sp.units_per_part;
    return sp;
}

}  // namespace kitrt_dev
