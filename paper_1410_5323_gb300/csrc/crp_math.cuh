// crp_math.cuh -- device arithmetic of the method that must reproduce the stated FP64
// reading bit for bit: Philox4x32-10 streams, exp/log by the stated reduction + series,
// table interpolation. Translation units that include this for the FP64 form are
// compiled with --fmad=false so every operation below is one IEEE-rounded operation.
#pragma once
#include <cstdint>
#include "crp_internal.h"

namespace crp {

constexpr double kC = 299792458.0;          // speed of light, m/s
constexpr double kMpC2 = 938272088.16;      // proton rest energy, eV (CODATA 2018)

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) ---------------------------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// U in (0,1): 52 random bits m = (w0 << 20) | (w1 >> 12), U = (m + 1/2) 2^-52 (exact).
__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long uid,
                                            uint32_t k, uint32_t tag) {
    const U4 w = philox10((uint32_t)uid, (uint32_t)(uid >> 32), k, tag, (uint32_t)seed,
                          (uint32_t)(seed >> 32));
    const unsigned long long m = ((unsigned long long)w.a << 20) | (unsigned long long)(w.b >> 12);
    return __dmul_rn(__dadd_rn((double)m, 0.5), 0x1p-52);
}

// Removed nucleon is a proton iff (w0 mod A) < Z, w0 from counter (uid, k, tag 1).
__device__ __forceinline__ int nucleon_proton(unsigned long long seed, unsigned long long uid,
                                              uint32_t k, int A, int Z) {
    const U4 w = philox10((uint32_t)uid, (uint32_t)(uid >> 32), k, 1u, (uint32_t)seed,
                          (uint32_t)(seed >> 32));
    return (int)(w.a % (uint32_t)A) < Z;
}

// ---- exp / log: Cody & Waite reduction, ln 2 = head (32 bits) + tail ------------------
constexpr double kLn2Hi = 0x1.62e42feep-1;
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

// exp(x) = 2^n e^r, |r| <= ln2/2, e^r by Taylor through r^14/14! in Horner order, every
// step one fused multiply-add; r = (x - n ln2_hi) - n ln2_lo with fused products.
__device__ __forceinline__ double crp_exp(double x) {
    if (x != x) return x;
    if (x > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.1332191019412) return 0.0;
    const double n = floor(__fma_rn(x, kInvLn2, 0.5));
    const double r = __fma_rn(-n, kLn2Lo, __fma_rn(-n, kLn2Hi, x));
    double p = 1.0 / 87178291200.0;
    p = __fma_rn(p, r, 1.0 / 6227020800.0);
    p = __fma_rn(p, r, 1.0 / 479001600.0);
    p = __fma_rn(p, r, 1.0 / 39916800.0);
    p = __fma_rn(p, r, 1.0 / 3628800.0);
    p = __fma_rn(p, r, 1.0 / 362880.0);
    p = __fma_rn(p, r, 1.0 / 40320.0);
    p = __fma_rn(p, r, 1.0 / 5040.0);
    p = __fma_rn(p, r, 1.0 / 720.0);
    p = __fma_rn(p, r, 1.0 / 120.0);
    p = __fma_rn(p, r, 1.0 / 24.0);
    p = __fma_rn(p, r, 1.0 / 6.0);
    p = __fma_rn(p, r, 0.5);
    p = __fma_rn(p, r, 1.0);
    p = __fma_rn(p, r, 1.0);
    return ldexp(p, (int)n);
}

// log(x) = e ln2 + log m, m in [sqrt(1/2), sqrt(2)); log m = 2s + 2s t with s = (m-1)/(m+1)
// and t = s^2/3 + ... + s^22/23 (fused Horner in s^2); e ln2_lo + log m and e ln2_hi + that
// fused (e ln2_hi is exact).
__device__ __forceinline__ double crp_log(double x) {
    if (x != x) return x;
    if (x < 0.0) return __longlong_as_double(0x7ff8000000000000LL);
    if (x == 0.0) return __longlong_as_double(0xfff0000000000000LL);
    if (isinf(x)) return x;
    int e;
    double m = frexp(x, &e);
    if (m < kSqrtHalf) { m = __dmul_rn(m, 2.0); e = e - 1; }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double s2 = __dmul_rn(s, s);
    double p = 1.0 / 23.0;
    p = __fma_rn(p, s2, 1.0 / 21.0);
    p = __fma_rn(p, s2, 1.0 / 19.0);
    p = __fma_rn(p, s2, 1.0 / 17.0);
    p = __fma_rn(p, s2, 1.0 / 15.0);
    p = __fma_rn(p, s2, 1.0 / 13.0);
    p = __fma_rn(p, s2, 1.0 / 11.0);
    p = __fma_rn(p, s2, 1.0 / 9.0);
    p = __fma_rn(p, s2, 1.0 / 7.0);
    p = __fma_rn(p, s2, 1.0 / 5.0);
    p = __fma_rn(p, s2, 1.0 / 3.0);
    const double t = __dmul_rn(s2, p);
    const double s_2 = __dmul_rn(2.0, s);
    const double log_m = __fma_rn(s_2, t, s_2);
    const double de = (double)e;
    return __fma_rn(de, kLn2Hi, __fma_rn(de, kLn2Lo, log_m));
}

}  // namespace crp
