// crp_fp64.cuh -- FP64 arithmetic of the method shared by the FP64 propagate kernel and the
// adjoint kernels: periodic trilinear lookup, Lorentz force, Cash & Karp (1990) attempt,
// error ratio. Translation units including it are compiled with --fmad=false so that every
// formula is evaluated exactly as written, in the stated order; the fused multiply-adds of
// the reading are explicit (__fma_rn).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "crp_internal.h"
#include "crp_math.cuh"

namespace crp {
namespace fp64 {

constexpr unsigned kFull = 0xffffffffu;

// Cash & Karp (1990) tableau; b - b* reduced to single rationals.
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 3.0 / 10.0, A42 = -9.0 / 10.0, A43 = 6.0 / 5.0;
constexpr double A51 = -11.0 / 54.0, A52 = 5.0 / 2.0, A53 = -70.0 / 27.0, A54 = 35.0 / 27.0;
constexpr double A61 = 1631.0 / 55296.0, A62 = 175.0 / 512.0, A63 = 575.0 / 13824.0,
                 A64 = 44275.0 / 110592.0, A65 = 253.0 / 4096.0;
constexpr double B1 = 37.0 / 378.0, B3 = 250.0 / 621.0, B4 = 125.0 / 594.0, B6 = 512.0 / 1771.0;
constexpr double E1 = -277.0 / 64512.0, E3 = 6925.0 / 370944.0, E4 = -6925.0 / 202752.0,
                 E5 = -277.0 / 14336.0, E6 = 277.0 / 7084.0;

struct V3 { double x, y, z; };

template <int L>
__device__ __forceinline__ V3 corner(const FieldDev& F, long long node) {
    V3 g;
    if constexpr (L == LAYOUT_F32X4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(F.data) + node);
        g.x = (double)v.x; g.y = (double)v.y; g.z = (double)v.z;
    } else if constexpr (L == LAYOUT_F64X4) {
        const double2* p = reinterpret_cast<const double2*>(F.data) + 2 * node;
        const double2 a = __ldg(p), b = __ldg(p + 1);
        g.x = a.x; g.y = a.y; g.z = b.x;
    } else if constexpr (L == LAYOUT_BF16X4) {
        const ushort4 v = __ldg(reinterpret_cast<const ushort4*>(F.data) + node);
        g.x = (double)__uint_as_float((unsigned)v.x << 16) * F.scale;
        g.y = (double)__uint_as_float((unsigned)v.y << 16) * F.scale;
        g.z = (double)__uint_as_float((unsigned)v.z << 16) * F.scale;
    } else {
        const ushort4 v = __ldg(reinterpret_cast<const ushort4*>(F.data) + node);
        g.x = (double)__half2float(__ushort_as_half(v.x)) * F.scale;
        g.y = (double)__half2float(__ushort_as_half(v.y)) * F.scale;
        g.z = (double)__half2float(__ushort_as_half(v.z)) * F.scale;
    }
    return g;
}

// floor(r) as an integer and as a double, from the bits of r with integer instructions only
// (GB300 rounds and converts FP64 values on its FP64 pipe, which the lookups' arithmetic
// already saturates). Exact for |r| < 2^63, where it equals floor() and its conversion;
// beyond that, and for infinities and NaN, i = 0 and fl = r (any index is wrapped into the
// grid afterwards).
__device__ __forceinline__ void floor_split(double r, long long& i, double& fl) {
    constexpr long long kSign = (long long)0x8000000000000000ull;
    constexpr long long kMant = 0xFFFFFFFFFFFFFll;
    const long long b = __double_as_longlong(r);
    const int ef = (int)((b >> 52) & 0x7FF);
    const bool neg = b < 0;
    const long long mag = b & ~kSign;
    if (ef < 1023) {                                   // |r| < 1: floor is 0, -0 or -1
        const bool m1 = neg && mag != 0;
        i = m1 ? -1 : 0;
        fl = __longlong_as_double(m1 ? (long long)0xBFF0000000000000ull : (b & kSign));
    } else if (ef < 1075) {                            // 1 <= |r| < 2^52: fb fraction bits
        const int fb = 1075 - ef;
        const long long fm = (1ll << fb) - 1;
        const long long n = ((mag & kMant) | (kMant + 1)) >> fb;       // |trunc r|
        if (!neg) {
            i = n;
            fl = __longlong_as_double(b & ~fm);
        } else if ((mag & fm) == 0) {
            i = -n;
            fl = r;
        } else {                                       // floor = -(n + 1), n + 1 <= 2^52
            const long long k = n + 1;
            const int p = 63 - __clzll(k);
            i = -k;
            fl = __longlong_as_double(kSign | ((long long)(1023 + p) << 52) | ((k << (52 - p)) & kMant));
        }
    } else if (ef < 1086) {                            // 2^52 <= |r| < 2^63: integral
        const long long n = ((mag & kMant) | (kMant + 1)) << (ef - 1075);
        i = neg ? -n : n;
        fl = r;
    } else {
        i = 0;
        fl = r;
    }
}

// One axis of the periodic lookup: r = x (1/spacing) - o (1/spacing) with one rounding (oi is
// the product o (1/spacing), rounded once), i0 = floor(r) mod n, weights (1 - f, f). P2: the
// caller guarantees n is a power of two, and the 64-bit modulo's code (inlined at every
// lookup, never run for such grids) is left out of the kernel.
template <bool P2 = false>
__device__ __forceinline__ void axis(double x, double oi, double inv, int n, int pow2,
                                     long long& i0, long long& i1, double& w0, double& w1) {
    const double r = __fma_rn(x, inv, -oi);
    long long i;
    double fl;
    floor_split(r, i, fl);
    const double fr = r - fl;
    long long a;
    if (P2 || pow2) a = i & (long long)(n - 1);
    else { a = i % n; if (a < 0) a += n; }
    i0 = a;
    i1 = (a + 1 == n) ? 0 : a + 1;
    w0 = 1.0 - fr;
    w1 = fr;
}

// Modulation value M(x): scalar periodic trilinear lookup on the modulation grid, corners
// in the order 000, 001, ..., 111, weight ((w_x * w_y) * w_z), each corner added with one
// rounding (fused multiply-add from 0).
__device__ __forceinline__ double modulation(const FieldDev& F, double x, double y, double z) {
    long long ix0, ix1, iy0, iy1, iz0, iz1;
    double wx0, wx1, wy0, wy1, wz0, wz1;
    axis(x, F.moix, F.m_inv_spacing, F.mnx, F.mpow2, ix0, ix1, wx0, wx1);
    axis(y, F.moiy, F.m_inv_spacing, F.mny, F.mpow2, iy0, iy1, wy0, wy1);
    axis(z, F.moiz, F.m_inv_spacing, F.mnz, F.mpow2, iz0, iz1, wz0, wz1);
    const long long ny = F.mny, nz = F.mnz;
    const float* M = F.mod;
    const long long r00 = (ix0 * ny + iy0) * nz, r01 = (ix0 * ny + iy1) * nz;
    const long long r10 = (ix1 * ny + iy0) * nz, r11 = (ix1 * ny + iy1) * nz;
    const double m0 = (double)__ldg(M + r00 + iz0), m1 = (double)__ldg(M + r00 + iz1);
    const double m2 = (double)__ldg(M + r01 + iz0), m3 = (double)__ldg(M + r01 + iz1);
    const double m4 = (double)__ldg(M + r10 + iz0), m5 = (double)__ldg(M + r10 + iz1);
    const double m6 = (double)__ldg(M + r11 + iz0), m7 = (double)__ldg(M + r11 + iz1);
    const double w00 = wx0 * wy0, w01 = wx0 * wy1, w10 = wx1 * wy0, w11 = wx1 * wy1;
    double m = __fma_rn(w00 * wz0, m0, 0.0);
    m = __fma_rn(w00 * wz1, m1, m);
    m = __fma_rn(w01 * wz0, m2, m);
    m = __fma_rn(w01 * wz1, m3, m);
    m = __fma_rn(w10 * wz0, m4, m);
    m = __fma_rn(w10 * wz1, m5, m);
    m = __fma_rn(w11 * wz0, m6, m);
    m = __fma_rn(w11 * wz1, m7, m);
    return m;
}

// Trilinear periodic lookup; corners summed in the order 000, 001, ..., 111 (x, y, z),
// weight ((w_x * w_y) * w_z), each corner added with one rounding (fused multiply-add from
// 0). With M, the result is scaled by the modulation value.
// With H, every lookup also folds its cell index into *hh (the visited-cell sequence of a
// trajectory; no effect on the arithmetic). P2: the vector grid's sizes are powers of two.
template <int L, bool H = false, bool M = false, bool P2 = false>
__device__ __forceinline__ V3 field_b(const FieldDev& F, double x, double y, double z,
                                      unsigned long long* hh = nullptr) {
    long long ix0, ix1, iy0, iy1, iz0, iz1;
    double wx0, wx1, wy0, wy1, wz0, wz1;
    axis<P2>(x, F.oix, F.inv_spacing, F.nx, F.pow2, ix0, ix1, wx0, wx1);
    axis<P2>(y, F.oiy, F.inv_spacing, F.ny, F.pow2, iy0, iy1, wy0, wy1);
    axis<P2>(z, F.oiz, F.inv_spacing, F.nz, F.pow2, iz0, iz1, wz0, wz1);
    const long long ny = F.ny, nz = F.nz;
    if constexpr (H) *hh = *hh * 0x9E3779B97F4A7C15ull + (unsigned long long)((ix0 * ny + iy0) * nz + iz0) + 1ull;
    const long long r00 = (ix0 * ny + iy0) * nz, r01 = (ix0 * ny + iy1) * nz;
    const long long r10 = (ix1 * ny + iy0) * nz, r11 = (ix1 * ny + iy1) * nz;
    const V3 g0 = corner<L>(F, r00 + iz0), g1 = corner<L>(F, r00 + iz1);
    const V3 g2 = corner<L>(F, r01 + iz0), g3 = corner<L>(F, r01 + iz1);
    const V3 g4 = corner<L>(F, r10 + iz0), g5 = corner<L>(F, r10 + iz1);
    const V3 g6 = corner<L>(F, r11 + iz0), g7 = corner<L>(F, r11 + iz1);
    const double w00 = wx0 * wy0, w01 = wx0 * wy1, w10 = wx1 * wy0, w11 = wx1 * wy1;
    double t;
    V3 B;
#define CRP_CORNER(g, acc0x, acc0y, acc0z)                                                    \
    B.x = __fma_rn(t, g.x, acc0x); B.y = __fma_rn(t, g.y, acc0y); B.z = __fma_rn(t, g.z, acc0z)
    t = w00 * wz0; CRP_CORNER(g0, 0.0, 0.0, 0.0);
    t = w00 * wz1; CRP_CORNER(g1, B.x, B.y, B.z);
    t = w01 * wz0; CRP_CORNER(g2, B.x, B.y, B.z);
    t = w01 * wz1; CRP_CORNER(g3, B.x, B.y, B.z);
    t = w10 * wz0; CRP_CORNER(g4, B.x, B.y, B.z);
    t = w10 * wz1; CRP_CORNER(g5, B.x, B.y, B.z);
    t = w11 * wz0; CRP_CORNER(g6, B.x, B.y, B.z);
    t = w11 * wz1; CRP_CORNER(g7, B.x, B.y, B.z);
#undef CRP_CORNER
    if constexpr (M) {
        const double m = modulation(F, x, y, z);
        B.x = m * B.x; B.y = m * B.y; B.z = m * B.z;
    }
    return B;
}

struct Y6 { double x, y, z, ux, uy, uz; };

// f(y) = (u, kappa u x B(x)); a cross-product component a b - c d as kappa fma(a, b, -(c d)).
template <int L, bool H = false, bool M = false, bool P2 = false>
__device__ __forceinline__ Y6 deriv(const FieldDev& F, double kappa, const Y6& y,
                                    unsigned long long* hh = nullptr) {
    const V3 B = field_b<L, H, M, P2>(F, y.x, y.y, y.z, hh);
    Y6 k;
    k.x = y.ux; k.y = y.uy; k.z = y.uz;
    k.ux = kappa * __fma_rn(y.uy, B.z, -(y.uz * B.y));
    k.uy = kappa * __fma_rn(y.uz, B.x, -(y.ux * B.z));
    k.uz = kappa * __fma_rn(y.ux, B.y, -(y.uy * B.x));
    return k;
}

// dst = y + h * sum, the final addition fused; the sums chain fused multiply-adds left to
// right from a plain first product (zero tableau entries, b2 = b5 = 0 and b2 - b*2 = 0, are
// not summed).
#define CRP_STAGE(dst, expr)                                                           \
    do {                                                                               \
        dst.x = __fma_rn(h, expr(x), y.x);    dst.y = __fma_rn(h, expr(y), y.y);        \
        dst.z = __fma_rn(h, expr(z), y.z);    dst.ux = __fma_rn(h, expr(ux), y.ux);     \
        dst.uy = __fma_rn(h, expr(uy), y.uy); dst.uz = __fma_rn(h, expr(uz), y.uz);     \
    } while (0)

// One Cash-Karp attempt of size h from y with k1 = f(y).
template <int L, bool H = false, bool M = false, bool P2 = false>
__device__ __forceinline__ void ck_attempt(const FieldDev& F, double kappa, const Y6& y,
                                           const Y6& k1, double h, Y6& y5, Y6& err,
                                           unsigned long long* hh = nullptr) {
    Y6 t;
#define S2(c) (A21 * k1.c)
    CRP_STAGE(t, S2);
    const Y6 k2 = deriv<L, H, M, P2>(F, kappa, t, hh);
#define S3(c) __fma_rn(A32, k2.c, A31 * k1.c)
    CRP_STAGE(t, S3);
    const Y6 k3 = deriv<L, H, M, P2>(F, kappa, t, hh);
#define S4(c) __fma_rn(A43, k3.c, __fma_rn(A42, k2.c, A41 * k1.c))
    CRP_STAGE(t, S4);
    const Y6 k4 = deriv<L, H, M, P2>(F, kappa, t, hh);
#define S5(c) __fma_rn(A54, k4.c, __fma_rn(A53, k3.c, __fma_rn(A52, k2.c, A51 * k1.c)))
    CRP_STAGE(t, S5);
    const Y6 k5 = deriv<L, H, M, P2>(F, kappa, t, hh);
#define S6(c) __fma_rn(A65, k5.c, __fma_rn(A64, k4.c, __fma_rn(A63, k3.c, __fma_rn(A62, k2.c, A61 * k1.c))))
    CRP_STAGE(t, S6);
    const Y6 k6 = deriv<L, H, M, P2>(F, kappa, t, hh);
#define SB(c) __fma_rn(B6, k6.c, __fma_rn(B4, k4.c, __fma_rn(B3, k3.c, B1 * k1.c)))
    CRP_STAGE(y5, SB);
#define SE(c) (h * __fma_rn(E6, k6.c, __fma_rn(E5, k5.c, __fma_rn(E4, k4.c, __fma_rn(E3, k3.c, E1 * k1.c)))))
    err.x = SE(x); err.y = SE(y); err.z = SE(z);
    err.ux = SE(ux); err.uy = SE(uy); err.uz = SE(uz);
#undef S2
#undef S3
#undef S4
#undef S5
#undef S6
#undef SB
#undef SE
}

// Compares, minima and maxima of step sizes and error sums on their bit patterns, with
// integer instructions (GB300 runs FP64 compares and min/max on its FP64 pipe). Each helper
// equals the IEEE operation on the operand domain it states.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
// v == 0.0 (either sign), any v
__device__ __forceinline__ bool is_zero(double v) { return (dbits(v) << 1) == 0; }
// a <= b for a in [+0, +inf] or a NaN of either sign, b in [+0, +inf]
__device__ __forceinline__ bool le_sum(double a, double b) {
    return (unsigned long long)dbits(a) <= (unsigned long long)dbits(b);
}
// a <= b for a not NaN, b in [+0, +inf]; a < b for a not NaN, b in (+0, +inf]
__device__ __forceinline__ bool le_pos(double a, double b) { return dbits(a) <= dbits(b); }
__device__ __forceinline__ bool lt_pos(double a, double b) { return dbits(a) < dbits(b); }
// a == b for a, b not NaN
__device__ __forceinline__ bool eq_num(double a, double b) {
    const long long x = dbits(a), y = dbits(b);
    return x == y || ((x | y) << 1) == 0;
}
// fmax(a, b) for a not NaN, b in (+0, +inf]
__device__ __forceinline__ double max_pos(double a, double b) { return lt_pos(a, b) ? b : a; }
// fmin(fmax(v, lo), hi) for 0 < lo <= hi < +inf and any v but a signaling NaN (a quiet NaN
// gives lo, as fmax does)
__device__ __forceinline__ double clampd(double v, double lo, double hi) {
    const long long x = dbits(v);
    if ((x & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll || x < dbits(lo)) return lo;
    return x > dbits(hi) ? hi : v;
}

// Error of an attempt, kept squared: sx = |dx|^2, su = |du|^2, each ((a0^2 + a1^2) + a2^2).
// Accept iff the step has zero length or sx <= (h tol)^2 and su <= tol^2 (r <= 1 for
// r = max(|dx|/h, |du|)/tol, compared as squares; a NaN sum rejects).
__device__ __forceinline__ void error_sums(const Y6& e, double& sx, double& su) {
    sx = __fma_rn(e.z, e.z, __fma_rn(e.y, e.y, e.x * e.x));
    su = __fma_rn(e.uz, e.uz, __fma_rn(e.uy, e.uy, e.ux * e.ux));
}

__device__ __forceinline__ bool error_accept(double sx, double su, double h, double tol, double tol2) {
    if (is_zero(h)) return true;
    const double ht = h * tol;
    return le_sum(sx, ht * ht) && le_sum(su, tol2);
}

// Step-size controller. The factor is a heuristic, so only its inputs (the FP64 error sums)
// and its application (h times the factor, in FP64) are FP64; the factor itself is FP32 on
// the FP32 pipe. ctrl_log2: log2 of a non-negative double from its bits -- exponent plus
// log2 of the top 23 significand bits m in [1, 2) (truncated), m reduced to
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh s through s^7, s = (m - 1)/(m + 1); -inf for zero
// and subnormals, +inf for infinity and NaN.
__device__ __forceinline__ float ctrl_log2(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((b >> 52) & 0x7FFu);
    if (ef == 0x7FF) return __int_as_float(0x7f800000);
    if (ef == 0) return __int_as_float((int)0xff800000u);
    int e = ef - 1023;
    float m = __uint_as_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFFu));
    if (m > 0x1.6a09e6p+0f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float q = 0x1.24924ap-3f;                                  // 1/7
    q = __fadd_rn(__fmul_rn(q, s2), 0x1.99999ap-3f);           // 1/5
    q = __fadd_rn(__fmul_rn(q, s2), 0x1.555556p-2f);           // 1/3
    q = __fadd_rn(__fmul_rn(q, s2), 1.0f);
    const float ln_m = __fmul_rn(__fmul_rn(2.0f, s), q);
    return __fadd_rn((float)e, __fmul_rn(ln_m, 0x1.715476p+0f));   // 1/ln 2
}

// log2 r = max(log2 sx / 2 - log2 h, log2 su / 2) - log2 tol.
__device__ __forceinline__ float ctrl_log2r(double sx, double su, double h, float lg_tol) {
    const float lx = __fmul_rn(0.5f, __fsub_rn(ctrl_log2(sx), __fmul_rn(2.0f, ctrl_log2(h))));
    const float lu = __fmul_rn(0.5f, ctrl_log2(su));
    return __fsub_rn(fmaxf(lx, lu), lg_tol);
}

// 2^y in FP32 for y in [-126, 126] (the caller clamps): 2^floor(y) exactly times e^(f ln 2)
// (f the fractional part) by Taylor through x^8/8! in Horner order, the product rounded once.
__device__ __forceinline__ float pow2_series(float y) {
    const float n = floorf(y);
    const float x = __fmul_rn(__fsub_rn(y, n), 0x1.62e430p-1f);   // ln 2
    float q = 0x1.a01a02p-16f;                                 // 1/8!
    q = __fadd_rn(__fmul_rn(q, x), 0x1.a01a02p-13f);           // 1/7!
    q = __fadd_rn(__fmul_rn(q, x), 0x1.6c16c2p-10f);           // 1/6!
    q = __fadd_rn(__fmul_rn(q, x), 0x1.111112p-7f);            // 1/5!
    q = __fadd_rn(__fmul_rn(q, x), 0x1.555556p-5f);            // 1/4!
    q = __fadd_rn(__fmul_rn(q, x), 0x1.555556p-3f);            // 1/3!
    q = __fadd_rn(__fmul_rn(q, x), 0.5f);
    q = __fadd_rn(__fmul_rn(q, x), 1.0f);
    q = __fadd_rn(__fmul_rn(q, x), 1.0f);
    const float p2 = __int_as_float(((int)n + 127) << 23);
    return __fmul_rn(q, p2);
}

// 0.95 r^p clamped to [lo, hi]: y = p log2 r clamped to [-8, 8] (a NaN y counts as -8).
__device__ __forceinline__ float ctrl_factor(float log2r, float p, float lo, float hi) {
    const float y = fminf(fmaxf(__fmul_rn(p, log2r), -8.0f), 8.0f);
    return fminf(fmaxf(__fmul_rn(0.95f, pow2_series(y)), lo), hi);
}

// Exact widening of a normal float (the clamped factors) to double with integer
// instructions (the hardware conversion issues on the FP64 pipe).
__device__ __forceinline__ double widen_normal(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned hi = (u & 0x80000000u) | ((((u >> 23) & 0xFFu) + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// Exact widening of any float: normals with integer instructions, zeros, subnormals,
// infinities and NaN (rare here) by the conversion.
__device__ __forceinline__ double widen_f32(float f) {
    const unsigned e = (__float_as_uint(f) >> 23) & 0xFFu;
    return (e == 0u || e == 0xFFu) ? (double)f : widen_normal(f);
}

// Tabulated loss and photo-disintegration rates at gamma0 = E / (A m_p c^2), in FP32 from the
// FP64 state (the rates are a tabulated heuristic): x = (log2 E - log2(A m_p c^2)) log10 2 with
// the bit-level log2 of the step controller (the product in FP64); t = (x - x0) inv_dx clamped
// to [0, n - 1], j = floor t (at most n - 2), v = T_j + (t - j)(T_{j+1} - T_j) over the FP32
// table copies; rate = 2^(v log2 10), the exponent clamped to [-126, 126] (normal results).
// Returns false if the species lies outside the tables.
__device__ __forceinline__ bool table_rates_f32(const TablesDev& t, int A, int Z, double E,
                                                float& r_loss, float& r_pd) {
    r_loss = 0.0f;
    r_pd = 0.0f;
    const int N = A - Z;
    if (Z < 0 || N < 0 || Z > t.z_max || N > t.n_max) return false;
    const long long sp = (long long)Z * (t.n_max + 1) + N;
    const float lg = __fsub_rn(ctrl_log2(E), ctrl_log2(__dmul_rn((double)A, kMpC2)));
    const float x = __fmul_rn(lg, 0x1.344136p-2f);                  // log10 2
    float tt = __fmul_rn(__fsub_rn(x, t.x0_f), t.inv_dx_f);
    tt = fminf(fmaxf(tt, 0.0f), (float)(t.n_nodes - 1));
    int j = (int)floorf(tt);
    if (j > t.n_nodes - 2) j = t.n_nodes - 2;
    const float fr = __fsub_rn(tt, (float)j);
    if (t.has_loss[sp]) {
        const float* T = t.loss_f + sp * t.n_nodes;
        const float a = __ldg(T + j), b = __ldg(T + j + 1);
        const float y = __fmul_rn(__fadd_rn(a, __fmul_rn(fr, __fsub_rn(b, a))), 0x1.a934f0p+1f);  // log2 10
        r_loss = pow2_series(fminf(fmaxf(y, -126.0f), 126.0f));
    }
    if (t.has_pd[sp]) {
        const float* T = t.pd_f + sp * t.n_nodes;
        const float a = __ldg(T + j), b = __ldg(T + j + 1);
        const float y = __fmul_rn(__fadd_rn(a, __fmul_rn(fr, __fsub_rn(b, a))), 0x1.a934f0p+1f);
        r_pd = pow2_series(fminf(fmaxf(y, -126.0f), 126.0f));
    }
    return true;
}


// Mirror fold of one coordinate into [lo, hi] (hi = lo + L, inv = 1/L): returns true when
// the number of reflections is odd (the direction component reverses).
__device__ __forceinline__ bool reflect_axis(double& x, double lo, double hi, double L, double inv) {
    if (!(x < lo || x > hi)) return false;
    const double t = (x - lo) * inv;
    const double k = floor(t);
    const double r = t - k;
    const bool odd = fmod(k, 2.0) != 0.0;
    x = odd ? hi - r * L : lo + r * L;
    return odd;
}

__device__ __forceinline__ bool finite6(const Y6& y) {
    auto fin = [](double v) { return ((unsigned long long)dbits(v) >> 52 & 0x7FFu) != 0x7FFu; };
    return fin(y.x) && fin(y.y) && fin(y.z) && fin(y.ux) && fin(y.uy) && fin(y.uz);
}


}  // namespace fp64
}  // namespace crp
