/*
 * crp_oracle.c -- plain FP64 CPU oracle for the 3D-mode propagation hot path of
 * "Cosmic ray propagation with CRPropa 3" (arXiv:1410.5323).
 *
 * TEST INFRASTRUCTURE: the slow, obviously correct reference the GPU path is checked
 * against. Only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant generator with the product library.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -pthread (no fused multiply-add, no
 * reassociation, so every FP64 operation is one IEEE-rounded operation in the order
 * written here).
 *
 * What each part follows (the paper gives the method qualitatively; the numerical
 * readings below are the ones stated in the design notes of this project):
 *   - per-step module sequence: propagation -> continuous loss -> interaction -> observer
 *     (Sec. 3.1, modular layout; modules called in turn until the particle is done);
 *   - step-size bidding, smallest bid wins (Sec. 3.1);
 *   - 3D deflection of charged nuclei in a gridded field (Sec. 2, Sec. 3.2 regular grids);
 *     equation of motion: ultra-relativistic Lorentz force in path length s,
 *     dx/ds = u, du/ds = (Z c / E) u x B;
 *   - integrator: Cash & Karp (1990) embedded RK4(5), 5th-order solution propagated;
 *   - continuous energy loss and photo-disintegration with nucleon secondaries (Sec. 2),
 *     from tabulated rates, sampled with Philox4x32-10 (Salmon et al. 2011).
 * Every function is pinned by a test that does not use this file's code (closed forms,
 * library routines, brute force, every bit pattern of the F16 storage); full
 * turbulent-field trajectories compose them and have no printed values in the paper.
 */
#include "crp_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- physical constants (readings; the paper states none) ---------------------- */
static const double C_LIGHT = 299792458.0;       /* m/s */
static const double MP_C2_EV = 938272088.16;     /* proton rest energy, eV (CODATA 2018) */

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5) ---------------- */
/* One round: two 32x32->64 multiplications, the high halves xored with the other
 * counter words and the round key, the words permuted. The key is bumped by the
 * Weyl constants (golden ratio, sqrt(3)-1) between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0,1) from counter (uid_lo, uid_hi, k, tag), key = seed:
 * 52 random bits m = (w0 << 20) | (w1 >> 12), U = (m + 1/2) * 2^-52 (exact in FP64). */
double orc_uniform(uint64_t seed, uint64_t uid, uint32_t k, uint32_t tag)
{
    uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), k, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t m = ((uint64_t)w[0] << 20) | (uint64_t)(w[1] >> 12);
    return ((double)m + 0.5) * 0x1p-52;
}

/* Photo-disintegration nucleon choice: the removed nucleon is a proton iff
 * (w0 mod A) < Z for the Philox word w0 of counter (uid, k, tag 1). */
static int nucleon_is_proton(uint64_t seed, uint64_t uid, uint32_t k, int32_t A, int32_t Z)
{
    uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), k, 1u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return (int32_t)(w[0] % (uint32_t)A) < Z;
}

/* ---- exp and log, evaluated by one stated algorithm ------------------------------
 * Cody & Waite (1980) argument reduction with ln 2 split into a 32-bit head (so that
 * n*head is exact) and a tail; the reduced argument goes through a truncated series.
 * Accuracy is pinned against the C library in the tests (<= 2 ulp). */
static const double LN2_HI = 0x1.62e42feep-1;           /* ln 2 truncated to 32 bits */
static const double LN2_LO = 0x1.a39ef35793c76p-33;     /* ln 2 - LN2_HI */
static const double INV_LN2 = 0x1.71547652b82fep+0;     /* 1/ln 2 */
static const double SQRT_HALF = 0x1.6a09e667f3bcdp-1;   /* sqrt(1/2) */

/* exp(x) = 2^n exp(r), x = n ln2 + r, |r| <= ln2/2; exp(r) by its Taylor series through
 * r^14/14! (truncation below 2^-60 on that interval), Horner order, each step one fused
 * multiply-add; r = (x - n ln2_hi) - n ln2_lo with the products fused (n ln2_hi is exact). */
double orc_exp(double x)
{
    if (x != x) return x;
    if (x > 709.782712893384) return INFINITY;
    if (x < -745.1332191019412) return 0.0;
    double n = floor(fma(x, INV_LN2, 0.5));
    double r = fma(-n, LN2_LO, fma(-n, LN2_HI, x));
    double p = 1.0 / 87178291200.0;          /* 1/14! */
    p = fma(p, r, 1.0 / 6227020800.0);       /* 1/13! */
    p = fma(p, r, 1.0 / 479001600.0);        /* 1/12! */
    p = fma(p, r, 1.0 / 39916800.0);         /* 1/11! */
    p = fma(p, r, 1.0 / 3628800.0);          /* 1/10! */
    p = fma(p, r, 1.0 / 362880.0);           /* 1/9!  */
    p = fma(p, r, 1.0 / 40320.0);            /* 1/8!  */
    p = fma(p, r, 1.0 / 5040.0);             /* 1/7!  */
    p = fma(p, r, 1.0 / 720.0);              /* 1/6!  */
    p = fma(p, r, 1.0 / 120.0);              /* 1/5!  */
    p = fma(p, r, 1.0 / 24.0);               /* 1/4!  */
    p = fma(p, r, 1.0 / 6.0);                /* 1/3!  */
    p = fma(p, r, 0.5);                      /* 1/2!  */
    p = fma(p, r, 1.0);                      /* 1/1!  */
    p = fma(p, r, 1.0);                      /* 1/0!  */
    return ldexp(p, (int)n);
}

/* log(x) = e ln2 + log(m), x = m 2^e with m in [sqrt(1/2), sqrt(2));
 * log(m) = 2 atanh(s) = 2s + 2s t, s = (m-1)/(m+1), |s| <= 0.1716, t = s^2/3 + s^4/5 + ...
 * through s^22/23 (Horner in s^2, fused), 2s + 2s t and e ln2_lo + log(m) fused, e ln2_hi
 * exact. */
double orc_log(double x)
{
    if (x != x) return x;
    if (x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (isinf(x)) return INFINITY;
    int e;
    double m = frexp(x, &e);
    if (m < SQRT_HALF) {
        m = m * 2.0;
        e = e - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 23.0;
    p = fma(p, s2, 1.0 / 21.0);
    p = fma(p, s2, 1.0 / 19.0);
    p = fma(p, s2, 1.0 / 17.0);
    p = fma(p, s2, 1.0 / 15.0);
    p = fma(p, s2, 1.0 / 13.0);
    p = fma(p, s2, 1.0 / 11.0);
    p = fma(p, s2, 1.0 / 9.0);
    p = fma(p, s2, 1.0 / 7.0);
    p = fma(p, s2, 1.0 / 5.0);
    p = fma(p, s2, 1.0 / 3.0);
    double t = s2 * p;                       /* s^2/3 + s^4/5 + ... */
    double s_2 = 2.0 * s;
    double log_m = fma(s_2, t, s_2);
    double de = (double)e;
    return fma(de, LN2_HI, fma(de, LN2_LO, log_m));
}

/* ---- field lookup: trilinear interpolation on a periodic regular grid (Sec. 3.2) --- */
static double bf16_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double f16_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int ex = (h >> 10) & 0x1f;
    int man = h & 0x3ff;
    double v;
    if (ex == 0) v = ldexp((double)man, -24);                       /* subnormal / zero */
    else if (ex == 31) v = man ? NAN : INFINITY;
    else v = ldexp((double)(man + 1024), ex - 25);
    return sign ? -v : v;
}

static double grid_at(const orc_field* f, int64_t i, int64_t j, int64_t k, int c)
{
    int64_t idx = ((i * f->ny + j) * f->nz + k) * 3 + c;
    switch (f->dtype) {
    case ORC_F64: return ((const double*)f->data)[idx];
    case ORC_F32: return (double)((const float*)f->data)[idx];
    case ORC_BF16: return bf16_to_double(((const uint16_t*)f->data)[idx]) * f->scale;
    default: return f16_to_double(((const uint16_t*)f->data)[idx]) * f->scale;
    }
}

/* Stored value of node (i, j, k), component c, widened to double (times the scale for
 * BF16/F16 storage): the value every lookup of that node reads (Sec. 3.2 regular grids). */
double orc_grid_value(const orc_field* f, int64_t i, int64_t j, int64_t k, int32_t c)
{
    return grid_at(f, i, j, k, c);
}

/* Modulation (Sec. 3.2): the scalar grid interpolated trilinearly, periodic over its own
 * extent (fractional index formed as for the field), corners summed in the order 000, ..., 111 with weight ((w_x * w_y) * w_z), each
 * corner added with one rounding, m = fma(w, M_corner, m) from m = 0. */
double orc_modulation_value(const orc_field* f, const double x[3])
{
    double inv = 1.0 / f->mod_spacing;
    int64_t dims[3] = {f->mod_nx, f->mod_ny, f->mod_nz};
    int64_t idx[3][2];
    double w[3][2];
    for (int a = 0; a < 3; ++a) {
        double r = fma(x[a], inv, -(f->mod_origin[a] * inv));
        double fl = floor(r);
        double fr = r - fl;
        int64_t i = (int64_t)fl;
        int64_t n = dims[a];
        int64_t i0 = ((i % n) + n) % n;
        idx[a][0] = i0;
        idx[a][1] = (i0 + 1) % n;
        w[a][0] = 1.0 - fr;
        w[a][1] = fr;
    }
    double m = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double wt = (w[0][a] * w[1][b]) * w[2][c];
                int64_t k = (idx[0][a] * f->mod_ny + idx[1][b]) * f->mod_nz + idx[2][c];
                double v = f->mod_dtype == ORC_F64 ? ((const double*)f->mod_data)[k]
                                                   : (double)((const float*)f->mod_data)[k];
                m = fma(wt, v, m);
            }
    return m;
}

/* Fractional index r = x (1/spacing) - origin (1/spacing), the product origin (1/spacing)
 * rounded once and r in one fused multiply-add; cell i0 = floor(r) wrapped modulo n;
 * weights (1 - f, f) with f = r - floor(r). B is the sum over the 8 cell corners, taken
 * in the order (a,b,c) = 000, 001, 010, ..., 111, of ((w_x,a * w_y,b) * w_z,c) * B_corner,
 * each corner added with one rounding: B = fma(w, B_corner, B) from B = 0. */
void orc_field_value(const orc_field* f, const double x[3], double B[3])
{
    double inv = 1.0 / f->spacing;
    int64_t dims[3] = {f->nx, f->ny, f->nz};
    int64_t idx[3][2];
    double w[3][2];
    for (int a = 0; a < 3; ++a) {
        double r = fma(x[a], inv, -(f->origin[a] * inv));
        double fl = floor(r);
        double fr = r - fl;
        int64_t i = (int64_t)fl;
        int64_t n = dims[a];
        int64_t i0 = ((i % n) + n) % n;
        idx[a][0] = i0;
        idx[a][1] = (i0 + 1) % n;
        w[a][0] = 1.0 - fr;
        w[a][1] = fr;
    }
    B[0] = 0.0; B[1] = 0.0; B[2] = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double wt = (w[0][a] * w[1][b]) * w[2][c];
                for (int q = 0; q < 3; ++q)
                    B[q] = fma(wt, grid_at(f, idx[0][a], idx[1][b], idx[2][c], q), B[q]);
            }
    if (f->mod_data) {
        double m = orc_modulation_value(f, x);
        for (int q = 0; q < 3; ++q) B[q] = m * B[q];
    }
}

/* ---- equation of motion (Sec. 2, 3D deflections) -------------------------------- */
/* y = (x, u); f(y) = (u, kappa u x B(x)), kappa = Z c / E (1/(T m)); each cross-product
 * component a b - c d as kappa * fma(a, b, -(c d)). */
void orc_deriv(const orc_field* f, double kappa, const double y[6], double k[6])
{
    double B[3];
    orc_field_value(f, y, B);
    k[0] = y[3];
    k[1] = y[4];
    k[2] = y[5];
    k[3] = kappa * fma(y[4], B[2], -(y[5] * B[1]));
    k[4] = kappa * fma(y[5], B[0], -(y[3] * B[2]));
    k[5] = kappa * fma(y[3], B[1], -(y[4] * B[0]));
}

/* ---- Cash & Karp (1990) embedded Runge-Kutta 4(5) tableau --------------------------- */
static const double CK_A[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0},
};
/* fifth-order weights b_i */
static const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
/* b_i - b*_i (fifth minus embedded fourth order), each reduced to one exact rational */
static const double CK_E[6] = {-277.0 / 64512.0, 0.0, 6925.0 / 370944.0, -6925.0 / 202752.0,
                               -277.0 / 14336.0, 277.0 / 7084.0};

/* One attempt of step h from y (k1 = f(y) given): stages y_i = y + h * sum_j a_ij k_j,
 * sums taken left to right; y5 = y + h * sum_i b_i k_i; err = h * sum_i (b_i - b*_i) k_i.
 * Every term after the first of a sum, and the final y + h * sum, is added with one rounding
 * (fused multiply-add); the first term and h * sum of err are plain products. */
void orc_ck_attempt(const orc_field* f, double kappa, const double y[6], const double k1[6],
                    double h, double y5[6], double err[6])
{
    double k[6][6];
    for (int c = 0; c < 6; ++c) k[0][c] = k1[c];
    for (int i = 1; i < 6; ++i) {
        double yt[6];
        for (int c = 0; c < 6; ++c) {
            double acc = CK_A[i][0] * k[0][c];
            for (int j = 1; j < i; ++j) acc = fma(CK_A[i][j], k[j][c], acc);
            yt[c] = fma(h, acc, y[c]);
        }
        orc_deriv(f, kappa, yt, k[i]);
    }
    for (int c = 0; c < 6; ++c) {
        double acc = CK_B5[0] * k[0][c];
        for (int j = 1; j < 6; ++j) acc = fma(CK_B5[j], k[j][c], acc);
        y5[c] = fma(h, acc, y[c]);
    }
    for (int c = 0; c < 6; ++c) {
        double acc = CK_E[0] * k[0][c];
        for (int j = 1; j < 6; ++j) acc = fma(CK_E[j], k[j][c], acc);
        err[c] = h * acc;
    }
}

/* Error of one attempt (Sec. 3.1: a step is kept when its estimated error is within the
 * requested accuracy), r = max(|dx|/h, |du|) / tol with Euclidean norms. The norms stay
 * squared: sx = |dx|^2 and su = |du|^2, each ((a0^2 + a1^2) + a2^2) with every square after
 * the first added with one rounding. */
void orc_error_sums(const double err[6], double* sx, double* su)
{
    *sx = fma(err[2], err[2], fma(err[1], err[1], err[0] * err[0]));
    *su = fma(err[5], err[5], fma(err[4], err[4], err[3] * err[3]));
}

/* r <= 1 compared as squares in FP64: sx <= (h tol)^2 and su <= tol^2, each product
 * rounded once; a zero-length step is always accepted (r = 0). A NaN sum rejects. */
int orc_error_accept(double sx, double su, double h, double tol)
{
    if (h == 0.0) return 1;
    double ht = h * tol;
    return sx <= ht * ht && su <= tol * tol;
}

/* ---- step-size controller (a heuristic: only its inputs and outputs are FP64) ----------
 * log2 of a non-negative double in FP32, from its bits: the unbiased exponent e plus log2 m
 * of the top 23 significand bits (truncated) m in [1, 2), reduced to [sqrt(1/2), sqrt(2)),
 * with ln m = 2 atanh s = 2 (s + s^3/3 + s^5/5 + s^7/7), s = (m - 1)/(m + 1) (truncation
 * error below 3e-8). Zero and subnormal inputs give -inf (no error), infinity and NaN +inf
 * (an infinite error). */
float orc_ctrl_log2(double v)
{
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    int ef = (int)((b >> 52) & 0x7FFu);
    if (ef == 0x7FF) return INFINITY;
    if (ef == 0) return -INFINITY;
    int e = ef - 1023;
    uint32_t mb = 0x3F800000u | (uint32_t)((b >> 29) & 0x7FFFFFu);
    float m;
    memcpy(&m, &mb, sizeof m);
    if (m > 0x1.6a09e6p+0f) {        /* sqrt(2) */
        m = m * 0.5f;
        e = e + 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float q = 0x1.24924ap-3f;        /* 1/7 */
    q = q * s2 + 0x1.99999ap-3f;     /* 1/5 */
    q = q * s2 + 0x1.555556p-2f;     /* 1/3 */
    q = q * s2 + 1.0f;
    float ln_m = (2.0f * s) * q;
    return (float)e + ln_m * 0x1.715476p+0f;    /* 1/ln 2 */
}

/* log2 r = max(log2 sx / 2 - log2 h, log2 su / 2) - log2 tol, in FP32. */
float orc_ctrl_log2r(double sx, double su, double h, double tol)
{
    float lx = 0.5f * (orc_ctrl_log2(sx) - 2.0f * orc_ctrl_log2(h));
    float lu = 0.5f * orc_ctrl_log2(su);
    return fmaxf(lx, lu) - orc_ctrl_log2(tol);
}

/* 2^y in FP32 for y in [-126, 126] (the caller clamps): 2^n exactly (n = floor y) times
 * e^(f ln 2), f = y - n in [0, 1), by Taylor through the 8th power in Horner order (truncation
 * error below 1e-7); the product q 2^n rounded once. */
static float pow2_series(float y)
{
    float n = floorf(y);
    float x = (y - n) * 0x1.62e430p-1f;         /* ln 2 */
    float q = 0x1.a01a02p-16f;                  /* 1/8! */
    q = q * x + 0x1.a01a02p-13f;                /* 1/7! */
    q = q * x + 0x1.6c16c2p-10f;                /* 1/6! */
    q = q * x + 0x1.111112p-7f;                 /* 1/5! */
    q = q * x + 0x1.555556p-5f;                 /* 1/4! */
    q = q * x + 0x1.555556p-3f;                 /* 1/3! */
    q = q * x + 0.5f;
    q = q * x + 1.0f;
    q = q * x + 1.0f;
    uint32_t pb = (uint32_t)((int)n + 127) << 23;
    float p2;
    memcpy(&p2, &pb, sizeof p2);
    return q * p2;
}

/* 0.95 r^p = 0.95 2^y with y = p log2 r clamped to [-8, 8] (beyond it every factor below is
 * clamped anyway), the result clamped to [lo, hi]. A NaN y counts as -8 (the smallest
 * factor). */
float orc_ctrl_factor(float log2r, float p, float lo, float hi)
{
    float y = fminf(fmaxf(p * log2r, -8.0f), 8.0f);
    return fminf(fmaxf(0.95f * pow2_series(y), lo), hi);
}

/* ---- tabulated rates (Sec. 2 interactions; synthetic tables) -----------------------
 * The rates are a heuristic input (tabulated, interpolated), so they are evaluated in FP32
 * from the FP64 state, by the same bit-level log2 and power-of-two series as the step
 * controller:
 *   x = (log2 E - log2(A m_p c^2)) log10(2), each log2 from the bits (orc_ctrl_log2; the
 *       product A m_p c^2 in FP64), i.e. x = log10 gamma0;
 *   t = (x - x0) inv_dx clamped to [0, n_nodes-1]; j = floor(t) (at most n_nodes-2);
 *   v = T_j + (t - j)(T_{j+1} - T_j) over the FP64 table entries rounded to FP32;
 *   rate = 2^(v log2 10), the exponent clamped to [-126, 126] (pow2_series).
 * Every operation is one FP32 rounding in the order written. Relative error of a rate
 * against the exact interpolation: below 2^-23 (|v log2 10| + 4), 2e-5 for the tables'
 * |v| < 40. Returns 0, or ORC_RANGE if the species is outside the table. */
int orc_rates_f32(const orc_tables* t, int32_t A, int32_t Z, double E, float* r_loss, float* r_pd)
{
    *r_loss = 0.0f;
    *r_pd = 0.0f;
    if (!t) return 0;
    int32_t N = A - Z;
    if (Z < 0 || N < 0 || Z > t->z_max || N > t->n_max) return ORC_RANGE;
    int64_t sp = (int64_t)Z * (t->n_max + 1) + N;
    float lg = orc_ctrl_log2(E) - orc_ctrl_log2((double)A * MP_C2_EV);
    float x = lg * 0x1.344136p-2f;                       /* log10 2 */
    float tt = (x - (float)t->x0) * (float)t->inv_dx;
    float tmax = (float)(t->n_nodes - 1);
    tt = fminf(fmaxf(tt, 0.0f), tmax);
    int32_t j = (int32_t)floorf(tt);
    if (j > t->n_nodes - 2) j = t->n_nodes - 2;
    float fr = tt - (float)j;
    if (t->has_loss[sp]) {
        const double* T = t->log10_loss + sp * t->n_nodes;
        float a = (float)T[j], b = (float)T[j + 1];
        float y = (a + fr * (b - a)) * 0x1.a934f0p+1f;   /* log2 10 */
        *r_loss = pow2_series(fminf(fmaxf(y, -126.0f), 126.0f));
    }
    if (t->has_pd[sp]) {
        const double* T = t->log10_pd + sp * t->n_nodes;
        float a = (float)T[j], b = (float)T[j + 1];
        float y = (a + fr * (b - a)) * 0x1.a934f0p+1f;
        *r_pd = pow2_series(fminf(fmaxf(y, -126.0f), 126.0f));
    }
    return 0;
}

/* The FP32 rates widened (exactly) to FP64. */
int orc_rates(const orc_tables* t, int32_t A, int32_t Z, double E, double* r_loss, double* r_pd)
{
    float rl = 0.0f, rp = 0.0f;
    int rc = orc_rates_f32(t, A, Z, E, &rl, &rp);
    *r_loss = (double)rl;
    *r_pd = (double)rp;
    return rc;
}

/* ---- source injection (Sec. 4: isotropic emission; sampled positions/directions are
 * inputs). Sets the per-particle bookkeeping: s = 0, no step proposal yet (+inf), first
 * optical depth tau = -ln U(uid, k = 0, tag 0), counters 0, u0 = u. ------------------- */
int orc_inject(orc_state* st, int64_t first, int64_t count, uint64_t seed, const orc_tables* t)
{
    if (!st || first < 0 || count < 0 || first + count > st->capacity) return ORC_ERR_INVALID_ARG;
    for (int64_t i = first; i < first + count; ++i) {
        if (st->uid[i] < 0 || st->uid[i] >= ((int64_t)1 << 32)) return ORC_ERR_INVALID_ARG;
        /* Z < 0: an antinucleus, for backward tracking (Sec. 3.3 galactic propagation:
         * cosmic rays propagated backwards from Earth); only without interaction tables */
        if (st->A[i] < 1 || st->Z[i] > st->A[i] || st->Z[i] < -st->A[i]) return ORC_ERR_INVALID_ARG;
        if (t && (st->Z[i] < 0 || st->Z[i] > t->z_max || st->A[i] - st->Z[i] > t->n_max))
            return ORC_ERR_INVALID_ARG;
        st->s[i] = 0.0;
        st->hprop[i] = INFINITY;
        st->tau[i] = -orc_log(orc_uniform(seed, (uint64_t)st->uid[i], 0u, 0u));
        st->u0x[i] = st->ux[i];
        st->u0y[i] = st->uy[i];
        st->u0z[i] = st->uz[i];
        st->n_int[i] = 0;
        st->status[i] = ORC_ACTIVE;
        st->n_steps[i] = 0;
        st->n_att[i] = 0;
    }
    if (first + count > st->n) st->n = first + count;
    return ORC_OK;
}

/* ---- one particle, module sequence per step (Sec. 3.1) ----------------------------- */
typedef struct {
    orc_state* st;
    const orc_field* fields;
    int32_t n_fields;
    const orc_tables* tab;
    const orc_params* p;
    int64_t next;             /* next slot to process (atomic) */
    int64_t end;
    int64_t reserved;         /* slot counter for secondaries (atomic) */
    int64_t accepted, attempted, finished, secondaries;   /* totals (atomic) */
    int32_t queue_full;
} orc_job;

static double clamp(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

/* Reflective boundary (Sec. 4: reflective boundary conditions make a finite volume stand
 * for sources at much larger distances). Along each axis the box is [o, o + L]. A position
 * outside it is folded back by mirror reflection at the faces: with t = (x - o) * (1/L) and
 * k = floor(t), the fractional part r = t - k gives x' = o + r L for even k and
 * x' = (o + L) - r L for odd k, and an odd k reverses the direction component. Returns 1 if
 * the component was reversed. Positions inside the box (faces included) are unchanged. */
static int reflect_axis(double* x, double o, double L)
{
    double hi = o + L;
    if (!(*x < o || *x > hi)) return 0;
    double t = (*x - o) * (1.0 / L);
    double k = floor(t);
    double r = t - k;
    int odd = fmod(k, 2.0) != 0.0;
    *x = odd ? hi - r * L : o + r * L;
    return odd;
}

/* Reflect position and direction after an accepted step; the initial direction u0 takes
 * the same sign flips, so that the deflection angle (u vs u0) is measured in the mirrored
 * frame in which the particle keeps moving. */
static void reflect_state(const orc_params* p, double y[6], orc_state* st, int64_t i)
{
    double* u0[3] = {st->u0x, st->u0y, st->u0z};
    for (int a = 0; a < 3; ++a) {
        if (reflect_axis(&y[a], p->box_origin[a], p->box_size[a])) {
            y[3 + a] = -y[3 + a];
            u0[a][i] = -u0[a][i];
        }
    }
}

static void propagate_one(orc_job* job, int64_t i)
{
    orc_state* st = job->st;
    const orc_params* p = job->p;
    const orc_tables* tab = job->tab;
    if (st->status[i] != ORC_ACTIVE) return;
    const orc_field* fld = &job->fields[st->grid_id[i]];

    double y[6] = {st->x[i], st->y[i], st->z[i], st->ux[i], st->uy[i], st->uz[i]};
    double E = st->E[i], s = st->s[i], hprop = st->hprop[i], tau = st->tau[i];
    int32_t A = st->A[i], Z = st->Z[i], n_int = st->n_int[i], status = ORC_ACTIVE;
    int64_t uid = st->uid[i], n_steps = st->n_steps[i], n_att = st->n_att[i];
    int64_t acc_total = 0, att_total = 0, taken = 0;

    while (status == ORC_ACTIVE && (p->max_steps <= 0 || taken < p->max_steps)) {
        /* rates at the start of the step (gamma0), FP32 */
        float rl_f = 0.0f, rpd_f = 0.0f;
        if (orc_rates_f32(tab, A, Z, E, &rl_f, &rpd_f) != 0) {
            status = ORC_RANGE;
            break;
        }
        double rl = (double)rl_f, rpd = (double)rpd_f;
        /* bids (Sec. 3.1): propagation, continuous loss, interaction, distance; lowest wins.
         * The loss and interaction bids are FP32 quotients (of heuristic inputs), widened:
         * 0.1 / R_loss and max(tau, 0) / R_pd with tau rounded to FP32. */
        double h_prop = fmin(fmax(hprop, p->hmin), p->hmax);
        double h_loss = rl_f > 0.0f ? (double)(0.1f / rl_f) : INFINITY;
        double h_int = rpd_f > 0.0f ? (double)((float)fmax(tau, 0.0) / rpd_f) : INFINITY;
        double h_dist = p->dmax - s;
        double h = h_prop;
        if (h_loss < h) h = h_loss;
        if (h_int < h) h = h_int;
        if (h_dist < h) h = h_dist;
        double h_first = h;

        /* propagation: Cash-Karp attempts until the FP64 error ratio is <= 1 */
        double kappa = (double)Z * C_LIGHT / E;
        double k1[6], y5[6], err[6], sx, su;
        orc_deriv(fld, kappa, y, k1);
        int rejected = 0;
        int64_t att_step = 0;
        for (;;) {
            orc_ck_attempt(fld, kappa, y, k1, h, y5, err);
            att_step += 1;
            orc_error_sums(err, &sx, &su);
            if (orc_error_accept(sx, su, h, p->tol) || h <= p->hmin) break;
            float shrink = orc_ctrl_factor(orc_ctrl_log2r(sx, su, h, p->tol), -0.25f, 0.1f, 1.0f);
            h = fmax(h * (double)shrink, p->hmin);
            rejected = 1;
        }
        int finite = 1;
        for (int c = 0; c < 6; ++c) finite &= isfinite(y5[c]) ? 1 : 0;
        if (!finite) {
            n_att += att_step;
            att_total += att_step;
            status = ORC_NAN;
            break;
        }

        /* split needs a free slot: reserve it before committing the step */
        int fires = (rpd > 0.0 && h == h_int);
        int64_t slot = -1;
        if (fires) {
            slot = __atomic_fetch_add(&job->reserved, 1, __ATOMIC_RELAXED);
            if (slot >= st->capacity) {
                __atomic_store_n(&job->queue_full, 1, __ATOMIC_RELAXED);
                break;      /* parked at the start of this step; resumable */
            }
        }

        /* accept */
        n_att += att_step;
        att_total += att_step;
        for (int c = 0; c < 6; ++c) y[c] = y5[c];
        if (p->boundary == ORC_BOUNDARY_REFLECT) reflect_state(p, y, st, i);
        int done = (h == h_dist);
        s = done ? p->dmax : s + h;
        n_steps += 1;
        acc_total += 1;
        taken += 1;
        float grow = (h == 0.0 || (sx == 0.0 && su == 0.0))
                         ? 5.0f : orc_ctrl_factor(orc_ctrl_log2r(sx, su, h, p->tol), -0.2f, 0.2f, 5.0f);
        double hnext = h * (double)grow;
        if (!rejected && h_first < h_prop) hnext = fmax(hnext, h_prop);
        hprop = clamp(hnext, p->hmin, p->hmax);

        /* continuous energy loss, rate at gamma0 */
        if (rl > 0.0) E = E * orc_exp(-h * rl);

        /* photo-disintegration: fires when the interaction bid was the step taken */
        if (rpd > 0.0) {
            if (fires) {
                uint32_t kk = (uint32_t)(n_int + 1);
                int proton = nucleon_is_proton(p->seed, (uint64_t)uid, kk, A, Z);
                int32_t dz = proton ? 1 : 0;
                double E_sec = E / (double)A;
                double E_par = E * (double)(A - 1) / (double)A;
                /* secondary nucleon: inherits x, u, s, u0; new uid */
                int64_t q = slot;
                st->x[q] = y[0]; st->y[q] = y[1]; st->z[q] = y[2];
                st->ux[q] = y[3]; st->uy[q] = y[4]; st->uz[q] = y[5];
                st->E[q] = E_sec;
                st->s[q] = s;
                st->hprop[q] = INFINITY;
                st->u0x[q] = st->u0x[i]; st->u0y[q] = st->u0y[i]; st->u0z[q] = st->u0z[i];
                st->A[q] = 1;
                st->Z[q] = dz;
                st->n_int[q] = 0;
                st->grid_id[q] = st->grid_id[i];
                st->uid[q] = ((int64_t)1 << 32) + uid * 64 + (int64_t)kk;
                st->tau[q] = -orc_log(orc_uniform(p->seed, (uint64_t)st->uid[q], 0u, 0u));
                st->n_steps[q] = 0;
                st->n_att[q] = 0;
                st->status[q] = done ? ORC_DONE : ORC_ACTIVE;
                __atomic_fetch_add(&job->secondaries, 1, __ATOMIC_RELAXED);
                if (done) __atomic_fetch_add(&job->finished, 1, __ATOMIC_RELAXED);
                /* parent */
                A = A - 1;
                Z = Z - dz;
                E = E_par;
                n_int = (int32_t)kk;
                tau = -orc_log(orc_uniform(p->seed, (uint64_t)uid, kk, 0u));
            } else {
                tau = tau - h * rpd;
            }
        }

        /* observer: trajectory-length limit */
        if (done) status = ORC_DONE;
    }

    st->x[i] = y[0]; st->y[i] = y[1]; st->z[i] = y[2];
    st->ux[i] = y[3]; st->uy[i] = y[4]; st->uz[i] = y[5];
    st->E[i] = E; st->s[i] = s; st->hprop[i] = hprop; st->tau[i] = tau;
    st->A[i] = A; st->Z[i] = Z; st->n_int[i] = n_int; st->status[i] = status;
    st->n_steps[i] = n_steps; st->n_att[i] = n_att;
    __atomic_fetch_add(&job->accepted, acc_total, __ATOMIC_RELAXED);
    __atomic_fetch_add(&job->attempted, att_total, __ATOMIC_RELAXED);
    if (status != ORC_ACTIVE) __atomic_fetch_add(&job->finished, 1, __ATOMIC_RELAXED);
}

static void* worker(void* arg)
{
    orc_job* job = (orc_job*)arg;
    for (;;) {
        int64_t i = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
        if (i >= job->end) break;
        propagate_one(job, i);
    }
    return NULL;
}

/* Propagate every active particle until it finishes or has taken max_steps accepted
 * steps in this call; secondaries created in the call are appended at slot n.. and
 * propagated in the same call. Particles are independent (Sec. 3.1), so threads take
 * them one at a time from a shared counter. stats = {accepted, attempted, finished,
 * secondaries}. Returns ORC_ERR_QUEUE_FULL if some split found no free slot (that
 * particle is parked at the start of the step and the call can be repeated). */
int orc_propagate(orc_state* st, const orc_field* fields, int32_t n_fields, const orc_tables* t,
                  const orc_params* p, int64_t stats[4])
{
    if (!st || !fields || n_fields < 1 || !p) return ORC_ERR_INVALID_ARG;
    if (!(p->tol > 0.0) || !(p->hmin > 0.0) || !(p->hmax >= p->hmin) || !(p->dmax > 0.0))
        return ORC_ERR_INVALID_ARG;
    if (p->boundary != ORC_BOUNDARY_NONE && p->boundary != ORC_BOUNDARY_REFLECT) return ORC_ERR_INVALID_ARG;
    if (p->boundary == ORC_BOUNDARY_REFLECT)
        for (int a = 0; a < 3; ++a)
            if (!(p->box_size[a] > 0.0) || !isfinite(p->box_size[a]) || !isfinite(p->box_origin[a]))
                return ORC_ERR_INVALID_ARG;
    for (int64_t i = 0; i < st->n; ++i)
        if (st->grid_id[i] < 0 || st->grid_id[i] >= n_fields) return ORC_ERR_INVALID_ARG;
    orc_job job;
    memset(&job, 0, sizeof job);
    job.st = st;
    job.fields = fields;
    job.n_fields = n_fields;
    job.tab = t;
    job.p = p;
    job.reserved = st->n;
    int nt = p->n_threads > 0 ? p->n_threads : 1;
    int64_t begin = 0;
    while (begin < st->n) {
        job.next = begin;
        job.end = st->n;
        if (nt == 1) {
            worker(&job);
        } else {
            pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
            int started = 0;
            for (int w = 0; w < nt; ++w)
                if (pthread_create(&th[w], NULL, worker, &job) == 0) started++;
                else break;
            if (started == 0) worker(&job);
            for (int w = 0; w < started; ++w) pthread_join(th[w], NULL);
            free(th);
        }
        begin = job.end;
        st->n = job.reserved < st->capacity ? job.reserved : st->capacity;
        job.reserved = st->n;
    }
    if (stats) {
        stats[0] = job.accepted;
        stats[1] = job.attempted;
        stats[2] = job.finished;
        stats[3] = job.secondaries;
    }
    return job.queue_full ? ORC_ERR_QUEUE_FULL : ORC_OK;
}


/* ==== frozen-step differentiation =====================================================
 * The controller and the bids are not differentiated: the accepted step sizes h_n of a
 * forward run are recorded and the map y_{n+1} = y_n + h_n sum_i b_i k_i (5th-order
 * Cash-Karp solution) is differentiated exactly for fixed h_n. */

/* Accepted steps of the propagation module alone (no distance, loss or interaction bids),
 * with the same attempt loop and controller as orc_propagate. */
int orc_record_steps(const orc_field* f, double kappa, const double y0[6], double tol, double hmin,
                     double hmax, int32_t n_steps, double* h_out, double yT[6])
{
    double y[6];
    for (int c = 0; c < 6; ++c) y[c] = y0[c];
    double hprop = INFINITY;
    for (int32_t n = 0; n < n_steps; ++n) {
        double h_prop = fmin(fmax(hprop, hmin), hmax);
        double h = h_prop;
        double k1[6], y5[6], err[6], sx, su;
        orc_deriv(f, kappa, y, k1);
        int rejected = 0;
        for (;;) {
            orc_ck_attempt(f, kappa, y, k1, h, y5, err);
            orc_error_sums(err, &sx, &su);
            if (orc_error_accept(sx, su, h, tol) || h <= hmin) break;
            float shrink = orc_ctrl_factor(orc_ctrl_log2r(sx, su, h, tol), -0.25f, 0.1f, 1.0f);
            h = fmax(h * (double)shrink, hmin);
            rejected = 1;
        }
        for (int c = 0; c < 6; ++c) y[c] = y5[c];
        h_out[n] = h;
        float grow = (h == 0.0 || (sx == 0.0 && su == 0.0))
                         ? 5.0f : orc_ctrl_factor(orc_ctrl_log2r(sx, su, h, tol), -0.2f, 0.2f, 5.0f);
        double hnext = h * (double)grow;
        if (!rejected && h < h_prop) hnext = fmax(hnext, h_prop);
        hprop = clamp(hnext, hmin, hmax);
    }
    for (int c = 0; c < 6; ++c) yT[c] = y[c];
    return 0;
}

/* One frozen step: the Cash-Karp 5th-order update with step h. */
static void frozen_step(const orc_field* f, double kappa, double y[6], double h)
{
    double k1[6], y5[6], err[6];
    orc_deriv(f, kappa, y, k1);
    orc_ck_attempt(f, kappa, y, k1, h, y5, err);
    for (int c = 0; c < 6; ++c) y[c] = y5[c];
}

void orc_frozen_forward(const orc_field* f, double kappa, const double y0[6], const double* h,
                        int32_t n_steps, double yT[6])
{
    double y[6];
    for (int c = 0; c < 6; ++c) y[c] = y0[c];
    for (int32_t n = 0; n < n_steps; ++n) frozen_step(f, kappa, y, h[n]);
    for (int c = 0; c < 6; ++c) yT[c] = y[c];
}

/* Trilinear lookup with the corner weights, the grid indices and the field's Jacobian. */
typedef struct {
    double B[3];
    double w[8];            /* corner weights, corner order 000, 001, ..., 111 */
    double J[3][3];         /* J[q][a] = d B_q / d x_a */
    int64_t node[8];
} orc_lookup;

static void lookup_full(const orc_field* f, const double x[3], orc_lookup* L)
{
    double inv = 1.0 / f->spacing;
    int64_t dims[3] = {f->nx, f->ny, f->nz};
    int64_t idx[3][2];
    double w[3][2], dwd[3][2];
    for (int a = 0; a < 3; ++a) {
        double r = fma(x[a], inv, -(f->origin[a] * inv));
        double fl = floor(r);
        double fr = r - fl;
        int64_t i = (int64_t)fl;
        int64_t n = dims[a];
        int64_t i0 = ((i % n) + n) % n;
        idx[a][0] = i0;
        idx[a][1] = (i0 + 1) % n;
        w[a][0] = 1.0 - fr;
        w[a][1] = fr;
        dwd[a][0] = -inv;
        dwd[a][1] = inv;
    }
    L->B[0] = 0.0; L->B[1] = 0.0; L->B[2] = 0.0;
    for (int q = 0; q < 3; ++q)
        for (int a = 0; a < 3; ++a) L->J[q][a] = 0.0;
    int c8 = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c, ++c8) {
                double wt = (w[0][a] * w[1][b]) * w[2][c];
                double dw[3];
                dw[0] = (dwd[0][a] * w[1][b]) * w[2][c];
                dw[1] = (w[0][a] * dwd[1][b]) * w[2][c];
                dw[2] = (w[0][a] * w[1][b]) * dwd[2][c];
                L->w[c8] = wt;
                L->node[c8] = (idx[0][a] * f->ny + idx[1][b]) * f->nz + idx[2][c];
                for (int q = 0; q < 3; ++q) {
                    double G = grid_at(f, idx[0][a], idx[1][b], idx[2][c], q);
                    L->B[q] = fma(wt, G, L->B[q]);     /* as orc_field_value */
                    for (int d = 0; d < 3; ++d) L->J[q][d] = fma(dw[d], G, L->J[q][d]);
                }
            }
}

/* Vector-Jacobian product of f(Y) = (u, kappa u x B(x)) with kbar = (abar, bbar):
 *   Bbar = kappa (bbar x u);  kappa_bar += bbar . (u x B);
 *   Ybar_u = abar + kappa (B x bbar);
 *   Ybar_x[a] = sum_q J[q][a] Bbar[q], with the field's Jacobian at Y,
 *   J[q][a] = d B_q / d x_a = sum_c (d w_c / d x_a) G_c[q] summed over the corners 000..111
 *   with one rounding per corner (fused multiply-add from 0);
 *   grid_bar[c] += w_c Bbar. */
static void vjp_f(const orc_field* f, double kappa, const double Y[6], const double kb[6],
                  double Yb[6], double* grid_bar, double* kappa_bar)
{
    orc_lookup L;
    lookup_full(f, Y, &L);
    const double* u = Y + 3;
    const double* bb = kb + 3;
    double Bb[3];
    Bb[0] = kappa * (bb[1] * u[2] - bb[2] * u[1]);
    Bb[1] = kappa * (bb[2] * u[0] - bb[0] * u[2]);
    Bb[2] = kappa * (bb[0] * u[1] - bb[1] * u[0]);
    double uxB0 = u[1] * L.B[2] - u[2] * L.B[1];
    double uxB1 = u[2] * L.B[0] - u[0] * L.B[2];
    double uxB2 = u[0] * L.B[1] - u[1] * L.B[0];
    *kappa_bar = *kappa_bar + ((bb[0] * uxB0 + bb[1] * uxB1) + bb[2] * uxB2);
    Yb[3] = kb[0] + kappa * (L.B[1] * bb[2] - L.B[2] * bb[1]);
    Yb[4] = kb[1] + kappa * (L.B[2] * bb[0] - L.B[0] * bb[2]);
    Yb[5] = kb[2] + kappa * (L.B[0] * bb[1] - L.B[1] * bb[0]);
    for (int a = 0; a < 3; ++a) Yb[a] = (L.J[0][a] * Bb[0] + L.J[1][a] * Bb[1]) + L.J[2][a] * Bb[2];
    for (int c = 0; c < 8; ++c) {
        if (grid_bar)
            for (int q = 0; q < 3; ++q)
                grid_bar[L.node[c] * 3 + q] = grid_bar[L.node[c] * 3 + q] + L.w[c] * Bb[q];
    }
}

/* Reverse pass through the recorded steps. lamT = dL/dy_T; grid_bar ([nx][ny][nz][3]) is
 * accumulated; y0_bar = dL/dy_0; kappa_bar = dL/dkappa (kappa is one constant per particle). */
void orc_adjoint(const orc_field* f, double kappa, const double y0[6], const double* h,
                 int32_t n_steps, const double lamT[6], double* grid_bar, double y0_bar[6],
                 double* kappa_bar)
{
    double* ys = (double*)malloc(sizeof(double) * 6 * (size_t)(n_steps + 1));
    for (int c = 0; c < 6; ++c) ys[c] = y0[c];
    for (int32_t n = 0; n < n_steps; ++n) {
        for (int c = 0; c < 6; ++c) ys[6 * (n + 1) + c] = ys[6 * n + c];
        frozen_step(f, kappa, ys + 6 * (n + 1), h[n]);
    }
    double lam[6];
    for (int c = 0; c < 6; ++c) lam[c] = lamT[c];
    *kappa_bar = 0.0;
    for (int32_t n = n_steps - 1; n >= 0; --n) {
        const double* y = ys + 6 * n;
        const double hn = h[n];
        /* stage states Y_1..Y_6 of this step */
        double k[6][6], Y[6][6];
        for (int c = 0; c < 6; ++c) Y[0][c] = y[c];
        orc_deriv(f, kappa, Y[0], k[0]);
        for (int i = 1; i < 6; ++i) {
            for (int c = 0; c < 6; ++c) {           /* the forward stage sums (orc_ck_attempt) */
                double acc = CK_A[i][0] * k[0][c];
                for (int j = 1; j < i; ++j) acc = fma(CK_A[i][j], k[j][c], acc);
                Y[i][c] = fma(hn, acc, y[c]);
            }
            orc_deriv(f, kappa, Y[i], k[i]);
        }
        /* adjoint of y' = y + h sum_i b_i k_i and of the stage sums, stages in reverse */
        double kb[6][6], yb[6];
        for (int i = 0; i < 6; ++i) {
            double hb = hn * CK_B5[i];
            for (int c = 0; c < 6; ++c) kb[i][c] = hb * lam[c];
        }
        for (int c = 0; c < 6; ++c) yb[c] = lam[c];
        for (int i = 5; i >= 0; --i) {
            double Yb[6];
            vjp_f(f, kappa, Y[i], kb[i], Yb, grid_bar, kappa_bar);
            for (int c = 0; c < 6; ++c) yb[c] = yb[c] + Yb[c];
            for (int j = 0; j < i; ++j) {
                double ha = hn * CK_A[i][j];
                for (int c = 0; c < 6; ++c) kb[j][c] = kb[j][c] + ha * Yb[c];
            }
        }
        for (int c = 0; c < 6; ++c) lam[c] = yb[c];
    }
    for (int c = 0; c < 6; ++c) y0_bar[c] = lam[c];
    free(ys);
}

/* ---- source spectrum (Sec. 4, Eq. 1) ---------------------------------------------------
 * dN_i/dE ~ x_i A_i^(alpha - 1) E^-alpha exp(-E / (Z_i R_cut)) on [E_min, E_max]. Sampled by
 * rejection from the cutoff-free joint law: species i with probability proportional to
 * w_i = x_i A_i^(alpha-1), E from E^-alpha by its inverse CDF, the pair kept with probability
 * exp(-E / (Z_i R_cut)); a rejected pair is redrawn whole, so the kept pairs follow Eq. 1
 * jointly. Random numbers: Philox counter (uid, k, tag 2) gives (U1, U2) for draw k,
 * (uid, k, tag 3) gives U3. Directions are isotropic by Marsaglia (1972): v1, v2 uniform in
 * (-1, 1) from counter (uid, k, tag 4), kept if s = v1^2 + v2^2 < 1, then
 * u = (2 v1 sqrt(1 - s), 2 v2 sqrt(1 - s), 1 - 2 s). */
static double uniform_words(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
    return ((double)m + 0.5) * 0x1p-52;
}

static void philox_words(uint64_t seed, uint64_t uid, uint32_t k, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), k, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

int orc_spectrum_check(const orc_spectrum* sp)
{
    if (!sp || sp->n_species < 1 || sp->n_species > ORC_MAX_SPECIES) return ORC_ERR_INVALID_ARG;
    if (!(sp->e_min_ev > 0.0) || !(sp->e_max_ev > sp->e_min_ev) || !isfinite(sp->e_max_ev))
        return ORC_ERR_INVALID_ARG;
    if (!(sp->rcut_v > 0.0) || !isfinite(sp->alpha)) return ORC_ERR_INVALID_ARG;
    double total = 0.0;
    for (int i = 0; i < sp->n_species; ++i) {
        if (sp->A[i] < 1 || sp->Z[i] < 1 || sp->Z[i] > sp->A[i] || !(sp->x[i] >= 0.0)) return ORC_ERR_INVALID_ARG;
        total += sp->x[i];
    }
    return total > 0.0 ? ORC_OK : ORC_ERR_INVALID_ARG;
}

int64_t orc_source_sample(const orc_spectrum* sp, uint64_t seed, uint64_t uid_base, int64_t n,
                          int32_t* A, int32_t* Z, double* E, double* ux, double* uy, double* uz)
{
    if (orc_spectrum_check(sp) != ORC_OK || n < 0) return -1;
    /* cumulative species weights w_i = x_i A_i^(alpha-1) */
    double cum[ORC_MAX_SPECIES];
    double acc = 0.0;
    for (int i = 0; i < sp->n_species; ++i) {
        double w = sp->x[i] * orc_exp((sp->alpha - 1.0) * orc_log((double)sp->A[i]));
        acc = acc + w;
        cum[i] = acc;
    }
    double W = acc;
    /* inverse CDF of E^-alpha: E = (lo + U (hi - lo))^(1/g), g = 1 - alpha, lo/hi = E_min/max^g;
     * alpha == 1: E = E_min exp(U ln(E_max/E_min)) */
    double g = 1.0 - sp->alpha;
    double lo = 0.0, hi = 0.0, lr = 0.0;
    if (g != 0.0) {
        lo = orc_exp(g * orc_log(sp->e_min_ev));
        hi = orc_exp(g * orc_log(sp->e_max_ev));
    } else {
        lr = orc_log(sp->e_max_ev / sp->e_min_ev);
    }
    int64_t failed = 0;
    for (int64_t p = 0; p < n; ++p) {
        uint64_t uid = uid_base + (uint64_t)p;
        int32_t a = 0, z = 0;
        double e = 0.0;
        for (uint32_t k = 0; k < ORC_SOURCE_DRAWS; ++k) {
            uint32_t w[4], v[4];
            philox_words(seed, uid, k, 2u, w);
            double u1 = uniform_words(w[0], w[1]);
            double u2 = uniform_words(w[2], w[3]);
            int s = sp->n_species - 1;
            double target = u1 * W;
            for (int i = 0; i < sp->n_species; ++i)
                if (target < cum[i]) { s = i; break; }
            double en = g != 0.0 ? orc_exp(orc_log(lo + u2 * (hi - lo)) / g)
                                 : sp->e_min_ev * orc_exp(u2 * lr);
            philox_words(seed, uid, k, 3u, v);
            double u3 = uniform_words(v[0], v[1]);
            if (u3 < orc_exp(-en / ((double)sp->Z[s] * sp->rcut_v))) {
                a = sp->A[s];
                z = sp->Z[s];
                e = en;
                break;
            }
        }
        double d[3] = {0.0, 0.0, 0.0};
        int have_dir = 0;
        for (uint32_t k = 0; k < ORC_SOURCE_DRAWS; ++k) {
            uint32_t w[4];
            philox_words(seed, uid, k, 4u, w);
            double v1 = 2.0 * uniform_words(w[0], w[1]) - 1.0;
            double v2 = 2.0 * uniform_words(w[2], w[3]) - 1.0;
            double s = v1 * v1 + v2 * v2;
            if (s < 1.0) {
                double r = 2.0 * sqrt(1.0 - s);
                d[0] = v1 * r;
                d[1] = v2 * r;
                d[2] = 1.0 - 2.0 * s;
                have_dir = 1;
                break;
            }
        }
        if (a == 0 || !have_dir) {
            failed += 1;
            a = 0;
            z = 0;
        }
        A[p] = a; Z[p] = z; E[p] = e;
        ux[p] = d[0]; uy[p] = d[1]; uz[p] = d[2];
    }
    return failed;
}

/* ---- arrival binning (Sec. 4, Fig. 4: HEALPix maps of arrival directions) ------------- */
static const double PI_D = 3.141592653589793;
static const double HALF_PI_D = 1.5707963267948966;
static const double QUARTER_PI_D = 0.7853981633974483;

/* atan2 by one stated algorithm (so that both implementations bin identically): reduce to
 * a = min(|x|,|y|) / max(|x|,|y|) in [0, 1]; for a > tan(pi/8) use atan a = pi/4 + atan b,
 * b = (a - 1)/(a + 1); then atan b = 2 atan c with c = b / (1 + sqrt(1 + b^2)), |c| <= 0.2;
 * atan c by its Taylor series through c^27/27 (Horner in c^2); undo the octant reduction. */
double orc_atan2(double y, double x)
{
    if (x != x || y != y) return NAN;
    double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    int swap = ay > ax;
    double a = swap ? ax / ay : ay / ax;
    double base = 0.0;
    double b = a;
    if (a > 0.41421356237309503) {
        b = (a - 1.0) / (a + 1.0);
        base = QUARTER_PI_D;
    }
    double c = b / (1.0 + sqrt(1.0 + b * b));
    double s = c * c;
    double p = -1.0 / 27.0;
    p = p * s + 1.0 / 25.0;
    p = p * s - 1.0 / 23.0;
    p = p * s + 1.0 / 21.0;
    p = p * s - 1.0 / 19.0;
    p = p * s + 1.0 / 17.0;
    p = p * s - 1.0 / 15.0;
    p = p * s + 1.0 / 13.0;
    p = p * s - 1.0 / 11.0;
    p = p * s + 1.0 / 9.0;
    p = p * s - 1.0 / 7.0;
    p = p * s + 1.0 / 5.0;
    p = p * s - 1.0 / 3.0;
    p = p * s + 1.0;
    double r = base + 2.0 * (c * p);
    if (swap) r = HALF_PI_D - r;
    if (x < 0.0) r = PI_D - r;
    if (y < 0.0) r = -r;
    return r;
}

/* HEALPix RING-scheme pixel of direction (x, y, z) (not necessarily unit) for resolution
 * nside (Gorski et al. 2005, ApJ 622, 759, Sec. 4): 12 nside^2 equal-area pixels on rings
 * 1 .. 4 nside - 1 from the north pole, numbered ring by ring and eastwards in phi.
 * With z = cos(theta) and t = phi / (pi/2) in [0, 4):
 *  |z| <= 2/3 (equatorial belt): pixel edges are the lines where
 *      A = nside (t - 3z/4 + 1/2) and B = nside (t + 3z/4 + 1/2) are integers; with
 *      jp = floor(A), jm = floor(B) the ring is i = 2 nside - (jm - jp) and the pixel in the
 *      ring j = (jp + jm + 1 - nside - s)/2 mod 4 nside, s = (i - nside + 1) mod 2 (rings with
 *      s = 0 have a pixel centred on phi = 0, the others are offset by half a pixel);
 *      index = 2 nside (nside - 1) + 4 nside (i - nside) + j.
 *  |z| > 2/3 (polar caps): with the equal-area radius sigma = nside sqrt(3 (1 - |z|)) and
 *      tp = t - floor(t), the ring counted from the pole is i = floor(tp sigma) +
 *      floor((1 - tp) sigma) + 1 (at most nside), its 4 i pixels split phi evenly:
 *      j = floor(t i); index = 2 i (i - 1) + j (north) or 12 nside^2 - 2 i (i + 1) + j (south).
 * Returns -1 for a zero or non-finite direction. */
int64_t orc_healpix_ring(int32_t nside, double x, double y, double z)
{
    double r = sqrt(x * x + y * y + z * z);
    if (!(r > 0.0) || !isfinite(r) || nside < 1) return -1;
    double zz = z / r;
    double phi = orc_atan2(y, x);
    if (phi < 0.0) phi = phi + 2.0 * PI_D;
    double t = phi / HALF_PI_D;
    if (t >= 4.0) t = t - 4.0;
    int64_t ns = nside;
    double dn = (double)nside;
    double az = fabs(zz);
    if (az <= 2.0 / 3.0) {
        double sg = 0.75 * zz;
        int64_t jp = (int64_t)floor(dn * (t - sg + 0.5));
        int64_t jm = (int64_t)floor(dn * (t + sg + 0.5));
        int64_t i = 2 * ns - (jm - jp);
        if (i < ns) i = ns;
        if (i > 3 * ns) i = 3 * ns;
        int64_t s = (i - ns + 1) & 1;
        int64_t j = (jp + jm + 1 - ns - s) / 2;
        int64_t m = 4 * ns;
        j = ((j % m) + m) % m;
        return 2 * ns * (ns - 1) + m * (i - ns) + j;
    }
    double tp = t - floor(t);
    double sigma = dn * sqrt(3.0 * (1.0 - az));
    int64_t i = (int64_t)floor(tp * sigma) + (int64_t)floor((1.0 - tp) * sigma) + 1;
    if (i > ns) i = ns;
    int64_t j = (int64_t)floor(t * (double)i);
    if (j >= 4 * i) j = 4 * i - 1;
    if (zz > 0.0) return 2 * i * (i - 1) + j;
    return 12 * ns * ns - 2 * i * (i + 1) + j;
}

/* Arrival map: every finished particle (status DONE) with E > e_min adds one count to the
 * pixel of its arrival direction, the direction it arrives from: -u. */
int orc_arrival_map(const orc_state* st, int32_t nside, double e_min_ev, uint64_t* map)
{
    if (!st || !map || nside < 1) return ORC_ERR_INVALID_ARG;
    for (int64_t i = 0; i < st->n; ++i) {
        if (st->status[i] != ORC_DONE || !(st->E[i] > e_min_ev)) continue;
        int64_t pix = orc_healpix_ring(nside, -st->ux[i], -st->uy[i], -st->uz[i]);
        if (pix >= 0) map[pix] += 1;
    }
    return ORC_OK;
}

/* ---- lenses (Sec. 3.3: per-rigidity sparse matrices that transform directions at the
 * galactic border into arrival directions at Earth, applied to whole distributions by
 * matrix-vector products) --------------------------------------------------------------
 * n_mat matrices of n_pix x n_pix in CSR form over shared arrays: matrix m, row p holds the
 * entries k in [row_ptr[m (n_pix + 1) + p], row_ptr[m (n_pix + 1) + p + 1]) with column
 * col[k] and value val[k] (single precision, as the lenses are stored). The observed maps are
 * y[p][b] = sum over m, then over k of row p of matrix m, of val[k] x[m][col[k]][b], for the
 * n_maps maps b of every rigidity bin m, summed in double precision with one rounding per
 * entry (acc = fma(val, x, acc)). */
int orc_lens_apply(int32_t n_pix, int32_t n_mat, const int64_t* row_ptr, const int32_t* col,
                   const float* val, const double* x, int32_t n_maps, double* y)
{
    if (n_pix < 1 || n_mat < 1 || n_maps < 1 || !row_ptr || !x || !y) return ORC_ERR_INVALID_ARG;
    for (int64_t p = 0; p < n_pix; ++p) {
        for (int32_t b = 0; b < n_maps; ++b) {
            double acc = 0.0;
            for (int32_t m = 0; m < n_mat; ++m) {
                const int64_t* rp = row_ptr + (int64_t)m * (n_pix + 1);
                const double* xm = x + (int64_t)m * n_pix * n_maps;
                for (int64_t k = rp[p]; k < rp[p + 1]; ++k)
                    acc = fma((double)val[k], xm[(int64_t)col[k] * n_maps + b], acc);
            }
            y[p * n_maps + b] = acc;
        }
    }
    return ORC_OK;
}

/* Rigidity-binned arrival maps at the galactic border, the input of a lens: every finished
 * charged particle (status DONE, Z > 0) with E > e_min and rigidity R = E/Z (V) in
 * [edges[m], edges[m+1]) adds one count to x[m][pixel of -u] (HEALPix RING, nside). */
int orc_lens_bin(const orc_state* st, int32_t nside, int32_t n_mat, const double* edges,
                 double e_min_ev, double* x)
{
    if (!st || !edges || !x || nside < 1 || n_mat < 1) return ORC_ERR_INVALID_ARG;
    int64_t n_pix = 12 * (int64_t)nside * nside;
    for (int64_t i = 0; i < st->n; ++i) {
        if (st->status[i] != ORC_DONE || st->Z[i] <= 0 || !(st->E[i] > e_min_ev)) continue;
        double R = st->E[i] / (double)st->Z[i];
        int32_t m = -1;
        for (int32_t q = 0; q < n_mat; ++q)
            if (edges[q] <= R && R < edges[q + 1]) { m = q; break; }
        if (m < 0) continue;
        int64_t pix = orc_healpix_ring(nside, -st->ux[i], -st->uy[i], -st->uz[i]);
        if (pix >= 0) x[(int64_t)m * n_pix + pix] += 1.0;
    }
    return ORC_OK;
}
