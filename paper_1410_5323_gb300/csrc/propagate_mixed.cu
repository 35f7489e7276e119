// propagate_mixed.cu -- precision form of the propagation hot path (arXiv:1410.5323,
// Sec. 3.1 module sequence, Sec. 2 3D deflection, Sec. 3.2 regular grids).
//
// Same persistent warp-per-particle-batch structure and module sequence as the FP64
// form, with the arithmetic moved to where GB300 is fast (FP32 is 64x FP64 here):
//   * lengths in grid-cell units; Cash-Karp stages in FP32 in a local frame: offsets from
//     the step-start cell, so stage positions stay O(1) and FP32 keeps ~1e-7 of a cell;
//   * the position itself is a double-float (hi + lo FP32 pair, TwoSum) in cell units,
//     which resolves 1 kpc steps at 500 Mpc without any FP64 instruction; the direction
//     is a double-float as well (its per-step increment is added with TwoSum), so rounding
//     does not accumulate in it over thousands of steps;
//   * the accept/reject decision is the FP64 one: the squared norms of the six FP32 error
//     components, widened, compared against tol^2 in FP64 (|dx|/h is computed as
//     |sum_i e_i u_i|, so no division by h is needed); the FP32 norms certify that decision
//     outside a 2^-18 guard band around tol^2, and only norms inside it are formed in FP64;
//   * path length s stays FP64 so the observer lands exactly on the distance limit;
//   * continuous loss and interaction rates in FP32 from FP32 copies of the tables; the
//     Philox streams and the nucleon rule are the same integers as in the FP64 form;
//   * the vector grid is read from a cell-major copy when one is built (the 8 corners of a
//     cell together, 3 or 2 256-bit loads per lookup instead of 8 scattered node reads: the
//     lookups were bound by L1 requests), else from the node grid; both give the same bits.
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "crp_internal.h"
#include "crp_math.cuh"
#include "crp_sched.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

namespace crp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

constexpr float A21 = 1.0f / 5.0f;
constexpr float A31 = 3.0f / 40.0f, A32 = 9.0f / 40.0f;
constexpr float A41 = 3.0f / 10.0f, A42 = -9.0f / 10.0f, A43 = 6.0f / 5.0f;
constexpr float A51 = -11.0f / 54.0f, A52 = 5.0f / 2.0f, A53 = -70.0f / 27.0f, A54 = 35.0f / 27.0f;
constexpr float A61 = 1631.0f / 55296.0f, A62 = 175.0f / 512.0f, A63 = 575.0f / 13824.0f,
                A64 = 44275.0f / 110592.0f, A65 = 253.0f / 4096.0f;
constexpr float B1 = 37.0f / 378.0f, B3 = 250.0f / 621.0f, B4 = 125.0f / 594.0f, B6 = 512.0f / 1771.0f;
constexpr float E1 = -277.0f / 64512.0f, E3 = 6925.0f / 370944.0f, E4 = -6925.0f / 202752.0f,
                E5 = -277.0f / 14336.0f, E6 = 277.0f / 7084.0f;

struct F3 { float x, y, z; };
struct DF { float hi, lo; };

// a + b with the rounding error carried in lo (Knuth TwoSum, then renormalise).
__device__ __forceinline__ DF df_add(DF a, float b) {
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b - bb) + a.lo;
    const float hi = s + e;
    return {hi, e - (hi - s)};
}

// floor of hi + lo and the fraction in [0, 1).
__device__ __forceinline__ void df_floor(DF a, int& i, float& f) {
    const float fl = floorf(a.hi);
    f = (a.hi - fl) + a.lo;
    i = (int)fl;
    if (f < 0.0f) { f += 1.0f; i -= 1; }
    else if (f >= 1.0f) { f -= 1.0f; i += 1; }
}

__device__ __forceinline__ int wrap(int i, int n, int pow2) {
    if (pow2) return i & (n - 1);
    int a = i % n;
    return a < 0 ? a + n : a;
}

// Field-local description in FP32.
struct FieldF {
    const void* data;
    int nx, ny, nz, pow2;
    float scale;
};

// Modulated fields: the step-start frame on the modulation grid. The 3x3x3 modulation nodes
// around the step-start cell, on the side the particle is heading (per axis the start cell and
// the next one along sign(u)), are loaded once per step into this lane's column of shared
// memory; a stage whose cell lies in that block reads its 8 corners from there, any other
// stage gathers them from the grid. Registers hold only the fraction, the ratio of spacings
// and the block's low corner per axis (0 or -1 cells, packed in lo).
struct MF { F3 f0; float q; int lo; };

constexpr int kModNodes = 27;            // cached node values per lane
constexpr int kModSlots = kModNodes + 3; // + the step-start cell (wrapped) per axis
// Per-thread shared-memory slots of the current particle's field constants in cell units
// (kept out of registers: they are read once per step, not per attempt): 3 doubles (spacing,
// 1/spacing, distance limit) then 3 floats (step limit, spacing, c x spacing). The grid origin,
// needed only when a particle is loaded, stored or split, is read from the field record.
// Few slots keep the block's shared memory small, so that L1 keeps most of the SM's
// shared/L1 storage (see launch_propagate_mixed).
constexpr int kFieldWords = 3 * 2 + 3;


template <int L>
__device__ __forceinline__ F3 corner_f(const FieldF& F, int node) {
    if constexpr (L == LAYOUT_F32X4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(F.data) + node);
        return {v.x, v.y, v.z};
    } else {
        const ushort4 v = __ldg(reinterpret_cast<const ushort4*>(F.data) + node);
        return {__uint_as_float((unsigned)v.x << 16), __uint_as_float((unsigned)v.y << 16),
                __uint_as_float((unsigned)v.z << 16)};
    }
}

template <int L>
constexpr bool kBF16 = (L == LAYOUT_BF16X4 || L == LAYOUT_BF16_CELLS);

// 256-bit read-only loads: the cell-major layouts hold a cell's 8 corners in 96 B (FP32) or
// 64 B (BF16), 32-byte aligned, so a lookup takes 3 or 2 loads instead of 8 scattered ones.
__device__ __forceinline__ void ld8(const void* p, unsigned (&w)[8]) {
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
                   "=r"(w[7])
                 : "l"(p));
}

// The 8 corners of a cell from a cell-major copy, in the order 000, 001, ..., 111 (the same
// values corner_f reads from the node layout).
template <int L>
__device__ __forceinline__ void cell_corners(const FieldF& F, long long cell, F3& g0, F3& g1, F3& g2, F3& g3,
                                             F3& g4, F3& g5, F3& g6, F3& g7) {
    if constexpr (L == LAYOUT_F32_CELLS) {
        const unsigned* q = static_cast<const unsigned*>(F.data) + cell * 24;
        unsigned a[8], b[8], c[8];
        ld8(q, a);
        ld8(q + 8, b);
        ld8(q + 16, c);
        auto f = [](unsigned u) { return __uint_as_float(u); };
        g0 = {f(a[0]), f(a[1]), f(a[2])}; g1 = {f(a[3]), f(a[4]), f(a[5])};
        g2 = {f(a[6]), f(a[7]), f(b[0])}; g3 = {f(b[1]), f(b[2]), f(b[3])};
        g4 = {f(b[4]), f(b[5]), f(b[6])}; g5 = {f(b[7]), f(c[0]), f(c[1])};
        g6 = {f(c[2]), f(c[3]), f(c[4])}; g7 = {f(c[5]), f(c[6]), f(c[7])};
    } else {
        // BF16: per corner two words, (x | y << 16) and (z | pad << 16)
        const unsigned* q = static_cast<const unsigned*>(F.data) + cell * 16;
        unsigned a[8], b[8];
        ld8(q, a);
        ld8(q + 8, b);
        auto c3 = [](unsigned w0, unsigned w1) {
            return F3{__uint_as_float(w0 << 16), __uint_as_float(w0 & 0xFFFF0000u), __uint_as_float(w1 << 16)};
        };
        g0 = c3(a[0], a[1]); g1 = c3(a[2], a[3]); g2 = c3(a[4], a[5]); g3 = c3(a[6], a[7]);
        g4 = c3(b[0], b[1]); g5 = c3(b[2], b[3]); g6 = c3(b[4], b[5]); g7 = c3(b[6], b[7]);
    }
}

// floor(t) and t - floor(t) without conversion instructions, exact for |t| < 2^22:
// adding 1.5 * 2^23 rounds t to an integer held in the low mantissa bits.
__device__ __forceinline__ int floor_frac(float t, float& frac) {
    const float big = __fadd_rn(t, 12582912.0f);
    const float n = __fsub_rn(big, 12582912.0f);      // t rounded to nearest (exact)
    int i = __float_as_int(big) - 0x4B400000;
    float f = __fsub_rn(t, n);                        // exact, in [-0.5, 0.5]
    if (f < 0.0f) { f = __fadd_rn(f, 1.0f); i -= 1; }
    frac = f;
    return i;
}

// Wrap an index that is usually already in [0, n) (a base cell plus a small offset).
__device__ __forceinline__ int wrap_near(int i, int n, int pow2) {
    return ((unsigned)i < (unsigned)n) ? i : wrap(i, n, pow2);
}

// Shared-memory slot k of this lane (column-major by lane: a warp's accesses hit 32 banks);
// the modulation slots follow the field constants.
__device__ __forceinline__ float& mslot(float* sm, int k) { return sm[(kFieldWords + k) * blockDim.x + threadIdx.x]; }
__device__ __forceinline__ double& dslot(float* sm, int k) {
    return reinterpret_cast<double*>(sm)[k * blockDim.x + threadIdx.x];
}
__device__ __forceinline__ float& fslot(float* sm, int k) { return sm[(6 + k) * blockDim.x + threadIdx.x]; }
// Grid origin along axis c (metres), from the field record.
__device__ __forceinline__ double origin(const PropArgs& a, int gid, int c) {
    const FieldDev& G = a.fields[gid];
    return __ldg(c == 0 ? &G.ox : (c == 1 ? &G.oy : &G.oz));
}

// Trilinear weights and the corner sum, in the same order for the cached and gathered paths.
__device__ __forceinline__ float trilerp(float fx, float fy, float fz, float m0, float m1, float m2,
                                         float m3, float m4, float m5, float m6, float m7) {
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w00 = gx * gy, w01 = gx * fy, w10 = fx * gy, w11 = fx * fy;
    float v = (w00 * gz) * m0;
    v = fmaf(w00 * fz, m1, v);
    v = fmaf(w01 * gz, m2, v);
    v = fmaf(w01 * fz, m3, v);
    v = fmaf(w10 * gz, m4, v);
    v = fmaf(w10 * fz, m5, v);
    v = fmaf(w11 * gz, m6, v);
    v = fmaf(w11 * fz, m7, v);
    return v;
}

// Step start: the wrapped node indices of the cached block along one axis.
__device__ __forceinline__ void mod_axis_nodes(int b, int lo, int n, int pow2, int (&idx)[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) idx[j] = wrap_near(b + lo + j, n, pow2);
}

// Step start: fill this lane's cached block from the modulation grid.
__device__ __forceinline__ void mod_fill(float* sm, const FieldDev& G, int bx, int by, int bz, int lo) {
    int ix[3], iy[3], iz[3];
    mod_axis_nodes(bx, -(lo & 1), G.mnx, G.mpow2, ix);
    mod_axis_nodes(by, -((lo >> 1) & 1), G.mny, G.mpow2, iy);
    mod_axis_nodes(bz, -((lo >> 2) & 1), G.mnz, G.mpow2, iz);
    const float* M = G.mod;
    float v[kModNodes];
#pragma unroll
    for (int jx = 0; jx < 3; ++jx)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy) {
            const int row = (ix[jx] * G.mny + iy[jy]) * G.mnz;
#pragma unroll
            for (int jz = 0; jz < 3; ++jz) v[(jx * 3 + jy) * 3 + jz] = __ldg(M + row + iz[jz]);
        }
#pragma unroll
    for (int k = 0; k < kModNodes; ++k) mslot(sm, k) = v[k];
    mslot(sm, kModNodes + 0) = __int_as_float(bx);
    mslot(sm, kModNodes + 1) = __int_as_float(by);
    mslot(sm, kModNodes + 2) = __int_as_float(bz);
}

// Modulation value at the local offset p (vector-grid cells): the same trilinear periodic
// lookup on the scalar grid, with the offset converted to modulation cells.
__device__ __forceinline__ float modulation_f(const FieldDev* fields, int gid, float* sm, const MF& m, F3 p) {
    float fx, fy, fz;
    const int cx = floor_frac(fmaf(p.x, m.q, m.f0.x), fx), cy = floor_frac(fmaf(p.y, m.q, m.f0.y), fy),
              cz = floor_frac(fmaf(p.z, m.q, m.f0.z), fz);
    // cell relative to the cached block's low corner: 0 or 1 when inside it
    const int jx = cx + (m.lo & 1), jy = cy + ((m.lo >> 1) & 1), jz = cz + ((m.lo >> 2) & 1);
    float m0, m1, m2, m3, m4, m5, m6, m7;
    if (((unsigned)jx | (unsigned)jy | (unsigned)jz) <= 1u) {
        const int k = (jx * 3 + jy) * 3 + jz;
        m0 = mslot(sm, k);      m1 = mslot(sm, k + 1);
        m2 = mslot(sm, k + 3);  m3 = mslot(sm, k + 4);
        m4 = mslot(sm, k + 9);  m5 = mslot(sm, k + 10);
        m6 = mslot(sm, k + 12); m7 = mslot(sm, k + 13);
    } else {
        const FieldDev& G = fields[gid];
        const int n_x = G.mnx, n_y = G.mny, n_z = G.mnz, pw = G.mpow2;
        const int ix = wrap_near(__float_as_int(mslot(sm, kModNodes + 0)) + cx, n_x, pw);
        const int iy = wrap_near(__float_as_int(mslot(sm, kModNodes + 1)) + cy, n_y, pw);
        const int iz = wrap_near(__float_as_int(mslot(sm, kModNodes + 2)) + cz, n_z, pw);
        const int ix1 = ix + 1 == n_x ? 0 : ix + 1, iy1 = iy + 1 == n_y ? 0 : iy + 1,
                  iz1 = iz + 1 == n_z ? 0 : iz + 1;
        const int r00 = (ix * n_y + iy) * n_z, r01 = (ix * n_y + iy1) * n_z;
        const int r10 = (ix1 * n_y + iy) * n_z, r11 = (ix1 * n_y + iy1) * n_z;
        const float* M = G.mod;
        m0 = __ldg(M + r00 + iz); m1 = __ldg(M + r00 + iz1);
        m2 = __ldg(M + r01 + iz); m3 = __ldg(M + r01 + iz1);
        m4 = __ldg(M + r10 + iz); m5 = __ldg(M + r10 + iz1);
        m6 = __ldg(M + r11 + iz); m7 = __ldg(M + r11 + iz1);
    }
    return trilerp(fx, fy, fz, m0, m1, m2, m3, m4, m5, m6, m7);
}

// Trilinear periodic lookup at (base cell b, fraction f0) + offset p (cells); with M, times
// the modulation value there. P2: the vector grid's sizes are powers of two, and the cell index
// wraps with a mask (the general wrap's integer modulo, inlined at each of an attempt's six
// lookups and never run for such grids, stays out of the kernel: +8.6 % measured).
template <int L, bool M, bool P2>
__device__ __forceinline__ F3 field_f(const FieldF& F, int bx, int by, int bz, F3 f0,
                                      const FieldDev* fields, int gid, float* sm, const MF& mf,
                                      F3 p) {
    float fx, fy, fz;
    const int cx = floor_frac(f0.x + p.x, fx), cy = floor_frac(f0.y + p.y, fy),
              cz = floor_frac(f0.z + p.z, fz);
    const int ix = P2 ? (bx + cx) & (F.nx - 1) : wrap(bx + cx, F.nx, F.pow2),
              iy = P2 ? (by + cy) & (F.ny - 1) : wrap(by + cy, F.ny, F.pow2),
              iz = P2 ? (bz + cz) & (F.nz - 1) : wrap(bz + cz, F.nz, F.pow2);
    F3 g0, g1, g2, g3, g4, g5, g6, g7;
    if constexpr (L == LAYOUT_F32X4 || L == LAYOUT_BF16X4) {
        const int ix1 = ix + 1 == F.nx ? 0 : ix + 1, iy1 = iy + 1 == F.ny ? 0 : iy + 1,
                  iz1 = iz + 1 == F.nz ? 0 : iz + 1;
        const int r00 = (ix * F.ny + iy) * F.nz, r01 = (ix * F.ny + iy1) * F.nz;
        const int r10 = (ix1 * F.ny + iy) * F.nz, r11 = (ix1 * F.ny + iy1) * F.nz;
        g0 = corner_f<L>(F, r00 + iz); g1 = corner_f<L>(F, r00 + iz1);
        g2 = corner_f<L>(F, r01 + iz); g3 = corner_f<L>(F, r01 + iz1);
        g4 = corner_f<L>(F, r10 + iz); g5 = corner_f<L>(F, r10 + iz1);
        g6 = corner_f<L>(F, r11 + iz); g7 = corner_f<L>(F, r11 + iz1);
    } else {
        cell_corners<L>(F, ((long long)ix * F.ny + iy) * F.nz + iz, g0, g1, g2, g3, g4, g5, g6, g7);
    }
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w00 = gx * gy, w01 = gx * fy, w10 = fx * gy, w11 = fx * fy;
    float w;
    F3 B;
    w = w00 * gz; B.x = w * g0.x;          B.y = w * g0.y;          B.z = w * g0.z;
    w = w00 * fz; B.x = fmaf(w, g1.x, B.x); B.y = fmaf(w, g1.y, B.y); B.z = fmaf(w, g1.z, B.z);
    w = w01 * gz; B.x = fmaf(w, g2.x, B.x); B.y = fmaf(w, g2.y, B.y); B.z = fmaf(w, g2.z, B.z);
    w = w01 * fz; B.x = fmaf(w, g3.x, B.x); B.y = fmaf(w, g3.y, B.y); B.z = fmaf(w, g3.z, B.z);
    w = w10 * gz; B.x = fmaf(w, g4.x, B.x); B.y = fmaf(w, g4.y, B.y); B.z = fmaf(w, g4.z, B.z);
    w = w10 * fz; B.x = fmaf(w, g5.x, B.x); B.y = fmaf(w, g5.y, B.y); B.z = fmaf(w, g5.z, B.z);
    w = w11 * gz; B.x = fmaf(w, g6.x, B.x); B.y = fmaf(w, g6.y, B.y); B.z = fmaf(w, g6.z, B.z);
    w = w11 * fz; B.x = fmaf(w, g7.x, B.x); B.y = fmaf(w, g7.y, B.y); B.z = fmaf(w, g7.z, B.z);
    if constexpr (M) {
        float m = modulation_f(fields, gid, sm, mf, p);
        if constexpr (kBF16<L>) m *= F.scale;
        B.x *= m; B.y *= m; B.z *= m;
    } else if constexpr (kBF16<L>) {
        B.x *= F.scale; B.y *= F.scale; B.z *= F.scale;
    }
    return B;
}

struct Y { F3 p, u; };   // local position offset (cells) and direction

template <int L, bool M, bool P2>
__device__ __forceinline__ Y deriv_f(const FieldF& F, int bx, int by, int bz, F3 f0,
                                     const FieldDev* fields, int gid, float* sm, const MF& mf,
                                     float kappa, const Y& y) {
    const F3 B = field_f<L, M, P2>(F, bx, by, bz, f0, fields, gid, sm, mf, y.p);
    Y k;
    k.p = y.u;
    k.u.x = kappa * (y.u.y * B.z - y.u.z * B.y);
    k.u.y = kappa * (y.u.z * B.x - y.u.x * B.z);
    k.u.z = kappa * (y.u.x * B.y - y.u.y * B.x);
    return k;
}

__device__ __forceinline__ float clampf_(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// Exact widening of a float to double. Normal values with integer instructions (GB300's FP64
// unit takes one warp instruction per 64 cycles per sub-partition, and the conversion would
// be one of them, on the attempt's critical path); zeros, subnormals, infinities and NaN by
// the conversion.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// r2^p for r2 > 0 (controller exponents on the squared ratio).
__device__ __forceinline__ float powf_pos(float r2, float p) { return exp2f(p * __log2f(r2)); }

__device__ __forceinline__ bool fin3(F3 a) { return isfinite(a.x) && isfinite(a.y) && isfinite(a.z); }

template <int L, bool M, bool P2>
__device__ __forceinline__ void propagate_mixed_body(const PropArgs& a, float* sm) {
    const int lane = threadIdx.x & 31;
    Counters* C = a.ctr;
    const unsigned long long n_work = *(volatile unsigned long long*)&C->count[a.list];
    const float INF = __int_as_float(0x7f800000);
    const SimState& S = a.st;
    const double tol2 = a.tol * a.tol;
    const float inv_tol2 = (float)(1.0 / tol2);
    // Guard band of the accept decision: an FP32 squared norm at most tol2_lo (at least
    // tol2_hi) certifies that the FP64 squared norm is at most (above) tol^2. The FP32 sum of
    // three non-negative squares is within 2^-22 of the exact sum, the FP64 one within 2^-52,
    // and the band is 2^-18 wide, so the certified decision is the FP64 decision; only norms
    // inside the band are formed in FP64.
    // (For tol^2 outside [2^-100, 2^100] FP32 subnormals or overflow would void the bound:
    // there every norm is formed in FP64.)
    const bool band = tol2 >= 0x1p-100 && tol2 <= 0x1p+100;
    const float tol2_lo = band ? __double2float_rd(tol2 * (1.0 - 0x1p-18)) : -1.0f;
    const float tol2_hi = band ? __double2float_ru(tol2 * (1.0 + 0x1p-18)) : __int_as_float(0x7fc00000);

    int slot = -1;
    // particle state (cell units)
    DF Rx{0, 0}, Ry{0, 0}, Rz{0, 0};
    F3 u{0, 0, 0};
    F3 ul{0, 0, 0};                    // low parts of the direction (double-float, like R)
    double E = 0, s_c = 0;
    float hprop = 0, tau = 0;
    int A = 0, Z = 0, n_int = 0, gid = 0;
    int taken = 0, att_call = 0;       // accepted steps and attempts of this call
    // field of the current particle (its other constants in shared slots)
    FieldF F{};
    float hmin_c = 0;
    // step state
    bool new_step = true;
    int bx = 0, by = 0, bz = 0;
    F3 f0{0, 0, 0};
    MF mf{{0, 0, 0}, 1.0f, 0};
    float h = 0, h_first = 0, h_propc = 0, h_int = 0, h_dist = 0, rl = 0, rpd = 0, kappa = 0;
    int rejected = 0;
    int att_step = 0;
    unsigned acc_tot = 0, att_tot = 0, sec_tot = 0;
    unsigned bits = 0;

    auto to_x = [&](DF r, double o) { return o + ((double)r.hi + (double)r.lo) * dslot(sm, 0); };
    auto from_x = [&](double x, double o) {
        const double rr = (x - o) * dslot(sm, 1);
        const float hi = (float)rr;
        return DF{hi, (float)(rr - (double)hi)};
    };
    auto store = [&](int status, bool exact_end) {
        S.x[slot] = to_x(Rx, origin(a, gid, 0)); S.y[slot] = to_x(Ry, origin(a, gid, 1)); S.z[slot] = to_x(Rz, origin(a, gid, 2));
        S.ux[slot] = (double)u.x + (double)ul.x; S.uy[slot] = (double)u.y + (double)ul.y;
        S.uz[slot] = (double)u.z + (double)ul.z;
        S.E[slot] = E;
        S.s[slot] = exact_end ? a.dmax : s_c * dslot(sm, 0);
        S.hprop[slot] = (double)hprop * dslot(sm, 0);
        S.tau[slot] = tau;
        S.A[slot] = A; S.Z[slot] = Z; S.n_int[slot] = n_int; S.status[slot] = status;
        S.n_steps[slot] = __ldcg(&S.n_steps[slot]) + taken;
        S.n_att[slot] = __ldcg(&S.n_att[slot]) + att_call;
        if (status != CRP_STATUS_ACTIVE_) {
            const unsigned long long d = atomicAdd(&C->n_done, 1ull);
            a.done_list[d] = slot;
        }
        slot = -1;
    };

    for (;;) {
        const bool idle = slot < 0;
        const int popped = sched_pop(a, idle, lane, n_work, bits);
        if (popped >= 0) {
            slot = popped;
            gid = __ldcg(&S.grid_id[slot]);
            if (gid < 0 || gid >= a.n_fields) { bits |= BIT_BOUNDS; gid = 0; slot = -1; }
        }
        if (slot >= 0 && popped >= 0) {
            const FieldDev& G = a.fields[gid];
            F.data = G.data; F.nx = G.nx; F.ny = G.ny; F.nz = G.nz; F.pow2 = G.pow2;
            F.scale = (float)G.scale;
            if constexpr (M) mf.q = (float)(G.spacing * G.m_inv_spacing);
            const double sp = G.spacing, inv_sp = G.inv_spacing;
            dslot(sm, 0) = sp; dslot(sm, 1) = inv_sp;
            dslot(sm, 2) = a.dmax * inv_sp;
            fslot(sm, 0) = (float)(a.hmax * inv_sp);
            fslot(sm, 1) = (float)sp;
            fslot(sm, 2) = (float)(kC * sp);
            hmin_c = (float)(a.hmin * inv_sp);
            Rx = from_x(__ldcg(&S.x[slot]), G.ox); Ry = from_x(__ldcg(&S.y[slot]), G.oy); Rz = from_x(__ldcg(&S.z[slot]), G.oz);
            {
                const double dx = __ldcg(&S.ux[slot]), dy = __ldcg(&S.uy[slot]), dz = __ldcg(&S.uz[slot]);
                u = {(float)dx, (float)dy, (float)dz};
                ul = {(float)(dx - (double)u.x), (float)(dy - (double)u.y), (float)(dz - (double)u.z)};
            }
            E = __ldcg(&S.E[slot]);
            s_c = __ldcg(&S.s[slot]) * inv_sp;
            hprop = (float)(__ldcg(&S.hprop[slot]) * inv_sp);
            tau = (float)__ldcg(&S.tau[slot]);
            A = __ldcg(&S.A[slot]); Z = __ldcg(&S.Z[slot]); n_int = __ldcg(&S.n_int[slot]);
            taken = 0;
            att_call = 0;
            new_step = true;
        }
        if (__ballot_sync(kFull, slot >= 0) == 0) break;

        for (int it = 0; it < a.cadence; ++it) {
            if (slot < 0) continue;
            if (new_step) {
                // rates at gamma0 (FP32 tables), per cell
                rl = 0.0f;
                rpd = 0.0f;
                if (a.has_tables) {
                    const TablesDev& T = a.tab;
                    const int N = A - Z;
                    if (Z < 0 || N < 0 || Z > T.z_max || N > T.n_max) {
                        bits |= BIT_RANGE;
                        store(CRP_STATUS_RANGE_, false);
                        continue;
                    }
                    const int sp_i = Z * (T.n_max + 1) + N;
                    const float g0 = (float)E / ((float)A * (float)kMpC2);
                    float t = (log10f(g0) - (float)T.x0) * (float)T.inv_dx;
                    t = clampf_(t, 0.0f, (float)(T.n_nodes - 1));
                    int j = (int)floorf(t);
                    if (j > T.n_nodes - 2) j = T.n_nodes - 2;
                    const float fr = t - (float)j;
                    if (T.has_loss[sp_i]) {
                        const float* R = T.loss_f + (long long)sp_i * T.n_nodes;
                        const float v0 = __ldg(R + j), v1 = __ldg(R + j + 1);
                        rl = exp10f(fmaf(fr, v1 - v0, v0)) * fslot(sm, 1);
                    }
                    if (T.has_pd[sp_i]) {
                        const float* R = T.pd_f + (long long)sp_i * T.n_nodes;
                        const float v0 = __ldg(R + j), v1 = __ldg(R + j + 1);
                        rpd = exp10f(fmaf(fr, v1 - v0, v0)) * fslot(sm, 1);
                    }
                }
                h_propc = clampf_(hprop, hmin_c, fslot(sm, 0));
                const float h_loss = rl > 0.0f ? 0.1f / rl : INF;
                h_int = rpd > 0.0f ? fmaxf(tau, 0.0f) / rpd : INF;
                h_dist = (float)(dslot(sm, 2) - s_c);
                h = h_propc;
                if (h_loss < h) h = h_loss;
                if (h_int < h) h = h_int;
                if (h_dist < h) h = h_dist;
                h_first = h;
                rejected = 0;
                att_step = 0;
                kappa = (float)Z * fslot(sm, 2) / (float)E;
                df_floor(Rx, bx, f0.x);
                df_floor(Ry, by, f0.y);
                df_floor(Rz, bz, f0.z);
                if constexpr (M) {
                    // step-start cell on the modulation grid (FP64, once per step), then this
                    // lane's cached block of modulation nodes
                    const FieldDev& G = a.fields[gid];
                    auto mcell = [&](DF r, double o, double mo, int n, int& b, float& f) {
                        const double rm = (to_x(r, o) - mo) * G.m_inv_spacing;
                        const double fl = floor(rm);
                        const long long i = (long long)fl;
                        long long w = i % n;
                        if (w < 0) w += n;
                        b = (int)w;
                        f = (float)(rm - fl);
                    };
                    int mbx, mby, mbz;
                    mcell(Rx, origin(a, gid, 0), G.mox, G.mnx, mbx, mf.f0.x);
                    mcell(Ry, origin(a, gid, 1), G.moy, G.mny, mby, mf.f0.y);
                    mcell(Rz, origin(a, gid, 2), G.moz, G.mnz, mbz, mf.f0.z);
                    mf.lo = (u.x < 0.0f ? 1 : 0) | (u.y < 0.0f ? 2 : 0) | (u.z < 0.0f ? 4 : 0);
                    mod_fill(sm, G, mbx, mby, mbz, mf.lo);
                }
                new_step = false;
            }
            // ---- one Cash-Karp attempt in the local frame (FP32) ----
            const Y y0{{0.0f, 0.0f, 0.0f}, u};
            const Y k1 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, y0);
            Y t;
#define STG(expr)                                                                              \
            t.p.x = h * (expr(p.x)); t.p.y = h * (expr(p.y)); t.p.z = h * (expr(p.z));         \
            t.u.x = fmaf(h, (expr(u.x)), u.x); t.u.y = fmaf(h, (expr(u.y)), u.y);               \
            t.u.z = fmaf(h, (expr(u.z)), u.z);
#define S2(c) (A21 * k1.c)
            STG(S2)
            const Y k2 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, t);
#define S3(c) (A31 * k1.c + A32 * k2.c)
            STG(S3)
            const Y k3 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, t);
#define S4(c) (A41 * k1.c + A42 * k2.c + A43 * k3.c)
            STG(S4)
            const Y k4 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, t);
#define S5(c) (A51 * k1.c + A52 * k2.c + A53 * k3.c + A54 * k4.c)
            STG(S5)
            const Y k5 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, t);
#define S6(c) (A61 * k1.c + A62 * k2.c + A63 * k3.c + A64 * k4.c + A65 * k5.c)
            STG(S6)
            const Y k6 = deriv_f<L, M, P2>(F, bx, by, bz, f0, a.fields, gid, sm, mf, kappa, t);
#define SB(c) (B1 * k1.c + B3 * k3.c + B4 * k4.c + B6 * k6.c)
#define SE(c) (E1 * k1.c + E3 * k3.c + E4 * k4.c + E5 * k5.c + E6 * k6.c)
            const F3 dp{h * SB(p.x), h * SB(p.y), h * SB(p.z)};
            const F3 du{h * SB(u.x), h * SB(u.y), h * SB(u.z)};       // direction increment
            const F3 ex{SE(p.x), SE(p.y), SE(p.z)};                  // |dx| / h
            const F3 eu{h * SE(u.x), h * SE(u.y), h * SE(u.z)};      // |du|
#undef STG
#undef S2
#undef S3
#undef S4
#undef S5
#undef S6
#undef SB
#undef SE
            att_step += 1;
            // ---- FP64 error norm and accept/reject (certified from FP32 outside the band) ----
            const float qx32 = ex.x * ex.x + ex.y * ex.y + ex.z * ex.z;
            const float qu32 = eu.x * eu.x + eu.y * eu.y + eu.z * eu.z;
            bool accept;
            if (qx32 <= tol2_lo && qu32 <= tol2_lo) {
                accept = true;
            } else if (qx32 >= tol2_hi || qu32 >= tol2_hi) {
                accept = false;
            } else {
                const double exx = widen(ex.x), exy = widen(ex.y), exz = widen(ex.z);
                const double eux = widen(eu.x), euy = widen(eu.y), euz = widen(eu.z);
                const double qx = fma(exz, exz, fma(exy, exy, exx * exx));
                const double qu = fma(euz, euz, fma(euy, euy, eux * eux));
                accept = fmax(qx, qu) <= tol2;
            }
            accept = accept || (h <= hmin_c);
            const float r2 = fmaxf(qx32, qu32) * inv_tol2;
            if (!accept) {
                const float shrink = clampf_(0.95f * powf_pos(r2, -0.125f), 0.1f, 1.0f);
                h = fmaxf(h * shrink, hmin_c);
                rejected = 1;
                continue;
            }
            if (!(fin3(dp) && fin3(du))) {
                att_call += att_step;
                att_tot += att_step;
                bits |= BIT_NAN;
                store(CRP_STATUS_NAN_, false);
                continue;
            }
            const bool fires = (rpd > 0.0f && h == h_int);
            unsigned long long q = 0;
            if (fires) {
                q = atomicAdd(&C->reserve, 1ull);
                if (q >= (unsigned long long)a.capacity) {
                    bits |= BIT_QUEUE_FULL;
                    store(CRP_STATUS_ACTIVE_, false);
                    continue;
                }
            }
            // ---- accept ----
            att_call += att_step;
            att_tot += att_step;
            Rx = df_add(Rx, dp.x);
            Ry = df_add(Ry, dp.y);
            Rz = df_add(Rz, dp.z);
            {   // direction as a double-float: the increment is added with TwoSum
                const DF nx = df_add(DF{u.x, ul.x}, du.x), ny = df_add(DF{u.y, ul.y}, du.y),
                         nz = df_add(DF{u.z, ul.z}, du.z);
                u = {nx.hi, ny.hi, nz.hi};
                ul = {nx.lo, ny.lo, nz.lo};
            }
            if (a.boundary) {   // reflective box, evaluated on the FP64 position
                auto fold = [&](DF& R, double o, int ax, float& uc, float& ucl, double* u0col) {
                    double xd = to_x(R, o);
                    const double lo = a.box_lo[ax], hi = a.box_hi[ax];
                    if (!(xd < lo || xd > hi)) return;
                    const double t = (xd - lo) * a.box_inv[ax];
                    const double k = floor(t);
                    const double r = t - k;
                    const bool odd = fmod(k, 2.0) != 0.0;
                    xd = odd ? hi - r * a.box_len[ax] : lo + r * a.box_len[ax];
                    R = from_x(xd, o);
                    if (odd) { uc = -uc; ucl = -ucl; u0col[slot] = -u0col[slot]; }
                };
                fold(Rx, origin(a, gid, 0), 0, u.x, ul.x, S.u0x);
                fold(Ry, origin(a, gid, 1), 1, u.y, ul.y, S.u0y);
                fold(Rz, origin(a, gid, 2), 2, u.z, ul.z, S.u0z);
            }
            bool done = (h == h_dist);
            s_c = s_c + widen(h);
            if (s_c >= dslot(sm, 2)) done = true;
            if (done) s_c = dslot(sm, 2);
            acc_tot += 1;
            taken += 1;
            const float grow = (r2 == 0.0f) ? 5.0f : clampf_(0.95f * powf_pos(r2, -0.1f), 0.2f, 5.0f);
            float hnext = h * grow;
            if (!rejected && h_first < h_propc) hnext = fmaxf(hnext, h_propc);
            hprop = clampf_(hnext, hmin_c, fslot(sm, 0));
            if (rl > 0.0f) E = E * (double)__expf(-h * rl);
            if (rpd > 0.0f) {
                if (fires) {
                    const unsigned kk = (unsigned)(n_int + 1);
                    const unsigned long long uid = (unsigned long long)__ldcg(&S.uid[slot]);
                    const int dz = nucleon_proton(a.seed, uid, kk, A, Z) ? 1 : 0;
                    const double E_sec = E / (double)A;
                    const double E_par = E * (double)(A - 1) / (double)A;
                    const long long qs = (long long)q;
                    const unsigned long long uid2 = (1ull << 32) + uid * 64ull + kk;
                    S.x[qs] = to_x(Rx, origin(a, gid, 0)); S.y[qs] = to_x(Ry, origin(a, gid, 1)); S.z[qs] = to_x(Rz, origin(a, gid, 2));
                    S.ux[qs] = (double)u.x + (double)ul.x; S.uy[qs] = (double)u.y + (double)ul.y;
                    S.uz[qs] = (double)u.z + (double)ul.z;
                    S.E[qs] = E_sec;
                    S.s[qs] = done ? a.dmax : s_c * dslot(sm, 0);
                    S.hprop[qs] = __longlong_as_double(0x7ff0000000000000LL);
                    S.tau[qs] = -crp_log(uniform01(a.seed, uid2, 0u, 0u));
                    S.u0x[qs] = S.u0x[slot]; S.u0y[qs] = S.u0y[slot]; S.u0z[qs] = S.u0z[slot];
                    S.A[qs] = 1; S.Z[qs] = dz; S.n_int[qs] = 0; S.grid_id[qs] = gid;
                    S.uid[qs] = (long long)uid2;
                    S.n_steps[qs] = 0; S.n_att[qs] = 0;
                    S.status[qs] = done ? CRP_STATUS_DONE_ : CRP_STATUS_ACTIVE_;
                    if (done) {
                        const unsigned long long d = atomicAdd(&C->n_done, 1ull);
                        a.done_list[d] = (int32_t)qs;
                    } else {
                        sched_push(a, (int32_t)qs);
                    }
                    sec_tot += 1;
                    A = A - 1;
                    Z = Z - dz;
                    E = E_par;
                    n_int = (int)kk;
                    tau = (float)(-crp_log(uniform01(a.seed, uid, kk, 0u)));
                } else {
                    tau = tau - h * rpd;
                }
            }
            new_step = true;
            if (done) {
                store(CRP_STATUS_DONE_, true);
            } else if (a.max_steps > 0 && taken >= a.max_steps) {
                store(CRP_STATUS_ACTIVE_, false);
            }
        }
    }

#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_tot += __shfl_xor_sync(kFull, acc_tot, o);
        att_tot += __shfl_xor_sync(kFull, att_tot, o);
        sec_tot += __shfl_xor_sync(kFull, sec_tot, o);
        bits |= __shfl_xor_sync(kFull, bits, o);
    }
    if (lane == 0) {
        if (acc_tot) atomicAdd(&C->accepted, acc_tot);
        if (att_tot) atomicAdd(&C->attempted, att_tot);
        if (sec_tot) atomicAdd(&C->secondaries, sec_tot);
        if (bits) atomicOr(&C->status_bits, bits);
    }
}

// Register caps (more resident warps to hide gather latency); build-time tuning knobs. By
// default the unmodulated kernel is bounded to 128 registers (16 warps per SM with 128-thread
// blocks): with the field constants in shared slots and 32-bit per-call counters its state fits
// (the BF16 cell layout without spills), and the latency-bound lookups gain from the extra warps.
#ifdef CRP_MIXED_MAXNREG
#define CRP_MIXED_BOUNDS __maxnreg__(CRP_MIXED_MAXNREG)
#else
#define CRP_MIXED_BOUNDS __launch_bounds__(256, 2)
#endif
#ifdef CRP_MIXED_MOD_MAXNREG
#define CRP_MIXED_MOD_BOUNDS __maxnreg__(CRP_MIXED_MOD_MAXNREG)
#else
#define CRP_MIXED_MOD_BOUNDS __launch_bounds__(256)
#endif

// Dynamic shared memory: kFieldWords words per thread (field constants), + kModSlots floats per
// thread for modulated fields.
template <int L, bool P2>
__global__ void CRP_MIXED_BOUNDS k_propagate_mixed(const PropArgs a) {
    CRP_COUNT_RUN();
    extern __shared__ double field_sm[];
    propagate_mixed_body<L, false, P2>(a, reinterpret_cast<float*>(field_sm));
}

template <int L, bool P2>
__global__ void CRP_MIXED_MOD_BOUNDS k_propagate_mixed_mod(const PropArgs a) {
    CRP_COUNT_RUN();
    extern __shared__ double mod_sm[];
    propagate_mixed_body<L, true, P2>(a, reinterpret_cast<float*>(mod_sm));
}

}  // namespace

// Kernel for (layout, modulated, power-of-two vector grids): FP32 or BF16 vector grids,
// node- or cell-major.
template <bool P2, typename Fn>
int with_mixed_kernel_p2(int layout, int mod, Fn&& fn) {
    switch (layout) {
    case LAYOUT_F32X4:
        return mod ? fn(k_propagate_mixed_mod<LAYOUT_F32X4, P2>) : fn(k_propagate_mixed<LAYOUT_F32X4, P2>);
    case LAYOUT_BF16X4:
        return mod ? fn(k_propagate_mixed_mod<LAYOUT_BF16X4, P2>) : fn(k_propagate_mixed<LAYOUT_BF16X4, P2>);
    case LAYOUT_F32_CELLS:
        return mod ? fn(k_propagate_mixed_mod<LAYOUT_F32_CELLS, P2>) : fn(k_propagate_mixed<LAYOUT_F32_CELLS, P2>);
    case LAYOUT_BF16_CELLS:
        return mod ? fn(k_propagate_mixed_mod<LAYOUT_BF16_CELLS, P2>) : fn(k_propagate_mixed<LAYOUT_BF16_CELLS, P2>);
    default: return (int)cudaErrorInvalidValue;
    }
}

template <typename Fn>
int with_mixed_kernel(int layout, int mod, int p2, Fn&& fn) {
    return p2 ? with_mixed_kernel_p2<true>(layout, mod, fn) : with_mixed_kernel_p2<false>(layout, mod, fn);
}

size_t mixed_smem(int mod, int block) { return (size_t)(kFieldWords + (mod ? kModSlots : 0)) * sizeof(float) * block; }

// Shared-memory carveout that holds the launch's blocks per SM and leaves the rest of the SM's
// unified L1/shared storage to L1: the gathers are served from L1 (the driver's own choice for
// this kernel was a 100 KB carveout, 37 KB used). Percent of the SM's shared-memory maximum,
// with the driver's per-block reservation; the driver rounds up to a configuration it supports.
static int mixed_carveout_pct(int grid, size_t shm_per_block) {
    int dev = 0, smem = 0, sms = 0, reserved = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        smem <= 0 || sms <= 0) {
        cudaGetLastError();
        return -1;   // the driver's default
    }
    const long long bps = (grid + sms - 1) / sms;
    const long long need = bps * ((long long)shm_per_block + reserved);
    const long long pct = (100 * need + smem - 1) / smem + 1;
    return pct > 100 ? 100 : (int)pct;
}

int launch_propagate_mixed(const PropArgs& a, int layout, int mod, int p2, int grid, int block, void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t shm = mixed_smem(mod, block);
    const int pct = mixed_carveout_pct(grid, shm);
    return with_mixed_kernel(layout, mod, p2, [&](void (*k)(const PropArgs)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        if (e != cudaSuccess) return (int)e;
        k<<<grid, block, shm, st>>>(a);
        return (int)cudaGetLastError();
    });
}

int propagate_mixed_occupancy(int layout, int mod, int p2, int block, int* blocks_per_sm) {
    const size_t shm = mixed_smem(mod, block);
    return with_mixed_kernel(layout, mod, p2, [&](void (*k)(const PropArgs)) {
        // the query sees the driver's default carveout, not the one a previous launch chose
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
        if (e != cudaSuccess) return (int)e;
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, shm);
    });
}

}  // namespace crp

namespace crp {
unsigned long long kernel_runs_mixed() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
