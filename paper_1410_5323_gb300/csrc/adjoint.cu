// adjoint.cu -- differentiation form of the propagation (arXiv:1410.5323 3D deflection,
// Sec. 2; regular grids, Sec. 3.2): reverse mode through a frozen step sequence.
//
// A forward pass with the adaptive Cash-Karp controller records the accepted step sizes
// h_n and checkpoints y = (x, u) every K steps. The map y_{n+1} = y_n + h_n sum_i b_i k_i
// is then differentiated exactly for fixed h_n: the states are recomputed from the
// checkpoints (all segments in parallel into a stage-state buffer when the device has room,
// else one segment at a time per particle), and the steps are reversed stage by stage with the
// vector-Jacobian product of f(y) = (u, kappa u x B(x)), which also yields dL/dkappa and
// scatters dL/dB into the grid gradient through the trilinear weights (FP64 atomics).
// Compiled with --fmad=false; per-particle arithmetic follows the oracle's order.
#include <cuda_runtime.h>

#include <algorithm>

#include "crp_fp64.cuh"
#include "crp_internal.h"
#include "crp_math.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

namespace crp {
namespace {

using namespace fp64;

__device__ __forceinline__ void load6(const double* a, long long n, long long i, Y6& y) {
    y.x = a[0 * n + i]; y.y = a[1 * n + i]; y.z = a[2 * n + i];
    y.ux = a[3 * n + i]; y.uy = a[4 * n + i]; y.uz = a[5 * n + i];
}
__device__ __forceinline__ void store6(double* a, long long n, long long i, const Y6& y) {
    a[0 * n + i] = y.x; a[1 * n + i] = y.y; a[2 * n + i] = y.z;
    a[3 * n + i] = y.ux; a[4 * n + i] = y.uy; a[5 * n + i] = y.uz;
}

// E = |p0| ((p_x^2 + p_y^2) + p_z^2, then sqrt), u0 = p0 / E, kappa = (Z c) / E; positions
// are copied from x0 unless it is NULL (then the position rows of y0 are left as they are).
__global__ void k_adj_init(const double* __restrict__ x0, const double* __restrict__ p0,
                           const int32_t* __restrict__ Z, double* __restrict__ y0,
                           double* __restrict__ kappa, double* __restrict__ E, long long n) {
    CRP_COUNT_RUN();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = p0[3 * i], py = p0[3 * i + 1], pz = p0[3 * i + 2];
    const double e = sqrt((px * px + py * py) + pz * pz);
    if (x0) {
        y0[0 * n + i] = x0[3 * i]; y0[1 * n + i] = x0[3 * i + 1]; y0[2 * n + i] = x0[3 * i + 2];
    }
    y0[3 * n + i] = px / e; y0[4 * n + i] = py / e; y0[5 * n + i] = pz / e;
    E[i] = e;
    kappa[i] = (double)Z[i] * kC / e;
}

template <int L, bool H = false>
__device__ __forceinline__ void frozen_step(const FieldDev& F, double kappa, Y6& y, double h,
                                            unsigned long long* hh = nullptr) {
    const Y6 k1 = deriv<L, H>(F, kappa, y, hh);
    Y6 y5, err;
    ck_attempt<L, H>(F, kappa, y, k1, h, y5, err, hh);
    y = y5;
}

// Frozen replay; with H also the hash of every cell its stages looked up (two replays with
// equal hashes stayed inside the same cells, where the map is smooth).
template <int L, bool H>
__global__ void k_adj_replay(FieldDev F, const double* __restrict__ y0, const double* __restrict__ kap,
                             const double* __restrict__ h, int n_steps, double* __restrict__ xT,
                             double* __restrict__ uT, unsigned long long* __restrict__ cell_hash,
                             long long n) {
    CRP_COUNT_RUN();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Y6 y;
    load6(y0, n, i, y);
    const double kappa = kap[i];
    unsigned long long hh = 0;
    for (int m = 0; m < n_steps; ++m) frozen_step<L, H>(F, kappa, y, h[(long long)m * n + i], &hh);
    xT[3 * i] = y.x; xT[3 * i + 1] = y.y; xT[3 * i + 2] = y.z;
    uT[3 * i] = y.ux; uT[3 * i + 1] = y.uy; uT[3 * i + 2] = y.uz;
    if (H) cell_hash[i] = hh;
}

// What the reverse sweep needs of one lookup: B, the corner weights and nodes, and the field's
// Jacobian J[q][a] = dB_q/dx_a = sum_c (dw_c/dx_a) G_c[q] (corners 000, 001, ..., 111, one
// rounding per corner; dw_c/dx_a = (d w_a) * w_b * w_c with d(1 - f) = -1/spacing,
// d f = 1/spacing). B is formed exactly as the forward lookup forms it.
struct Look {
    double B[3], w[8], J[3][3];
    long long node[8];
};

// P2: the grid's sizes are powers of two (indices wrap with a mask, as in field_b).
template <int L, bool P2 = false>
__device__ __forceinline__ void lookup_jac(const FieldDev& F, double x, double y, double z, Look& o) {
    long long ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    axis<P2>(x, F.oix, F.inv_spacing, F.nx, F.pow2, ix[0], ix[1], wx[0], wx[1]);
    axis<P2>(y, F.oiy, F.inv_spacing, F.ny, F.pow2, iy[0], iy[1], wy[0], wy[1]);
    axis<P2>(z, F.oiz, F.inv_spacing, F.nz, F.pow2, iz[0], iz[1], wz[0], wz[1]);
    const double dd[2] = {-F.inv_spacing, F.inv_spacing};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        o.B[q] = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) o.J[q][d] = 0.0;
    }
    int c8 = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c, ++c8) {
                const double wab = wx[a] * wy[b];
                const double wt = wab * wz[c];
                const double dw[3] = {(dd[a] * wy[b]) * wz[c], (wx[a] * dd[b]) * wz[c], wab * dd[c]};
                o.w[c8] = wt;
                o.node[c8] = (ix[a] * F.ny + iy[b]) * F.nz + iz[c];
                const V3 g = corner<L>(F, o.node[c8]);
                const double G[3] = {g.x, g.y, g.z};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    o.B[q] = __fma_rn(wt, G[q], o.B[q]);      // as the forward lookup
#pragma unroll
                    for (int d = 0; d < 3; ++d) o.J[q][d] = __fma_rn(dw[d], G[q], o.J[q][d]);
                }
            }
}

// Vector-Jacobian product of f(Y) = (u, kappa u x B(x)) with cotangent kb = (abar, bbar), from
// the stage's direction u, field B, Jacobian J, corner weights w and nodes:
//   Bbar = kappa (bbar x u); kappa_bar += bbar . (u x B); Ybar_u = abar + kappa (B x bbar);
//   Ybar_x = J^T Bbar; grid_bar[node_c] += w_c Bbar (FP64 atomics).
__device__ __forceinline__ void vjp_apply(double kappa, double ux, double uy, double uz, const double B[3],
                                          const double J[3][3], const double w[8], const long long node[8],
                                          const Y6& kb, Y6& Yb, double* __restrict__ grid_bar,
                                          double& kappa_bar) {
    const double Bb0 = kappa * (kb.uy * uz - kb.uz * uy);
    const double Bb1 = kappa * (kb.uz * ux - kb.ux * uz);
    const double Bb2 = kappa * (kb.ux * uy - kb.uy * ux);
    const double uxB0 = uy * B[2] - uz * B[1];
    const double uxB1 = uz * B[0] - ux * B[2];
    const double uxB2 = ux * B[1] - uy * B[0];
    kappa_bar = kappa_bar + ((kb.ux * uxB0 + kb.uy * uxB1) + kb.uz * uxB2);
    Yb.ux = kb.x + kappa * (B[1] * kb.uz - B[2] * kb.uy);
    Yb.uy = kb.y + kappa * (B[2] * kb.ux - B[0] * kb.uz);
    Yb.uz = kb.z + kappa * (B[0] * kb.uy - B[1] * kb.ux);
    Yb.x = (J[0][0] * Bb0 + J[1][0] * Bb1) + J[2][0] * Bb2;
    Yb.y = (J[0][1] * Bb0 + J[1][1] * Bb1) + J[2][1] * Bb2;
    Yb.z = (J[0][2] * Bb0 + J[1][2] * Bb1) + J[2][2] * Bb2;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double* gp = grid_bar + node[c] * 3;
        atomicAdd(gp + 0, w[c] * Bb0);
        atomicAdd(gp + 1, w[c] * Bb1);
        atomicAdd(gp + 2, w[c] * Bb2);
    }
}

// Vector-Jacobian product of f at stage state Y (lookup on the fly).
template <int L>
__device__ __forceinline__ void vjp_f(const FieldDev& F, double kappa, const Y6& Y, const Y6& kb,
                                      Y6& Yb, double* __restrict__ grid_bar, double& kappa_bar) {
    Look o;
    lookup_jac<L>(F, Y.x, Y.y, Y.z, o);
    vjp_apply(kappa, Y.ux, Y.uy, Y.uz, o.B, o.J, o.w, o.node, kb, Yb, grid_bar, kappa_bar);
}

__device__ __forceinline__ void axpy6(Y6& acc, double s, const Y6& v) {
    acc.x = acc.x + s * v.x; acc.y = acc.y + s * v.y; acc.z = acc.z + s * v.z;
    acc.ux = acc.ux + s * v.ux; acc.uy = acc.uy + s * v.uy; acc.uz = acc.uz + s * v.uz;
}
__device__ __forceinline__ void fmaxpy6(Y6& acc, double s, const Y6& v) {
    acc.x = __fma_rn(s, v.x, acc.x); acc.y = __fma_rn(s, v.y, acc.y); acc.z = __fma_rn(s, v.z, acc.z);
    acc.ux = __fma_rn(s, v.ux, acc.ux); acc.uy = __fma_rn(s, v.uy, acc.uy); acc.uz = __fma_rn(s, v.uz, acc.uz);
}
__device__ __forceinline__ Y6 scale6(double s, const Y6& v) {
    return {s * v.x, s * v.y, s * v.z, s * v.ux, s * v.uy, s * v.uz};
}
__device__ __forceinline__ void add6(Y6& acc, const Y6& v) {
    acc.x = acc.x + v.x; acc.y = acc.y + v.y; acc.z = acc.z + v.z;
    acc.ux = acc.ux + v.ux; acc.uy = acc.uy + v.uy; acc.uz = acc.uz + v.uz;
}

__constant__ double cA[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
__constant__ double cB5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
constexpr double cB5h[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};

// The six stage states Y_0 = y_m, ..., Y_5 of step m (the forward stage sums: acc = A[i][0]
// k1, then fused A[i][j] k_j for j < i; y + h acc fused).
template <int L>
__device__ __forceinline__ void stage_states(const FieldDev& F, double kappa, const Y6& y, double hn, Y6 (&Y)[6]) {
    Y6 k[6];
    Y[0] = y;
    k[0] = deriv<L>(F, kappa, y);
    for (int i = 1; i < 6; ++i) {
        Y6 acc = scale6(cA[i][0], k[0]);
        for (int j = 1; j < i; ++j) fmaxpy6(acc, cA[i][j], k[j]);
        Y[i] = {__fma_rn(hn, acc.x, y.x), __fma_rn(hn, acc.y, y.y), __fma_rn(hn, acc.z, y.z),
                __fma_rn(hn, acc.ux, y.ux), __fma_rn(hn, acc.uy, y.uy), __fma_rn(hn, acc.uz, y.uz)};
        if (i < 5) k[i] = deriv<L>(F, kappa, Y[i]);
    }
}

// One reverse step from the stage states: lam = dL/dy_{m+1} in, dL/dy_m out.
template <int L>
__device__ void reverse_step(const FieldDev& F, double kappa, const Y6 (&Y)[6], double hn, Y6& lam,
                             double* __restrict__ grid_bar, double& kappa_bar) {
    Y6 kb[6];
    for (int i = 0; i < 6; ++i) kb[i] = scale6(hn * cB5[i], lam);
    Y6 yb = lam;
    for (int i = 5; i >= 0; --i) {
        Y6 Yb;
        vjp_f<L>(F, kappa, Y[i], kb[i], Yb, grid_bar, kappa_bar);
        add6(yb, Yb);
        for (int j = 0; j < i; ++j) axpy6(kb[j], hn * cA[i][j], Yb);
    }
    lam = yb;
}

template <int L>
__device__ __forceinline__ void adjoint_step(const FieldDev& F, double kappa, const Y6& y, double hn, Y6& lam,
                                             double* __restrict__ grid_bar, double& kappa_bar) {
    Y6 Y[6];
    stage_states<L>(F, kappa, y, hn, Y);
    reverse_step<L>(F, kappa, Y, hn, lam, grid_bar, kappa_bar);
}

// Stage records: for every step m and stage s of chain i, what the reverse sweep applies
// (all of it a function of the stage state alone): the direction u, B, the Jacobian J and
// the corner weights (kRecD doubles at rec_d[((m * 6 + s) * kRecD + k) * n + i]) and the
// corner nodes (kRecN int32 at rec_n[((m * 6 + s) * kRecN + k) * n + i]).
constexpr int kRecD = 3 + 3 + 9 + 8;
constexpr int kRecN = 8;
static_assert(kAdjRecordBytes == 6 * (kRecD * sizeof(double) + kRecN * sizeof(int32_t)), "record size");

__device__ __forceinline__ void put_rec(double* __restrict__ rec_d, int32_t* __restrict__ rec_n, long long n,
                                        long long i, int m, int st, const Y6& Y, const Look& o) {
    double* d = rec_d + ((long long)(m * 6 + st) * kRecD) * n + i;
    d[0 * n] = Y.ux; d[1 * n] = Y.uy; d[2 * n] = Y.uz;
    d[3 * n] = o.B[0]; d[4 * n] = o.B[1]; d[5 * n] = o.B[2];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) d[(6 + 3 * q + a) * n] = o.J[q][a];
#pragma unroll
    for (int c = 0; c < 8; ++c) d[(15 + c) * n] = o.w[c];
    int32_t* q = rec_n + ((long long)(m * 6 + st) * kRecN) * n + i;
#pragma unroll
    for (int c = 0; c < 8; ++c) q[c * n] = (int32_t)o.node[c];
}

// f(Y) from its lookup, exactly as deriv() forms it.
__device__ __forceinline__ Y6 deriv_from(double kappa, const Y6& y, const Look& o) {
    Y6 k;
    k.x = y.ux; k.y = y.uy; k.z = y.uz;
    k.ux = kappa * __fma_rn(y.uy, o.B[2], -(y.uz * o.B[1]));
    k.uy = kappa * __fma_rn(y.uz, o.B[0], -(y.ux * o.B[2]));
    k.uz = kappa * __fma_rn(y.ux, o.B[1], -(y.uy * o.B[0]));
    return k;
}

// Stage records of the segments [sg0, sg0 + n_seg): thread (particle i, segment sg)
// recomputes its segment from the checkpoint. Each step evaluates f at its six stage states
// with the forward stage sums (as ck_attempt) and advances y by the 5th-order update, so the
// states are the frozen forward's, bit for bit.
template <int L, bool P2>
__global__ void k_adj_records(FieldDev F, const double* __restrict__ kap, const double* __restrict__ h,
                              const double* __restrict__ ck, double* __restrict__ rec_d,
                              int32_t* __restrict__ rec_n, int n_steps, int K, int sg0, int n_seg,
                              long long n) {
    CRP_COUNT_RUN();
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n * n_seg) return;
    const long long i = t % n;
    const int sg = sg0 + (int)(t / n);
    const double kappa = kap[i];
    const int m0 = sg * K, m1 = min(m0 + K, n_steps);
    Y6 y;
    load6(ck + (long long)sg * 6 * n, n, i, y);
    for (int m = m0; m < m1; ++m) {
        const double h_ = h[(long long)m * n + i];
        Look o;
        Y6 t_;
        lookup_jac<L, P2>(F, y.x, y.y, y.z, o);
        put_rec(rec_d, rec_n, n, i, m, 0, y, o);
        const Y6 k1 = deriv_from(kappa, y, o);
#define ADJ_STAGE(dst, expr)                                                                \
        do {                                                                                \
            dst.x = __fma_rn(h_, expr(x), y.x);    dst.y = __fma_rn(h_, expr(y), y.y);      \
            dst.z = __fma_rn(h_, expr(z), y.z);    dst.ux = __fma_rn(h_, expr(ux), y.ux);   \
            dst.uy = __fma_rn(h_, expr(uy), y.uy); dst.uz = __fma_rn(h_, expr(uz), y.uz);   \
        } while (0)
#define R2(c) (A21 * k1.c)
        ADJ_STAGE(t_, R2);
        lookup_jac<L, P2>(F, t_.x, t_.y, t_.z, o);
        put_rec(rec_d, rec_n, n, i, m, 1, t_, o);
        const Y6 k2 = deriv_from(kappa, t_, o);
#define R3(c) __fma_rn(A32, k2.c, A31 * k1.c)
        ADJ_STAGE(t_, R3);
        lookup_jac<L, P2>(F, t_.x, t_.y, t_.z, o);
        put_rec(rec_d, rec_n, n, i, m, 2, t_, o);
        const Y6 k3 = deriv_from(kappa, t_, o);
#define R4(c) __fma_rn(A43, k3.c, __fma_rn(A42, k2.c, A41 * k1.c))
        ADJ_STAGE(t_, R4);
        lookup_jac<L, P2>(F, t_.x, t_.y, t_.z, o);
        put_rec(rec_d, rec_n, n, i, m, 3, t_, o);
        const Y6 k4 = deriv_from(kappa, t_, o);
#define R5(c) __fma_rn(A54, k4.c, __fma_rn(A53, k3.c, __fma_rn(A52, k2.c, A51 * k1.c)))
        ADJ_STAGE(t_, R5);
        lookup_jac<L, P2>(F, t_.x, t_.y, t_.z, o);
        put_rec(rec_d, rec_n, n, i, m, 4, t_, o);
        const Y6 k5 = deriv_from(kappa, t_, o);
#define R6(c) __fma_rn(A65, k5.c, __fma_rn(A64, k4.c, __fma_rn(A63, k3.c, __fma_rn(A62, k2.c, A61 * k1.c))))
        ADJ_STAGE(t_, R6);
        lookup_jac<L, P2>(F, t_.x, t_.y, t_.z, o);
        put_rec(rec_d, rec_n, n, i, m, 5, t_, o);
        const Y6 k6 = deriv_from(kappa, t_, o);
#define RB(c) __fma_rn(B6, k6.c, __fma_rn(B4, k4.c, __fma_rn(B3, k3.c, B1 * k1.c)))
        Y6 y5;
        ADJ_STAGE(y5, RB);
        y = y5;
#undef ADJ_STAGE
#undef R2
#undef R3
#undef R4
#undef R5
#undef R6
#undef RB
    }
}

template <int L>
__global__ void k_adj_backward(FieldDev F, const double* __restrict__ kap, const double* __restrict__ h,
                               const double* __restrict__ ck, double* __restrict__ seg, int n_steps,
                               int K, const double* __restrict__ uT_bar, double* __restrict__ grid_bar,
                               double* __restrict__ y0_bar, double* __restrict__ kappa_bar_out,
                               long long n) {
    CRP_COUNT_RUN();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double kappa = kap[i];
    Y6 lam{0.0, 0.0, 0.0, uT_bar[3 * i], uT_bar[3 * i + 1], uT_bar[3 * i + 2]};
    double kappa_bar = 0.0;
    const int n_seg = (n_steps + K - 1) / K;
    for (int sg = n_seg - 1; sg >= 0; --sg) {
        const int m0 = sg * K, m1 = min(m0 + K, n_steps);
        Y6 y;
        load6(ck + (long long)sg * 6 * n, n, i, y);
        store6(seg, n, i, y);
        for (int m = m0; m < m1; ++m) {          // recompute the segment from its checkpoint
            frozen_step<L>(F, kappa, y, h[(long long)m * n + i]);
            store6(seg + (long long)(m - m0 + 1) * 6 * n, n, i, y);
        }
        for (int m = m1 - 1; m >= m0; --m) {
            Y6 ym;
            load6(seg + (long long)(m - m0) * 6 * n, n, i, ym);
            adjoint_step<L>(F, kappa, ym, h[(long long)m * n + i], lam, grid_bar, kappa_bar);
        }
    }
    store6(y0_bar, n, i, lam);
    kappa_bar_out[i] = kappa_bar;
}

// dL/dp0 = (ubar0 - (u0 . ubar0) u0) / E + Ebar u0 with Ebar = -(kappa_bar * kappa) / E;
// dL/dx0 = xbar0.
__global__ void k_adj_p0bar(const double* __restrict__ y0, const double* __restrict__ kap,
                            const double* __restrict__ E, const double* __restrict__ y0_bar,
                            const double* __restrict__ kappa_bar, double* __restrict__ p0_bar,
                            double* __restrict__ x0_bar, long long n) {
    CRP_COUNT_RUN();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Y6 y, yb;
    load6(y0, n, i, y);
    load6(y0_bar, n, i, yb);
    const double e = E[i];
    const double dot = (y.ux * yb.ux + y.uy * yb.uy) + y.uz * yb.uz;
    const double Eb = -(kappa_bar[i] * kap[i]) / e;
    p0_bar[3 * i] = (yb.ux - dot * y.ux) / e + Eb * y.ux;
    p0_bar[3 * i + 1] = (yb.uy - dot * y.uy) / e + Eb * y.uy;
    p0_bar[3 * i + 2] = (yb.uz - dot * y.uz) / e + Eb * y.uz;
    if (x0_bar) {
        x0_bar[3 * i] = yb.x; x0_bar[3 * i + 1] = yb.y; x0_bar[3 * i + 2] = yb.z;
    }
}

// ---- team form: three lanes per particle ----------------------------------------------------
// GB300 issues one FP64 warp instruction per 64 cycles per SM sub-partition, whatever the
// number of active lanes, and the forward and reverse sweeps have one chain per particle: their
// time is each lane's FP64 instruction count. A team of three lanes (lanes 3t, 3t+1, 3t+2; ten
// teams per warp) shares one particle: lane c owns component c of the position and direction,
// of every stage state, stage derivative and cotangent, forms axis c of each lookup, a share of
// the corner weights, B_c and the c-th Lorentz component. Values of the whole particle (error
// sums, accept decision, step size, kappa_bar) are formed by the same operations in all three
// lanes. Every value is the one the one-lane form computes, so the results are the same bits.
constexpr int kTeams = 10;

struct Team {
    unsigned mask;   // the team's lanes
    int l0, c;       // its first lane, this lane's component
    double oi;       // origin / spacing along axis c (rounded once), grid size along it
    int nn;
    __device__ __forceinline__ double get(double v, int k) const { return __shfl_sync(mask, v, l0 + k); }
    __device__ __forceinline__ long long get(long long v, int k) const { return __shfl_sync(mask, v, l0 + k); }
    __device__ __forceinline__ int nx1() const { return c == 2 ? 0 : c + 1; }
    __device__ __forceinline__ int nx2() const { return c == 0 ? 2 : c - 1; }
};

// B_c at the team's stage position (lane c holds its coordinate xc): the periodic trilinear
// lookup of field_b, with the axes, the corner weights and the corner loads split over the
// team. FP64 node copy: component c of node k at ((const double*)data)[4k + c].
template <bool P2>
__device__ __forceinline__ double field_team(const FieldDev& F, const Team& T, double xc) {
    long long i0, i1;
    const double oi = T.oi;
    const int nn = T.nn;
    double w0, w1;
    axis<P2>(xc, oi, F.inv_spacing, nn, F.pow2, i0, i1, w0, w1);
    const long long ix0 = T.get(i0, 0), ix1 = T.get(i1, 0), iy0 = T.get(i0, 1), iy1 = T.get(i1, 1);
    const long long iz0 = T.get(i0, 2), iz1 = T.get(i1, 2);
    const double wx0 = T.get(w0, 0), wx1 = T.get(w1, 0), wy0 = T.get(w0, 1), wy1 = T.get(w1, 1);
    const double wz0 = T.get(w0, 2), wz1 = T.get(w1, 2);
    // lane 0 forms w00, w01 and t0..t3, lane 1 w10, w11 and t4..t7 (lane 2 repeats lane 1)
    const double wxa = T.c == 0 ? wx0 : wx1;
    const double wA = wxa * wy0, wB = wxa * wy1;
    const double tA0 = wA * wz0, tA1 = wA * wz1, tB0 = wB * wz0, tB1 = wB * wz1;
    const double t0 = T.get(tA0, 0), t1 = T.get(tA1, 0), t2 = T.get(tB0, 0), t3 = T.get(tB1, 0);
    const double t4 = T.get(tA0, 1), t5 = T.get(tA1, 1), t6 = T.get(tB0, 1), t7 = T.get(tB1, 1);
    const long long ny = F.ny, nz = F.nz;
    const long long r00 = (ix0 * ny + iy0) * nz, r01 = (ix0 * ny + iy1) * nz;
    const long long r10 = (ix1 * ny + iy0) * nz, r11 = (ix1 * ny + iy1) * nz;
    const double* G = reinterpret_cast<const double*>(F.data) + T.c;
    const double g0 = __ldg(G + 4 * (r00 + iz0)), g1 = __ldg(G + 4 * (r00 + iz1));
    const double g2 = __ldg(G + 4 * (r01 + iz0)), g3 = __ldg(G + 4 * (r01 + iz1));
    const double g4 = __ldg(G + 4 * (r10 + iz0)), g5 = __ldg(G + 4 * (r10 + iz1));
    const double g6 = __ldg(G + 4 * (r11 + iz0)), g7 = __ldg(G + 4 * (r11 + iz1));
    double B = __fma_rn(t0, g0, 0.0);
    B = __fma_rn(t1, g1, B);
    B = __fma_rn(t2, g2, B);
    B = __fma_rn(t3, g3, B);
    B = __fma_rn(t4, g4, B);
    B = __fma_rn(t5, g5, B);
    B = __fma_rn(t6, g6, B);
    B = __fma_rn(t7, g7, B);
    return B;
}

// Component c of f(Y) = (u, kappa u x B(x)): (ku_c = kappa fma(u_{c+1}, B_{c+2}, -(u_{c+2} B_{c+1}))).
template <bool P2>
__device__ __forceinline__ void deriv_team(const FieldDev& F, const Team& T, double kappa, double yx,
                                           double yu, double& kx, double& ku) {
    const double B = field_team<P2>(F, T, yx);
    const double u1 = T.get(yu, T.nx1()), u2 = T.get(yu, T.nx2());
    const double B1 = T.get(B, T.nx1()), B2 = T.get(B, T.nx2());
    kx = yu;
    ku = kappa * __fma_rn(u1, B2, -(u2 * B1));
}

__device__ __forceinline__ Team make_team(long long n, long long& i, bool& active, const FieldDev* F = nullptr) {
    const int lane = threadIdx.x & 31;
    const int team = lane / 3;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    i = warp * kTeams + team;
    active = lane < 3 * kTeams && i < n;
    Team T;
    T.l0 = 3 * team;
    T.c = lane - T.l0;
    T.mask = 7u << T.l0;
    T.oi = 0.0;
    T.nn = 1;
    if (F) {
        T.oi = T.c == 0 ? F->oix : (T.c == 1 ? F->oiy : F->oiz);
        T.nn = T.c == 0 ? F->nx : (T.c == 1 ? F->ny : F->nz);
    }
    return T;
}

// Forward with the propagation module's controller only, in team form; records h_n and the
// checkpoints of every K-th step (the oracle's frozen forward, value for value).
template <bool P2>
__global__ void k_adj_record_team(FieldDev F, const double* __restrict__ y0, const double* __restrict__ kap,
                                  double tol, double hmin, double hmax, int n_steps, int K,
                                  double* __restrict__ h_out, double* __restrict__ ck,
                                  double* __restrict__ xT, double* __restrict__ uT, long long n) {
    CRP_COUNT_RUN();
    long long i;
    bool active;
    const Team T = make_team(n, i, active, &F);
    if (!active) return;
    const int c = T.c;
    double yx = y0[(long long)c * n + i], yu = y0[(long long)(3 + c) * n + i];
    const double kappa = kap[i];
    const double tol2 = tol * tol;
    const float lg_tol = ctrl_log2(tol);
    // one attempt per iteration: teams that retry a step and teams that start one run the
    // attempt together (a rejection in one team does not make the warp repeat it for the rest)
    double hprop = __longlong_as_double(0x7ff0000000000000LL);
    double h = 0.0, h_prop = 0.0, k1x = 0.0, k1u = 0.0;
    int m = 0, rejected = 0;
    bool new_step = true;
    while (m < n_steps) {
        if (new_step) {
            if (m % K == 0) {
                double* q = ck + (long long)(m / K) * 6 * n;
                q[(long long)c * n + i] = yx;
                q[(long long)(3 + c) * n + i] = yu;
            }
            h_prop = clampd(hprop, hmin, hmax);
            h = h_prop;
            deriv_team<P2>(F, T, kappa, yx, yu, k1x, k1u);
            rejected = 0;
            new_step = false;
        }
        double tx, tu, k2x, k2u, k3x, k3u, k4x, k4u, k5x, k5u, k6x, k6u;
        tx = __fma_rn(h, A21 * k1x, yx); tu = __fma_rn(h, A21 * k1u, yu);
        deriv_team<P2>(F, T, kappa, tx, tu, k2x, k2u);
#define T3(k) __fma_rn(A32, k2##k, A31 * k1##k)
        tx = __fma_rn(h, T3(x), yx); tu = __fma_rn(h, T3(u), yu);
        deriv_team<P2>(F, T, kappa, tx, tu, k3x, k3u);
#define T4(k) __fma_rn(A43, k3##k, __fma_rn(A42, k2##k, A41 * k1##k))
        tx = __fma_rn(h, T4(x), yx); tu = __fma_rn(h, T4(u), yu);
        deriv_team<P2>(F, T, kappa, tx, tu, k4x, k4u);
#define T5(k) __fma_rn(A54, k4##k, __fma_rn(A53, k3##k, __fma_rn(A52, k2##k, A51 * k1##k)))
        tx = __fma_rn(h, T5(x), yx); tu = __fma_rn(h, T5(u), yu);
        deriv_team<P2>(F, T, kappa, tx, tu, k5x, k5u);
#define T6(k) __fma_rn(A65, k5##k, __fma_rn(A64, k4##k, __fma_rn(A63, k3##k, __fma_rn(A62, k2##k, A61 * k1##k))))
        tx = __fma_rn(h, T6(x), yx); tu = __fma_rn(h, T6(u), yu);
        deriv_team<P2>(F, T, kappa, tx, tu, k6x, k6u);
#define TB(k) __fma_rn(B6, k6##k, __fma_rn(B4, k4##k, __fma_rn(B3, k3##k, B1 * k1##k)))
#define TE(k) (h * __fma_rn(E6, k6##k, __fma_rn(E5, k5##k, __fma_rn(E4, k4##k, __fma_rn(E3, k3##k, E1 * k1##k)))))
        const double y5x = __fma_rn(h, TB(x), yx), y5u = __fma_rn(h, TB(u), yu);
        const double ex = TE(x), eu = TE(u);
#undef T3
#undef T4
#undef T5
#undef T6
#undef TB
#undef TE
        // squared norms ((e0^2 + e1^2) + e2^2) with fused products, as error_sums
        const double ex0 = T.get(ex, 0), ex1 = T.get(ex, 1), ex2 = T.get(ex, 2);
        const double eu0 = T.get(eu, 0), eu1 = T.get(eu, 1), eu2 = T.get(eu, 2);
        const double sx = __fma_rn(ex2, ex2, __fma_rn(ex1, ex1, ex0 * ex0));
        const double su = __fma_rn(eu2, eu2, __fma_rn(eu1, eu1, eu0 * eu0));
        if (!(error_accept(sx, su, h, tol, tol2) || le_pos(h, hmin))) {
            const float shrink = ctrl_factor(ctrl_log2r(sx, su, h, lg_tol), -0.25f, 0.1f, 1.0f);
            h = max_pos(h * widen_normal(shrink), hmin);
            rejected = 1;
            continue;
        }
        yx = y5x;
        yu = y5u;
        if (c == 0) h_out[(long long)m * n + i] = h;
        const float grow = (is_zero(h) || (is_zero(sx) && is_zero(su)))
                               ? 5.0f : ctrl_factor(ctrl_log2r(sx, su, h, lg_tol), -0.2f, 0.2f, 5.0f);
        double hnext = h * widen_normal(grow);
        if (!rejected && lt_pos(h, h_prop)) hnext = max_pos(hnext, h_prop);
        hprop = clampd(hnext, hmin, hmax);
        ++m;
        new_step = true;
    }
    xT[3 * i + c] = yx;
    uT[3 * i + c] = yu;
}

// Reverse sweep over the stage records in team form: lane c owns component c of the cotangents.
// Per stage: Bbar_c = kappa (bbar_{c+1} u_{c+2} - bbar_{c+2} u_{c+1}); kappa_bar += ((p0 + p1) + p2)
// with p_k = bbar_k (u x B)_k; Ybar_u_c = abar_c + kappa (B_{c+1} bbar_{c+2} - B_{c+2} bbar_{c+1});
// Ybar_x_c = (J[0][c] Bbar_0 + J[1][c] Bbar_1) + J[2][c] Bbar_2; lane c scatters w_k Bbar_c.
// One stage's record, the part lane c applies: u_{c+1}, u_{c+2}, B_{c+1}, B_{c+2}, column c of J,
// the corner weights and nodes. Loaded one stage ahead of its use (the sweep runs one warp per
// sub-partition, so registers do not limit occupancy here).
struct RecT {
    double u1, u2, B1, B2, J0, J1, J2, w[8];
    int32_t node[8];
};

__device__ __forceinline__ RecT load_rec_team(const double* __restrict__ rec_d, const int32_t* __restrict__ rec_n,
                                              long long n, long long i, int m, int st, const Team& T) {
    const int c = T.c, c1 = T.nx1(), c2 = T.nx2();
    const double* d = rec_d + ((long long)(m * 6 + st) * kRecD) * n + i;
    const int32_t* q = rec_n + ((long long)(m * 6 + st) * kRecN) * n + i;
    RecT r;
    r.u1 = __ldcs(d + c1 * n); r.u2 = __ldcs(d + c2 * n);
    r.B1 = __ldcs(d + (3 + c1) * n); r.B2 = __ldcs(d + (3 + c2) * n);
    r.J0 = __ldcs(d + (6 + c) * n); r.J1 = __ldcs(d + (9 + c) * n); r.J2 = __ldcs(d + (12 + c) * n);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        r.w[k] = __ldcs(d + (15 + k) * n);
        r.node[k] = __ldcs(q + k * n);
    }
    return r;
}

__device__ __forceinline__ void vjp_rec_team(const RecT& r, double kappa, const Team& T, double kbx, double kbu,
                                             double& Ybx, double& Ybu, double* __restrict__ grid_bar,
                                             double& kappa_bar) {
    const int c = T.c;
    const double bb1 = T.get(kbu, T.nx1()), bb2 = T.get(kbu, T.nx2());
    const double Bb = kappa * (bb1 * r.u2 - bb2 * r.u1);
    const double uxB = r.u1 * r.B2 - r.u2 * r.B1;
    const double p = kbu * uxB;
    const double p0 = T.get(p, 0), p1 = T.get(p, 1), p2 = T.get(p, 2);
    kappa_bar = kappa_bar + ((p0 + p1) + p2);
    Ybu = kbx + kappa * (r.B1 * bb2 - r.B2 * bb1);
    const double Bb0 = T.get(Bb, 0), Bb1 = T.get(Bb, 1), Bb2 = T.get(Bb, 2);
    Ybx = (r.J0 * Bb0 + r.J1 * Bb1) + r.J2 * Bb2;
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(grid_bar + (long long)r.node[k] * 3 + c, r.w[k] * Bb);
}

__global__ void k_adj_reverse_team(const double* __restrict__ kap, const double* __restrict__ h,
                                   const double* __restrict__ rec_d, const int32_t* __restrict__ rec_n,
                                   int m_hi, int m_lo, int first, const double* __restrict__ uT_bar,
                                   double* __restrict__ grid_bar, double* __restrict__ y0_bar,
                                   double* __restrict__ kappa_bar_out, long long n) {
    CRP_COUNT_RUN();
    long long i;
    bool active;
    const Team T = make_team(n, i, active);
    if (!active) return;
    const int c = T.c;
    const double kappa = kap[i];
    // steps m_hi - 1 down to m_lo; a later range continues from the cotangents the previous
    // one left in y0_bar and kappa_bar_out (the same values in the same order as one sweep)
    double lx = 0.0, lu = uT_bar[3 * i + c];
    double kappa_bar = 0.0;
    if (!first) {
        lx = y0_bar[(long long)c * n + i];
        lu = y0_bar[(long long)(3 + c) * n + i];
        kappa_bar = kappa_bar_out[i];
    }
    for (int m = m_hi - 1; m >= m_lo; --m) {
        if (m > m_lo) {   // the previous step's records into L2, a third of the lines per lane
            const double* d = rec_d + ((long long)(m - 1) * 6 * kRecD) * n + i;
            for (int k = c; k < 6 * kRecD; k += 3) asm volatile("prefetch.global.L2 [%0];" ::"l"(d + k * n));
            const int32_t* q = rec_n + ((long long)(m - 1) * 6 * kRecN) * n + i;
            for (int k = c; k < 6 * kRecN; k += 3) asm volatile("prefetch.global.L2 [%0];" ::"l"(q + k * n));
        }
        const double hn = h[(long long)m * n + i];
        // stage cotangents kb_s = (h b_s) lam, per component
        const double s0 = hn * cB5h[0], s1 = hn * cB5h[1], s2 = hn * cB5h[2], s3 = hn * cB5h[3],
                     s4 = hn * cB5h[4], s5 = hn * cB5h[5];
        double k0x = s0 * lx, k0u = s0 * lu, k1x = s1 * lx, k1u = s1 * lu, k2x = s2 * lx, k2u = s2 * lu;
        double k3x = s3 * lx, k3u = s3 * lu, k4x = s4 * lx, k4u = s4 * lu;
        const double k5x = s5 * lx, k5u = s5 * lu;
        double ybx = lx, ybu = lu, Yx, Yu;
        // each stage's record is loaded before the previous stage is applied
        RecT cur = load_rec_team(rec_d, rec_n, n, i, m, 5, T), nxt;
#define AX(kx, ku, a) do { const double ha = hn * (a); kx = kx + ha * Yx; ku = ku + ha * Yu; } while (0)
        nxt = load_rec_team(rec_d, rec_n, n, i, m, 4, T);
        vjp_rec_team(cur, kappa, T, k5x, k5u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
        AX(k0x, k0u, A61); AX(k1x, k1u, A62); AX(k2x, k2u, A63); AX(k3x, k3u, A64); AX(k4x, k4u, A65);
        cur = load_rec_team(rec_d, rec_n, n, i, m, 3, T);
        vjp_rec_team(nxt, kappa, T, k4x, k4u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
        AX(k0x, k0u, A51); AX(k1x, k1u, A52); AX(k2x, k2u, A53); AX(k3x, k3u, A54);
        nxt = load_rec_team(rec_d, rec_n, n, i, m, 2, T);
        vjp_rec_team(cur, kappa, T, k3x, k3u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
        AX(k0x, k0u, A41); AX(k1x, k1u, A42); AX(k2x, k2u, A43);
        cur = load_rec_team(rec_d, rec_n, n, i, m, 1, T);
        vjp_rec_team(nxt, kappa, T, k2x, k2u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
        AX(k0x, k0u, A31); AX(k1x, k1u, A32);
        nxt = load_rec_team(rec_d, rec_n, n, i, m, 0, T);
        vjp_rec_team(cur, kappa, T, k1x, k1u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
        AX(k0x, k0u, A21);
        vjp_rec_team(nxt, kappa, T, k0x, k0u, Yx, Yu, grid_bar, kappa_bar);
        ybx = ybx + Yx; ybu = ybu + Yu;
#undef AX
        lx = ybx;
        lu = ybu;
    }
    // every lane has read its state above before any lane of the team writes it here
    __syncwarp(T.mask);
    y0_bar[(long long)c * n + i] = lx;
    y0_bar[(long long)(3 + c) * n + i] = lu;
    if (c == 0) kappa_bar_out[i] = kappa_bar;
}

int team_blocks(long long n) { return (int)((n + kTeams - 1) / kTeams); }   // one warp per block

int blocks(long long n) { return (int)((n + 127) / 128); }

// Kernels with one thread per chain run one warp per block: 4096 chains are then 128 blocks
// spread over 128 SMs instead of 32 blocks of four warps on 32 SMs (each warp's sequential
// chain is bound by its SM's FP64 pipe and lookup latency, not by occupancy).
constexpr int kChainBlock = 32;
int chain_blocks(long long n) { return (int)((n + kChainBlock - 1) / kChainBlock); }

}  // namespace

int adj_init(const double* x0, const double* p0, const int32_t* Z, double* y0, double* kappa,
             double* E, long long n, void* stream) {
    k_adj_init<<<blocks(n), 128, 0, (cudaStream_t)stream>>>(x0, p0, Z, y0, kappa, E, n);
    return (int)cudaGetLastError();
}

int adj_record(const FieldDev& F, const double* y0, const double* kappa, double tol, double hmin,
               double hmax, int n_steps, int K, double* h, double* ck, double* xT, double* uT,
               long long n, void* stream) {
    auto k = F.pow2 ? k_adj_record_team<true> : k_adj_record_team<false>;
    k<<<team_blocks(n), 32, 0, (cudaStream_t)stream>>>(F, y0, kappa, tol, hmin, hmax, n_steps, K, h, ck,
                                                        xT, uT, n);
    return (int)cudaGetLastError();
}

int adj_replay(const FieldDev& F, const double* y0, const double* kappa, const double* h, int n_steps,
               double* xT, double* uT, unsigned long long* cell_hash, long long n, void* stream) {
    if (cell_hash)
        k_adj_replay<LAYOUT_F64X4, true><<<chain_blocks(n), kChainBlock, 0, (cudaStream_t)stream>>>(
            F, y0, kappa, h, n_steps, xT, uT, cell_hash, n);
    else
        k_adj_replay<LAYOUT_F64X4, false><<<chain_blocks(n), kChainBlock, 0, (cudaStream_t)stream>>>(
            F, y0, kappa, h, n_steps, xT, uT, nullptr, n);
    return (int)cudaGetLastError();
}

int adj_backward(const FieldDev& F, const double* kappa, const double* h, const double* ck,
                 double* seg, double* stages, int n_steps, int K, const double* uT_bar, double* grid_bar,
                 double* y0_bar, double* kappa_bar, long long n, void* stream, void* aux_stream,
                 void* const* events, int n_events) {
    if (stages) {
        // Stage records in chunks of checkpoint segments, last chunk first, on the auxiliary
        // stream; the reverse sweep takes each chunk once its event has fired. The records
        // kernel (FP64-throughput-bound, many threads) then runs beside the reverse sweep
        // (one warp per ten chains, latency-bound). Without an auxiliary stream: one chunk.
        // A chunk of C segments is n * C threads; C is the smallest that still gives every SM
        // about one 128-thread block (fewer blocks leave SMs idle for the chunk's whole run).
        const cudaStream_t st = (cudaStream_t)stream, aux = (cudaStream_t)aux_stream;
        const int S = (n_steps + K - 1) / K;
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
        const long long c_min = std::max(1ll, (long long)((0.8 * sms * 128.0 + (double)n - 1.0) / (double)n));
        int J = (aux && n_events >= 2) ? (int)std::min<long long>(n_events - 1, S / c_min) : 1;
        J = std::max(1, J);
        const int C = (S + J - 1) / J;
        J = (S + C - 1) / C;
        double* rec_d = stages;
        int32_t* rec_n = reinterpret_cast<int32_t*>(stages + (size_t)n_steps * 6 * kRecD * (size_t)n);
        const cudaStream_t rs = J > 1 ? aux : st;
        cudaError_t e = cudaSuccess;
        if (J > 1) {
            e = cudaEventRecord((cudaEvent_t)events[0], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, (cudaEvent_t)events[0], 0);
            if (e != cudaSuccess) return (int)e;
        }
        for (int j = 0; j < J; ++j) {
            const int hi = S - j * C, lo = std::max(0, hi - C);
            auto k = F.pow2 ? k_adj_records<LAYOUT_F64X4, true> : k_adj_records<LAYOUT_F64X4, false>;
            k<<<blocks(n * (hi - lo)), 128, 0, rs>>>(F, kappa, h, ck, rec_d, rec_n, n_steps, K, lo, hi - lo, n);
            e = cudaGetLastError();
            if (e == cudaSuccess && J > 1) e = cudaEventRecord((cudaEvent_t)events[1 + j], aux);
            if (e != cudaSuccess) return (int)e;
        }
        for (int j = 0; j < J; ++j) {
            const int hi = S - j * C, lo = std::max(0, hi - C);
            if (J > 1) {
                e = cudaStreamWaitEvent(st, (cudaEvent_t)events[1 + j], 0);
                if (e != cudaSuccess) return (int)e;
            }
            k_adj_reverse_team<<<team_blocks(n), 32, 0, st>>>(
                kappa, h, rec_d, rec_n, std::min(hi * K, n_steps), lo * K, j == 0 ? 1 : 0, uT_bar,
                grid_bar, y0_bar, kappa_bar, n);
            e = cudaGetLastError();
            if (e != cudaSuccess) return (int)e;
        }
        return 0;
    }
    k_adj_backward<LAYOUT_F64X4><<<chain_blocks(n), kChainBlock, 0, (cudaStream_t)stream>>>(
        F, kappa, h, ck, seg, n_steps, K, uT_bar, grid_bar, y0_bar, kappa_bar, n);
    return (int)cudaGetLastError();
}

int adj_p0bar(const double* y0, const double* kappa, const double* E, const double* y0_bar,
              const double* kappa_bar, double* p0_bar, double* x0_bar, long long n, void* stream) {
    k_adj_p0bar<<<blocks(n), 128, 0, (cudaStream_t)stream>>>(y0, kappa, E, y0_bar, kappa_bar, p0_bar,
                                                             x0_bar, n);
    return (int)cudaGetLastError();
}

}  // namespace crp

namespace crp {
unsigned long long kernel_runs_adjoint() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
