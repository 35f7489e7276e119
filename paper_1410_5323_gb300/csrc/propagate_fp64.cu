// propagate_fp64.cu -- FP64 form of the propagation hot path (arXiv:1410.5323, Sec. 3.1
// module sequence, Sec. 2 3D deflection, Sec. 3.2 regular grids).
//
// Persistent, warp-per-particle-batch kernel: each lane holds one particle in registers;
// one loop iteration is one Cash-Karp attempt, so lanes that reject and lanes that start
// a new step stay converged. Idle lanes are refilled from a global work counter with one
// warp-aggregated atomic (ballot + popc); finished particles are appended to the done
// list; secondaries reserve a slot atomically and go to the other work list, which a
// second launch of this kernel processes.
//
// Compiled with --fmad=false: every FP64 expression is evaluated as written, in the same
// order as the stated reading, so results are bit-identical to the FP64 oracle.
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "crp_internal.h"
#include "crp_math.cuh"
#include "crp_sched.cuh"

namespace crp {
namespace {

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

// One axis of the periodic lookup: r = (x - o)*(1/spacing), i0 = floor(r) mod n, weights.
__device__ __forceinline__ void axis(double x, double o, double inv, int n, int pow2,
                                     long long& i0, long long& i1, double& w0, double& w1) {
    const double r = (x - o) * inv;
    const double fl = floor(r);
    const double fr = r - fl;
    const long long i = (long long)fl;
    long long a;
    if (pow2) a = i & (long long)(n - 1);
    else { a = i % n; if (a < 0) a += n; }
    i0 = a;
    i1 = (a + 1 == n) ? 0 : a + 1;
    w0 = 1.0 - fr;
    w1 = fr;
}

// Trilinear periodic lookup; corners summed in the order 000, 001, ..., 111 (x, y, z),
// weight ((w_x * w_y) * w_z).
template <int L>
__device__ __forceinline__ V3 field_b(const FieldDev& F, double x, double y, double z) {
    long long ix0, ix1, iy0, iy1, iz0, iz1;
    double wx0, wx1, wy0, wy1, wz0, wz1;
    axis(x, F.ox, F.inv_spacing, F.nx, F.pow2, ix0, ix1, wx0, wx1);
    axis(y, F.oy, F.inv_spacing, F.ny, F.pow2, iy0, iy1, wy0, wy1);
    axis(z, F.oz, F.inv_spacing, F.nz, F.pow2, iz0, iz1, wz0, wz1);
    const long long ny = F.ny, nz = F.nz;
    const long long r00 = (ix0 * ny + iy0) * nz, r01 = (ix0 * ny + iy1) * nz;
    const long long r10 = (ix1 * ny + iy0) * nz, r11 = (ix1 * ny + iy1) * nz;
    const V3 g0 = corner<L>(F, r00 + iz0), g1 = corner<L>(F, r00 + iz1);
    const V3 g2 = corner<L>(F, r01 + iz0), g3 = corner<L>(F, r01 + iz1);
    const V3 g4 = corner<L>(F, r10 + iz0), g5 = corner<L>(F, r10 + iz1);
    const V3 g6 = corner<L>(F, r11 + iz0), g7 = corner<L>(F, r11 + iz1);
    const double w00 = wx0 * wy0, w01 = wx0 * wy1, w10 = wx1 * wy0, w11 = wx1 * wy1;
    double t;
    V3 B;
    t = w00 * wz0; B.x = t * g0.x;       B.y = t * g0.y;       B.z = t * g0.z;
    t = w00 * wz1; B.x = B.x + t * g1.x; B.y = B.y + t * g1.y; B.z = B.z + t * g1.z;
    t = w01 * wz0; B.x = B.x + t * g2.x; B.y = B.y + t * g2.y; B.z = B.z + t * g2.z;
    t = w01 * wz1; B.x = B.x + t * g3.x; B.y = B.y + t * g3.y; B.z = B.z + t * g3.z;
    t = w10 * wz0; B.x = B.x + t * g4.x; B.y = B.y + t * g4.y; B.z = B.z + t * g4.z;
    t = w10 * wz1; B.x = B.x + t * g5.x; B.y = B.y + t * g5.y; B.z = B.z + t * g5.z;
    t = w11 * wz0; B.x = B.x + t * g6.x; B.y = B.y + t * g6.y; B.z = B.z + t * g6.z;
    t = w11 * wz1; B.x = B.x + t * g7.x; B.y = B.y + t * g7.y; B.z = B.z + t * g7.z;
    return B;
}

struct Y6 { double x, y, z, ux, uy, uz; };

// f(y) = (u, kappa u x B(x))
template <int L>
__device__ __forceinline__ Y6 deriv(const FieldDev& F, double kappa, const Y6& y) {
    const V3 B = field_b<L>(F, y.x, y.y, y.z);
    Y6 k;
    k.x = y.ux; k.y = y.uy; k.z = y.uz;
    k.ux = kappa * (y.uy * B.z - y.uz * B.y);
    k.uy = kappa * (y.uz * B.x - y.ux * B.z);
    k.uz = kappa * (y.ux * B.y - y.uy * B.x);
    return k;
}

#define CRP_STAGE(dst, expr)                                                           \
    do {                                                                               \
        dst.x = y.x + h * (expr(x));  dst.y = y.y + h * (expr(y));                      \
        dst.z = y.z + h * (expr(z));  dst.ux = y.ux + h * (expr(ux));                   \
        dst.uy = y.uy + h * (expr(uy)); dst.uz = y.uz + h * (expr(uz));                 \
    } while (0)

// One Cash-Karp attempt of size h from y with k1 = f(y).
template <int L>
__device__ __forceinline__ void ck_attempt(const FieldDev& F, double kappa, const Y6& y,
                                           const Y6& k1, double h, Y6& y5, Y6& err) {
    Y6 t;
#define S2(c) (A21 * k1.c)
    CRP_STAGE(t, S2);
    const Y6 k2 = deriv<L>(F, kappa, t);
#define S3(c) (A31 * k1.c + A32 * k2.c)
    CRP_STAGE(t, S3);
    const Y6 k3 = deriv<L>(F, kappa, t);
#define S4(c) (A41 * k1.c + A42 * k2.c + A43 * k3.c)
    CRP_STAGE(t, S4);
    const Y6 k4 = deriv<L>(F, kappa, t);
#define S5(c) (A51 * k1.c + A52 * k2.c + A53 * k3.c + A54 * k4.c)
    CRP_STAGE(t, S5);
    const Y6 k5 = deriv<L>(F, kappa, t);
#define S6(c) (A61 * k1.c + A62 * k2.c + A63 * k3.c + A64 * k4.c + A65 * k5.c)
    CRP_STAGE(t, S6);
    const Y6 k6 = deriv<L>(F, kappa, t);
#define SB(c) (B1 * k1.c + B3 * k3.c + B4 * k4.c + B6 * k6.c)
    CRP_STAGE(y5, SB);
#define SE(c) (h * (E1 * k1.c + E3 * k3.c + E4 * k4.c + E5 * k5.c + E6 * k6.c))
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

__device__ __forceinline__ double error_ratio(const Y6& e, double h, double tol) {
    if (h == 0.0) return 0.0;
    const double ex = sqrt((e.x * e.x + e.y * e.y) + e.z * e.z) / h;
    const double eu = sqrt((e.ux * e.ux + e.uy * e.uy) + e.uz * e.uz);
    return fmax(ex, eu) / tol;
}

__device__ __forceinline__ double clampd(double v, double lo, double hi) {
    return fmin(fmax(v, lo), hi);
}

__device__ __forceinline__ bool finite6(const Y6& y) {
    return isfinite(y.x) && isfinite(y.y) && isfinite(y.z) && isfinite(y.ux) &&
           isfinite(y.uy) && isfinite(y.uz);
}

template <int L>
__global__ void __launch_bounds__(256) k_propagate_fp64(const PropArgs a) {
    const int lane = threadIdx.x & 31;
    Counters* C = a.ctr;
    const unsigned long long n_work = *(volatile unsigned long long*)&C->count[a.list];
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    const SimState& S = a.st;

    int slot = -1;
    Y6 y{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double E = 0, s = 0, hprop = 0, tau = 0;
    int A = 0, Z = 0, n_int = 0, gid = 0;
    unsigned long long uid = 0;
    long long n_steps = 0, n_att = 0, taken = 0;
    bool new_step = true;
    double h = 0, h_first = 0, h_propc = 0, h_int = 0, h_dist = 0, rl = 0, rpd = 0;
    int rejected = 0;
    long long att_step = 0;
    unsigned long long acc_tot = 0, att_tot = 0, sec_tot = 0;
    unsigned bits = 0;

    auto store = [&](int status) {
        S.x[slot] = y.x; S.y[slot] = y.y; S.z[slot] = y.z;
        S.ux[slot] = y.ux; S.uy[slot] = y.uy; S.uz[slot] = y.uz;
        S.E[slot] = E; S.s[slot] = s; S.hprop[slot] = hprop; S.tau[slot] = tau;
        S.A[slot] = A; S.Z[slot] = Z; S.n_int[slot] = n_int; S.status[slot] = status;
        S.n_steps[slot] = n_steps; S.n_att[slot] = n_att;
        if (status != CRP_STATUS_ACTIVE_) {
            const unsigned long long d = atomicAdd(&C->n_done, 1ull);
            a.done_list[d] = slot;
        }
        slot = -1;
    };

    for (;;) {
        // ---- refill idle lanes from the work list (one atomic per warp) ----
        const bool idle = slot < 0;
        const int popped = sched_pop(a, idle, lane, n_work, bits);
        if (popped >= 0) {
            slot = popped;
            y.x = __ldcg(&S.x[slot]); y.y = __ldcg(&S.y[slot]); y.z = __ldcg(&S.z[slot]);
            y.ux = __ldcg(&S.ux[slot]); y.uy = __ldcg(&S.uy[slot]); y.uz = __ldcg(&S.uz[slot]);
            E = __ldcg(&S.E[slot]); s = __ldcg(&S.s[slot]); hprop = __ldcg(&S.hprop[slot]); tau = __ldcg(&S.tau[slot]);
            A = __ldcg(&S.A[slot]); Z = __ldcg(&S.Z[slot]); n_int = __ldcg(&S.n_int[slot]); gid = __ldcg(&S.grid_id[slot]);
            uid = (unsigned long long)__ldcg(&S.uid[slot]);
            n_steps = __ldcg(&S.n_steps[slot]); n_att = __ldcg(&S.n_att[slot]);
            taken = 0;
            new_step = true;
        }
        if (__ballot_sync(kFull, slot >= 0) == 0) break;

        for (int it = 0; it < a.cadence; ++it) {
            if (slot < 0) continue;
            const FieldDev& F = a.fields[gid];
            // ---- bids (Sec. 3.1): lowest of propagation, loss, interaction, distance ----
            if (new_step) {
                if (a.has_tables) {
                    if (!table_rates(a.tab, A, Z, E, rl, rpd)) {
                        bits |= BIT_RANGE;
                        store(CRP_STATUS_RANGE_);
                        continue;
                    }
                } else {
                    rl = 0.0;
                    rpd = 0.0;
                }
                h_propc = clampd(hprop, a.hmin, a.hmax);
                const double h_loss = rl > 0.0 ? 0.1 / rl : INF;
                h_int = rpd > 0.0 ? fmax(tau, 0.0) / rpd : INF;
                h_dist = a.dmax - s;
                h = h_propc;
                if (h_loss < h) h = h_loss;
                if (h_int < h) h = h_int;
                if (h_dist < h) h = h_dist;
                h_first = h;
                rejected = 0;
                att_step = 0;
                new_step = false;
            }
            // ---- propagation: one Cash-Karp attempt ----
            const double kappa = (double)Z * kC / E;
            const Y6 k1 = deriv<L>(F, kappa, y);
            Y6 y5, err;
            ck_attempt<L>(F, kappa, y, k1, h, y5, err);
            att_step += 1;
            const double r = error_ratio(err, h, a.tol);
            if (!(r <= 1.0 || h <= a.hmin)) {
                const double shrink = clampd(0.95 * crp_exp(-0.25 * crp_log(r)), 0.1, 1.0);
                h = fmax(h * shrink, a.hmin);
                rejected = 1;
                continue;
            }
            if (!finite6(y5)) {
                n_att += att_step;
                att_tot += att_step;
                bits |= BIT_NAN;
                store(CRP_STATUS_NAN_);
                continue;
            }
            const bool fires = (rpd > 0.0 && h == h_int);
            unsigned long long q = 0;
            if (fires) {
                q = atomicAdd(&C->reserve, 1ull);
                if (q >= (unsigned long long)a.capacity) {
                    bits |= BIT_QUEUE_FULL;      // parked at the start of this step
                    store(CRP_STATUS_ACTIVE_);
                    continue;
                }
            }
            // ---- accept ----
            n_att += att_step;
            att_tot += att_step;
            y = y5;
            const bool done = (h == h_dist);
            s = done ? a.dmax : s + h;
            n_steps += 1;
            acc_tot += 1;
            taken += 1;
            const double grow = (r == 0.0) ? 5.0 : clampd(0.95 * crp_exp(-0.2 * crp_log(r)), 0.2, 5.0);
            double hnext = h * grow;
            if (!rejected && h_first < h_propc) hnext = fmax(hnext, h_propc);
            hprop = clampd(hnext, a.hmin, a.hmax);
            // ---- continuous loss at gamma0 ----
            if (rl > 0.0) E = E * crp_exp(-h * rl);
            // ---- photo-disintegration ----
            if (rpd > 0.0) {
                if (fires) {
                    const unsigned kk = (unsigned)(n_int + 1);
                    const int dz = nucleon_proton(a.seed, uid, kk, A, Z) ? 1 : 0;
                    const double E_sec = E / (double)A;
                    const double E_par = E * (double)(A - 1) / (double)A;
                    const long long qs = (long long)q;
                    const unsigned long long uid2 = (1ull << 32) + uid * 64ull + kk;
                    S.x[qs] = y.x; S.y[qs] = y.y; S.z[qs] = y.z;
                    S.ux[qs] = y.ux; S.uy[qs] = y.uy; S.uz[qs] = y.uz;
                    S.E[qs] = E_sec; S.s[qs] = s;
                    S.hprop[qs] = INF;
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
                    tau = -crp_log(uniform01(a.seed, uid, kk, 0u));
                } else {
                    tau = tau - h * rpd;
                }
            }
            new_step = true;
            // ---- observer ----
            if (done) {
                store(CRP_STATUS_DONE_);
            } else if (a.max_steps > 0 && taken >= a.max_steps) {
                store(CRP_STATUS_ACTIVE_);
            }
        }
    }

    // ---- statistics: warp reduction, one atomic per warp ----
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

}  // namespace

int launch_propagate_fp64(const PropArgs& a, int layout, int grid, int block, void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (layout) {
    case LAYOUT_F32X4: k_propagate_fp64<LAYOUT_F32X4><<<grid, block, 0, st>>>(a); break;
    case LAYOUT_F64X4: k_propagate_fp64<LAYOUT_F64X4><<<grid, block, 0, st>>>(a); break;
    case LAYOUT_BF16X4: k_propagate_fp64<LAYOUT_BF16X4><<<grid, block, 0, st>>>(a); break;
    case LAYOUT_F16X4: k_propagate_fp64<LAYOUT_F16X4><<<grid, block, 0, st>>>(a); break;
    default: return -1;
    }
    return (int)cudaGetLastError();
}

int propagate_fp64_occupancy(int layout, int block, int* blocks_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (layout) {
    case LAYOUT_F32X4:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate_fp64<LAYOUT_F32X4>, block, 0);
        break;
    case LAYOUT_F64X4:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate_fp64<LAYOUT_F64X4>, block, 0);
        break;
    case LAYOUT_BF16X4:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate_fp64<LAYOUT_BF16X4>, block, 0);
        break;
    case LAYOUT_F16X4:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate_fp64<LAYOUT_F16X4>, block, 0);
        break;
    default: break;
    }
    return (int)e;
}

}  // namespace crp
