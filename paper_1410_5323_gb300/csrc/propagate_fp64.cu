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
// order as the stated reading, so results are bit-identical to the FP64 oracle. Work that
// the reading leaves to the implementation stays off the FP64 pipe, which bounds this
// kernel: the lookup's floors and indices are integer operations on the bits of the grid
// coordinate, the step-size factor is FP32 (from the bits of the FP64 error sums), and the
// compares, minima and maxima of step sizes and error sums are integer operations on their
// bits (exact on the operand domains the helpers state).
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include "crp_internal.h"
#include "crp_math.cuh"
#include "crp_sched.cuh"
#include "crp_fp64.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

namespace crp {
namespace {

using namespace fp64;

// Register cap, a build-time tuning knob (-DCRP_FP64_MAXNREG=N). Unset by default: capping
// the 170-register kernel at 168 (12 instead of 8 warps per SM, no spills) measured 1.6 %
// slower, since the FP64 pipe, not latency, bounds it.
#ifdef CRP_FP64_MAXNREG
#define CRP_FP64_BOUNDS __maxnreg__(CRP_FP64_MAXNREG)
#else
#define CRP_FP64_BOUNDS __launch_bounds__(256)
#endif

template <int L, bool M, bool P2>
__global__ void CRP_FP64_BOUNDS k_propagate_fp64(const PropArgs a) {
    CRP_COUNT_RUN();
    const int lane = threadIdx.x & 31;
    Counters* C = a.ctr;
    const unsigned long long n_work = *(volatile unsigned long long*)&C->count[a.list];
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    const SimState& S = a.st;

    int slot = -1;
    Y6 y{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    Y6 k1{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // derivative at the step start
    double E = 0, s = 0, hprop = 0, tau = 0;
    int A = 0, Z = 0, n_int = 0, gid = 0;
    unsigned long long uid = 0;
    long long n_steps = 0, n_att = 0, taken = 0;
    bool new_step = true;
    double h = 0, h_first = 0, h_propc = 0, h_int = 0, h_dist = 0, rl = 0, rpd = 0, kappa = 0;
    const double tol2 = a.tol * a.tol;
    const float lg_tol = ctrl_log2(a.tol);
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
            if (gid < 0 || gid >= a.n_fields) { bits |= BIT_BOUNDS; slot = -1; }
        }
        if (__ballot_sync(kFull, slot >= 0) == 0) break;

        for (int it = 0; it < a.cadence; ++it) {
            if (slot < 0) continue;
            const FieldDev& F = a.fields[gid];
            // ---- bids (Sec. 3.1): lowest of propagation, loss, interaction, distance ----
            if (new_step) {
                float rl_f = 0.0f, rpd_f = 0.0f;
                if (a.has_tables && !table_rates_f32(a.tab, A, Z, E, rl_f, rpd_f)) {
                    bits |= BIT_RANGE;
                    store(CRP_STATUS_RANGE_);
                    continue;
                }
                // FP32 rates (normal or zero) widened; loss and interaction bids as FP32 quotients
                rl = rl_f > 0.0f ? widen_normal(rl_f) : 0.0;
                rpd = rpd_f > 0.0f ? widen_normal(rpd_f) : 0.0;
                h_propc = clampd(hprop, a.hmin, a.hmax);
                const double h_loss = rl_f > 0.0f ? widen_f32(__fdiv_rn(0.1f, rl_f)) : INF;
                h_int = rpd_f > 0.0f ? widen_f32(__fdiv_rn(__double2float_rn(fmax(tau, 0.0)), rpd_f)) : INF;
                h_dist = a.dmax - s;
                h = h_propc;
                if (lt_pos(h_loss, h)) h = h_loss;
                if (lt_pos(h_int, h)) h = h_int;
                if (dbits(h_dist) < dbits(h)) h = h_dist;   // h_dist is never -0
                h_first = h;
                kappa = (double)Z * kC / E;   // E and Z are constant within a step
                k1 = deriv<L, false, M, P2>(F, kappa, y);   // rejected attempts reuse k1
                rejected = 0;
                att_step = 0;
                new_step = false;
            }
            // ---- propagation: one Cash-Karp attempt ----
            Y6 y5, err;
            ck_attempt<L, false, M, P2>(F, kappa, y, k1, h, y5, err);
            att_step += 1;
            double sx, su;
            error_sums(err, sx, su);
            if (!(error_accept(sx, su, h, a.tol, tol2) || le_pos(h, a.hmin))) {
                const float shrink = ctrl_factor(ctrl_log2r(sx, su, h, lg_tol), -0.25f, 0.1f, 1.0f);
                h = max_pos(h * widen_normal(shrink), a.hmin);
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
            const bool fires = (dbits(rpd) > 0 && eq_num(h, h_int));
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
            if (a.boundary) {   // reflective box: fold the position, flip u (and u0) per odd axis
                if (reflect_axis(y.x, a.box_lo[0], a.box_hi[0], a.box_len[0], a.box_inv[0])) {
                    y.ux = -y.ux; S.u0x[slot] = -S.u0x[slot];
                }
                if (reflect_axis(y.y, a.box_lo[1], a.box_hi[1], a.box_len[1], a.box_inv[1])) {
                    y.uy = -y.uy; S.u0y[slot] = -S.u0y[slot];
                }
                if (reflect_axis(y.z, a.box_lo[2], a.box_hi[2], a.box_len[2], a.box_inv[2])) {
                    y.uz = -y.uz; S.u0z[slot] = -S.u0z[slot];
                }
            }
            const bool done = eq_num(h, h_dist);
            s = done ? a.dmax : s + h;
            n_steps += 1;
            acc_tot += 1;
            taken += 1;
            const float grow = (is_zero(h) || (is_zero(sx) && is_zero(su)))
                                   ? 5.0f : ctrl_factor(ctrl_log2r(sx, su, h, lg_tol), -0.2f, 0.2f, 5.0f);
            double hnext = h * widen_normal(grow);
            if (!rejected && lt_pos(h_first, h_propc)) hnext = max_pos(hnext, h_propc);
            hprop = clampd(hnext, a.hmin, a.hmax);
            // ---- continuous loss at gamma0 ----
            if (dbits(rl) > 0) E = E * crp_exp(-h * rl);
            // ---- photo-disintegration ----
            if (dbits(rpd) > 0) {
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

// Kernel for (layout, modulated, power-of-two vector grids): the FP64 form reads FP64 or
// FP32 vector grids; a modulated field is read through its FP64 copy only.
template <bool P2, typename Fn>
int with_fp64_kernel_p2(int layout, int mod, Fn&& fn) {
    if (mod) {
        if (layout != LAYOUT_F64X4) return (int)cudaErrorInvalidValue;
        return fn(k_propagate_fp64<LAYOUT_F64X4, true, P2>);
    }
    switch (layout) {
    case LAYOUT_F32X4: return fn(k_propagate_fp64<LAYOUT_F32X4, false, P2>);
    case LAYOUT_F64X4: return fn(k_propagate_fp64<LAYOUT_F64X4, false, P2>);
    case LAYOUT_BF16X4: return fn(k_propagate_fp64<LAYOUT_BF16X4, false, P2>);
    case LAYOUT_F16X4: return fn(k_propagate_fp64<LAYOUT_F16X4, false, P2>);
    default: return (int)cudaErrorInvalidValue;
    }
}

template <typename Fn>
int with_fp64_kernel(int layout, int mod, int p2, Fn&& fn) {
    return p2 ? with_fp64_kernel_p2<true>(layout, mod, fn) : with_fp64_kernel_p2<false>(layout, mod, fn);
}

int launch_propagate_fp64(const PropArgs& a, int layout, int mod, int p2, int grid, int block, void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return with_fp64_kernel(layout, mod, p2, [&](void (*k)(const PropArgs)) {
        k<<<grid, block, 0, st>>>(a);
        return (int)cudaGetLastError();
    });
}

int propagate_fp64_occupancy(int layout, int mod, int p2, int block, int* blocks_per_sm) {
    return with_fp64_kernel(layout, mod, p2, [&](void (*k)(const PropArgs)) {
        return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, 0);
    });
}

}  // namespace crp

namespace crp {
unsigned long long kernel_runs_fp64() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
