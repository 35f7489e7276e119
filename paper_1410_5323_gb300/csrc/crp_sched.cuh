// crp_sched.cuh -- work distribution for the persistent propagate kernels: a warp refills
// its idle lanes with one claim on a global counter (ballot + popc), first from the fixed
// work list of the launch, then from the list of secondaries pushed during this launch.
// A pushed entry is published with a release store after the particle's state is written;
// a reader claims positions below the push count with a CAS (never past it) and waits,
// bounded, for the entry to appear with an acquire load. A wait that runs out sets a
// status bit instead of hanging; nothing here traps.
#pragma once
#include <cuda/atomic>

#include "crp_internal.h"

namespace crp {

constexpr unsigned kSchedFull = 0xffffffffu;
constexpr int kPublishWaitLimit = 1 << 22;     // iterations of 64 ns sleeps (~0.3 s)
constexpr int kClaimRetryLimit = 64;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

// Waits, at most `limit` times 64 ns, for a non-negative value to be published at p (acquire
// loads). Returns false if it never appeared; the caller turns that into a status bit.
__device__ __forceinline__ bool bounded_acquire_wait(int32_t* p, int limit, int32_t& v) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> e(*p);
    for (int t = 0; t < limit; ++t) {
        v = e.load(cuda::memory_order_acquire);
        if (v >= 0) return true;
        __nanosleep(64);
    }
    return false;
}

// Append slot q to the list the launch pushes into (secondaries).
__device__ __forceinline__ void sched_push(const PropArgs& a, int32_t q) {
    const int L = 1 - a.list;
    const unsigned long long p = atomicAdd(&a.ctr->count[L], 1ull);
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> e(a.lists[L][p]);
    e.store(q, cuda::memory_order_release);
}

// Returns the slot this lane should load next, or -1. Lanes with idle == false get -1.
__device__ __forceinline__ int sched_pop(const PropArgs& a, bool idle, int lane,
                                        unsigned long long n_work, unsigned& bits) {
    const unsigned im = __ballot_sync(kSchedFull, idle);
    if (!im) return -1;
    Counters* C = a.ctr;
    const int L = a.list, P = 1 - a.list;
    unsigned long long base = 0;
    unsigned got = 0, from = 0;
    if (lane == 0) {
        const unsigned need = (unsigned)__popc(im);
        if (ld_volatile(&C->head[L]) < n_work) {
            base = atomicAdd(&C->head[L], (unsigned long long)need);
            if (base < n_work) got = (unsigned)min((unsigned long long)need, n_work - base);
        }
        if (got == 0 && a.pickup) {   // secondaries pushed so far in this launch
            from = 1;
            for (int t = 0; t < kClaimRetryLimit; ++t) {
                const unsigned long long h = ld_volatile(&C->head[P]);
                const unsigned long long c = ld_volatile(&C->count[P]);
                if (h >= c) break;
                const unsigned take = (unsigned)min((unsigned long long)need, c - h);
                if (atomicCAS(&C->head[P], h, h + take) == h) {
                    base = h;
                    got = take;
                    break;
                }
            }
        }
    }
    base = __shfl_sync(kSchedFull, base, 0);
    got = __shfl_sync(kSchedFull, got, 0);
    from = __shfl_sync(kSchedFull, from, 0);
    if (!idle) return -1;
    const unsigned rank = (unsigned)__popc(im & ((1u << lane) - 1u));
    if (rank >= got) return -1;
    const unsigned long long pos = base + rank;
    if (from == 0) {
        const int32_t v = a.lists[L][pos];
        if (v < 0 || v >= a.capacity) { bits |= BIT_BOUNDS; return -1; }
        return v;
    }
    int32_t v = -1;
    if (!bounded_acquire_wait(a.lists[P] + pos, kPublishWaitLimit, v)) {
        bits |= BIT_TIMEOUT;   // the entry never appeared: reported by crp_sync
        return -1;
    }
    if (v >= a.capacity) { bits |= BIT_BOUNDS; return -1; }
    return v;
}

}  // namespace crp
