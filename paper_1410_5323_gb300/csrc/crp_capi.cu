// crp_capi.cu -- the C ABI of libcrp.so (declared in include/crp.h): handles, argument
// checks, device memory, and the small bookkeeping kernels around the propagate kernels
// (grid layout, injection initialisation, work-list compaction, list swap, observer gather).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <atomic>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "crp.h"
#include "crp_internal.h"
#include "crp_math.cuh"
#include "crp_sched.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

static_assert(CRP_STATUS_ACTIVE == crp::CRP_STATUS_ACTIVE_, "status numbering");
static_assert(CRP_STATUS_DONE == crp::CRP_STATUS_DONE_, "status numbering");
static_assert(CRP_STATUS_NAN == crp::CRP_STATUS_NAN_, "status numbering");
static_assert(CRP_STATUS_RANGE == crp::CRP_STATUS_RANGE_, "status numbering");

using namespace crp;

namespace {

thread_local std::string g_detail;

int fail(int code, const std::string& msg) {
    g_detail = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    g_detail = std::string(where) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? CRP_ERR_OOM : CRP_ERR_CUDA;
}

// Device allocations of the library go through here. crp_debug_fail_allocations(n) makes
// the next n of them fail as out of memory (fault injection for tests).
std::atomic<int> g_fail_allocs{0};

template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// NVTX range over one library call (visible in Nsight timelines; no cost without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define CRP_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ---- K1: grid layout (one 4-wide vector per node) --------------------------------------
template <class In, class Out>
__global__ void k_layout(const In* __restrict__ in, Out* __restrict__ out, long long n_nodes);

template <>
__global__ void k_layout<float, float4>(const float* __restrict__ in, float4* __restrict__ out,
                                         long long n) {
    CRP_COUNT_RUN();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0.0f);
}
template <>
__global__ void k_layout<double, double2>(const double* __restrict__ in, double2* __restrict__ out,
                                           long long n) {
    CRP_COUNT_RUN();   // two double2 per node
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        out[2 * i] = make_double2(in[3 * i], in[3 * i + 1]);
        out[2 * i + 1] = make_double2(in[3 * i + 2], 0.0);
    }
}
template <>
__global__ void k_layout<unsigned short, ushort4>(const unsigned short* __restrict__ in,
                                                  ushort4* __restrict__ out, long long n) {
    CRP_COUNT_RUN();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = make_ushort4(in[3 * i], in[3 * i + 1], in[3 * i + 2], 0);
}

// Cell-major copy of a 4-wide FP32 or BF16 node layout for the precision form: cell
// (i, j, k) holds its corners (i+a, j+b, k+c) mod n in the order 4a + 2b + c; FP32 keeps 3
// floats per corner (96 B per cell), BF16 the 4 halves of the node (64 B per cell).
__global__ void k_cells(const void* __restrict__ in, int bf16, int nx, int ny, int nz, void* __restrict__ out) {
    CRP_COUNT_RUN();
    const long long n = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c / ((long long)ny * nz)), j = (int)((c / nz) % ny), k = (int)(c % nz);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int a = q >> 2, b = (q >> 1) & 1, d = q & 1;
            const long long node = ((long long)((i + a) % nx) * ny + (j + b) % ny) * nz + (k + d) % nz;
            if (bf16) {
                static_cast<ushort4*>(out)[c * 8 + q] = static_cast<const ushort4*>(in)[node];
            } else {
                const float4 v = static_cast<const float4*>(in)[node];
                float* o = static_cast<float*>(out) + c * 24 + 3 * q;
                o[0] = v.x; o[1] = v.y; o[2] = v.z;
            }
        }
    }
}

// Widen a 4-wide FP32 / BF16 / F16 node layout to FP64 pairs (x, y | z, 0), with the exact
// per-corner expression the FP64 kernel would otherwise evaluate on every lookup.
__global__ void k_widen(const void* __restrict__ in, int layout, double scale,
                        double2* __restrict__ out, long long n) {
    CRP_COUNT_RUN();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double x, y, z;
        if (layout == LAYOUT_F32X4) {
            const float4 v = reinterpret_cast<const float4*>(in)[i];
            x = (double)v.x; y = (double)v.y; z = (double)v.z;
        } else if (layout == LAYOUT_BF16X4) {
            const ushort4 v = reinterpret_cast<const ushort4*>(in)[i];
            x = (double)__uint_as_float((unsigned)v.x << 16) * scale;
            y = (double)__uint_as_float((unsigned)v.y << 16) * scale;
            z = (double)__uint_as_float((unsigned)v.z << 16) * scale;
        } else {
            const ushort4 v = reinterpret_cast<const ushort4*>(in)[i];
            x = (double)__half2float(__ushort_as_half(v.x)) * scale;
            y = (double)__half2float(__ushort_as_half(v.y)) * scale;
            z = (double)__half2float(__ushort_as_half(v.z)) * scale;
        }
        out[2 * i] = make_double2(x, y);
        out[2 * i + 1] = make_double2(z, 0.0);
    }
}

// ---- injection: per-particle bookkeeping (Philox tau draw), validation ----------------
__global__ void k_inject_init(SimState S, long long first, long long n, int uid_given,
                              int gid_given, unsigned long long uid_base, int n_fields,
                              int has_tables, int z_max, int n_max, unsigned long long seed,
                              int32_t* done_list, Counters* C) {
    CRP_COUNT_RUN();
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = first + k;
        if (!uid_given) S.uid[i] = (long long)(uid_base + (unsigned long long)k);
        if (!gid_given) S.grid_id[i] = 0;
        const int A = S.A[i], Z = S.Z[i];
        const long long uid = S.uid[i];
        bool ok = A >= 1 && Z >= -A && Z <= A && uid >= 0 && uid < (1ll << 32) &&
                  S.grid_id[i] >= 0 && S.grid_id[i] < n_fields;
        if (has_tables && (Z < 0 || Z > z_max || A - Z > n_max)) ok = false;
        S.s[i] = 0.0;
        S.hprop[i] = INF;
        S.tau[i] = -crp_log(uniform01(seed, (unsigned long long)uid, 0u, 0u));
        S.u0x[i] = S.ux[i];
        S.u0y[i] = S.uy[i];
        S.u0z[i] = S.uz[i];
        S.n_int[i] = 0;
        S.n_steps[i] = 0;
        S.n_att[i] = 0;
        S.status[i] = ok ? CRP_STATUS_ACTIVE_ : CRP_STATUS_RANGE_;
        if (!ok) {   // stopped at injection; reported by crp_sync as INVALID_ARG
            atomicOr(&C->status_bits, BIT_INVALID);
            const unsigned long long d = atomicAdd(&C->n_done, 1ull);
            done_list[d] = (int32_t)i;
        }
    }
}

__global__ void k_set_used(Counters* C, unsigned long long n_used, unsigned long long n_prim) {
    CRP_COUNT_RUN();
    C->n_used = n_used;
    C->reserve = n_used;
    C->n_primaries = n_prim;
}

// ---- propagate bookkeeping ----------------------------------------------------------------
__global__ void k_prepare(Counters* C) {
    CRP_COUNT_RUN();
    C->count[0] = 0;
    C->count[1] = 0;
    C->head[0] = 0;
    C->head[1] = 0;
    C->reserve = C->n_used;
}

// ---- work list in order of expected cost (longest first) ------------------------------
// Bucket by rigidity E/Z (step size grows with the gyro-radius, so low rigidity means many
// steps): 4 buckets per octave from 2^50 V, neutral particles last. A counting sort:
// histogram, exclusive scan, scatter with one atomic per (warp, bucket).
constexpr int kBuckets = 64;

__device__ __forceinline__ int cost_bucket(double E, int Z) {
    if (Z <= 0) return kBuckets - 1;
    const float b = 4.0f * (__log2f((float)E / (float)Z) - 50.0f);
    return b < 0.0f ? 0 : (b > (float)(kBuckets - 2) ? kBuckets - 2 : (int)b);
}

__device__ __forceinline__ int sort_key(double E, int Z, int gid, int grid_major) {
    return grid_major ? gid * kBuckets + cost_bucket(E, Z) : cost_bucket(E, Z);
}

__global__ void k_cost_hist(const int32_t* __restrict__ status, const double* __restrict__ E,
                            const int32_t* __restrict__ Zc, const int32_t* __restrict__ gid,
                            int grid_major, int n_buckets, int use_shared,
                            unsigned* __restrict__ hist, const Counters* C) {
    CRP_COUNT_RUN();
    extern __shared__ unsigned sh[];
    if (use_shared) {
        for (int b = threadIdx.x; b < n_buckets; b += blockDim.x) sh[b] = 0;
        __syncthreads();
    }
    const long long n = (long long)*(volatile const unsigned long long*)&C->n_used;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (status[i] != CRP_STATUS_ACTIVE_) continue;
        const int k = sort_key(E[i], Zc[i], gid[i], grid_major);
        if (use_shared) atomicAdd(&sh[k], 1u);
        else atomicAdd(&hist[k], 1u);
    }
    if (use_shared) {
        __syncthreads();
        for (int b = threadIdx.x; b < n_buckets; b += blockDim.x)
            if (sh[b]) atomicAdd(&hist[b], sh[b]);
    }
}

// Exclusive scan of the histogram (one block of 1024 threads), clearing it for next time.
__global__ void k_cost_scan(unsigned* hist, unsigned* offs, int n_buckets, Counters* C) {
    CRP_COUNT_RUN();
    __shared__ unsigned part[1024];
    const int t = threadIdx.x;
    const int chunk = (n_buckets + blockDim.x - 1) / blockDim.x;
    const int b0 = t * chunk, b1 = min(b0 + chunk, n_buckets);
    unsigned sum = 0;
    for (int b = b0; b < b1; ++b) sum += hist[b];
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        unsigned acc = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const unsigned v = part[k];
            part[k] = acc;
            acc += v;
        }
        C->count[0] = acc;
    }
    __syncthreads();
    unsigned acc = part[t];
    for (int b = b0; b < b1; ++b) {
        offs[b] = acc;
        acc += hist[b];
        hist[b] = 0;
    }
}

__global__ void k_cost_scatter(const int32_t* __restrict__ status, const double* __restrict__ E,
                               const int32_t* __restrict__ Zc, const int32_t* __restrict__ gid,
                               int grid_major, unsigned* __restrict__ offs,
                               int32_t* __restrict__ list, const Counters* C) {
    CRP_COUNT_RUN();
    const long long n = (long long)*(volatile const unsigned long long*)&C->n_used;
    const int lane = threadIdx.x & 31;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool act = i < n && status[i] == CRP_STATUS_ACTIVE_;
        const int b = act ? sort_key(E[i], Zc[i], gid[i], grid_major) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        if (act) {
            const int leader = __ffs(grp) - 1;
            unsigned p0 = 0;
            if (lane == leader) p0 = atomicAdd(&offs[b], (unsigned)__popc(grp));
            p0 = __shfl_sync(grp, p0, leader);
            list[p0 + __popc(grp & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
}

// Work list 0 <- slots [0, n_used) with status ACTIVE, in slot order within each warp
// (warp-aggregated append).
__global__ void k_build_worklist(const int32_t* __restrict__ status, int32_t* __restrict__ list,
                                 Counters* C) {
    CRP_COUNT_RUN();
    const unsigned long long n = *(volatile unsigned long long*)&C->n_used;
    const int lane = threadIdx.x & 31;
    for (long long base = blockIdx.x * (long long)blockDim.x; base < (long long)n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool act = i < (long long)n && status[i] == CRP_STATUS_ACTIVE_;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (!m) continue;
        unsigned long long p0 = 0;
        if (lane == 0) p0 = atomicAdd(&C->count[0], (unsigned long long)__popc(m));
        p0 = __shfl_sync(0xffffffffu, p0, 0);
        if (act) list[p0 + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    }
}

// After a propagate launch over list `from`: fix the slot count, reset the pop head and
// the list that the next launch pushes into.
__global__ void k_swap(Counters* C, long long capacity, int from) {
    CRP_COUNT_RUN();
    const unsigned long long r = C->reserve;
    C->n_used = r < (unsigned long long)capacity ? r : (unsigned long long)capacity;
    C->reserve = C->n_used;
    C->head[from] = 0;      // the other list keeps its head: the next launch continues it
    C->count[from] = 0;
    C->launches += 1;
}

// ---- observer gather ----------------------------------------------------------------------
struct ObsCols {
    int64_t* uid;
    int32_t *A, *Z, *n_int, *status;
    double *E, *x, *y, *z, *ux, *uy, *uz, *u0x, *u0y, *u0z, *s;
    int64_t *n_steps, *n_att;
};

__global__ void k_observe(SimState S, const int32_t* __restrict__ done, long long first,
                          long long n, ObsCols o) {
    CRP_COUNT_RUN();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int32_t i = done[first + k];
        if (o.uid) o.uid[k] = S.uid[i];
        if (o.A) o.A[k] = S.A[i];
        if (o.Z) o.Z[k] = S.Z[i];
        if (o.n_int) o.n_int[k] = S.n_int[i];
        if (o.status) o.status[k] = S.status[i];
        if (o.E) o.E[k] = S.E[i];
        if (o.x) o.x[k] = S.x[i];
        if (o.y) o.y[k] = S.y[i];
        if (o.z) o.z[k] = S.z[i];
        if (o.ux) o.ux[k] = S.ux[i];
        if (o.uy) o.uy[k] = S.uy[i];
        if (o.uz) o.uz[k] = S.uz[i];
        if (o.u0x) o.u0x[k] = S.u0x[i];
        if (o.u0y) o.u0y[k] = S.u0y[i];
        if (o.u0z) o.u0z[k] = S.u0z[i];
        if (o.s) o.s[k] = S.s[i];
        if (o.n_steps) o.n_steps[k] = S.n_steps[i];
        if (o.n_att) o.n_att[k] = S.n_att[i];
    }
}

int grid_for(long long n, int block, int max_blocks) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// Column table for SimState: element size and pointer slot.
struct ColInfo { int size; };
const ColInfo kCols[CRP_N_COLS] = {
    {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8}, {8},   // f64 0..12
    {4}, {4}, {4}, {4}, {4},                                           // i32 13..17
    {8}, {8}, {8}};                                                    // i64 18..20

void** col_ptr(SimState& S, int c) {
    void** f[CRP_N_COLS] = {(void**)&S.x, (void**)&S.y, (void**)&S.z, (void**)&S.ux,
                            (void**)&S.uy, (void**)&S.uz, (void**)&S.E, (void**)&S.s,
                            (void**)&S.hprop, (void**)&S.tau, (void**)&S.u0x, (void**)&S.u0y,
                            (void**)&S.u0z, (void**)&S.A, (void**)&S.Z, (void**)&S.n_int,
                            (void**)&S.status, (void**)&S.grid_id, (void**)&S.uid,
                            (void**)&S.n_steps, (void**)&S.n_att};
    return f[c];
}

}  // namespace

// ---- handles ------------------------------------------------------------------------------
namespace {
// One validated propagate call: kernel arguments and launch shape.
struct Plan {
    PropArgs a{};
    int grid = 0, block = 0, order = 0, mixed = 0, n_buckets = 0, layout = 0, mod = 0;
    int p2 = 0;   // every field's vector grid has power-of-two sizes
};

}  // namespace

struct crp_field {
    FieldDev dev;
    void* mem = nullptr;
    long long nodes = 0;
    void* mem64 = nullptr;   // FP64 copy for the FP64 form (built on first use)
    FieldDev dev64{};
    void* memc = nullptr;    // cell-major copy for the precision form (built on first use)
    void* modmem = nullptr;  // modulation grid, FP32 (crp_field_modulate)
};

struct crp_tables {
    TablesDev dev;
    void* mem = nullptr;
};

struct crp_sim {
    std::vector<FieldDev> host_fields;
    std::vector<crp_field*> handles;
    FieldDev* d_fields = nullptr;
    FieldDev* d_fields64 = nullptr;     // FP64 copies, for the FP64 form
    FieldDev* d_fields_cells = nullptr; // cell-major copies, for the precision form
    int layout = LAYOUT_F32X4;
    int mod = 0;                        // 1: every field carries a modulation grid
    int boundary = CRP_BOUNDARY_NONE;   // crp_sim_set_boundary
    double box_origin[3] = {0, 0, 0}, box_size[3] = {0, 0, 0};
    const crp_tables* tables = nullptr;
    unsigned long long seed = 0;
    long long capacity = 0;
    SimState st{};
    int32_t* lists[2] = {nullptr, nullptr};
    int32_t* done_list = nullptr;
    Counters* ctr = nullptr;
    unsigned* sort_scratch = nullptr;   // [hist n_buckets][offsets n_buckets]
    cudaStream_t last = nullptr;
    cudaGraph_t loop_graph = nullptr;   // crp_propagate_loop, cached for one plan
    cudaGraphExec_t loop_exec = nullptr;
    Plan loop_plan{};
    int loop_max_slices = 0;
    int sms = 0;
};

namespace {

void free_state(SimState& S) {
    for (int c = 0; c < CRP_N_COLS; ++c) {
        void** p = col_ptr(S, c);
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

int alloc_state(SimState& S, long long cap) {
    for (int c = 0; c < CRP_N_COLS; ++c) {
        void** p = col_ptr(S, c);
        cudaError_t e = dev_malloc(p, (size_t)cap * kCols[c].size);
        if (e != cudaSuccess) {
            free_state(S);
            return cuda_fail(e, "cudaMalloc(state)");
        }
    }
    return CRP_OK;
}

int sync_stream(crp_sim* s) {
    cudaError_t e = cudaStreamSynchronize(s->last);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return CRP_OK;
}

int read_counters(crp_sim* s, Counters* h) {
    int rc = sync_stream(s);
    if (rc) return rc;
    CRP_CUDA(cudaMemcpy(h, s->ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
    return CRP_OK;
}

}  // namespace

extern "C" {

const char* crp_version(void) { return "crp 1 sm_103a"; }

const char* crp_error_string(int32_t code) {
    switch (code) {
    case CRP_OK: return "ok";
    case CRP_ERR_INVALID_ARG: return "invalid argument";
    case CRP_ERR_OOM: return "device allocation failed";
    case CRP_ERR_CUDA: return "CUDA runtime error";
    case CRP_ERR_QUEUE_FULL: return "secondary queue full (resumable after crp_sim_reserve)";
    case CRP_ERR_TIMEOUT: return "wait limit reached";
    case CRP_ERR_NAN_STATE: return "non-finite particle state";
    case CRP_ERR_TABLE_RANGE: return "species outside the interaction tables";
    default: return "unknown error";
    }
}

const char* crp_last_error_detail(void) { return g_detail.c_str(); }

int crp_field_create(const void* grid, int32_t dtype, int32_t is_device, int32_t nx, int32_t ny,
                     int32_t nz, double spacing_m, const double origin_m[3], float scale,
                     crp_field** out) {
    NvtxRange nvtx_("crp_field_create");
    if (!out) return fail(CRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !origin_m) return fail(CRP_ERR_INVALID_ARG, "grid or origin is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(CRP_ERR_INVALID_ARG, "grid sizes must be >= 1");
    const long long nodes = (long long)nx * ny * nz;
    if (nodes >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "grid above 2^31 nodes");
    if (!(spacing_m > 0.0) || !std::isfinite(spacing_m))
        return fail(CRP_ERR_INVALID_ARG, "spacing must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin_m[a])) return fail(CRP_ERR_INVALID_ARG, "origin not finite");
    int elem, layout, out_elem;
    switch (dtype) {
    case CRP_DTYPE_F64: elem = 8; layout = LAYOUT_F64X4; out_elem = 32; break;
    case CRP_DTYPE_F32: elem = 4; layout = LAYOUT_F32X4; out_elem = 16; break;
    case CRP_DTYPE_BF16: elem = 2; layout = LAYOUT_BF16X4; out_elem = 8; break;
    case CRP_DTYPE_F16: elem = 2; layout = LAYOUT_F16X4; out_elem = 8; break;
    default: return fail(CRP_ERR_INVALID_ARG, "unknown dtype");
    }
    if ((dtype == CRP_DTYPE_BF16 || dtype == CRP_DTYPE_F16) && !(std::isfinite(scale) && scale != 0.0f))
        return fail(CRP_ERR_INVALID_ARG, "scale must be finite and non-zero");
    int ndev = 0;
    CRP_CUDA(cudaGetDeviceCount(&ndev));
    const size_t in_bytes = (size_t)nodes * 3 * elem;
    const void* src = grid;
    void* staging = nullptr;
    if (!is_device) {
        CRP_CUDA(dev_malloc(&staging, in_bytes));
        cudaError_t e = cudaMemcpy(staging, grid, in_bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(staging); return cuda_fail(e, "cudaMemcpy(grid)"); }
        src = staging;
    }
    crp_field* f = new crp_field();
    cudaError_t e = dev_malloc(&f->mem, (size_t)nodes * out_elem);
    if (e != cudaSuccess) {
        if (staging) cudaFree(staging);
        delete f;
        return cuda_fail(e, "cudaMalloc(field)");
    }
    const int block = 256;
    const int gridn = grid_for(nodes, block, 65535);
    switch (dtype) {
    case CRP_DTYPE_F64: k_layout<double, double2><<<gridn, block>>>((const double*)src, (double2*)f->mem, nodes); break;
    case CRP_DTYPE_F32: k_layout<float, float4><<<gridn, block>>>((const float*)src, (float4*)f->mem, nodes); break;
    default: k_layout<unsigned short, ushort4><<<gridn, block>>>((const unsigned short*)src, (ushort4*)f->mem, nodes); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (staging) cudaFree(staging);
    if (e != cudaSuccess) {
        cudaFree(f->mem);
        delete f;
        return cuda_fail(e, "field layout kernel");
    }
    f->nodes = nodes;
    FieldDev& d = f->dev;
    d.data = f->mem;
    d.layout = layout;
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.pow2 = (is_pow2(nx) && is_pow2(ny) && is_pow2(nz)) ? 1 : 0;
    d.inv_spacing = 1.0 / spacing_m;
    d.spacing = spacing_m;
    d.ox = origin_m[0]; d.oy = origin_m[1]; d.oz = origin_m[2];
    d.oix = d.ox * d.inv_spacing; d.oiy = d.oy * d.inv_spacing; d.oiz = d.oz * d.inv_spacing;
    d.scale = (dtype == CRP_DTYPE_BF16 || dtype == CRP_DTYPE_F16) ? (double)scale : 1.0;
    d.mod = nullptr;
    *out = f;
    return CRP_OK;
}

int crp_field_modulate(crp_field* field, const void* mod, int32_t dtype, int32_t is_device,
                       int32_t nx, int32_t ny, int32_t nz, double spacing_m, const double origin_m[3]) {
    NvtxRange nvtx_("crp_field_modulate");
    if (!field || !mod || !origin_m) return fail(CRP_ERR_INVALID_ARG, "field, modulation or origin is NULL");
    if (dtype != CRP_DTYPE_F32) return fail(CRP_ERR_INVALID_ARG, "modulation grids are FP32");
    if (nx < 1 || ny < 1 || nz < 1) return fail(CRP_ERR_INVALID_ARG, "grid sizes must be >= 1");
    const long long nodes = (long long)nx * ny * nz;
    if (nodes >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "grid above 2^31 nodes");
    if (!(spacing_m > 0.0) || !std::isfinite(spacing_m))
        return fail(CRP_ERR_INVALID_ARG, "spacing must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin_m[a])) return fail(CRP_ERR_INVALID_ARG, "origin not finite");
    if (field->modmem) return fail(CRP_ERR_INVALID_ARG, "field already modulated");
    void* m = nullptr;
    CRP_CUDA(dev_malloc(&m, (size_t)nodes * sizeof(float)));
    cudaError_t e = cudaMemcpy(m, mod, (size_t)nodes * sizeof(float),
                               is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(m); return cuda_fail(e, "cudaMemcpy(modulation)"); }
    field->modmem = m;
    FieldDev& d = field->dev;
    d.mod = (const float*)m;
    d.mnx = nx; d.mny = ny; d.mnz = nz;
    d.mpow2 = (is_pow2(nx) && is_pow2(ny) && is_pow2(nz)) ? 1 : 0;
    d.m_inv_spacing = 1.0 / spacing_m;
    d.m_spacing = spacing_m;
    d.mox = origin_m[0]; d.moy = origin_m[1]; d.moz = origin_m[2];
    d.moix = d.mox * d.m_inv_spacing; d.moiy = d.moy * d.m_inv_spacing; d.moiz = d.moz * d.m_inv_spacing;
    return CRP_OK;
}

int crp_field_destroy(crp_field* field) {
    if (!field) return fail(CRP_ERR_INVALID_ARG, "field is NULL");
    if (field->mem) cudaFree(field->mem);
    if (field->mem64) cudaFree(field->mem64);
    if (field->memc) cudaFree(field->memc);
    if (field->modmem) cudaFree(field->modmem);
    delete field;
    return CRP_OK;
}

int crp_tables_create(int32_t z_max, int32_t n_max, int32_t n_nodes, double x0, double inv_dx,
                      const double* log10_loss, const double* log10_pd, const uint8_t* has_loss,
                      const uint8_t* has_pd, crp_tables** out) {
    NvtxRange nvtx_("crp_tables_create");
    if (!out) return fail(CRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!log10_loss || !log10_pd || !has_loss || !has_pd)
        return fail(CRP_ERR_INVALID_ARG, "NULL table pointer");
    if (z_max < 0 || n_max < 0 || n_nodes < 2 || !(inv_dx > 0.0) || !std::isfinite(x0))
        return fail(CRP_ERR_INVALID_ARG, "bad table geometry");
    const long long n_sp = (long long)(z_max + 1) * (n_max + 1);
    for (long long sp = 0; sp < n_sp; ++sp) {
        for (int j = 0; j < n_nodes; ++j) {
            if (has_loss[sp] && !std::isfinite(log10_loss[sp * n_nodes + j]))
                return fail(CRP_ERR_INVALID_ARG, "non-finite value in a loss row");
            if (has_pd[sp] && !std::isfinite(log10_pd[sp * n_nodes + j]))
                return fail(CRP_ERR_INVALID_ARG, "non-finite value in a PD row");
        }
    }
    int ndev = 0;
    CRP_CUDA(cudaGetDeviceCount(&ndev));
    const size_t vb = (size_t)n_sp * n_nodes * sizeof(double);
    const size_t fb = (size_t)n_sp * n_nodes * sizeof(float);
    const size_t total = 2 * vb + 2 * fb + 2 * (size_t)n_sp + 64;
    std::vector<float> lf((size_t)n_sp * n_nodes), pf((size_t)n_sp * n_nodes);
    for (size_t i = 0; i < lf.size(); ++i) {
        lf[i] = (float)log10_loss[i];
        pf[i] = (float)log10_pd[i];
    }
    crp_tables* t = new crp_tables();
    cudaError_t e = dev_malloc(&t->mem, total);
    if (e != cudaSuccess) { delete t; return cuda_fail(e, "cudaMalloc(tables)"); }
    char* base = (char*)t->mem;
    e = cudaMemcpy(base, log10_loss, vb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + vb, log10_pd, vb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 2 * vb, lf.data(), fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 2 * vb + fb, pf.data(), fb, cudaMemcpyHostToDevice);
    char* flags = base + 2 * vb + 2 * fb;
    if (e == cudaSuccess) e = cudaMemcpy(flags, has_loss, n_sp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(flags + n_sp, has_pd, n_sp, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(t->mem); delete t; return cuda_fail(e, "cudaMemcpy(tables)"); }
    TablesDev& d = t->dev;
    d.loss = (const double*)base;
    d.pd = (const double*)(base + vb);
    d.loss_f = (const float*)(base + 2 * vb);
    d.pd_f = (const float*)(base + 2 * vb + fb);
    d.has_loss = (const uint8_t*)flags;
    d.has_pd = (const uint8_t*)(flags + n_sp);
    d.z_max = z_max; d.n_max = n_max; d.n_nodes = n_nodes;
    d.x0 = x0; d.inv_dx = inv_dx;
    d.x0_f = (float)x0; d.inv_dx_f = (float)inv_dx;
    *out = t;
    return CRP_OK;
}

int crp_tables_destroy(crp_tables* tables) {
    if (!tables) return fail(CRP_ERR_INVALID_ARG, "tables is NULL");
    if (tables->mem) cudaFree(tables->mem);
    delete tables;
    return CRP_OK;
}

int crp_sim_create(const crp_field* const* fields, int32_t n_fields, const crp_tables* tables,
                   uint64_t seed, int64_t capacity, crp_sim** out) {
    NvtxRange nvtx_("crp_sim_create");
    if (!out) return fail(CRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!fields || n_fields < 1) return fail(CRP_ERR_INVALID_ARG, "need at least one field");
    for (int i = 0; i < n_fields; ++i)
        if (!fields[i]) return fail(CRP_ERR_INVALID_ARG, "NULL field handle");
    if (capacity < 1 || capacity >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "capacity out of range");
    const int layout = fields[0]->dev.layout;
    const int mod = fields[0]->dev.mod ? 1 : 0;
    for (int i = 1; i < n_fields; ++i) {
        if (fields[i]->dev.layout != layout)
            return fail(CRP_ERR_INVALID_ARG, "all fields of a simulation need the same dtype");
        if ((fields[i]->dev.mod ? 1 : 0) != mod)
            return fail(CRP_ERR_INVALID_ARG, "all fields of a simulation are modulated, or none");
    }
    int ndev = 0;
    CRP_CUDA(cudaGetDeviceCount(&ndev));
    crp_sim* s = new crp_sim();
    s->layout = layout;
    s->mod = mod;
    s->tables = tables;
    s->seed = seed;
    s->capacity = capacity;
    s->sms = device_sms();
    for (int i = 0; i < n_fields; ++i) {
        s->host_fields.push_back(fields[i]->dev);
        s->handles.push_back(const_cast<crp_field*>(fields[i]));
    }
    int rc = alloc_state(s->st, capacity);
    cudaError_t e = cudaSuccess;
    if (rc == CRP_OK) e = dev_malloc(&s->d_fields, sizeof(FieldDev) * n_fields);
    if (rc == CRP_OK && e == cudaSuccess)
        e = cudaMemcpy(s->d_fields, s->host_fields.data(), sizeof(FieldDev) * n_fields, cudaMemcpyHostToDevice);
    if (rc == CRP_OK && e == cudaSuccess) e = dev_malloc(&s->lists[0], sizeof(int32_t) * capacity);
    if (rc == CRP_OK && e == cudaSuccess) e = dev_malloc(&s->lists[1], sizeof(int32_t) * capacity);
    if (rc == CRP_OK && e == cudaSuccess) e = dev_malloc(&s->done_list, sizeof(int32_t) * capacity);
    if (rc == CRP_OK && e == cudaSuccess) e = dev_malloc(&s->ctr, sizeof(Counters));
    if (rc == CRP_OK && e == cudaSuccess) e = cudaMemset(s->ctr, 0, sizeof(Counters));
    const size_t sort_bytes = 2 * (size_t)kBuckets * n_fields * sizeof(unsigned);
    if (rc == CRP_OK && e == cudaSuccess) e = dev_malloc(&s->sort_scratch, sort_bytes);
    if (rc == CRP_OK && e == cudaSuccess) e = cudaMemset(s->sort_scratch, 0, sort_bytes);
    if (rc != CRP_OK || e != cudaSuccess) {
        crp_sim_destroy(s);
        return rc != CRP_OK ? rc : cuda_fail(e, "crp_sim_create allocations");
    }
    *out = s;
    return CRP_OK;
}

int crp_sim_set_boundary(crp_sim* s, int32_t kind, const double origin_m[3], const double size_m[3]) {
    if (!s) return fail(CRP_ERR_INVALID_ARG, "sim is NULL");
    if (kind == CRP_BOUNDARY_NONE) {
        s->boundary = CRP_BOUNDARY_NONE;
        return CRP_OK;
    }
    if (kind != CRP_BOUNDARY_REFLECT) return fail(CRP_ERR_INVALID_ARG, "unknown boundary kind");
    if (!origin_m || !size_m) return fail(CRP_ERR_INVALID_ARG, "origin or size is NULL");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(origin_m[c]) || !(size_m[c] > 0.0) || !std::isfinite(size_m[c]))
            return fail(CRP_ERR_INVALID_ARG, "box origin must be finite, sizes finite and > 0");
    s->boundary = kind;
    for (int c = 0; c < 3; ++c) {
        s->box_origin[c] = origin_m[c];
        s->box_size[c] = size_m[c];
    }
    return CRP_OK;
}

int crp_sim_grid_layout(const crp_sim* s, int32_t* layout) {
    if (!s || !layout) return fail(CRP_ERR_INVALID_ARG, "sim or layout is NULL");
    *layout = s->d_fields_cells ? CRP_GRID_CELLS : CRP_GRID_NODES;
    return CRP_OK;
}

int crp_sim_destroy(crp_sim* s) {
    if (!s) return fail(CRP_ERR_INVALID_ARG, "sim is NULL");
    if (s->last) cudaStreamSynchronize(s->last);
    free_state(s->st);
    if (s->d_fields) cudaFree(s->d_fields);
    if (s->d_fields64) cudaFree(s->d_fields64);
    if (s->d_fields_cells) cudaFree(s->d_fields_cells);
    if (s->lists[0]) cudaFree(s->lists[0]);
    if (s->lists[1]) cudaFree(s->lists[1]);
    if (s->done_list) cudaFree(s->done_list);
    if (s->ctr) cudaFree(s->ctr);
    if (s->sort_scratch) cudaFree(s->sort_scratch);
    if (s->loop_exec) cudaGraphExecDestroy(s->loop_exec);
    if (s->loop_graph) cudaGraphDestroy(s->loop_graph);
    delete s;
    return CRP_OK;
}

int crp_sim_reset(crp_sim* s) {
    NvtxRange nvtx_("crp_sim_reset");
    if (!s) return fail(CRP_ERR_INVALID_ARG, "sim is NULL");
    int rc = sync_stream(s);
    if (rc) return rc;
    CRP_CUDA(cudaMemset(s->ctr, 0, sizeof(Counters)));
    CRP_CUDA(cudaDeviceSynchronize());
    return CRP_OK;
}

int crp_sim_reserve(crp_sim* s, int64_t capacity) {
    NvtxRange nvtx_("crp_sim_reserve");
    if (!s) return fail(CRP_ERR_INVALID_ARG, "sim is NULL");
    if (capacity >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "capacity out of range");
    if (capacity <= s->capacity) return CRP_OK;
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    SimState ns{};
    rc = alloc_state(ns, capacity);
    if (rc) return rc;
    int32_t *l0 = nullptr, *l1 = nullptr, *dl = nullptr;
    cudaError_t e = dev_malloc(&l0, sizeof(int32_t) * capacity);
    if (e == cudaSuccess) e = dev_malloc(&l1, sizeof(int32_t) * capacity);
    if (e == cudaSuccess) e = dev_malloc(&dl, sizeof(int32_t) * capacity);
    for (int c = 0; c < CRP_N_COLS && e == cudaSuccess; ++c)
        e = cudaMemcpy(*col_ptr(ns, c), *col_ptr(s->st, c), (size_t)h.n_used * kCols[c].size,
                       cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dl, s->done_list, sizeof(int32_t) * h.n_done, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        free_state(ns);
        if (l0) cudaFree(l0);
        if (l1) cudaFree(l1);
        if (dl) cudaFree(dl);
        return cuda_fail(e, "crp_sim_reserve");
    }
    free_state(s->st);
    cudaFree(s->lists[0]);
    cudaFree(s->lists[1]);
    cudaFree(s->done_list);
    s->st = ns;
    s->lists[0] = l0;
    s->lists[1] = l1;
    s->done_list = dl;
    s->capacity = capacity;
    return CRP_OK;
}

int crp_source_inject(crp_sim* s, const crp_particles* p, int64_t n, void* stream) {
    NvtxRange nvtx_("crp_source_inject");
    if (!s || !p) return fail(CRP_ERR_INVALID_ARG, "sim or particles is NULL");
    if (n < 0) return fail(CRP_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return CRP_OK;
    if (!p->x || !p->y || !p->z || !p->ux || !p->uy || !p->uz || !p->E || !p->A || !p->Z)
        return fail(CRP_ERR_INVALID_ARG, "NULL particle column");
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    if ((long long)h.n_used + n > s->capacity)
        return fail(CRP_ERR_INVALID_ARG, "injection exceeds the simulation capacity");
    const int n_fields = (int)s->host_fields.size();
    const TablesDev* tab = s->tables ? &s->tables->dev : nullptr;
    // host columns: validate before touching the device (a branch-free pass over all
    // particles, then, only if it found an invalid one, the pass that names the error)
    bool bad = false;
    if (!p->is_device) {
        const int zmax = tab ? tab->z_max : 0, nmax = tab ? tab->n_max : 0;
        const bool t = tab != nullptr;
        auto scan = [&](long long lo, long long hi) {
            unsigned acc = 0;
            for (long long i = lo; i < hi; ++i) {
                const int A = p->A[i], Z = p->Z[i];
                acc |= (unsigned)(A < 1) | (unsigned)(Z < -A) | (unsigned)(Z > A) |
                       (unsigned)(t & ((Z < 0) | (Z > zmax) | (A - Z > nmax)));
            }
            if (p->uid)
                for (long long i = lo; i < hi; ++i)
                    acc |= (unsigned)((unsigned long long)p->uid[i] >= (1ull << 32));
            if (p->grid_id)
                for (long long i = lo; i < hi; ++i)
                    acc |= (unsigned)((unsigned)p->grid_id[i] >= (unsigned)n_fields);
            return acc;
        };
        // one host core reads these columns at a fraction of the memory bandwidth: large
        // batches are scanned by several threads (chunks of at least 2^20 particles)
        const long long kChunk = 1ll << 20;
        long long nt = std::min<long long>(n / kChunk, std::max(1u, std::thread::hardware_concurrency()));
        nt = std::max(1ll, std::min(nt, 32ll));
        unsigned acc = 0;
        if (nt == 1) {
            acc = scan(0, n);
        } else {
            std::vector<unsigned> part((size_t)nt, 0u);
            std::vector<std::thread> th;
            bool spawned = true;
            try {
                th.reserve((size_t)nt);
                for (long long k = 0; k < nt; ++k)
                    th.emplace_back([&, k] { part[(size_t)k] = scan(n * k / nt, n * (k + 1) / nt); });
            } catch (...) {   // no threads to be had: the whole scan on this one
                spawned = false;
            }
            for (auto& x : th) x.join();
            if (spawned) {
                for (unsigned v : part) acc |= v;
            } else {
                acc = scan(0, n);
            }
        }
        if (!p->uid) acc |= (unsigned)(h.n_primaries + (unsigned long long)n > (1ull << 32));
        bad = acc != 0;
    }
    if (bad) {
        for (long long i = 0; i < n; ++i) {
            const int A = p->A[i], Z = p->Z[i];
            if (A < 1 || Z < -A || Z > A) return fail(CRP_ERR_INVALID_ARG, "particle with invalid A/Z");
            if (tab && (Z < 0 || Z > tab->z_max || A - Z > tab->n_max))
                return fail(CRP_ERR_INVALID_ARG, "species outside the interaction tables (antinuclei take none)");
            const long long uid = p->uid ? p->uid[i] : (long long)(h.n_primaries + i);
            if (uid < 0 || uid >= (1ll << 32)) return fail(CRP_ERR_INVALID_ARG, "uid outside [0, 2^32)");
            if (p->grid_id && (p->grid_id[i] < 0 || p->grid_id[i] >= n_fields))
                return fail(CRP_ERR_INVALID_ARG, "grid_id out of range");
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = p->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const long long f = (long long)h.n_used;
    struct { const void* src; int col; } cp[] = {
        {p->x, CRP_COL_X}, {p->y, CRP_COL_Y}, {p->z, CRP_COL_Z}, {p->ux, CRP_COL_UX},
        {p->uy, CRP_COL_UY}, {p->uz, CRP_COL_UZ}, {p->E, CRP_COL_E}, {p->A, CRP_COL_A},
        {p->Z, CRP_COL_Z_CHARGE}, {p->uid, CRP_COL_UID}, {p->grid_id, CRP_COL_GRID_ID}};
    for (auto& c : cp) {
        if (!c.src) continue;
        char* dst = (char*)*col_ptr(s->st, c.col) + f * kCols[c.col].size;
        CRP_CUDA(cudaMemcpyAsync(dst, c.src, (size_t)n * kCols[c.col].size, kind, st));
    }
    const int block = 256;
    k_inject_init<<<grid_for(n, block, 4096), block, 0, st>>>(
        s->st, f, n, p->uid ? 1 : 0, p->grid_id ? 1 : 0, h.n_primaries, n_fields, tab ? 1 : 0,
        tab ? tab->z_max : 0, tab ? tab->n_max : 0, s->seed, s->done_list, s->ctr);
    CRP_CUDA(cudaGetLastError());
    k_set_used<<<1, 1, 0, st>>>(s->ctr, h.n_used + n, h.n_primaries + (p->uid ? 0 : n));
    CRP_CUDA(cudaGetLastError());
    s->last = st;
    return CRP_OK;
}

int crp_source_sample(crp_sim* s, const crp_spectrum* sp, const double* x, const double* y,
                      const double* z, const int32_t* grid_id, int32_t is_device, int64_t n,
                      void* stream) {
    NvtxRange nvtx_("crp_source_sample");
    if (!s || !sp) return fail(CRP_ERR_INVALID_ARG, "sim or spectrum is NULL");
    if (n < 0) return fail(CRP_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return CRP_OK;
    if (!x || !y || !z) return fail(CRP_ERR_INVALID_ARG, "NULL position column");
    if (sp->n_species < 1 || sp->n_species > CRP_MAX_SPECIES)
        return fail(CRP_ERR_INVALID_ARG, "n_species outside [1, CRP_MAX_SPECIES]");
    if (!(sp->e_min_ev > 0.0) || !(sp->e_max_ev > sp->e_min_ev) || !std::isfinite(sp->e_max_ev) ||
        !(sp->rcut_v > 0.0) || !std::isfinite(sp->alpha))
        return fail(CRP_ERR_INVALID_ARG, "need 0 < e_min < e_max, rcut > 0, finite alpha");
    double total = 0.0;
    for (int i = 0; i < sp->n_species; ++i) {
        if (sp->A[i] < 1 || sp->Z[i] < 1 || sp->Z[i] > sp->A[i] || !(sp->x[i] >= 0.0) || !std::isfinite(sp->x[i]))
            return fail(CRP_ERR_INVALID_ARG, "species need 1 <= Z <= A and abundance >= 0");
        total += sp->x[i];
    }
    if (!(total > 0.0)) return fail(CRP_ERR_INVALID_ARG, "abundances are all zero");
    const TablesDev* tab = s->tables ? &s->tables->dev : nullptr;
    for (int i = 0; i < sp->n_species; ++i)
        if (tab && (sp->Z[i] > tab->z_max || sp->A[i] - sp->Z[i] > tab->n_max))
            return fail(CRP_ERR_INVALID_ARG, "species outside the interaction tables");
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    if ((long long)h.n_used + n > s->capacity)
        return fail(CRP_ERR_INVALID_ARG, "injection exceeds the simulation capacity");
    if (h.n_primaries + (unsigned long long)n > (1ull << 32))
        return fail(CRP_ERR_INVALID_ARG, "uids would exceed 2^32");
    const int n_fields = (int)s->host_fields.size();
    if (!is_device && grid_id)
        for (long long i = 0; i < n; ++i)
            if (grid_id[i] < 0 || grid_id[i] >= n_fields) return fail(CRP_ERR_INVALID_ARG, "grid_id out of range");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const long long f = (long long)h.n_used;
    struct { const void* src; int col; } cp[] = {
        {x, CRP_COL_X}, {y, CRP_COL_Y}, {z, CRP_COL_Z}, {grid_id, CRP_COL_GRID_ID}};
    for (auto& c : cp) {
        if (!c.src) continue;
        char* dst = (char*)*col_ptr(s->st, c.col) + f * kCols[c.col].size;
        CRP_CUDA(cudaMemcpyAsync(dst, c.src, (size_t)n * kCols[c.col].size, kind, st));
    }
    int e = launch_source_sample(s->st, f, n, h.n_primaries, *sp, s->seed, grid_for(n, 128, 8192), st);
    if (e) return cuda_fail((cudaError_t)e, "source sampling kernel");
    const int block = 256;
    k_inject_init<<<grid_for(n, block, 4096), block, 0, st>>>(
        s->st, f, n, 1, grid_id ? 1 : 0, h.n_primaries, n_fields, tab ? 1 : 0,
        tab ? tab->z_max : 0, tab ? tab->n_max : 0, s->seed, s->done_list, s->ctr);
    CRP_CUDA(cudaGetLastError());
    k_set_used<<<1, 1, 0, st>>>(s->ctr, h.n_used + n, h.n_primaries + n);
    CRP_CUDA(cudaGetLastError());
    s->last = st;
    return CRP_OK;
}

int crp_healpix_ring(int32_t nside, const double* u, int64_t n, int64_t* pix, void* stream) {
    NvtxRange nvtx_("crp_healpix_ring");
    if (nside < 1 || nside > 8192) return fail(CRP_ERR_INVALID_ARG, "nside outside [1, 8192]");
    if (n < 0) return fail(CRP_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return CRP_OK;
    if (!u || !pix) return fail(CRP_ERR_INVALID_ARG, "NULL direction or pixel buffer");
    int e = launch_healpix(nside, u, n, (long long*)pix, grid_for(n, 256, 8192), stream);
    if (e) return cuda_fail((cudaError_t)e, "healpix kernel");
    return CRP_OK;
}

int crp_arrival_map(crp_sim* s, int32_t nside, double e_min_ev, uint64_t* map, void* stream) {
    NvtxRange nvtx_("crp_arrival_map");
    if (!s || !map) return fail(CRP_ERR_INVALID_ARG, "sim or map is NULL");
    if (nside < 1 || nside > 8192) return fail(CRP_ERR_INVALID_ARG, "nside outside [1, 8192]");
    if (e_min_ev != e_min_ev) return fail(CRP_ERR_INVALID_ARG, "e_min is NaN");
    const int grid = (s->sms > 0 ? s->sms : 1) * 4;
    int e = launch_arrival_map(s->st, s->ctr, nside, e_min_ev, (unsigned long long*)map, grid, stream);
    if (e) return cuda_fail((cudaError_t)e, "arrival map kernel");
    s->last = reinterpret_cast<cudaStream_t>(stream);
    return CRP_OK;
}

}  // extern "C"

extern "C" {

int crp_kernel_runs(uint64_t* count) {
    if (!count) return fail(CRP_ERR_INVALID_ARG, "count is NULL");
    CRP_CUDA(cudaDeviceSynchronize());
    *count = kernel_runs_capi() + kernel_runs_fp64() + kernel_runs_mixed() + kernel_runs_adjoint() +
             kernel_runs_sources() + kernel_runs_lens();
    return CRP_OK;
}

int crp_debug_fail_allocations(int32_t n) {
    if (n < 0) return fail(CRP_ERR_INVALID_ARG, "n < 0");
    g_fail_allocs.store(n);
    return CRP_OK;
}

}  // extern "C"

namespace {

// Waits on a device flag with the scheduler's bounded wait; *status = 1 if the wait ran out.
__global__ void k_selftest_wait(int32_t* flag, int limit, int* status) {
    CRP_COUNT_RUN();
    int32_t v = -1;
    *status = bounded_acquire_wait(flag, limit, v) ? 0 : 1;
}

}  // namespace

extern "C" int crp_selftest_wait(int32_t limit, int32_t preset, void* stream) {
    NvtxRange nvtx_("crp_selftest_wait");
    if (limit < 1) return fail(CRP_ERR_INVALID_ARG, "limit must be >= 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t* flag = nullptr;
    CRP_CUDA(dev_malloc(&flag, 2 * sizeof(int32_t)));
    int* status = reinterpret_cast<int*>(flag + 1);
    const int32_t init[2] = {preset, -1};
    cudaError_t e = cudaMemcpyAsync(flag, init, sizeof init, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 1, 0, st>>>(flag, limit, status);
        e = cudaGetLastError();
    }
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "crp_selftest_wait");
    if (h == 1) return fail(CRP_ERR_TIMEOUT, "self-test wait limit reached (expected when the flag is never set)");
    return CRP_OK;
}

struct crp_lens {
    int n_pix = 0, n_mat = 0, group = 32;
    long long nnz = 0;
    void* mem = nullptr;                 // [row_ptr | col | val | edges]
    const long long* rp = nullptr;      // row starts (multiples of 4) of the merged rows
    const int* rl = nullptr;            // row lengths
    const int* col = nullptr;
    const float* val = nullptr;
    const double* edges = nullptr;
};

extern "C" {

int crp_lens_create(int32_t n_pix, int32_t n_mat, const int64_t* row_ptr, const int32_t* col,
                    const float* val, const double* edges, crp_lens** out) {
    NvtxRange nvtx_("crp_lens_create");
    if (!out) return fail(CRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_pix < 1 || n_mat < 1) return fail(CRP_ERR_INVALID_ARG, "n_pix and n_mat must be >= 1");
    if (!row_ptr) return fail(CRP_ERR_INVALID_ARG, "row_ptr is NULL");
    const long long rows = (long long)n_mat * (n_pix + 1);
    if (row_ptr[0] != 0) return fail(CRP_ERR_INVALID_ARG, "row_ptr must start at 0");
    for (long long m = 0; m < n_mat; ++m) {
        const int64_t* r = row_ptr + m * (n_pix + 1);
        if (m > 0 && r[0] != row_ptr[m * (n_pix + 1) - 1])
            return fail(CRP_ERR_INVALID_ARG, "each matrix must start where the previous one ends");
        for (long long q = 0; q < n_pix; ++q)
            if (r[q + 1] < r[q]) return fail(CRP_ERR_INVALID_ARG, "row_ptr decreases");
    }
    const long long nnz = row_ptr[rows - 1];
    if (nnz > 0 && (!col || !val)) return fail(CRP_ERR_INVALID_ARG, "col or val is NULL");
    if ((long long)n_mat * n_pix >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "n_mat * n_pix above 2^31");
    for (long long k = 0; k < nnz; ++k)
        if (col[k] < 0 || col[k] >= n_pix) return fail(CRP_ERR_INVALID_ARG, "column out of range");
    if (edges)
        for (int m = 0; m <= n_mat; ++m)
            if (!(edges[m] > 0.0) || !std::isfinite(edges[m]) || (m > 0 && !(edges[m] > edges[m - 1])))
                return fail(CRP_ERR_INVALID_ARG, "edges must be positive, finite, strictly increasing");
    // row-merged form: row p = the row-p segments of matrices 0 .. n_mat-1 in order, columns
    // offset by m n_pix into the stacked maps; each row starts on a 4-entry boundary (16-byte
    // vector loads), rl holds its length, and the padding (column 0, value 0) is never summed
    std::vector<long long> mrs((size_t)n_pix + 1, 0);
    std::vector<int> mrl((size_t)n_pix, 0);
    for (long long q = 0; q < n_pix; ++q) {
        long long len = 0;
        for (long long m = 0; m < n_mat; ++m) {
            const int64_t* r = row_ptr + m * (n_pix + 1);
            len += r[q + 1] - r[q];
        }
        if (len >= (1ll << 31)) return fail(CRP_ERR_INVALID_ARG, "a merged row above 2^31 entries");
        mrl[q] = (int)len;
        mrs[q + 1] = mrs[q] + (len + 3) / 4 * 4;
    }
    const long long padded = mrs[n_pix];
    std::vector<int> mcol((size_t)padded, 0);
    std::vector<float> mval((size_t)padded, 0.0f);
    for (long long q = 0; q < n_pix; ++q) {
        long long o = mrs[q];
        for (long long m = 0; m < n_mat; ++m) {
            const int64_t* r = row_ptr + m * (n_pix + 1);
            for (long long k = r[q]; k < r[q + 1]; ++k, ++o) {
                mcol[o] = (int)(m * n_pix + col[k]);
                mval[o] = val[k];
            }
        }
    }
    const size_t b_rp = (size_t)(n_pix + 1) * 8, b_rl = (size_t)n_pix * 4;
    const size_t b_col = (size_t)padded * 4, b_val = (size_t)padded * 4;
    const size_t b_e = edges ? (size_t)(n_mat + 1) * 8 : 0;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    crp_lens* L = new crp_lens();
    cudaError_t e = dev_malloc(&L->mem, up(b_rp) + up(b_rl) + up(b_col) + up(b_val) + up(b_e) + 256);
    if (e != cudaSuccess) { delete L; return cuda_fail(e, "cudaMalloc(lens)"); }
    char* base = (char*)L->mem;
    size_t off = 0;
    L->rp = (const long long*)(base + off); off += up(b_rp);
    L->rl = (const int*)(base + off); off += up(b_rl);
    L->col = (const int*)(base + off); off += up(b_col);
    L->val = (const float*)(base + off); off += up(b_val);
    L->edges = edges ? (const double*)(base + off) : nullptr;
    struct { const void* src; const void* dst; size_t n; } cp[] = {
        {mrs.data(), L->rp, b_rp}, {mrl.data(), L->rl, b_rl}, {mcol.data(), L->col, b_col},
        {mval.data(), L->val, b_val}, {edges, L->edges, b_e}};
    for (auto& c : cp) {
        if (!c.n) continue;
        e = cudaMemcpy(const_cast<void*>(c.dst), c.src, c.n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(L->mem); delete L; return cuda_fail(e, "cudaMemcpy(lens)"); }
    }
    L->n_pix = n_pix;
    L->n_mat = n_mat;
    L->nnz = nnz;
    // lanes per row for one map: the mean merged row length in 4-entry vectors, rounded up to
    // a power of two in [4, 32]
    const double mean = (double)padded / 4.0 / (double)n_pix;
    int g = 4;
    while (g < 32 && g < mean) g *= 2;
    L->group = g;
    *out = L;
    return CRP_OK;
}

int crp_lens_set_group(crp_lens* L, int32_t g) {
    if (!L) return fail(CRP_ERR_INVALID_ARG, "lens is NULL");
    if (g != 4 && g != 8 && g != 16 && g != 32) return fail(CRP_ERR_INVALID_ARG, "lanes per row must be 4, 8, 16 or 32");
    L->group = g;
    return CRP_OK;
}

int crp_lens_destroy(crp_lens* L) {
    if (!L) return fail(CRP_ERR_INVALID_ARG, "lens is NULL");
    if (L->mem) cudaFree(L->mem);
    delete L;
    return CRP_OK;
}

int crp_lens_apply(const crp_lens* L, const double* x, double* y, int32_t n_maps, void* stream) {
    NvtxRange nvtx_("crp_lens_apply");
    if (!L || !x || !y) return fail(CRP_ERR_INVALID_ARG, "lens, x or y is NULL");
    if (n_maps < 1) return fail(CRP_ERR_INVALID_ARG, "n_maps must be >= 1");
    int e = launch_lens_apply(L->n_pix, n_maps, L->group, L->rp, L->rl, L->col, L->val, x, y, device_sms(), stream);
    if (e) return cuda_fail((cudaError_t)e, "lens kernel");
    return CRP_OK;
}

int crp_lens_bin(const crp_lens* L, crp_sim* s, int32_t nside, double e_min_ev, double* x, void* stream) {
    NvtxRange nvtx_("crp_lens_bin");
    if (!L || !s || !x) return fail(CRP_ERR_INVALID_ARG, "lens, sim or x is NULL");
    if (!L->edges) return fail(CRP_ERR_INVALID_ARG, "lens has no rigidity edges");
    if (nside < 1 || nside > 8192 || 12ll * nside * nside != L->n_pix)
        return fail(CRP_ERR_INVALID_ARG, "lens n_pix must be 12 nside^2");
    if (e_min_ev != e_min_ev) return fail(CRP_ERR_INVALID_ARG, "e_min is NaN");
    const int grid = (s->sms > 0 ? s->sms : 1) * 4;
    int e = launch_lens_bin(s->st, s->ctr, nside, L->n_mat, L->edges, e_min_ev, x, grid, stream);
    if (e) return cuda_fail((cudaError_t)e, "lens binning kernel");
    s->last = reinterpret_cast<cudaStream_t>(stream);
    return CRP_OK;
}

}  // extern "C"

namespace {

// FP64 descriptor of a field: the field itself for FP64 grids, else an FP64 copy of the
// vector grid (built on first use) with the field's geometry and modulation.
int field_fp64_desc(crp_field* f, FieldDev& out) {
    if (f->dev.layout == LAYOUT_F64X4) { out = f->dev; return CRP_OK; }
    if (!f->mem64) {
        void* m = nullptr;
        CRP_CUDA(dev_malloc(&m, (size_t)f->nodes * 32));
        k_widen<<<grid_for(f->nodes, 256, 65535), 256>>>(f->mem, f->dev.layout, f->dev.scale,
                                                         (double2*)m, f->nodes);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { cudaFree(m); return cuda_fail(e, "field widening"); }
        f->mem64 = m;
    }
    out = f->dev;
    out.data = f->mem64;
    out.layout = LAYOUT_F64X4;
    f->dev64 = out;
    return CRP_OK;
}

// Build (once per field) the FP64 copies and this simulation's descriptor array for them.
int ensure_fp64_fields(crp_sim* s) {
    if (s->d_fields64) return CRP_OK;
    int rc = sync_stream(s);
    if (rc) return rc;
    std::vector<FieldDev> d64;
    for (size_t i = 0; i < s->handles.size(); ++i) {
        FieldDev F;
        rc = field_fp64_desc(s->handles[i], F);
        if (rc) return rc;
        // the modulation as it was when the simulation was created
        const FieldDev& H = s->host_fields[i];
        F.mod = H.mod; F.mnx = H.mnx; F.mny = H.mny; F.mnz = H.mnz; F.mpow2 = H.mpow2;
        F.m_inv_spacing = H.m_inv_spacing; F.m_spacing = H.m_spacing;
        F.mox = H.mox; F.moy = H.moy; F.moz = H.moz;
        F.moix = H.moix; F.moiy = H.moiy; F.moiz = H.moiz;
        d64.push_back(F);
    }
    void* d = nullptr;
    CRP_CUDA(dev_malloc(&d, sizeof(FieldDev) * d64.size()));
    cudaError_t e = cudaMemcpy(d, d64.data(), sizeof(FieldDev) * d64.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "cudaMemcpy(fields64)"); }
    s->d_fields64 = (FieldDev*)d;
    return CRP_OK;
}

// Cell-major copies (precision form): bytes they need beyond what is already built.
long long cells_bytes_needed(const crp_sim* s) {
    long long need = 0;
    for (const crp_field* f : s->handles)
        if (!f->memc) need += f->nodes * (f->dev.layout == LAYOUT_BF16X4 ? 64 : 96);
    return need;
}

// Build (once per field) the cell-major copies and this simulation's descriptor array for
// them (geometry and modulation as when the simulation was created).
int ensure_cell_fields(crp_sim* s) {
    if (s->d_fields_cells) return CRP_OK;
    int rc = sync_stream(s);
    if (rc) return rc;
    std::vector<FieldDev> dc;
    for (size_t i = 0; i < s->handles.size(); ++i) {
        crp_field* f = s->handles[i];
        const bool bf16 = f->dev.layout == LAYOUT_BF16X4;
        if (!f->memc) {
            void* m = nullptr;
            CRP_CUDA(dev_malloc(&m, (size_t)f->nodes * (bf16 ? 64 : 96)));
            k_cells<<<grid_for(f->nodes, 256, 65535), 256>>>(f->mem, bf16 ? 1 : 0, f->dev.nx, f->dev.ny,
                                                              f->dev.nz, m);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) { cudaFree(m); return cuda_fail(e, "cell-major copy"); }
            f->memc = m;
        }
        FieldDev F = s->host_fields[i];
        F.data = f->memc;
        F.layout = bf16 ? LAYOUT_BF16_CELLS : LAYOUT_F32_CELLS;
        dc.push_back(F);
    }
    void* d = nullptr;
    CRP_CUDA(dev_malloc(&d, sizeof(FieldDev) * dc.size()));
    cudaError_t e = cudaMemcpy(d, dc.data(), sizeof(FieldDev) * dc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "cudaMemcpy(fields cells)"); }
    s->d_fields_cells = (FieldDev*)d;
    return CRP_OK;
}

int make_plan(crp_sim* s, const crp_params* prm, double tol, double hmin, double hmax,
              double dmax, Plan& P) {
    if (!s || !prm) return fail(CRP_ERR_INVALID_ARG, "sim or params is NULL");
    if (!(tol > 0.0) || !(hmin > 0.0) || !(hmax >= hmin) || !(dmax > 0.0) || !std::isfinite(hmax) ||
        !std::isfinite(dmax))
        return fail(CRP_ERR_INVALID_ARG, "need tolerance > 0, 0 < min_step <= max_step, max_distance > 0");
    if (prm->form != CRP_FORM_FP64 && prm->form != CRP_FORM_MIXED)
        return fail(CRP_ERR_INVALID_ARG, "unknown form");
    if (prm->form == CRP_FORM_MIXED && s->layout != LAYOUT_F32X4 && s->layout != LAYOUT_BF16X4)
        return fail(CRP_ERR_INVALID_ARG, "the mixed form reads FP32 or BF16 grids");
    const bool mixed = prm->form == CRP_FORM_MIXED;
    const int order = prm->order == CRP_ORDER_DEFAULT ? CRP_ORDER_COST : prm->order;
    const int pickup = prm->pickup == CRP_PICKUP_DEFAULT ? CRP_PICKUP_OFF : prm->pickup;
    if (order != CRP_ORDER_SLOT && order != CRP_ORDER_COST && order != CRP_ORDER_GRID)
        return fail(CRP_ERR_INVALID_ARG, "unknown order");
    if (pickup != CRP_PICKUP_OFF && pickup != CRP_PICKUP_ON) return fail(CRP_ERR_INVALID_ARG, "unknown pickup");
    const int block = prm->block_size > 0 ? prm->block_size : 128;
    if (block % 32 || block > 256) return fail(CRP_ERR_INVALID_ARG, "block_size must be a multiple of 32, <= 256");
    // the FP64 form reads FP64 copies of the grids (no per-corner widening on the FP64 pipe)
    const FieldDev* fields = s->d_fields;
    int layout = s->layout;
    if (!mixed && layout != LAYOUT_F64X4) {
        int rc = ensure_fp64_fields(s);
        if (rc) return rc;
        fields = s->d_fields64;
        layout = LAYOUT_F64X4;
    }
    if (prm->grid_layout != CRP_GRID_AUTO && prm->grid_layout != CRP_GRID_NODES &&
        prm->grid_layout != CRP_GRID_CELLS)
        return fail(CRP_ERR_INVALID_ARG, "unknown grid_layout");
    if (mixed && prm->grid_layout != CRP_GRID_NODES) {
        bool use = true;
        if (!s->d_fields_cells) {
            size_t free_b = 0, total_b = 0;
            CRP_CUDA(cudaMemGetInfo(&free_b, &total_b));
            const long long need = cells_bytes_needed(s);
            const bool fits = (double)need + 4.0 * (1ll << 30) <= (double)free_b;
            if (!fits && prm->grid_layout == CRP_GRID_CELLS)
                return fail(CRP_ERR_OOM, "cell-major grid copies do not fit in free device memory");
            use = fits;
        }
        if (use) {
            int rc = ensure_cell_fields(s);
            if (rc) return rc;
            fields = s->d_fields_cells;
            layout = layout == LAYOUT_BF16X4 ? LAYOUT_BF16_CELLS : LAYOUT_F32_CELLS;
        }
    }
    int p2 = 1;   // the mask-wrap kernels when every vector grid's sizes are powers of two
    for (const FieldDev& hf : s->host_fields) p2 &= hf.pow2 ? 1 : 0;
    int bps = prm->blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        const int oe = mixed ? propagate_mixed_occupancy(layout, s->mod, p2, block, &occ)
                             : propagate_fp64_occupancy(layout, s->mod, p2, block, &occ);
        if (oe != 0 || occ < 1) occ = 1;
        bps = occ;
    }
    P.grid = (s->sms > 0 ? s->sms : 1) * bps;
    P.block = block;
    P.order = order;
    P.mixed = mixed ? 1 : 0;
    P.layout = layout;
    P.mod = s->mod;
    P.p2 = p2;
    P.n_buckets = order == CRP_ORDER_GRID ? kBuckets * (int)s->host_fields.size() : kBuckets;
    PropArgs& a = P.a;
    a.st = s->st;
    a.fields = fields;
    a.n_fields = (int)s->host_fields.size();
    a.has_tables = s->tables ? 1 : 0;
    if (s->tables) a.tab = s->tables->dev;
    a.tol = tol; a.hmin = hmin; a.hmax = hmax; a.dmax = dmax;
    a.seed = s->seed;
    a.max_steps = prm->max_steps;
    a.capacity = s->capacity;
    // default cadence: 2 attempts between refill checks in the precision form (measured +1.5 %
    // on the 10^6-nuclei workload), 1 in the FP64 form; results do not depend on it
    a.cadence = prm->cadence > 0 ? prm->cadence : (prm->form == CRP_FORM_MIXED ? 2 : 1);
    a.pickup = pickup == CRP_PICKUP_ON ? 1 : 0;
    a.lists[0] = s->lists[0];
    a.lists[1] = s->lists[1];
    a.done_list = s->done_list;
    a.ctr = s->ctr;
    a.boundary = s->boundary == CRP_BOUNDARY_REFLECT ? 1 : 0;
    for (int c = 0; c < 3; ++c) {
        a.box_lo[c] = s->box_origin[c];
        a.box_hi[c] = s->box_origin[c] + s->box_size[c];
        a.box_len[c] = s->box_size[c];
        a.box_inv[c] = s->boundary == CRP_BOUNDARY_REFLECT ? 1.0 / s->box_size[c] : 0.0;
    }
    return CRP_OK;
}

// The launch sequence of one propagate call (no host synchronisation; capturable).
int enqueue(crp_sim* s, const Plan& P, cudaStream_t st) {
    PropArgs a = P.a;
    k_prepare<<<1, 1, 0, st>>>(s->ctr);
    CRP_CUDA(cudaGetLastError());
    const int sgrid = (s->sms > 0 ? s->sms : 1) * 4;
    if (P.order == CRP_ORDER_SLOT) {
        k_build_worklist<<<sgrid, 256, 0, st>>>(s->st.status, s->lists[0], s->ctr);
    } else {
        const int grid_major = P.order == CRP_ORDER_GRID ? 1 : 0;
        // fixed regions sized for the largest bucket count: [hist | offsets]; the scan leaves
        // hist zeroed for the next build, whatever order that build uses
        const int max_buckets = kBuckets * (int)s->host_fields.size();
        unsigned* hist = s->sort_scratch;
        unsigned* offs = s->sort_scratch + max_buckets;
        const size_t shm = (size_t)P.n_buckets * sizeof(unsigned);
        k_cost_hist<<<sgrid, 256, shm <= 48 * 1024 ? shm : 0, st>>>(
            s->st.status, s->st.E, s->st.Z, s->st.grid_id, grid_major, P.n_buckets,
            shm <= 48 * 1024 ? 1 : 0, hist, s->ctr);
        k_cost_scan<<<1, 1024, 0, st>>>(hist, offs, P.n_buckets, s->ctr);
        k_cost_scatter<<<sgrid, 256, 0, st>>>(s->st.status, s->st.E, s->st.Z, s->st.grid_id,
                                              grid_major, offs, s->lists[0], s->ctr);
    }
    CRP_CUDA(cudaGetLastError());
    // generation 1: the work list (and, with pickup, secondaries it pushes once the list
    // runs dry); generation 2: the secondaries left. Nucleon secondaries never split, so two
    // launches finish the call. The push list starts filled with -1.
    for (int gen = 0; gen < 2; ++gen) {
        if (a.pickup) CRP_CUDA(cudaMemsetAsync(s->lists[1 - gen], 0xff, sizeof(int32_t) * s->capacity, st));
        a.list = gen;
        int e = P.mixed ? launch_propagate_mixed(a, P.layout, P.mod, P.p2, P.grid, P.block, st)
                        : launch_propagate_fp64(a, P.layout, P.mod, P.p2, P.grid, P.block, st);
        if (e) return cuda_fail((cudaError_t)e, "propagate kernel launch");
        k_swap<<<1, 1, 0, st>>>(s->ctr, s->capacity, gen);
        CRP_CUDA(cudaGetLastError());
    }
    return CRP_OK;
}

// Device-side loop control for crp_propagate_loop.
__global__ void k_loop_init(Counters* C) {
    CRP_COUNT_RUN();
    C->slices = 0;
    C->prev_accepted = C->accepted;
}

__global__ void k_loop_cond(Counters* C, cudaGraphConditionalHandle h, long long max_slices) {
    CRP_COUNT_RUN();
    C->slices += 1;
    const bool active = C->n_used > C->n_done;
    const bool progressed = C->accepted != C->prev_accepted;
    C->prev_accepted = C->accepted;
    const bool go = active && C->status_bits == 0 && progressed && (long long)C->slices < max_slices;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

bool same_plan(const Plan& x, const Plan& y) {
    return std::memcmp(&x.a, &y.a, sizeof(PropArgs)) == 0 && x.grid == y.grid &&
           x.block == y.block && x.order == y.order && x.mixed == y.mixed && x.n_buckets == y.n_buckets &&
           x.p2 == y.p2 &&
           x.layout == y.layout;
}

}  // namespace

extern "C" {

int crp_propagate(crp_sim* s, const crp_params* prm, double tol, double hmin, double hmax,
                  double dmax, void* stream) {
    NvtxRange nvtx_("crp_propagate");
    Plan P;
    int rc = make_plan(s, prm, tol, hmin, hmax, dmax, P);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rc = enqueue(s, P, st);
    if (rc) return rc;
    s->last = st;
    return CRP_OK;
}

int crp_propagate_loop(crp_sim* s, const crp_params* prm, double tol, double hmin, double hmax,
                       double dmax, int32_t max_slices, void* stream) {
    NvtxRange nvtx_("crp_propagate_loop");
    Plan P;
    int rc = make_plan(s, prm, tol, hmin, hmax, dmax, P);
    if (rc) return rc;
    if (max_slices < 1) return fail(CRP_ERR_INVALID_ARG, "max_slices must be >= 1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!s->loop_exec || !same_plan(P, s->loop_plan) || s->loop_max_slices != max_slices) {
        if (s->loop_exec) { cudaGraphExecDestroy(s->loop_exec); s->loop_exec = nullptr; }
        if (s->loop_graph) { cudaGraphDestroy(s->loop_graph); s->loop_graph = nullptr; }
        cudaGraph_t g = nullptr;
        CRP_CUDA(cudaGraphCreate(&g, 0));
        s->loop_graph = g;
        // init node
        cudaKernelNodeParams kp{};
        Counters* ctr = s->ctr;
        void* init_args[] = {&ctr};
        kp.func = (void*)k_loop_init;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = init_args;
        cudaGraphNode_t init_node;
        CRP_CUDA(cudaGraphAddKernelNode(&init_node, g, nullptr, 0, &kp));
        // while node; its body is the captured propagate sequence plus the condition kernel
        cudaGraphConditionalHandle h;
        CRP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cond_node;
        CRP_CUDA(cudaGraphAddNode(&cond_node, g, &init_node, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t cs;
        CRP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(e, "cudaStreamBeginCaptureToGraph"); }
        rc = enqueue(s, P, cs);
        k_loop_cond<<<1, 1, 0, cs>>>(s->ctr, h, (long long)max_slices);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cs, &captured);
        cudaStreamDestroy(cs);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        CRP_CUDA(cudaGraphInstantiate(&s->loop_exec, g, 0));
        s->loop_plan = P;
        s->loop_max_slices = max_slices;
    }
    CRP_CUDA(cudaGraphLaunch(s->loop_exec, st));
    s->last = st;
    return CRP_OK;
}

int crp_sync(crp_sim* s, double timeout_s) {
    NvtxRange nvtx_("crp_sync");
    if (!s) return fail(CRP_ERR_INVALID_ARG, "sim is NULL");
    if (timeout_s > 0) {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            cudaError_t e = cudaStreamQuery(s->last);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (dt > timeout_s) return fail(CRP_ERR_TIMEOUT, "crp_sync wait limit reached");
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    }
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    const unsigned b = h.status_bits;
    if (b) {
        unsigned zero = 0;
        CRP_CUDA(cudaMemcpy(&s->ctr->status_bits, &zero, sizeof zero, cudaMemcpyHostToDevice));
    }
    if (b & BIT_QUEUE_FULL) return fail(CRP_ERR_QUEUE_FULL, "secondary queue full");
    if (b & BIT_NAN) return fail(CRP_ERR_NAN_STATE, "non-finite particle state");
    if (b & BIT_RANGE) return fail(CRP_ERR_TABLE_RANGE, "species outside tables");
    if (b & BIT_INVALID) return fail(CRP_ERR_INVALID_ARG, "invalid particle in injection");
    if (b & BIT_TIMEOUT) return fail(CRP_ERR_TIMEOUT, "a pushed secondary never appeared in its list");
    if (b & BIT_BOUNDS) return fail(CRP_ERR_CUDA, "a work-list entry or grid id was out of range (skipped)");
    return CRP_OK;
}

int crp_sim_counts(crp_sim* s, int64_t counts[8]) {
    if (!s || !counts) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    counts[0] = (int64_t)h.n_used;
    counts[1] = (int64_t)(h.n_used - h.n_done);
    counts[2] = (int64_t)h.n_done;
    counts[3] = (int64_t)h.accepted;
    counts[4] = (int64_t)h.attempted;
    counts[5] = (int64_t)h.secondaries;
    counts[6] = (int64_t)h.launches;
    counts[7] = (int64_t)h.status_bits;
    return CRP_OK;
}

int crp_read_state(crp_sim* s, int32_t column, void* dst, int32_t dst_is_device, int64_t first,
                   int64_t count) {
    NvtxRange nvtx_("crp_read_state");
    if (!s || !dst) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (column < 0 || column >= CRP_N_COLS) return fail(CRP_ERR_INVALID_ARG, "unknown column");
    if (first < 0 || count < 0 || first + count > s->capacity)
        return fail(CRP_ERR_INVALID_ARG, "slot range outside the simulation");
    int rc = sync_stream(s);
    if (rc) return rc;
    const char* src = (const char*)*col_ptr(s->st, column) + first * kCols[column].size;
    CRP_CUDA(cudaMemcpy(dst, src, (size_t)count * kCols[column].size,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return CRP_OK;
}

int crp_observe(crp_sim* s, const crp_observer* o, int64_t first, int64_t capacity, int64_t* n_out) {
    NvtxRange nvtx_("crp_observe");
    if (!s || !o || !n_out) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (first < 0 || capacity < 0) return fail(CRP_ERR_INVALID_ARG, "negative range");
    *n_out = 0;
    Counters h;
    int rc = read_counters(s, &h);
    if (rc) return rc;
    long long n = (long long)h.n_done - first;
    if (n <= 0) return CRP_OK;
    if (n > capacity) n = capacity;
    ObsCols d{o->uid, o->A, o->Z, o->n_int, o->status, o->E, o->x, o->y, o->z, o->ux, o->uy,
              o->uz, o->u0x, o->u0y, o->u0z, o->s, o->n_steps, o->n_att};
    void* tmp = nullptr;
    ObsCols t = d;
    // Host columns in pinned (page-locked) memory are written by the gather kernel directly,
    // through their device addresses; other host memory goes through a staging block.
    bool direct = !o->is_device;
    if (direct) {
        void** cols[] = {(void**)&t.uid, (void**)&t.A, (void**)&t.Z, (void**)&t.n_int,
                         (void**)&t.status, (void**)&t.E, (void**)&t.x, (void**)&t.y,
                         (void**)&t.z, (void**)&t.ux, (void**)&t.uy, (void**)&t.uz,
                         (void**)&t.u0x, (void**)&t.u0y, (void**)&t.u0z, (void**)&t.s,
                         (void**)&t.n_steps, (void**)&t.n_att};
        for (void** c : cols) {
            if (!*c) continue;
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, *c) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
                !pa.devicePointer) {
                cudaGetLastError();
                direct = false;
                break;
            }
            *c = pa.devicePointer;
        }
        if (!direct) t = d;
    }
    if (!o->is_device && !direct) {   // gather on the device into one staging block, then copy out
        size_t off = 0;
        const size_t sz8 = (size_t)n * 8, sz4 = (size_t)n * 4;
        CRP_CUDA(dev_malloc(&tmp, 13 * sz8 + 4 * sz4 + 2 * sz8));
        char* b = (char*)tmp;
        auto take8 = [&](void* want) -> void* { if (!want) return nullptr; void* r = b + off; off += sz8; return r; };
        auto take4 = [&](void* want) -> void* { if (!want) return nullptr; void* r = b + off; off += sz4; return r; };
        t.uid = (int64_t*)take8(d.uid);
        t.E = (double*)take8(d.E); t.x = (double*)take8(d.x); t.y = (double*)take8(d.y);
        t.z = (double*)take8(d.z); t.ux = (double*)take8(d.ux); t.uy = (double*)take8(d.uy);
        t.uz = (double*)take8(d.uz); t.u0x = (double*)take8(d.u0x); t.u0y = (double*)take8(d.u0y);
        t.u0z = (double*)take8(d.u0z); t.s = (double*)take8(d.s);
        t.n_steps = (int64_t*)take8(d.n_steps); t.n_att = (int64_t*)take8(d.n_att);
        t.A = (int32_t*)take4(d.A); t.Z = (int32_t*)take4(d.Z);
        t.n_int = (int32_t*)take4(d.n_int); t.status = (int32_t*)take4(d.status);
    }
    k_observe<<<grid_for(n, 256, 4096), 256>>>(s->st, s->done_list, first, n, t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !o->is_device && !direct) {
        struct { void* dst; void* src; size_t sz; } cps[] = {
            {d.uid, t.uid, 8}, {d.E, t.E, 8}, {d.x, t.x, 8}, {d.y, t.y, 8}, {d.z, t.z, 8},
            {d.ux, t.ux, 8}, {d.uy, t.uy, 8}, {d.uz, t.uz, 8}, {d.u0x, t.u0x, 8},
            {d.u0y, t.u0y, 8}, {d.u0z, t.u0z, 8}, {d.s, t.s, 8}, {d.n_steps, t.n_steps, 8},
            {d.n_att, t.n_att, 8}, {d.A, t.A, 4}, {d.Z, t.Z, 4}, {d.n_int, t.n_int, 4},
            {d.status, t.status, 4}};
        for (auto& c : cps)
            if (c.dst && e == cudaSuccess) e = cudaMemcpy(c.dst, c.src, (size_t)n * c.sz, cudaMemcpyDeviceToHost);
    }
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "crp_observe");
    *n_out = n;
    return CRP_OK;
}

}  // extern "C"

// ---- propagation without allocation: scratch in a static device array ---------------------
// Layout: [Counters | pad to 256] [FieldDev | pad to 256] [work list 0] [work list 1]
// [done list], each list CRP_NOALLOC_MAX_PARTICLES int32 entries.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CRP_NOALLOC_SCRATCH_BYTES];
static_assert(sizeof(Counters) <= 256 && sizeof(FieldDev) <= 256, "scratch header layout");

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};   // device address of the array, per device ordinal

__global__ void k_noalloc_setup(Counters* C, FieldDev* F, FieldDev f, unsigned long long n) {
    CRP_COUNT_RUN();
    Counters z{};
    z.n_used = n;
    z.reserve = n;
    *C = z;
    *F = f;
}

}  // namespace

extern "C" int crp_propagate_noalloc(const void* grid, int32_t nx, int32_t ny, int32_t nz,
                                     double spacing_m, const double origin_m[3],
                                     const crp_state_columns* cols, int64_t n, uint64_t seed,
                                     double tol, double hmin, double hmax, double dmax,
                                     int64_t max_steps, void* stream) {
    NvtxRange nvtx_("crp_propagate_noalloc");
    if (!grid || !origin_m || !cols) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n > CRP_NOALLOC_MAX_PARTICLES)
        return fail(CRP_ERR_INVALID_ARG, "n outside [0, CRP_NOALLOC_MAX_PARTICLES]");
    if (((uintptr_t)grid) % 16) return fail(CRP_ERR_INVALID_ARG, "grid must be 16-byte aligned");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1ll << 31))
        return fail(CRP_ERR_INVALID_ARG, "grid sizes out of range");
    if (!(spacing_m > 0.0) || !std::isfinite(spacing_m))
        return fail(CRP_ERR_INVALID_ARG, "spacing must be finite and > 0");
    if (!(tol > 0.0) || !(hmin > 0.0) || !(hmax >= hmin) || !(dmax > 0.0) ||
        !std::isfinite(hmax) || !std::isfinite(dmax))
        return fail(CRP_ERR_INVALID_ARG, "need tolerance > 0, 0 < min_step <= max_step, max_distance > 0");
    const crp_state_columns& c = *cols;
    const void* req[] = {c.x, c.y, c.z, c.ux, c.uy, c.uz, c.E, c.s, c.hprop, c.tau, c.u0x,
                         c.u0y, c.u0z, c.A, c.Z, c.n_int, c.status, c.grid_id, c.uid,
                         c.n_steps, c.n_att};
    for (const void* q : req)
        if (!q) return fail(CRP_ERR_INVALID_ARG, "NULL state column");
    if (n == 0) return CRP_OK;
    int dev = 0;
    CRP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CRP_ERR_CUDA, "device ordinal above 63");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    Counters* ctr = (Counters*)base;
    FieldDev* fdev = (FieldDev*)((char*)base + 256);
    int32_t* l0 = (int32_t*)((char*)base + 512);
    int32_t* l1 = l0 + CRP_NOALLOC_MAX_PARTICLES;
    int32_t* done = l1 + CRP_NOALLOC_MAX_PARTICLES;

    FieldDev f{};
    f.data = grid;
    f.layout = LAYOUT_F32X4;
    f.nx = nx; f.ny = ny; f.nz = nz;
    f.pow2 = (is_pow2(nx) && is_pow2(ny) && is_pow2(nz)) ? 1 : 0;
    f.inv_spacing = 1.0 / spacing_m;
    f.spacing = spacing_m;
    f.ox = origin_m[0]; f.oy = origin_m[1]; f.oz = origin_m[2];
    f.oix = f.ox * f.inv_spacing; f.oiy = f.oy * f.inv_spacing; f.oiz = f.oz * f.inv_spacing;
    f.scale = 1.0;
    SimState S{c.x, c.y, c.z, c.ux, c.uy, c.uz, c.E, c.s, c.hprop, c.tau, c.u0x, c.u0y, c.u0z,
               c.A, c.Z, c.n_int, c.status, c.grid_id, c.uid, c.n_steps, c.n_att};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int sms = device_sms() > 0 ? device_sms() : 1;

    k_noalloc_setup<<<1, 1, 0, st>>>(ctr, fdev, f, (unsigned long long)n);
    CRP_CUDA(cudaGetLastError());
    k_inject_init<<<grid_for(n, 256, 4096), 256, 0, st>>>(S, 0, n, 1, 0, 0ull, 1, 0, 0, 0, seed,
                                                          done, ctr);
    CRP_CUDA(cudaGetLastError());
    k_prepare<<<1, 1, 0, st>>>(ctr);
    CRP_CUDA(cudaGetLastError());
    k_build_worklist<<<sms * 4, 256, 0, st>>>(S.status, l0, ctr);
    CRP_CUDA(cudaGetLastError());
    const int block = 128;
    int occ = 0;
    if (propagate_fp64_occupancy(LAYOUT_F32X4, 0, f.pow2, block, &occ) != 0 || occ < 1) occ = 1;
    PropArgs a{};
    a.st = S;
    a.fields = fdev;
    a.n_fields = 1;
    a.has_tables = 0;
    a.tol = tol; a.hmin = hmin; a.hmax = hmax; a.dmax = dmax;
    a.seed = seed;
    a.max_steps = max_steps;
    a.capacity = n;
    a.cadence = 1;
    a.lists[0] = l0;
    a.lists[1] = l1;
    a.done_list = done;
    a.ctr = ctr;
    for (int gen = 0; gen < 2; ++gen) {
        a.list = gen;
        int e = launch_propagate_fp64(a, LAYOUT_F32X4, 0, f.pow2, sms * occ, block, st);
        if (e) return cuda_fail((cudaError_t)e, "propagate kernel launch");
        k_swap<<<1, 1, 0, st>>>(ctr, n, gen);
        CRP_CUDA(cudaGetLastError());
    }
    CRP_CUDA(cudaStreamSynchronize(st));
    unsigned bits = 0;
    CRP_CUDA(cudaMemcpy(&bits, &ctr->status_bits, sizeof bits, cudaMemcpyDeviceToHost));
    // every device status bit is an error here, mapped to the codes crp_sync uses
    if (bits & BIT_QUEUE_FULL) return fail(CRP_ERR_QUEUE_FULL, "secondary queue full");
    if (bits & BIT_NAN) return fail(CRP_ERR_NAN_STATE, "non-finite particle state");
    if (bits & BIT_RANGE) return fail(CRP_ERR_TABLE_RANGE, "species outside tables");
    if (bits & BIT_INVALID) return fail(CRP_ERR_INVALID_ARG, "invalid particle");
    if (bits & BIT_TIMEOUT) return fail(CRP_ERR_TIMEOUT, "a pushed secondary never appeared in its list");
    if (bits & BIT_BOUNDS)
        return fail(CRP_ERR_CUDA, "a work-list entry was out of range and skipped (overlapping calls?)");
    if (bits) return fail(CRP_ERR_CUDA, "unknown device status bit");
    return CRP_OK;
}

// ---- differentiation through a frozen step sequence -----------------------------------------
struct crp_adjoint {
    crp_field* field = nullptr;
    long long n = 0;
    int n_steps = 0, K = 0, n_ck = 0;
    double *y0 = nullptr, *kappa = nullptr, *E = nullptr, *h = nullptr, *ck = nullptr;
    double *seg = nullptr, *y0_bar = nullptr, *kappa_bar = nullptr, *y0_tmp = nullptr;
    double *kappa_tmp = nullptr, *E_tmp = nullptr;
    double* stages = nullptr;            // stage records of every step (kAdjRecordBytes each), if room
    int32_t* Z = nullptr;
    bool recorded = false;
    // the backward pass forms the stage records in chunks on `aux` beside the reverse sweep
    static constexpr int kEvents = 9;   // up to 8 chunks
    cudaStream_t aux = nullptr;
    cudaEvent_t ev[kEvents] = {};
    int n_ev = 0;
};

namespace {

void adj_free(crp_adjoint* a) {
    double* ds[] = {a->y0, a->kappa, a->E, a->h, a->ck, a->seg, a->y0_bar, a->kappa_bar, a->y0_tmp,
                    a->kappa_tmp, a->E_tmp, a->stages};
    for (double* p : ds)
        if (p) cudaFree(p);
    if (a->Z) cudaFree(a->Z);
    for (int k = 0; k < a->n_ev; ++k) cudaEventDestroy(a->ev[k]);
    if (a->aux) cudaStreamDestroy(a->aux);
}

}  // namespace

extern "C" {

int crp_adjoint_create(const crp_field* field, int64_t n, int32_t n_steps, int32_t K, crp_adjoint** out) {
    NvtxRange nvtx_("crp_adjoint_create");
    if (!out) return fail(CRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!field || n < 1 || n_steps < 1 || K < 1) return fail(CRP_ERR_INVALID_ARG, "need field, n >= 1, n_steps >= 1, checkpoint_every >= 1");
    if (field->dev.mod) return fail(CRP_ERR_INVALID_ARG, "the adjoint takes unmodulated fields");
    crp_adjoint* a = new crp_adjoint();
    a->field = const_cast<crp_field*>(field);
    a->n = n;
    a->n_steps = n_steps;
    a->K = K;
    a->n_ck = (n_steps + K - 1) / K;
    struct { double** p; size_t count; } al[] = {
        {&a->y0, 6 * (size_t)n}, {&a->kappa, (size_t)n}, {&a->E, (size_t)n},
        {&a->h, (size_t)n_steps * n}, {&a->ck, (size_t)a->n_ck * 6 * n}, {&a->seg, (size_t)(K + 1) * 6 * n},
        {&a->y0_bar, 6 * (size_t)n}, {&a->kappa_bar, (size_t)n}, {&a->y0_tmp, 6 * (size_t)n},
        {&a->kappa_tmp, (size_t)n}, {&a->E_tmp, (size_t)n}};
    for (auto& q : al) {
        cudaError_t e = dev_malloc(q.p, q.count * sizeof(double));
        if (e != cudaSuccess) { adj_free(a); delete a; return cuda_fail(e, "cudaMalloc(adjoint)"); }
    }
    cudaError_t e = dev_malloc(&a->Z, sizeof(int32_t) * n);
    if (e != cudaSuccess) { adj_free(a); delete a; return cuda_fail(e, "cudaMalloc(adjoint Z)"); }
    FieldDev F;
    int rc = field_fp64_desc(a->field, F);
    if (rc) { adj_free(a); delete a; return rc; }
    // stage records of all steps (kAdjRecordBytes per step and particle) when they fit in half
    // of the free memory and the grid's node indices fit in int32: every segment's records are
    // then formed in parallel and the serial reverse sweep only applies them
    size_t free_b = 0, total_b = 0;
    const size_t st_bytes = kAdjRecordBytes * (size_t)n_steps * (size_t)n;
    const long long nodes = (long long)F.nx * F.ny * F.nz;
    if (nodes < (1ll << 31) && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && st_bytes <= free_b / 2) {
        if (dev_malloc(&a->stages, st_bytes) != cudaSuccess) {
            a->stages = nullptr;
            cudaGetLastError();
        }
    }
    if (a->stages) {   // without a stream and events the records form in one chunk
        if (cudaStreamCreateWithFlags(&a->aux, cudaStreamNonBlocking) == cudaSuccess) {
            while (a->n_ev < crp_adjoint::kEvents &&
                   cudaEventCreateWithFlags(&a->ev[a->n_ev], cudaEventDisableTiming) == cudaSuccess)
                ++a->n_ev;
        } else {
            a->aux = nullptr;
        }
        cudaGetLastError();
    }
    *out = a;
    return CRP_OK;
}

int crp_adjoint_destroy(crp_adjoint* a) {
    if (!a) return fail(CRP_ERR_INVALID_ARG, "adjoint is NULL");
    cudaDeviceSynchronize();
    adj_free(a);
    delete a;
    return CRP_OK;
}

int crp_adjoint_forward(crp_adjoint* a, const double* x0, const double* p0, const int32_t* Z,
                        double tol, double hmin, double hmax, double* xT, double* uT, void* stream) {
    NvtxRange nvtx_("crp_adjoint_forward");
    if (!a || !x0 || !p0 || !Z || !xT || !uT) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (!(tol > 0.0) || !(hmin > 0.0) || !(hmax >= hmin) || !std::isfinite(hmax))
        return fail(CRP_ERR_INVALID_ARG, "need tolerance > 0 and 0 < min_step <= max_step");
    FieldDev F;
    int rc = field_fp64_desc(a->field, F);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CRP_CUDA(cudaMemcpyAsync(a->Z, Z, sizeof(int32_t) * a->n, cudaMemcpyDeviceToDevice, st));
    int e = adj_init(x0, p0, a->Z, a->y0, a->kappa, a->E, a->n, st);
    if (e) return cuda_fail((cudaError_t)e, "adjoint init");
    e = adj_record(F, a->y0, a->kappa, tol, hmin, hmax, a->n_steps, a->K, a->h, a->ck, xT, uT, a->n, st);
    if (e) return cuda_fail((cudaError_t)e, "adjoint forward");
    a->recorded = true;
    return CRP_OK;
}

int crp_adjoint_replay(crp_adjoint* a, const crp_field* field, const double* p0, double* xT,
                       double* uT, uint64_t* cell_hash, void* stream) {
    NvtxRange nvtx_("crp_adjoint_replay");
    if (!a || !xT || !uT) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (!a->recorded) return fail(CRP_ERR_INVALID_ARG, "no recorded forward pass");
    crp_field* f = field ? const_cast<crp_field*>(field) : a->field;
    if (f->dev.nx != a->field->dev.nx || f->dev.ny != a->field->dev.ny || f->dev.nz != a->field->dev.nz)
        return fail(CRP_ERR_INVALID_ARG, "replay field has another grid geometry");
    if (f->dev.mod) return fail(CRP_ERR_INVALID_ARG, "the adjoint takes unmodulated fields");
    FieldDev F;
    int rc = field_fp64_desc(f, F);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double* y0 = a->y0;
    const double* kap = a->kappa;
    if (p0) {   // new directions and kappa; positions as recorded
        CRP_CUDA(cudaMemcpyAsync(a->y0_tmp, a->y0, sizeof(double) * 3 * a->n, cudaMemcpyDeviceToDevice, st));
        int e = adj_init(nullptr, p0, a->Z, a->y0_tmp, a->kappa_tmp, a->E_tmp, a->n, st);
        if (e) return cuda_fail((cudaError_t)e, "replay init");
        y0 = a->y0_tmp;
        kap = a->kappa_tmp;
    }
    int e = adj_replay(F, y0, kap, a->h, a->n_steps, xT, uT, (unsigned long long*)cell_hash, a->n, st);
    if (e) return cuda_fail((cudaError_t)e, "adjoint replay");
    return CRP_OK;
}

int crp_adjoint_backward(crp_adjoint* a, const double* uT_bar, double* grid_bar, double* p0_bar,
                         double* x0_bar, void* stream) {
    NvtxRange nvtx_("crp_adjoint_backward");
    if (!a || !uT_bar || !grid_bar || !p0_bar) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    if (!a->recorded) return fail(CRP_ERR_INVALID_ARG, "no recorded forward pass");
    FieldDev F;
    int rc = field_fp64_desc(a->field, F);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int e = adj_backward(F, a->kappa, a->h, a->ck, a->seg, a->stages, a->n_steps, a->K, uT_bar, grid_bar,
                         a->y0_bar, a->kappa_bar, a->n, st, a->aux, reinterpret_cast<void* const*>(a->ev),
                         a->n_ev);
    if (e) return cuda_fail((cudaError_t)e, "adjoint backward");
    e = adj_p0bar(a->y0, a->kappa, a->E, a->y0_bar, a->kappa_bar, p0_bar, x0_bar, a->n, st);
    if (e) return cuda_fail((cudaError_t)e, "adjoint p0 gradient");
    return CRP_OK;
}

int crp_adjoint_read_steps(crp_adjoint* a, double* h, int32_t is_device) {
    if (!a || !h) return fail(CRP_ERR_INVALID_ARG, "NULL argument");
    CRP_CUDA(cudaDeviceSynchronize());
    CRP_CUDA(cudaMemcpy(h, a->h, sizeof(double) * a->n * a->n_steps,
                        is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return CRP_OK;
}

}  // extern "C"

namespace crp {
unsigned long long kernel_runs_capi() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
