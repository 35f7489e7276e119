// lens.cu -- lenses (arXiv:1410.5323 Sec. 3.3): per-rigidity sparse matrices that map
// directions at the galactic border to arrival directions at Earth, applied to whole arrival
// distributions by sparse matrix-vector products, and the rigidity-binned maps they take.
//
// y[p][b] = sum_m (M_m x_m)[p][b] over all n_mat matrices in one launch. The matrices are CSR
// (single-precision values, as lenses are stored); each entry enters the FP64 sum with one
// rounding, acc = fma(v, x, acc). On the device the lens is kept row-merged: row p holds the
// row-p segments of matrices 0, 1, ..., n_mat-1 one after the other, with columns offset by
// m n_pix into the stacked maps x[m][c] -- the same entries in the same order as the
// per-matrix form, but one contiguous run per output row, so a warp streams it with
// independent loads. The launch is bound by streaming the lens from HBM (8 bytes per entry);
// the stacked maps (n_mat x n_pix doubles per map) stay in L2.
//   one map  : a group of G lanes per output row, each lane every G-th group of four
//              entries of the row (rows padded to start on 16 bytes), the group reduces at
//              the end (G from the mean merged row length);
//   n_maps>1 : a warp per (row, 32 consecutive maps); lanes own maps, entries are read once
//              per warp (broadcast), and every map sums its row in stored order.
// Compiled with --fmad=false; the fused multiply-adds are explicit.
#include <cuda_runtime.h>

#include "crp.h"
#include "crp_internal.h"
#include "crp_sky.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

namespace crp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Exact FP32 -> FP64 widening of a stored value with integer instructions only. GB300 runs
// the hardware conversion on its FP64 pipe, which the fused multiply-adds already saturate.
// Normal: exponent rebiased by 1023 - 127, mantissa to the top of the 52 bits; zero: zero;
// subnormal m 2^-149: normalised with a leading-zero count; infinity and NaN: exponent 0x7FF,
// payload kept. Every branch is integer arithmetic, so a predicated select costs no FP64 issue.
__device__ __forceinline__ double widen_f32(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned e = (u >> 23) & 0xFFu;
    unsigned m = u & 0x7FFFFFu;
    unsigned ed;
    if (e == 0xFFu) {
        ed = 0x7FFu;
    } else if (e != 0u) {
        ed = e + 896u;
    } else if (m == 0u) {
        ed = 0u;
    } else {
        const unsigned sh = (unsigned)__clz((int)m) - 8u;   // moves the leading 1 to bit 23
        m = (m << sh) & 0x7FFFFFu;
        ed = 897u - sh;
    }
    const unsigned hi = (u & 0x80000000u) | (ed << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}

// Rows start on a 4-entry boundary (rs[p] is a multiple of 4) and hold rl[p] entries; the
// padding between rows is never read as an entry. One map: each lane of a G-lane group loads
// four entries (16-byte col and val vectors) per iteration.
template <int G>
__global__ void __launch_bounds__(256) k_lens_apply_vec(int n_pix, const long long* __restrict__ rs,
                                                        const int* __restrict__ rl, const int* __restrict__ col,
                                                        const float* __restrict__ val,
                                                        const double* __restrict__ x, double* __restrict__ y) {
    CRP_COUNT_RUN();
    const int lane = threadIdx.x & (G - 1);
    constexpr int kGroups = 32 / G;                              // rows per warp
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int4* col4 = reinterpret_cast<const int4*>(col);
    const float4* val4 = reinterpret_cast<const float4*>(val);
    // the loop bound is the same for every lane of a warp, so all lanes reach the shuffles
    for (long long base = warp * kGroups; base < n_pix; base += n_warps * kGroups) {
        const long long p = base + ((threadIdx.x & 31) / G);
        double acc = 0.0;
        if (p < n_pix) {
            const long long q0 = __ldg(rs + p) >> 2;
            const int len = __ldg(rl + p);
            const long long q1 = q0 + ((len + 3) >> 2);
#pragma unroll 2
            for (long long q = q0 + lane; q < q1; q += G) {
                const int4 c = __ldcs(col4 + q);
                const float4 v = __ldcs(val4 + q);
                const int left = len - (int)((q - q0) << 2);       // entries of the row from 4q on
                acc = __fma_rn(widen_f32(v.x), __ldg(x + c.x), acc);
                if (left > 1) acc = __fma_rn(widen_f32(v.y), __ldg(x + c.y), acc);
                if (left > 2) acc = __fma_rn(widen_f32(v.z), __ldg(x + c.z), acc);
                if (left > 3) acc = __fma_rn(widen_f32(v.w), __ldg(x + c.w), acc);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc = acc + __shfl_xor_sync(kFull, acc, o, G);
        if (lane == 0 && p < n_pix) y[p] = acc;
    }
}

__global__ void __launch_bounds__(256) k_lens_apply_maps(int n_pix, int n_maps, const long long* __restrict__ rs,
                                                         const int* __restrict__ rl, const int* __restrict__ col,
                                                         const float* __restrict__ val,
                                                         const double* __restrict__ x, double* __restrict__ y) {
    CRP_COUNT_RUN();
    const int lane = threadIdx.x & 31;
    const int chunks = (n_maps + 31) / 32;
    const long long warps = (long long)gridDim.x * blockDim.x / 32;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; w < (long long)n_pix * chunks;
         w += warps) {
        const long long p = w / chunks;
        const int b = (int)(w % chunks) * 32 + lane;
        const bool on = b < n_maps;
        double acc = 0.0;
        const long long k0 = __ldg(rs + p), k1 = k0 + __ldg(rl + p);
#pragma unroll 4
        for (long long k = k0; k < k1; ++k) {
            const double v = widen_f32(__ldg(val + k));
            const int c = __ldg(col + k);
            if (on) acc = __fma_rn(v, __ldg(x + (long long)c * n_maps + b), acc);
        }
        if (on) y[p * n_maps + b] = acc;
    }
}

// Rigidity-binned arrival maps: finished charged particles above e_min, bin of R = E/Z among
// the lens edges (binary search; the bin m with edges[m] <= R < edges[m+1]), pixel of -u.
__global__ void k_lens_bin(SimState S, const Counters* C, int nside, int n_mat, const double* __restrict__ edges,
                           double e_min, double* __restrict__ x) {
    CRP_COUNT_RUN();
    const long long n_pix = 12ll * nside * nside;
    const long long n = (long long)C->n_used;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (S.status[i] != CRP_STATUS_DONE_ || S.Z[i] <= 0 || !(S.E[i] > e_min)) continue;
        const double R = S.E[i] / (double)S.Z[i];
        if (!(edges[0] <= R && R < edges[n_mat])) continue;
        int lo = 0, hi = n_mat;              // edges[lo] <= R < edges[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (edges[mid] <= R) lo = mid; else hi = mid;
        }
        const long long p = sky::healpix_ring(nside, -S.ux[i], -S.uy[i], -S.uz[i]);
        if (p < 0 || p >= n_pix) continue;
        atomicAdd(x + (long long)lo * n_pix + p, 1.0);
    }
}

}  // namespace

int launch_lens_apply(int n_pix, int n_maps, int group, const long long* rs, const int* rl, const int* col,
                      const float* val, const double* x, double* y, int sms, void* stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int block = 256;
    if (n_maps == 1) {
        const long long threads = ((long long)n_pix * group + 31) / 32 * 32;
        long long blocks = (threads + block - 1) / block;
        const long long cap = (long long)sms * 8 * 16;
        if (blocks > cap) blocks = cap;
        switch (group) {
        case 4: k_lens_apply_vec<4><<<(int)blocks, block, 0, st>>>(n_pix, rs, rl, col, val, x, y); break;
        case 8: k_lens_apply_vec<8><<<(int)blocks, block, 0, st>>>(n_pix, rs, rl, col, val, x, y); break;
        case 16: k_lens_apply_vec<16><<<(int)blocks, block, 0, st>>>(n_pix, rs, rl, col, val, x, y); break;
        default: k_lens_apply_vec<32><<<(int)blocks, block, 0, st>>>(n_pix, rs, rl, col, val, x, y); break;
        }
    } else {
        const long long warps = (long long)n_pix * ((n_maps + 31) / 32);
        long long blocks = (warps * 32 + block - 1) / block;
        const long long cap = (long long)sms * 8 * 16;
        if (blocks > cap) blocks = cap;
        k_lens_apply_maps<<<(int)blocks, block, 0, st>>>(n_pix, n_maps, rs, rl, col, val, x, y);
    }
    return (int)cudaGetLastError();
}

int launch_lens_bin(const SimState& S, const Counters* C, int nside, int n_mat, const double* edges, double e_min,
                    double* x, int grid, void* stream) {
    k_lens_bin<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(S, C, nside, n_mat, edges, e_min, x);
    return (int)cudaGetLastError();
}

}  // namespace crp

namespace crp {
unsigned long long kernel_runs_lens() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
