// sources.cu -- Sec. 4 sources (Eq. 1 spectrum, isotropic emission) and arrival maps (Fig. 4:
// HEALPix maps of arrival directions). Compiled with --fmad=false: every expression is
// evaluated as written, so species, energies, directions and pixel indices are identical to
// the FP64 reading.
#include <cuda_runtime.h>

#include "crp.h"
#include "crp_internal.h"
#include "crp_math.cuh"
#include "crp_sky.cuh"

// Runs of this file's kernels (diagnostics: each launch adds one, from its first thread).
namespace {
__device__ unsigned long long g_kernel_runs = 0;
}

namespace crp {
namespace {

__device__ __forceinline__ double uniform_words(uint32_t hi, uint32_t lo) {
    const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
    return ((double)m + 0.5) * 0x1p-52;
}

__device__ __forceinline__ U4 words(unsigned long long seed, unsigned long long uid, uint32_t k,
                                    uint32_t tag) {
    return philox10((uint32_t)uid, (uint32_t)(uid >> 32), k, tag, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// One draw per particle and thread. Per particle: species and energy from Eq. 1 by rejection
// from the cutoff-free joint law, then an isotropic direction (Marsaglia 1972).
__global__ void k_source_sample(SimState S, long long first, long long n, unsigned long long uid_base,
                                crp_spectrum sp, unsigned long long seed) {
    CRP_COUNT_RUN();
    // cumulative species weights w_i = x_i A_i^(alpha-1); inverse-CDF constants of E^-alpha
    double cum[CRP_MAX_SPECIES];
    double acc = 0.0;
    for (int i = 0; i < sp.n_species; ++i) {
        acc = acc + sp.x[i] * crp_exp((sp.alpha - 1.0) * crp_log((double)sp.A[i]));
        cum[i] = acc;
    }
    const double W = acc;
    const double g = 1.0 - sp.alpha;
    double lo = 0.0, hi = 0.0, lr = 0.0;
    if (g != 0.0) {
        lo = crp_exp(g * crp_log(sp.e_min_ev));
        hi = crp_exp(g * crp_log(sp.e_max_ev));
    } else {
        lr = crp_log(sp.e_max_ev / sp.e_min_ev);
    }
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long slot = first + p;
        const unsigned long long uid = uid_base + (unsigned long long)p;
        int a = 0, z = 0;
        double e = 0.0;
        for (uint32_t k = 0; k < CRP_SOURCE_DRAWS; ++k) {
            const U4 w = words(seed, uid, k, 2u);
            const double u1 = uniform_words(w.a, w.b);
            const double u2 = uniform_words(w.c, w.d);
            int s = sp.n_species - 1;
            const double target = u1 * W;
            for (int i = 0; i < sp.n_species; ++i)
                if (target < cum[i]) { s = i; break; }
            const double en = g != 0.0 ? crp_exp(crp_log(lo + u2 * (hi - lo)) / g)
                                       : sp.e_min_ev * crp_exp(u2 * lr);
            const U4 v = words(seed, uid, k, 3u);
            const double u3 = uniform_words(v.a, v.b);
            if (u3 < crp_exp(-en / ((double)sp.Z[s] * sp.rcut_v))) {
                a = sp.A[s];
                z = sp.Z[s];
                e = en;
                break;
            }
        }
        double dx = 0.0, dy = 0.0, dz = 0.0;
        bool have_dir = false;
        for (uint32_t k = 0; k < CRP_SOURCE_DRAWS; ++k) {
            const U4 w = words(seed, uid, k, 4u);
            const double v1 = 2.0 * uniform_words(w.a, w.b) - 1.0;
            const double v2 = 2.0 * uniform_words(w.c, w.d) - 1.0;
            const double s2 = v1 * v1 + v2 * v2;
            if (s2 < 1.0) {
                const double r = 2.0 * sqrt(1.0 - s2);
                dx = v1 * r;
                dy = v2 * r;
                dz = 1.0 - 2.0 * s2;
                have_dir = true;
                break;
            }
        }
        if (!have_dir) { a = 0; z = 0; }    // A = 0: flagged invalid by the injection kernel
        S.uid[slot] = (long long)uid;
        S.A[slot] = a;
        S.Z[slot] = z;
        S.E[slot] = e;
        S.ux[slot] = dx;
        S.uy[slot] = dy;
        S.uz[slot] = dz;
    }
}

__global__ void k_healpix(int nside, const double* __restrict__ u, long long n, long long* __restrict__ pix) {
    CRP_COUNT_RUN();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        pix[k] = sky::healpix_ring(nside, u[3 * k], u[3 * k + 1], u[3 * k + 2]);
}

// Arrival map over the used slots. With `shared`, each block counts into a shared copy of
// the map (12 nside^2 32-bit counters) and adds its non-zero pixels to the global map once.
__global__ void k_arrival_map(SimState S, const Counters* C, int nside, double e_min, int shared,
                              unsigned long long* __restrict__ map) {
    CRP_COUNT_RUN();
    extern __shared__ unsigned int smap[];
    const long long npix = 12ll * nside * nside;
    if (shared) {
        for (long long q = threadIdx.x; q < npix; q += blockDim.x) smap[q] = 0u;
        __syncthreads();
    }
    const long long n = (long long)C->n_used;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (S.status[i] != CRP_STATUS_DONE_ || !(S.E[i] > e_min)) continue;
        const long long p = sky::healpix_ring(nside, -S.ux[i], -S.uy[i], -S.uz[i]);
        if (p < 0 || p >= npix) continue;
        if (shared) atomicAdd(&smap[p], 1u);
        else atomicAdd(&map[p], 1ull);
    }
    if (shared) {
        __syncthreads();
        for (long long q = threadIdx.x; q < npix; q += blockDim.x)
            if (smap[q]) atomicAdd(&map[q], (unsigned long long)smap[q]);
    }
}

}  // namespace

int launch_source_sample(const SimState& S, long long first, long long n, unsigned long long uid_base,
                         const crp_spectrum& sp, unsigned long long seed, int grid, void* stream) {
    k_source_sample<<<grid, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(S, first, n, uid_base, sp, seed);
    return (int)cudaGetLastError();
}

int launch_healpix(int nside, const double* u, long long n, long long* pix, int grid, void* stream) {
    k_healpix<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(nside, u, n, pix);
    return (int)cudaGetLastError();
}

int launch_arrival_map(const SimState& S, const Counters* C, int nside, double e_min,
                       unsigned long long* map, int grid, void* stream) {
    const long long npix = 12ll * nside * nside;
    const bool shared = npix * 4 <= 48 * 1024;
    k_arrival_map<<<grid, 256, shared ? (size_t)npix * 4 : 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        S, C, nside, e_min, shared ? 1 : 0, map);
    return (int)cudaGetLastError();
}

}  // namespace crp

namespace crp {
unsigned long long kernel_runs_sources() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_kernel_runs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}
}  // namespace crp
