// crp_internal.h -- device-side data structures shared by the host library (crp_capi.cu)
// and the kernels. Not part of the public ABI.
#pragma once
#include <cstdint>

#include "crp.h"

namespace crp {

// Grid layouts in device memory: one 4-wide vector per node, node index
// (i*ny + j)*nz + k, the 4th lane unused (padding keeps every corner one aligned load).
enum Layout : int32_t { LAYOUT_F32X4 = 0, LAYOUT_F64X4 = 1, LAYOUT_BF16X4 = 2, LAYOUT_F16X4 = 3,
                        // cell-major copies for the precision form: the 8 corners of cell
                        // (i, j, k) at cell index (i*ny + j)*nz + k, corner (a, b, c) at 4a + 2b + c;
                        // FP32: 3 floats per corner (96 B per cell), BF16: 4 halves (64 B)
                        LAYOUT_F32_CELLS = 4, LAYOUT_BF16_CELLS = 5 };

struct FieldDev {
    const void* data;
    int32_t layout;
    int32_t nx, ny, nz;
    int32_t pow2;            // 1 if nx, ny, nz are all powers of two
    int32_t pad_;
    double inv_spacing;      // 1/spacing, rounded once
    double spacing;
    double ox, oy, oz;
    double oix, oiy, oiz;    // origin * (1/spacing), rounded once
    double scale;            // BF16/F16 multiplier (1 otherwise)
    // Modulation grid (Sec. 3.2 modulated grids): B(x) = M(x) b(x) with M a scalar FP32
    // periodic grid, node (i,j,k) at (i*mny + j)*mnz + k; nullptr when the field has none.
    const float* mod;
    int32_t mnx, mny, mnz, mpow2;
    double m_inv_spacing, m_spacing;
    double mox, moy, moz;
    double moix, moiy, moiz; // modulation origin * (1/spacing), rounded once
};

struct TablesDev {
    const double* loss;      // [species][n_nodes] log10 rate
    const double* pd;
    const float* loss_f;     // FP32 copies (precision form)
    const float* pd_f;
    const uint8_t* has_loss;
    const uint8_t* has_pd;
    int32_t z_max, n_max, n_nodes, pad_;
    double x0, inv_dx;
    float x0_f, inv_dx_f;    // the same rounded to FP32 (FP32 rate evaluation)
};

struct SimState {            // structure of arrays, `capacity` slots
    double *x, *y, *z, *ux, *uy, *uz, *E, *s, *hprop, *tau, *u0x, *u0y, *u0z;
    int32_t *A, *Z, *n_int, *status, *grid_id;
    int64_t *uid, *n_steps, *n_att;
};

// Particle status values (same numbers as CRP_STATUS_* in the public header).
constexpr int32_t CRP_STATUS_ACTIVE_ = 0;
constexpr int32_t CRP_STATUS_DONE_ = 1;
constexpr int32_t CRP_STATUS_NAN_ = 2;
constexpr int32_t CRP_STATUS_RANGE_ = 3;

// Device status bits.
enum : uint32_t {
    BIT_QUEUE_FULL = 1u,
    BIT_NAN = 2u,
    BIT_RANGE = 4u,
    BIT_INVALID = 8u,
    BIT_TIMEOUT = 16u,
    BIT_BOUNDS = 32u,       // a work-list entry or grid id out of range (skipped)
};

struct Counters {
    unsigned long long n_used;       // slots in use
    unsigned long long reserve;      // slot reservation counter during a launch
    unsigned long long count[2];     // entries in work list 0 / 1
    unsigned long long head[2];      // next position to pop, per work list
    unsigned long long n_done;       // entries in the done list
    unsigned long long accepted;     // cumulative accepted steps
    unsigned long long attempted;    // cumulative attempted steps
    unsigned long long secondaries;  // cumulative secondaries created
    unsigned long long launches;     // propagate kernel launches
    unsigned long long n_primaries;  // primaries injected (default uids)
    unsigned long long slices;       // slices run by the current propagate loop
    unsigned long long prev_accepted;
    unsigned int status_bits;
    unsigned int pad_;
};

struct PropArgs {
    SimState st;
    const FieldDev* fields;
    int32_t n_fields;
    int32_t has_tables;
    TablesDev tab;
    double tol, hmin, hmax, dmax;
    unsigned long long seed;
    long long max_steps;
    long long capacity;
    int32_t cadence;
    int32_t pickup;                  // take secondaries pushed during the launch
    int32_t list;                    // process list `list`, push secondaries to 1 - list
    int32_t* lists[2];
    int32_t* done_list;
    Counters* ctr;
    // reflective box (boundary = 1): per axis origin, origin + size, size, 1/size
    int32_t boundary;
    int32_t pad_;
    double box_lo[3], box_hi[3], box_len[3], box_inv[3];
};

// Launchers (defined in the kernel translation units).
// Sources and arrival maps (sources.cu).
int launch_source_sample(const SimState& S, long long first, long long n, unsigned long long uid_base,
                         const crp_spectrum& sp, unsigned long long seed, int grid, void* stream);
int launch_healpix(int nside, const double* u, long long n, long long* pix, int grid, void* stream);
int launch_arrival_map(const SimState& S, const Counters* C, int nside, double e_min,
                       unsigned long long* map, int grid, void* stream);

// Lenses (lens.cu).
int launch_lens_apply(int n_pix, int n_maps, int group, const long long* rs, const int* rl, const int* col,
                      const float* val, const double* x, double* y, int sms, void* stream);
int launch_lens_bin(const SimState& S, const Counters* C, int nside, int n_mat, const double* edges, double e_min,
                    double* x, int grid, void* stream);

// `mod`: 1 for simulations whose fields carry a modulation grid.
// p2: every vector grid of the launch has power-of-two sizes (the kernels then wrap cell
// indices with a mask; with p2 = 0 they take the general wrap, valid for any size).
int launch_propagate_fp64(const PropArgs& a, int layout, int mod, int p2, int grid, int block, void* stream);
int propagate_fp64_occupancy(int layout, int mod, int p2, int block, int* blocks_per_sm);
int launch_propagate_mixed(const PropArgs& a, int layout, int mod, int p2, int grid, int block, void* stream);
int propagate_mixed_occupancy(int layout, int mod, int p2, int block, int* blocks_per_sm);

// Diagnostics: every kernel counts its runs in a device counter of its own translation unit
// (one atomic per launch, by the first thread of the first block); kernel_runs_*() read them.
#define CRP_COUNT_RUN()                                                                         \
    do {                                                                                        \
        if ((threadIdx.x | threadIdx.y | threadIdx.z | blockIdx.x | blockIdx.y | blockIdx.z) == 0) \
            atomicAdd(&g_kernel_runs, 1ull);                                                    \
    } while (0)
unsigned long long kernel_runs_capi();
unsigned long long kernel_runs_fp64();
unsigned long long kernel_runs_mixed();
unsigned long long kernel_runs_adjoint();
unsigned long long kernel_runs_sources();
unsigned long long kernel_runs_lens();

// Adjoint launchers (adjoint.cu). Arrays are component-major [component][n] for y,
// [step][n] for h, [checkpoint][6][n] for checkpoints. `stages`, when not NULL, holds the
// stage records of every step: per step and particle kAdjRecordBytes (6 stages x (23 FP64:
// direction, field, Jacobian, corner weights + 8 int32 corner nodes)), doubles first.
constexpr size_t kAdjRecordBytes = 6 * (23 * sizeof(double) + 8 * sizeof(int32_t));
int adj_init(const double* x0, const double* p0, const int32_t* Z, double* y0, double* kappa,
             double* E, long long n, void* stream);
int adj_record(const FieldDev& F, const double* y0, const double* kappa, double tol, double hmin,
               double hmax, int n_steps, int K, double* h, double* ck, double* xT, double* uT,
               long long n, void* stream);
int adj_replay(const FieldDev& F, const double* y0, const double* kappa, const double* h, int n_steps,
               double* xT, double* uT, unsigned long long* cell_hash, long long n, void* stream);
// With `stages`, the records are formed in up to n_events - 1 chunks on `aux_stream` (events[0]
// orders it after `stream`, events[1 + j] hands chunk j to the reverse sweep on `stream`);
// aux_stream NULL: one chunk on `stream`.
int adj_backward(const FieldDev& F, const double* kappa, const double* h, const double* ck,
                 double* seg, double* stages, int n_steps, int K, const double* uT_bar, double* grid_bar,
                 double* y0_bar, double* kappa_bar, long long n, void* stream, void* aux_stream,
                 void* const* events, int n_events);
int adj_p0bar(const double* y0, const double* kappa, const double* E, const double* y0_bar,
              const double* kappa_bar, double* p0_bar, double* x0_bar, long long n, void* stream);

}  // namespace crp
