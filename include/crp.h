/*
 * crp.h -- C ABI of the GB300 3D-mode cosmic-ray propagation library (libcrp.so).
 *
 * Method: "Cosmic ray propagation with CRPropa 3" (arXiv:1410.5323). The library
 * advances batches of independent charged nuclei through a periodic gridded magnetic
 * field; every particle runs the per-step module sequence of Sec. 3.1 (propagation
 * with step-size bidding, continuous energy loss, photo-disintegration with nucleon
 * secondaries, observer) with the 3D deflection of Sec. 2 on the regular grids of
 * Sec. 3.2.
 *
 * Conventions for every entry point:
 *   - Units: lengths in metres, energies in eV, magnetic field in tesla.
 *   - Return value: CRP_OK (0) or a negative CRP_ERR_* code; crp_error_string() names
 *     it and crp_last_error_detail() gives the last failure's text (thread-local).
 *   - Pointers marked "host or device" are device pointers when the accompanying
 *     is_device flag is non-zero, host pointers otherwise. The library never keeps a
 *     caller pointer after the call returns (it copies), except where stated.
 *   - The library owns the device memory behind every handle; the caller owns every
 *     buffer it passes in.
 *   - `stream` is a cudaStream_t passed as void* (NULL: the legacy default stream).
 *     Calls taking a stream are asynchronous with respect to the host; crp_sync()
 *     waits and turns the device status word into a return code.
 *   - There is no CPU fallback: without a usable CUDA device every call that needs
 *     one returns CRP_ERR_CUDA.
 */
#ifndef CRP_H
#define CRP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define CRP_OK 0
#define CRP_ERR_INVALID_ARG (-1)   /* bad argument; nothing was changed */
#define CRP_ERR_OOM (-2)           /* device allocation failed */
#define CRP_ERR_CUDA (-3)          /* a CUDA runtime call failed (no device, launch error) */
#define CRP_ERR_QUEUE_FULL (-4)    /* a split found no free particle slot: the parent is
                                      parked at the start of that step; grow the simulation
                                      with crp_sim_reserve() and call crp_propagate() again */
#define CRP_ERR_TIMEOUT (-5)       /* crp_sync() wait limit reached (work still running) */
#define CRP_ERR_NAN_STATE (-6)     /* a particle state became non-finite; that particle was
                                      stopped with status CRP_STATUS_NAN */
#define CRP_ERR_TABLE_RANGE (-7)   /* a species fell outside the interaction tables; that
                                      particle was stopped with status CRP_STATUS_RANGE */

/* ---- enumerations ------------------------------------------------------------------ */
#define CRP_DTYPE_F64 0
#define CRP_DTYPE_F32 1
#define CRP_DTYPE_BF16 2
#define CRP_DTYPE_F16 3

#define CRP_FORM_FP64 0     /* FP64 stages, FP64 lookups; bit-identical to the FP64 reading. On
                               first use it builds an FP64 copy of each FP32/BF16/F16 grid
                               (32 B per node, kept with the field) so that no widening runs
                               on the FP64 pipe per lookup */
#define CRP_FORM_MIXED 1    /* FP32 local-frame stages, FP64 position and error norm */

#define CRP_STATUS_ACTIVE 0
#define CRP_STATUS_DONE 1   /* reached the trajectory-length limit (observer) */
#define CRP_STATUS_NAN 2
#define CRP_STATUS_RANGE 3

/* Particle-state columns for crp_read_state(). */
#define CRP_COL_X 0         /* f64 */
#define CRP_COL_Y 1
#define CRP_COL_Z 2
#define CRP_COL_UX 3
#define CRP_COL_UY 4
#define CRP_COL_UZ 5
#define CRP_COL_E 6
#define CRP_COL_S 7         /* path length travelled, m */
#define CRP_COL_HPROP 8     /* next propagation-step proposal, m (+inf before the first step) */
#define CRP_COL_TAU 9       /* remaining optical depth to the next photo-disintegration */
#define CRP_COL_U0X 10
#define CRP_COL_U0Y 11
#define CRP_COL_U0Z 12
#define CRP_COL_A 13        /* i32 */
#define CRP_COL_Z_CHARGE 14 /* i32 */
#define CRP_COL_N_INT 15    /* i32: photo-disintegrations so far */
#define CRP_COL_STATUS 16   /* i32: CRP_STATUS_* */
#define CRP_COL_GRID_ID 17  /* i32 */
#define CRP_COL_UID 18      /* i64 */
#define CRP_COL_N_STEPS 19  /* i64: accepted steps */
#define CRP_COL_N_ATT 20    /* i64: attempted Cash-Karp steps */
#define CRP_N_COLS 21

typedef struct crp_field crp_field;
typedef struct crp_tables crp_tables;
typedef struct crp_sim crp_sim;

/* ---- field (Sec. 3.2: regular Cartesian vector grid, periodic) ----------------------
 * grid: [nx][ny][nz][3] B values (C order, component fastest), dtype CRP_DTYPE_*,
 * host or device. Node (i,j,k) sits at origin_m + (i,j,k)*spacing_m; the grid repeats
 * with period (nx,ny,nz)*spacing_m. B = value (F32/F64) or value*scale (BF16/F16).
 * The library copies the grid into its own device layout (one float4/double4/half4
 * per node) and keeps nothing of the caller's buffer.
 * Errors: INVALID_ARG for NULL pointers, non-positive sizes, spacing <= 0, unknown
 * dtype, or a grid above 2^31 nodes; OOM; CUDA. */
int crp_field_create(const void* grid, int32_t dtype, int32_t is_device, int32_t nx,
                     int32_t ny, int32_t nz, double spacing_m, const double origin_m[3],
                     float scale, crp_field** out);
int crp_field_destroy(crp_field* field);

/* Modulated grid (Sec. 3.2, used so in Sec. 4): a small high-resolution vector grid b,
 * repeated periodically, times a large low-resolution scalar grid M that carries the
 * large-scale structure: B(x) = M(x) * b(x). M is interpolated trilinearly and periodically
 * over its own extent, exactly like b: fractional index r = (x - origin_m) / spacing_m per
 * axis, corners 000..111 weighted ((w_x w_y) w_z), and the product is taken after both
 * lookups (the FP64 form evaluates m * B_c for each component c).
 * mod: nx*ny*nz FP32 values (dtype must be CRP_DTYPE_F32), node (i,j,k) at (i*ny + j)*nz + k,
 * host (is_device = 0) or device memory; copied, the caller keeps ownership. A field takes
 * one modulation for its lifetime; simulations created from the field before this call keep
 * the unmodulated field. All fields of one simulation are modulated, or none (crp_sim_create
 * returns INVALID_ARG otherwise). The adjoint entry points reject modulated fields.
 * Errors: INVALID_ARG (NULL pointer, dtype not F32, sizes < 1, above 2^31 nodes, spacing
 * <= 0 or not finite, origin not finite, field already modulated); OOM; CUDA. */
int crp_field_modulate(crp_field* field, const void* mod, int32_t dtype, int32_t is_device,
                       int32_t nx, int32_t ny, int32_t nz, double spacing_m,
                       const double origin_m[3]);

/* ---- interaction tables (Sec. 2: pair-production loss, photo-disintegration) --------
 * Species s = Z*(n_max+1) + (A-Z), Z in [0,z_max], A-Z in [0,n_max]. Row s holds
 * n_nodes values of log10(rate in 1/m) on x = log10(gamma) = x0 + j/inv_dx, with
 * gamma = E/(A m_p c^2). log10_loss is the continuous-loss rate 1/lambda_loss,
 * log10_pd the photo-disintegration rate. has_loss[s] / has_pd[s] == 0 mark
 * identically-zero rates (the row is then ignored). All pointers are host pointers.
 * Errors: INVALID_ARG for NULL pointers, n_nodes < 2, inv_dx <= 0, non-finite values
 * in a flagged row; OOM; CUDA. */
int crp_tables_create(int32_t z_max, int32_t n_max, int32_t n_nodes, double x0, double inv_dx,
                      const double* log10_loss, const double* log10_pd,
                      const uint8_t* has_loss, const uint8_t* has_pd, crp_tables** out);
int crp_tables_destroy(crp_tables* tables);

/* ---- simulation -----------------------------------------------------------------------
 * fields: n_fields field handles (a particle's grid_id picks one); tables: NULL for no
 * interactions; seed: Philox key for interaction sampling; capacity: particle slots
 * (primaries + secondaries). The handles must outlive the simulation.
 * Errors: INVALID_ARG (n_fields < 1, NULL field, capacity < 1 or >= 2^31); OOM; CUDA. */
int crp_sim_create(const crp_field* const* fields, int32_t n_fields, const crp_tables* tables,
                   uint64_t seed, int64_t capacity, crp_sim** out);
/* Grow to `capacity` slots, keeping every particle (resumes after CRP_ERR_QUEUE_FULL).
 * Synchronises the simulation's last stream. */
int crp_sim_reserve(crp_sim* sim, int64_t capacity);
int crp_sim_destroy(crp_sim* sim);
/* Forget every particle (slots, done list, step counters, status word) and keep the
 * allocations, fields, tables and seed; uids continue from 0 again. Synchronises. */
int crp_sim_reset(crp_sim* sim);

/* Reflective boundary (Sec. 4: reflective boundary conditions let a finite volume stand for
 * sources at much larger distances). With CRP_BOUNDARY_REFLECT, after every accepted step a
 * position outside the box [origin_m, origin_m + size_m] (per axis, faces included in the
 * box) is folded back by mirror reflection: t = (x - o) * (1/L), k = floor(t), r = t - k,
 * x' = o + r L for even k, (o + L) - r L for odd k; an odd k reverses that component of the
 * direction and of the initial direction u0 (deflection angles stay in the mirrored frame).
 * Secondaries inherit the folded state. Applies to later crp_propagate / crp_propagate_loop
 * calls of this simulation; CRP_BOUNDARY_NONE (origin/size ignored, may be NULL) removes it.
 * Errors: INVALID_ARG (NULL sim, unknown kind, a size <= 0 or not finite, origin not finite). */
#define CRP_BOUNDARY_NONE 0
#define CRP_BOUNDARY_REFLECT 1
int crp_sim_set_boundary(crp_sim* sim, int32_t kind, const double origin_m[3], const double size_m[3]);

/* ---- source injection (Sec. 4: sources emit isotropically; positions/directions/
 * energies come from the caller) ----------------------------------------------------------
 * Appends n particles after the ones already present. Each needs A >= 1, -A <= Z <= A
 * (Z < 0: an antinucleus, for backward tracking from the observer, Sec. 3.3; only in a
 * simulation without tables), a species inside the tables (if any), uid < 2^32 (uid == NULL: uids continue the
 * count of primaries injected so far), 0 <= grid_id < n_fields (grid_id == NULL: 0).
 * The library initialises s = 0, no step proposal, the first optical depth
 * tau = -ln U(uid, 0, tag 0) (Philox), u0 = u, counters 0, status active.
 * Errors: INVALID_ARG (NULL columns, n < 0, capacity exceeded, an invalid particle when
 * the columns are host pointers; with device columns invalid particles are reported by
 * crp_sync as INVALID_ARG); CUDA. */
typedef struct {
    const double *x, *y, *z;
    const double *ux, *uy, *uz;
    const double* E;
    const int32_t *A, *Z;
    const int64_t* uid;        /* may be NULL */
    const int32_t* grid_id;    /* may be NULL */
    int32_t is_device;
    int32_t pad_;
} crp_particles;
int crp_source_inject(crp_sim* sim, const crp_particles* particles, int64_t n, void* stream);

/* ---- propagation (Sec. 3.1 module sequence; Sec. 2 3D deflection) ----------------------
 * Advances every active particle until it reaches max_distance_m (status DONE), or has
 * taken params->max_steps accepted steps in this call (stays active; a later call resumes
 * it bit-identically), or fails (NAN / RANGE). Secondaries created in the call are
 * propagated in the same call. Per step: bids h = min(clamp(proposal, min_step_m,
 * max_step_m), 0.1/R_loss, tau/R_pd, max_distance_m - s); Cash-Karp RK4(5) attempts
 * until the FP64 error ratio max(|dx|/h, |du|)/tolerance <= 1 (or h <= min_step_m);
 * continuous loss; photo-disintegration when the interaction bid was the step; observer.
 * Asynchronous on `stream`. Errors: INVALID_ARG (tolerance <= 0, min_step_m <= 0,
 * max_step_m < min_step_m, max_distance_m <= 0, unknown form); CUDA (launch failure). */
/* Grid layout read by the precision form (CRP_FORM_MIXED; the FP64 form always reads its
 * FP64 node copy). NODES: one 4-wide vector per node (16 B FP32, 8 B BF16), 8 scattered
 * corner reads per lookup. CELLS: a cell-major copy holding the 8 corners of every cell
 * contiguously (FP32: 8 x 3 floats = 96 B; BF16: 8 x 4 halves = 64 B), periodic wrap
 * included, read with 3 (FP32) or 2 (BF16) 32-byte loads per lookup; it takes 6x (FP32) or
 * 8x (BF16) the node grid's device memory, is built on first use and freed with the field,
 * and gives results identical to NODES (the same corner values in the same arithmetic).
 * AUTO: CELLS when the copies of all the simulation's fields fit in free device memory with
 * 4 GiB to spare, else NODES. CELLS when they do not fit: CRP_ERR_OOM. */
#define CRP_GRID_AUTO 0
#define CRP_GRID_NODES 1
#define CRP_GRID_CELLS 2

/* The layout the precision form reads under CRP_GRID_AUTO: CRP_GRID_CELLS once the
 * simulation's cell-major copies are built (by a precision-form call that found room for
 * them), else CRP_GRID_NODES. sim and layout non-NULL, else CRP_ERR_INVALID_ARG. */
int crp_sim_grid_layout(const crp_sim* sim, int32_t* layout);

typedef struct {
    int32_t form;            /* CRP_FORM_FP64 or CRP_FORM_MIXED */
    int32_t block_size;      /* threads per block, multiple of 32; 0: default */
    int32_t blocks_per_sm;   /* 0: the occupancy limit */
    int32_t cadence;         /* attempts between refill checks; 0: default (2 in the precision form, 1 in FP64) */
    int64_t max_steps;       /* accepted steps per particle per call; <= 0: no limit */
    int32_t order;           /* work-list order: CRP_ORDER_* (0: default = CRP_ORDER_COST) */
    int32_t pickup;          /* secondaries created in a launch: CRP_PICKUP_* (0: default = OFF) */
    int32_t grid_layout;     /* precision form: CRP_GRID_* (0: default = AUTO) */
    int32_t pad_;
} crp_params;
/* Scheduling choices (never change a particle's result, only when it runs). */
#define CRP_ORDER_DEFAULT 0
#define CRP_ORDER_SLOT 1         /* slot (injection) order */
#define CRP_ORDER_COST 2         /* lowest rigidity E/Z first: expected longest first */
#define CRP_ORDER_GRID 3         /* by grid_id, then lowest rigidity first: concurrent particles
                                    share field realisations (cache locality over many grids) */
#define CRP_PICKUP_DEFAULT 0
#define CRP_PICKUP_OFF 1         /* secondaries wait for the second launch */
#define CRP_PICKUP_ON 2          /* idle warps take secondaries pushed earlier in the launch */
int crp_propagate(crp_sim* sim, const crp_params* params, double tolerance, double min_step_m,
                  double max_step_m, double max_distance_m, void* stream);

/* The batching form of the propagation: slices of params->max_steps accepted steps per
 * particle (must be > 0 to make slices; <= 0 runs everything in one slice), repeated on the
 * device until no particle is active, the device status word reports an error, a slice
 * made no progress, or max_slices slices ran. Between slices the work list is rebuilt from
 * the active particles, so long-lived particles are packed into full warps again. The whole
 * loop is one CUDA graph (a conditional while node around the captured propagate sequence),
 * built on the first call and reused while the arguments and the simulation's buffers are
 * unchanged: one graph launch, no host round trip per slice. Results are the same as
 * repeated crp_propagate calls with the same max_steps. Asynchronous on `stream`.
 * Errors: as crp_propagate; INVALID_ARG for max_slices < 1; CUDA. */
int crp_propagate_loop(crp_sim* sim, const crp_params* params, double tolerance,
                       double min_step_m, double max_step_m, double max_distance_m,
                       int32_t max_slices, void* stream);

/* Wait for the simulation's last stream (at most timeout_s seconds; <= 0: no limit),
 * then return the first device-side error as a code: QUEUE_FULL, NAN_STATE,
 * TABLE_RANGE, INVALID_ARG, or CRP_OK. Clears the reported bits. */
int crp_sync(crp_sim* sim, double timeout_s);

/* counts[8] = {slots in use, active, done, accepted steps, attempted steps, secondaries
 * created, propagate kernel launches, device status bits}; the step counters are
 * cumulative over the simulation. Synchronises. */
int crp_sim_counts(crp_sim* sim, int64_t counts[8]);

/* Copy `count` entries of column `column` (CRP_COL_*) starting at slot `first` into dst
 * (host or device). Element type as listed with the CRP_COL_* values. Synchronises when
 * dst is a host pointer. Errors: INVALID_ARG (range, column). */
int crp_read_state(crp_sim* sim, int32_t column, void* dst, int32_t dst_is_device,
                   int64_t first, int64_t count);

/* ---- observer records (Sec. 3.1 observers) ---------------------------------------------
 * Copies the records of particles that have finished (status != ACTIVE), in the order
 * they finished, starting at the `first`-th finished particle, at most `capacity`
 * records; *n_out receives the number written. Caller-allocated columns, host or device;
 * NULL columns are skipped. Host columns that are all page-locked (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) are written by the gather kernel directly; other host
 * columns go through a device staging block (allocated and freed by the call). The call
 * waits for the device; columns must hold `capacity` entries. */
typedef struct {
    int64_t* uid;
    int32_t *A, *Z, *n_int, *status;
    double *E, *x, *y, *z, *ux, *uy, *uz, *u0x, *u0y, *u0z, *s;
    int64_t *n_steps, *n_att;
    int32_t is_device;
    int32_t pad_;
} crp_observer;
int crp_observe(crp_sim* sim, const crp_observer* out, int64_t first, int64_t capacity,
                int64_t* n_out);

/* ---- differentiation through a frozen step sequence (Sec. 2 deflection, Sec. 3.2 grid) --
 * The FP64 propagation module alone (no loss, interactions or distance limit) for n
 * particles through one field: crp_adjoint_forward records the accepted step sizes h_n of
 * n_steps steps with the adaptive Cash-Karp controller and checkpoints (x, u) every
 * checkpoint_every steps; crp_adjoint_backward differentiates the map with the recorded h_n
 * held fixed (the controller is not differentiated), recomputing each segment from its
 * checkpoint. Initial momenta p0 are in eV/c: E = |p0|, u0 = p0/E, kappa = Z c / E.
 * All array arguments are device pointers; [n][3] arrays are row-major.
 * Memory owned by the handle: 8 B x n x (n_steps + 6 (n_steps / checkpoint_every + 1) +
 * 6 (checkpoint_every + 1) + 20), plus 1296 B x n x n_steps for the stage records of every
 * step (direction, field, Jacobian, corner weights and corner nodes of its six stages) when
 * that fits in half of the device's free memory at creation and the grid has fewer than 2^31
 * nodes. With the records, the backward pass forms them for all checkpoint segments in
 * parallel, in chunks on a CUDA stream the handle owns (ordered after the caller's stream,
 * and the caller's stream after it, with events the handle owns), while the reverse sweep
 * consumes the chunks already formed; without them it recomputes one segment at a time
 * inside the reverse sweep. The results are the same either way. */
typedef struct crp_adjoint crp_adjoint;
int crp_adjoint_create(const crp_field* field, int64_t n, int32_t n_steps,
                       int32_t checkpoint_every, crp_adjoint** out);
int crp_adjoint_destroy(crp_adjoint* adj);
/* x0, p0: [n][3]; Z: [n]; outputs xT, uT: [n][3] after n_steps accepted steps. */
int crp_adjoint_forward(crp_adjoint* adj, const double* x0, const double* p0, const int32_t* Z,
                        double tolerance, double min_step_m, double max_step_m, double* xT,
                        double* uT, void* stream);
/* The recorded step sequence again, on `field` (NULL: the handle's; otherwise same grid
 * geometry) and/or from other initial momenta p0 ([n][3], NULL: the recorded ones), x0 as
 * recorded. For finite differences and sensitivity studies. cell_hash (may be NULL) receives
 * per particle a hash of the cell of every stage lookup: the trilinear field is only
 * continuous across cell faces, so a difference quotient is a derivative only where the
 * perturbed replays visit the same cells. */
int crp_adjoint_replay(crp_adjoint* adj, const crp_field* field, const double* p0, double* xT,
                       double* uT, uint64_t* cell_hash, void* stream);
/* uT_bar = dL/du_T [n][3]. grid_bar: [nx][ny][nz][3] FP64, accumulated (the caller zeroes
 * it); p0_bar = dL/dp0 [n][3]; x0_bar = dL/dx0 [n][3] (may be NULL). */
int crp_adjoint_backward(crp_adjoint* adj, const double* uT_bar, double* grid_bar, double* p0_bar,
                         double* x0_bar, void* stream);
/* Recorded step sizes, [n_steps][n] (host or device). */
int crp_adjoint_read_steps(crp_adjoint* adj, double* h, int32_t is_device);

/* ---- sources with the Sec. 4 spectrum (Eq. 1) ---------------------------------------------
 * dN_i/dE ~ x_i A_i^(alpha-1) E^-alpha exp(-E / (Z_i rcut_v)) on [e_min_ev, e_max_ev] for
 * species i = (A_i, Z_i, x_i), i < n_species <= CRP_MAX_SPECIES (Sec. 4 uses alpha = 1.8,
 * rcut_v = 10^19.8 V and H, He-4, N-14, Fe-56 with x = 1, 0.5, 0.3, 0.1). */
#define CRP_MAX_SPECIES 8
typedef struct {
    int32_t n_species;
    int32_t A[CRP_MAX_SPECIES], Z[CRP_MAX_SPECIES];   /* 1 <= Z <= A */
    int32_t pad_;
    double x[CRP_MAX_SPECIES];                        /* relative abundances, >= 0, not all 0 */
    double alpha;                                     /* spectral index */
    double rcut_v;                                    /* cutoff rigidity, V */
    double e_min_ev, e_max_ev;                        /* 0 < e_min < e_max */
} crp_spectrum;

/* Appends n primaries at the given positions (x, y, z: n metres each; grid_id: n values or
 * NULL for 0; host or device memory per is_device) whose species, energy and direction the
 * library draws on the device: species i with weight x_i A_i^(alpha-1) and E from E^-alpha
 * by its inverse CDF, the pair kept with probability exp(-E / (Z_i rcut_v)) and redrawn whole
 * otherwise (so the kept pairs follow Eq. 1 jointly), the direction isotropic by Marsaglia's
 * method. Random numbers: Philox4x32-10 keyed by the simulation seed, counter (uid, draw k,
 * tag) with tag 2 for (species, energy), 3 for the acceptance, 4 for the direction; uids
 * continue the count of primaries; powers and exponentials by the library's exp/log. A
 * particle whose CRP_SOURCE_DRAWS draws were all rejected is stopped at injection and
 * reported by crp_sync as INVALID_ARG. Then as crp_source_inject (s = 0, u0 = u, ...).
 * Errors: INVALID_ARG (NULL sim, spec or position column, n < 0, capacity exceeded, invalid
 * spectrum, a species outside the tables); CUDA. */
#define CRP_SOURCE_DRAWS 64
int crp_source_sample(crp_sim* sim, const crp_spectrum* spec, const double* x, const double* y,
                      const double* z, const int32_t* grid_id, int32_t is_device, int64_t n,
                      void* stream);

/* ---- arrival maps (Sec. 4, Fig. 4) -------------------------------------------------------
 * HEALPix RING-scheme pixel (Gorski et al. 2005) of each direction u[k] = (x, y, z) (device,
 * [n][3], not necessarily unit) for 1 <= nside <= 8192; pix: n int64 (device), -1 for a zero
 * or non-finite direction. phi comes from the library's atan2 (octant reduction, tan(pi/8)
 * split, half-angle step, Taylor series through c^27), so that maps are reproducible. */
int crp_healpix_ring(int32_t nside, const double* u, int64_t n, int64_t* pix, void* stream);
/* Adds to map (device, 12 nside^2 uint64, the caller zeroes it) one count per finished
 * particle (status DONE) with E > e_min_ev in the pixel of its arrival direction -u. */
int crp_arrival_map(crp_sim* sim, int32_t nside, double e_min_ev, uint64_t* map, void* stream);

/* ---- lenses (Sec. 3.3) ----------------------------------------------------------------------
 * A lens is a set of n_mat sparse matrices, one per rigidity bin, that map cosmic-ray
 * directions at the galactic border (columns) to arrival directions at Earth (rows), both
 * binned into n_pix pixels (12 nside^2 for HEALPix RING maps). CSR over shared arrays:
 * matrix m, row p holds entries k in [row_ptr[m (n_pix + 1) + p], row_ptr[m (n_pix + 1) + p + 1])
 * with column col[k] in [0, n_pix) and value val[k] (single precision, as lenses are
 * stored). The matrices are stored one after the other: row_ptr starts at 0, is
 * nondecreasing inside each matrix, and each matrix starts where the previous one ends;
 * nnz = the last offset. edges: n_mat + 1 strictly increasing positive rigidities in V, the
 * bin limits used by crp_lens_bin (NULL: no binning). All host pointers, copied to the device.
 * Errors: INVALID_ARG (sizes < 1, NULL arrays, offsets or columns out of range, bad edges);
 * OOM; CUDA. */
typedef struct crp_lens crp_lens;
int crp_lens_create(int32_t n_pix, int32_t n_mat, const int64_t* row_ptr, const int32_t* col,
                    const float* val, const double* edges, crp_lens** out);
int crp_lens_destroy(crp_lens* lens);
/* Lanes that share one row when a single map is applied: 4, 8, 16 or 32 (a tuning choice; the
 * default is the mean merged row length in 4-entry vectors, rounded up to a power of two in
 * [4, 32]). The sum stays within the same FP64 bound for any choice. Errors: INVALID_ARG. */
int crp_lens_set_group(crp_lens* lens, int32_t lanes_per_row);
/* Observed maps through the lens: y[p][b] = sum over m of (M_m x_m)[p][b] in FP64, each
 * entry added with one rounding (fused multiply-add), for n_maps maps at once. x: device,
 * [n_mat][n_pix][n_maps] FP64 (map b of rigidity bin m at the galactic border); y: device,
 * [n_pix][n_maps] FP64, overwritten. For several maps each row sums its entries in stored
 * order (matrix 0's row first); for one map the lanes that share a row add partial sums in an
 * unspecified order. */
int crp_lens_apply(const crp_lens* lens, const double* x, double* y, int32_t n_maps, void* stream);
/* The lens input from a simulation: adds to x (device, [n_mat][12 nside^2] FP64; the caller
 * zeroes it; needs n_pix = 12 nside^2) one count per finished particle with Z > 0 and
 * E > e_min_ev, in rigidity bin m (edges[m] <= E/Z < edges[m+1]; outside all bins: none) and
 * the HEALPix RING pixel of -u. */
int crp_lens_bin(const crp_lens* lens, crp_sim* sim, int32_t nside, double e_min_ev, double* x,
                 void* stream);

/* ---- diagnostics and fault injection (no counterpart in the paper) ----------------------
 * crp_debug_fail_allocations(n): the library's next n device allocations fail as if the device
 * were out of memory (every entry point that allocates then returns CRP_ERR_OOM and frees
 * what it had taken); 0 disarms. For testing the error paths without exhausting a GPU.
 * crp_selftest_wait(limit, preset, stream): runs the kernels' bounded wait (limit polls of
 * 64 ns) on a device flag initialised to `preset`; a flag that is never set (preset < 0)
 * makes the wait run out and the call return CRP_ERR_TIMEOUT, preset >= 0 returns CRP_OK.
 * Synchronises `stream`; the context stays usable either way. */
int crp_debug_fail_allocations(int32_t n);
int crp_selftest_wait(int32_t limit, int32_t preset, void* stream);

/* crp_kernel_runs(count): how many of this library's kernels have run on the current device
 * since the library was loaded, including those launched from inside the propagate loop's
 * CUDA graph (every kernel counts its own launches on the device). Synchronises the device;
 * *count is written on CRP_OK. For benchmarks and tests (no counterpart in the paper). */
int crp_kernel_runs(uint64_t* count);

/* ---- propagation that allocates nothing -------------------------------------------------
 * This entry point has no counterpart in the paper; it exists for callers that must not
 * have this library allocate device memory. Some host programs own every byte of GPU
 * memory themselves: a framework with its own pooled allocator, where a library's
 * cudaMalloc would fragment the pool or fail against a budget the host already handed
 * out, or a long-running service whose device footprint is fixed at start-up. Such
 * callers cannot use crp_sim_create / crp_field_create, which allocate. Here the caller
 * passes every input and output buffer, and the bookkeeping the propagate kernel needs
 * (counters, work lists, done list) lives in one static device array inside the library,
 * of CRP_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds until
 * the process exits.
 *
 * What it does: for particles 0..n-1 in `cols` (device pointers, each column at least n
 * entries; the caller fills x, y, z, ux, uy, uz, E, A, Z and uid < 2^32) it initialises
 * the bookkeeping columns exactly as crp_source_inject does (grid_id = 0) and propagates
 * them in the FP64 form without interactions through one field, exactly as
 * crp_propagate does, to max_distance_m or max_steps accepted steps (<= 0: no limit).
 * The field is `grid_f32x4`: a device pointer, 16-byte aligned, to nx*ny*nz float4 nodes
 * (x, y, z components, fourth lane ignored), node (i,j,k) at index (i*ny + j)*nz + k.
 * The call synchronises `stream` (it waits for the work to finish), reads the device
 * status word back and returns CRP_OK or that status as the code crp_sync would give:
 * CRP_ERR_NAN_STATE (non-finite state), CRP_ERR_INVALID_ARG (an invalid particle),
 * CRP_ERR_CUDA (a work-list entry out of range was skipped, e.g. when two calls overlap
 * on the shared array; particles may then be left unpropagated), CRP_ERR_TIMEOUT,
 * CRP_ERR_QUEUE_FULL, CRP_ERR_TABLE_RANGE (not reachable without interactions).
 *
 * Limits and sharing: n <= CRP_NOALLOC_MAX_PARTICLES, else CRP_ERR_INVALID_ARG and nothing
 * runs. The first call on a device looks up the static array's device address (once per
 * device, with that device current). Every call reuses the same array and clears what
 * must start at zero, so calls that overlap on the GPU (from several host threads or
 * streams) race: serialise them.
 * It never calls cudaMalloc, cudaFree or any allocating routine. */
#define CRP_NOALLOC_MAX_PARTICLES 262144
#define CRP_NOALLOC_SCRATCH_BYTES (512 + 3 * 4 * CRP_NOALLOC_MAX_PARTICLES)
typedef struct {
    double *x, *y, *z, *ux, *uy, *uz, *E, *s, *hprop, *tau, *u0x, *u0y, *u0z;
    int32_t *A, *Z, *n_int, *status, *grid_id;
    int64_t *uid, *n_steps, *n_att;
} crp_state_columns;
int crp_propagate_noalloc(const void* grid_f32x4, int32_t nx, int32_t ny, int32_t nz,
                          double spacing_m, const double origin_m[3],
                          const crp_state_columns* cols, int64_t n, uint64_t seed,
                          double tolerance, double min_step_m, double max_step_m,
                          double max_distance_m, int64_t max_steps, void* stream);

const char* crp_error_string(int32_t code);
const char* crp_last_error_detail(void);

/* Library build identifier, e.g. "crp 1 sm_103a". */
const char* crp_version(void);

#ifdef __cplusplus
}
#endif
#endif
