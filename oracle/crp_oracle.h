/*
 * crp_oracle.h -- plain FP64 CPU oracle for the 3D-mode propagation hot path of
 * "Cosmic ray propagation with CRPropa 3" (arXiv:1410.5323).
 *
 * TEST INFRASTRUCTURE. This library is the checker the GPU path is compared against.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg load it;
 * the product library never links, loads or calls it, and it shares no code with it.
 *
 * Units: lengths in metres, energies in eV, magnetic field in tesla.
 * Every function names the passage of the paper (section / equation) it follows;
 * the paper states the method only qualitatively, so every constant not in the
 * paper is a stated reading (Cash & Karp 1990 for the integrator, Salmon et al. 2011
 * for Philox4x32-10, Cody & Waite 1980 for the exp/log argument reduction).
 */
#ifndef CRP_ORACLE_H
#define CRP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Particle status values (shared meaning with the product library, separate code). */
#define ORC_ACTIVE 0
#define ORC_DONE 1        /* reached the trajectory-length limit (observer, paper Sec. 3.1) */
#define ORC_NAN 2         /* state became non-finite; particle stopped */
#define ORC_RANGE 3       /* species outside the interaction tables; particle stopped */

/* Return codes of orc_propagate / orc_inject. */
#define ORC_OK 0
#define ORC_ERR_INVALID_ARG (-1)
#define ORC_ERR_QUEUE_FULL (-4)

/* Grid storage types. */
#define ORC_F64 0
#define ORC_F32 1
#define ORC_BF16 2
#define ORC_F16 3

/* Regular periodic Cartesian vector grid (paper Sec. 3.2): node (i,j,k) sits at
 * origin + (i,j,k)*spacing and holds B at data[((i*ny + j)*nz + k)*3 + c]. */
typedef struct {
    const void* data;
    int32_t dtype;
    int32_t nx, ny, nz;
    int32_t pad_;
    double spacing;
    double origin[3];
    double scale;       /* multiplies BF16/F16 values; ignored for F32/F64 */
    /* Optional modulation (Sec. 3.2 modulated grids): a scalar periodic grid M, node (i,j,k)
     * at mod_origin + (i,j,k)*mod_spacing holding mod_data[(i*mod_ny + j)*mod_nz + k]
     * (F32 or F64); B(x) = M(x) * b(x) with both interpolated trilinearly. NULL: none. */
    const void* mod_data;
    int32_t mod_dtype;
    int32_t mod_nx, mod_ny, mod_nz;
    double mod_spacing;
    double mod_origin[3];
} orc_field;

/* Interaction tables on x = log10(Lorentz factor): node j at x0 + j/inv_dx.
 * Species index = Z*(n_max+1) + (A-Z). Values are log10 of a rate in 1/m.
 * has_* == 0 marks a species whose rate is identically zero. */
typedef struct {
    int32_t z_max, n_max, n_nodes, pad_;
    double x0, inv_dx;
    const double* log10_loss;   /* continuous-loss rate 1/lambda_loss  [species][n_nodes] */
    const double* log10_pd;     /* photo-disintegration rate            [species][n_nodes] */
    const uint8_t* has_loss;
    const uint8_t* has_pd;
} orc_tables;

typedef struct {
    double tol;          /* Cash-Karp error tolerance */
    double hmin, hmax;   /* propagation step limits, m */
    double dmax;         /* trajectory-length limit (observer), m */
    uint64_t seed;       /* Philox key */
    int64_t max_steps;   /* accepted steps per particle per call; <= 0: no limit */
    int32_t n_threads;   /* <= 0: one */
    int32_t boundary;    /* ORC_BOUNDARY_NONE or ORC_BOUNDARY_REFLECT */
    double box_origin[3];/* reflective box [origin, origin + size] per axis, m */
    double box_size[3];
} orc_params;

enum { ORC_BOUNDARY_NONE = 0, ORC_BOUNDARY_REFLECT = 1 };

/* Particle state, structure of arrays, `capacity` slots; slots [0, n) are in use. */
typedef struct {
    double *x, *y, *z, *ux, *uy, *uz, *E, *s, *hprop, *tau, *u0x, *u0y, *u0z;
    int32_t *A, *Z, *n_int, *status, *grid_id;
    int64_t *uid, *n_steps, *n_att;
    int64_t capacity;
    int64_t n;
} orc_state;

/* Source spectrum of Sec. 4, Eq. 1 (species i: mass A_i, charge Z_i, abundance x_i). */
#define ORC_MAX_SPECIES 8
#define ORC_SOURCE_DRAWS 64     /* draws per particle before a sample counts as failed */
typedef struct {
    int32_t n_species;
    int32_t A[ORC_MAX_SPECIES], Z[ORC_MAX_SPECIES];
    int32_t pad_;
    double x[ORC_MAX_SPECIES];
    double alpha;        /* spectral index */
    double rcut_v;       /* cutoff rigidity, V (E cutoff Z_i * rcut_v in eV) */
    double e_min_ev, e_max_ev;
} orc_spectrum;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint64_t seed, uint64_t uid, uint32_t k, uint32_t tag);
double orc_exp(double x);
double orc_log(double x);
void orc_field_value(const orc_field* f, const double x[3], double B[3]);
double orc_grid_value(const orc_field* f, int64_t i, int64_t j, int64_t k, int32_t c);
double orc_modulation_value(const orc_field* f, const double x[3]);
void orc_deriv(const orc_field* f, double kappa, const double y[6], double k[6]);
void orc_ck_attempt(const orc_field* f, double kappa, const double y[6], const double k1[6],
                    double h, double y5[6], double err[6]);
void orc_error_sums(const double err[6], double* sx, double* su);
int orc_error_accept(double sx, double su, double h, double tol);
float orc_ctrl_log2(double v);
float orc_ctrl_log2r(double sx, double su, double h, double tol);
float orc_ctrl_factor(float log2r, float p, float lo, float hi);
int orc_rates_f32(const orc_tables* t, int32_t A, int32_t Z, double E, float* r_loss, float* r_pd);
int orc_rates(const orc_tables* t, int32_t A, int32_t Z, double E, double* r_loss, double* r_pd);
int orc_inject(orc_state* st, int64_t first, int64_t count, uint64_t seed, const orc_tables* t);
int orc_propagate(orc_state* st, const orc_field* fields, int32_t n_fields, const orc_tables* t,
                  const orc_params* p, int64_t stats[4]);

/* Frozen-step differentiation (adjoint of the Cash-Karp map with recorded steps).
 * y = (x, u); kappa = Z c / E. */
int orc_record_steps(const orc_field* f, double kappa, const double y0[6], double tol, double hmin,
                     double hmax, int32_t n_steps, double* h_out, double yT[6]);
void orc_frozen_forward(const orc_field* f, double kappa, const double y0[6], const double* h,
                        int32_t n_steps, double yT[6]);
void orc_adjoint(const orc_field* f, double kappa, const double y0[6], const double* h,
                 int32_t n_steps, const double lamT[6], double* grid_bar, double y0_bar[6],
                 double* kappa_bar);

/* Sources (Sec. 4, Eq. 1) and arrival binning (HEALPix RING scheme). */
int orc_spectrum_check(const orc_spectrum* sp);
int64_t orc_source_sample(const orc_spectrum* sp, uint64_t seed, uint64_t uid_base, int64_t n,
                          int32_t* A, int32_t* Z, double* E, double* ux, double* uy, double* uz);
double orc_atan2(double y, double x);
int64_t orc_healpix_ring(int32_t nside, double x, double y, double z);
int orc_arrival_map(const orc_state* st, int32_t nside, double e_min_ev, uint64_t* map);

/* Lenses (Sec. 3.3): per-rigidity sparse matrices applied to arrival distributions. */
int orc_lens_apply(int32_t n_pix, int32_t n_mat, const int64_t* row_ptr, const int32_t* col,
                   const float* val, const double* x, int32_t n_maps, double* y);
int orc_lens_bin(const orc_state* st, int32_t nside, int32_t n_mat, const double* edges,
                 double e_min_ev, double* x);

#ifdef __cplusplus
}
#endif

#endif
