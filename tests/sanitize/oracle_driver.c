/* Exercises every oracle entry point on small inputs; built with AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_oracle_sanitizers.py. Exit status 0 = clean. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "crp_oracle.h"

#define N 8
#define MAXP 4096

static double uni(uint64_t* s)
{
    *s = *s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(*s >> 11) * 0x1p-53;
}

int main(void)
{
    uint64_t rs = 12345;
    /* vector grid N^3 x 3 (F32) and a modulation grid 5 x 6 x 7 */
    float* g = malloc(sizeof(float) * N * N * N * 3);
    for (int i = 0; i < N * N * N * 3; ++i) g[i] = (float)((uni(&rs) - 0.5) * 2e-13);
    float* m = malloc(sizeof(float) * 5 * 6 * 7);
    for (int i = 0; i < 5 * 6 * 7; ++i) m[i] = (float)(0.5 + uni(&rs));
    const double MPC = 3.0856775814913673e22;
    orc_field f;
    memset(&f, 0, sizeof f);
    f.data = g; f.dtype = ORC_F32; f.nx = f.ny = f.nz = N;
    f.spacing = 0.25 * MPC;
    f.mod_data = m; f.mod_dtype = ORC_F32; f.mod_nx = 5; f.mod_ny = 6; f.mod_nz = 7;
    f.mod_spacing = 0.7 * MPC;

    /* tables: constant loss and photo-disintegration rates for Z <= 26, N <= 30 */
    const int zmax = 26, nmax = 30, nodes = 201;
    const int nsp = (zmax + 1) * (nmax + 1);
    double* ll = malloc(sizeof(double) * nsp * nodes);
    double* lp = malloc(sizeof(double) * nsp * nodes);
    uint8_t* hl = calloc(nsp, 1);
    uint8_t* hp = calloc(nsp, 1);
    for (int s = 0; s < nsp; ++s) {
        int Z = s / (nmax + 1), A = Z + s % (nmax + 1);
        hl[s] = Z > 0;
        hp[s] = A > 1;
        for (int j = 0; j < nodes; ++j) {
            ll[s * nodes + j] = log10(1.0 / (300.0 * MPC)) + 0.001 * j;
            lp[s * nodes + j] = log10(1.0 / (5.0 * MPC));
        }
    }
    orc_tables t = {zmax, nmax, nodes, 0, 6.0, 25.0, ll, lp, hl, hp};

    /* state: 64 primaries (He, N, Fe), room for their nucleons */
    orc_state st;
    memset(&st, 0, sizeof st);
    double** dcols[] = {&st.x, &st.y, &st.z, &st.ux, &st.uy, &st.uz, &st.E, &st.s, &st.hprop,
                        &st.tau, &st.u0x, &st.u0y, &st.u0z};
    for (size_t c = 0; c < sizeof dcols / sizeof dcols[0]; ++c) *dcols[c] = calloc(MAXP, sizeof(double));
    int32_t** icols[] = {&st.A, &st.Z, &st.n_int, &st.status, &st.grid_id};
    for (size_t c = 0; c < sizeof icols / sizeof icols[0]; ++c) *icols[c] = calloc(MAXP, sizeof(int32_t));
    int64_t** lcols[] = {&st.uid, &st.n_steps, &st.n_att};
    for (size_t c = 0; c < sizeof lcols / sizeof lcols[0]; ++c) *lcols[c] = calloc(MAXP, sizeof(int64_t));
    st.capacity = MAXP;
    const int np = 64;
    const int32_t As[3] = {4, 14, 56}, Zs[3] = {2, 7, 26};
    for (int i = 0; i < np; ++i) {
        double w = 2 * uni(&rs) - 1, ph = 6.283185307179586 * uni(&rs), sw = sqrt(1 - w * w);
        st.x[i] = uni(&rs) * 2 * MPC; st.y[i] = uni(&rs) * 2 * MPC; st.z[i] = uni(&rs) * 2 * MPC;
        st.ux[i] = sw * cos(ph); st.uy[i] = sw * sin(ph); st.uz[i] = w;
        st.E[i] = 1e19 * (1 + uni(&rs));
        st.A[i] = As[i % 3]; st.Z[i] = Zs[i % 3]; st.uid[i] = i;
    }
    if (orc_inject(&st, 0, np, 7, &t) != ORC_OK) return 2;
    orc_params p;
    memset(&p, 0, sizeof p);
    p.tol = 1e-4; p.hmin = 1e-3 * MPC; p.hmax = MPC; p.dmax = 20 * MPC; p.seed = 7; p.n_threads = 2;
    p.boundary = ORC_BOUNDARY_REFLECT;
    for (int a = 0; a < 3; ++a) { p.box_origin[a] = 0.0; p.box_size[a] = 3 * MPC; }
    int64_t stats[4];
    if (orc_propagate(&st, &f, 1, &t, &p, stats) != ORC_OK) return 3;
    if (stats[3] <= 0) return 4;

    /* sources, sky, maps, lenses */
    orc_spectrum sp;
    memset(&sp, 0, sizeof sp);
    sp.n_species = 4;
    const int32_t sa[4] = {1, 4, 14, 56}, sz[4] = {1, 2, 7, 26};
    const double sx[4] = {1, 0.5, 0.3, 0.1};
    for (int i = 0; i < 4; ++i) { sp.A[i] = sa[i]; sp.Z[i] = sz[i]; sp.x[i] = sx[i]; }
    sp.alpha = 1.8; sp.rcut_v = pow(10.0, 19.8); sp.e_min_ev = 1e18; sp.e_max_ev = 1e21;
    int32_t A[100], Z[100];
    double E[100], ux[100], uy[100], uz[100];
    if (orc_source_sample(&sp, 3, 0, 100, A, Z, E, ux, uy, uz) != 0) return 5;
    for (int i = 0; i < 100; ++i)
        if (orc_healpix_ring(64, ux[i], uy[i], uz[i]) < 0) return 6;
    uint64_t map[12 * 4 * 4];
    memset(map, 0, sizeof map);
    if (orc_arrival_map(&st, 4, 1e18, map) != ORC_OK) return 7;
    const int npix = 48, nmat = 2;
    int64_t rp[2 * 49];
    int32_t col[2 * 48];
    float val[2 * 48];
    for (int mm = 0; mm < nmat; ++mm)
        for (int q = 0; q <= npix; ++q) rp[mm * (npix + 1) + q] = mm * npix + q;
    for (int k = 0; k < nmat * npix; ++k) { col[k] = (k * 7) % npix; val[k] = 0.5f; }
    double xm[2 * 48], ym[48];
    for (int k = 0; k < nmat * npix; ++k) xm[k] = k;
    if (orc_lens_apply(npix, nmat, rp, col, val, xm, 1, ym) != ORC_OK) return 8;
    const double edges[3] = {1e17, 1e19, 1e21};
    double xb[2 * 12 * 4 * 4];
    memset(xb, 0, sizeof xb);
    if (orc_lens_bin(&st, 4, 2, edges, 1e18, xb) != ORC_OK) return 9;

    /* frozen steps and the adjoint */
    f.mod_data = NULL;
    double y0[6] = {MPC, MPC, MPC, 1, 0, 0}, yT[6], h[40], lam[6] = {0, 0, 0, 1, 0, 0}, y0b[6], kb;
    const double kappa = 299792458.0 / 1e19;
    if (orc_record_steps(&f, kappa, y0, 1e-4, 1e-3 * MPC, MPC, 40, h, yT) != ORC_OK) return 10;
    orc_frozen_forward(&f, kappa, y0, h, 40, yT);
    double* gb = calloc(N * N * N * 3, sizeof(double));
    orc_adjoint(&f, kappa, y0, h, 40, lam, gb, y0b, &kb);
    printf("ok %lld accepted, %lld secondaries\n", (long long)stats[0], (long long)stats[3]);
    free(gb); free(g); free(m); free(ll); free(lp); free(hl); free(hp);
    for (size_t c = 0; c < sizeof dcols / sizeof dcols[0]; ++c) free(*dcols[c]);
    for (size_t c = 0; c < sizeof icols / sizeof icols[0]; ++c) free(*icols[c]);
    for (size_t c = 0; c < sizeof lcols / sizeof lcols[0]; ++c) free(*lcols[c]);
    return 0;
}
