/*
 * swdg_oracle.h -- plain FP64 CPU oracle for the sub-grid DG shallow-water
 * operator and its IMEX Runge-Kutta stage update (Arpaia, Orlando, Ferrarin,
 * Bonaventura, "High-order adaptive discontinuous finite elements for the
 * shallow water equations with sub-grid irregular bathymetry", arXiv 2505.18743).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this code: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library; both sides receive the same seeded inputs and nothing else.
 *
 * Every routine evaluates the paper's definitions directly: each basis
 * function at each point, dense per-cell matrices solved by Gaussian
 * elimination, and each sub-grid integral as an explicit sum over the pixels
 * that overlap the sampling rectangle.  No sum factorisation, no fast paths.
 *
 * Conventions (shared with the library only through the documented C-ABI
 * semantics, not through code):
 *   - cell K = [x0, x0+hx] x [y0, y0+hy], reference coordinates in [0,1]^2;
 *   - nodal DoFs on the (r+1)^2 Gauss-Lobatto support points, index a + (r+1) b,
 *     x fastest (Sec. 3.2);
 *   - nbr[K][f][s]: faces f = 0 W, 1 E, 2 S, 3 N; slot s = 0 is the neighbour
 *     (or -1-tag for a boundary face), slot 1 the second fine neighbour of a
 *     2:1 hanging face (ordered by increasing tangential coordinate) or -1;
 *   - raster: row-major [ny][nx], value z_b = bathymetry depth, positive down,
 *     so h = max(zeta + z_b, 0) (Eq. zeta2depth-2).
 */
#ifndef SWDG_ORACLE_H
#define SWDG_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora ora;

typedef struct {
    int degree;          /* r in 1..3 */
    int subgrid_mode;    /* 0: S (pixel sub-cells), 1: P (point samples) */
    int tableau;         /* 0 RK32/TR-BDF2 IMEX, 1 SSP33, 2 RK44, 3 forward Euler */
    double g, eps_vel, h_lim, eps0, cfl;
    int newton_max;
    double newton_tol;
} ora_config;

/* create / destroy; the oracle copies every input */
ora* ora_create(const ora_config* cfg, int64_t n_cells, const double* x0y0,
                const double* hxhy, const int32_t* nbr, const double* raster,
                int64_t nx, int64_t ny, double xo, double yo, double dx, double dy);
void ora_destroy(ora* o);
const char* ora_error(void);

int ora_set_boundary(ora* o, int tag, int kind, double amp, double period, double phase);
int ora_set_manning(ora* o, const double* n_per_cell);
/* tracer numerical diffusivity nu_c per cell (Eq. numdiff: -sum_K int nu_c h
 * grad c . grad psi_i added to R); NULL: none (the default) */
int ora_set_tracer_diffusivity(ora* o, const double* nu);
int ora_set_state(ora* o, const double* zeta, const double* qx, const double* qy, const double* c);
int ora_get_state(const ora* o, double* zeta, double* qx, double* qy, double* c);
int ora_get_flags(const ora* o, uint8_t* flags);

/* residual (F, G, R, L of Eqs. mass_rhs, discharge_rhs, r_concentration,
 * discharge_rhs_implicit) of the current state at time t, for all cells or the
 * listed ones (cells == NULL: all; outputs then [n][nd], else [n_sel][nd]) */
int ora_residual(ora* o, double t, int64_t n_sel, const int64_t* cells, double* F,
                 double* Gx, double* Gy, double* R, double* Lx, double* Ly);
/* C_cfl * min J_K / (lambda l_Gamma) over all face points of the current state */
int ora_cfl_dt(ora* o, double t, double* dt);
/* the degree switch of Eq. criteria_p with its remap (start of a step) */
int ora_degree_switch(ora* o);
/* n time steps; dt_or_neg < 0: CFL time step */
int ora_step(ora* o, int n_steps, double dt_or_neg, double* t_inout);
/* mass, tracer mass, min h, r-cells, max Newton its (last step), positivity
 * violations (cumulative), last dt, t */
int ora_diagnostics(ora* o, double out[8]);
int ora_gauges(const ora* o, int n, const double* xy, double* zeta_out);
/* Definition 3.1: lake at rest at elevation zeta0 */
int ora_lake_at_rest(const ora* o, double zeta0, double* zeta_out);
/* per-cell wet mass Hbar_K (Eq. positivity-7) of the current state */
int ora_cell_mass(const ora* o, double* hbar);

/* unit-level hooks used by the pins */
int ora_rule(int kind, int n, double* nodes, double* weights); /* 0 GL, 1 GLL on [0,1] */
/* V and A of Sec. 3.3 on the physical rectangle [X0,X1]x[Y0,Y1] (mode S) */
int ora_subgrid_rect(const ora* o, double X0, double X1, double Y0, double Y1,
                     double eta, double* V, double* A);
/* V, A at point p of point set s (0 vol GL, 1 mass GLL, 2 momentum GL) of cell K */
int ora_subgrid_point(const ora* o, int64_t K, int set, int p, double eta, double* V, double* A);
/* bathymetry depth at a physical point by bilinear interpolation (mode P) */
double ora_zb_point(const ora* o, double x, double y);
/* one face point of the Rusanov flux with hydrostatic reconstruction (Eqs.
 * lxf_parameter, velocity, hydro_rec, hydro_rec_vars) in mode P:
 * in = {zm, qxm, qym, cm, zbm, zp, qxp, qyp, cp, zbp, nx, ny},
 * out = {F, Gx, Gy, R, lambda, hstar_m, hstar_p} */
int ora_face_flux_p(const ora* o, const double in[12], double out[7]);
int ora_tableau(int tableau, int* s, double* a, double* at, double* b, double* bt, double* c);

#ifdef __cplusplus
}
#endif
#endif
