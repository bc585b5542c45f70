/*
 * swdg.h -- C-ABI of the GB300 (sm_103a) sub-grid DG shallow-water hot path.
 *
 * Method: Arpaia, Orlando, Ferrarin, Bonaventura, "High-order adaptive
 * discontinuous finite elements for the shallow water equations with sub-grid
 * irregular bathymetry" (arXiv 2505.18743).  The library evaluates the
 * matrix-free DG operator of Sec. 3.2 (continuity F, Eq. mass_rhs; momentum G,
 * Eq. discharge_rhs; friction L, Eq. discharge_rhs_implicit; tracer R,
 * Eq. r_concentration) with wet depth and wet area taken from the bathymetry
 * pixels (Sec. 3.3), and advances it with the IMEX Runge-Kutta stage update of
 * Sec. 3.1 (Eqs. imex_shw, algebraic_elevation, newton, algebraic_discharge,
 * algebraic_concentration) and the degree switch of Eq. criteria_p.
 *
 * Conventions
 *  - Every call returns SWDG_OK (0) or a negative SWDG_E* code; the message of
 *    the last failure is kept per context (swdg_last_error).
 *  - The caller owns every buffer it passes; the library copies inputs and
 *    owns all the device memory it allocates.  Nothing is thread-safe per
 *    context.
 *  - `where` selects host (SWDG_HOST) or device (SWDG_DEVICE) pointers.
 *    Device pointers must be valid on the context's stream; the library
 *    synchronises that stream before returning from every call except
 *    swdg_step, which only synchronises to read the status word.
 *  - Cell K = [x0, x0+hx] x [y0, y0+hy].  Nodal DoFs sit on the (r+1)^2
 *    Gauss-Lobatto support points, index a + (r+1) b with x fastest; per-field
 *    arrays are [n_cells][(r+1)^2] float64.
 *  - Faces f = 0 W, 1 E, 2 S, 3 N.  nbr[K][f][0] is the neighbour across f, or
 *    -1 - tag (tag in 0..15) on a boundary face; nbr[K][f][1] is -1, except on
 *    the coarse side of a 2:1 (hanging) face, where slots 0 and 1 are the two
 *    fine neighbours by increasing tangential coordinate.  A fine cell lists
 *    the coarse cell in slot 0.  Each fine half face is integrated with its
 *    own r+2 Gauss-Lobatto points; the coarse side evaluates its polynomial
 *    there and its sub-grid operator on the strip under each point.
 *  - Bathymetry z_b is a depth, positive down: water depth h = max(zeta+z_b, 0)
 *    (Eq. zeta2depth-2).
 *  - Device-side failures never trap: kernels record them in a status word
 *    that swdg_step reads back.
 */
#ifndef SWDG_H
#define SWDG_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWDG_OK 0
#define SWDG_EINVAL (-1)      /* bad argument, size or mesh */
#define SWDG_ECUDA (-2)       /* a CUDA call failed */
#define SWDG_ENEWTON (-3)     /* reserved: Newton did not converge (counted, not fatal) */
#define SWDG_EPOSITIVITY (-4) /* reserved: a cell mass went negative (counted, not fatal) */
#define SWDG_ENAN (-5)        /* a non-finite value appeared in the state */
#define SWDG_ESTATE (-6)      /* call out of order (no mesh, no bathymetry, no state) */

#define SWDG_HOST 0
#define SWDG_DEVICE 1

#define SWDG_BC_WALL 0  /* mirrored ghost state: zero normal mass flux */
#define SWDG_BC_TIDE 1  /* imposed elevation amp*sin(2 pi t/period + phase), q+ = q- */

#define SWDG_PIX_F32 0
#define SWDG_PIX_F64 1

typedef struct swdg_ctx swdg_ctx;

typedef struct {
    int degree;       /* r in 1..3 (Q_r space of Sec. 3.2) */
    int precision;    /* 0: FP64 everywhere (the plain method);
                         1: FP32-bulk -- the momentum, friction and flux arithmetic
                         of the residual in FP32, while the elevation, the sub-grid
                         integrals, the hydrostatic reconstruction, the continuity
                         and tracer test integrals and every stage solve stay FP64
                         (mass, tracer mass, c = 1 and the lake at rest keep FP64
                         round-off; other results carry FP32 error) */
    int subgrid_mode; /* 0: S, each quadrature point owns the sub-cell given by the
                         cumulative weights and integrates max(eta+z_b,0) over its
                         pixels; 1: P, z_b sampled at the point by bilinear
                         interpolation of pixel centres (Sec. 5) */
    int tableau;      /* 0 RK32 + TR-BDF2 IMEX (Table tab:imex_rk2_butch), 1 SSP33
                         (Table tab:rk3), 2 RK44 (Table tab:rk4), 3 forward Euler;
                         1-3 take the friction term explicitly */
    double g;          /* gravity, m s^-2 */
    double eps_vel;    /* epsilon of the desingularised velocity, Eq. velocity */
    double h_lim;      /* depth threshold of the degree switch, Eq. criteria_p */
    double eps0;       /* dry-start lift of Eq. initial_guess */
    double cfl;        /* dt = cfl * min J_K / (lambda l_Gamma), Eq. deltat_fe */
    int newton_max;    /* iteration cap of the per-cell Newton solve (>= 1) */
    double newton_tol; /* stop when sum|dzeta| <= tol * sum(1 + |zeta| + max|z_b|), or
                          when every pixel of the cell is wet at two successive
                          iterates (H is then affine between them and the last
                          iterate is the solution); 0 disables the first test */
    void* stream;      /* cudaStream_t to run on, or NULL for the legacy stream */
} swdg_config;

/* Create a context on the current CUDA device.  Validates cfg. */
int swdg_create(const swdg_config* cfg, swdg_ctx** out);

/* Upload an axis-aligned quadrilateral mesh (Sec. 3.2): x0y0, hxhy [n][2]
 * float64 host arrays; nbr [n][4][2] int32 host array (see Conventions).
 * Errors: SWDG_EINVAL for n < 1, non-positive sizes, out-of-range neighbours,
 * boundary tags >= 16, non-mutual neighbours, or faces that are neither
 * conforming nor an exact 2:1 split. */
int swdg_upload_mesh(swdg_ctx* ctx, int64_t n_cells, const double* x0y0, const double* hxhy,
                     const int32_t* nbr);

/* Upload the bathymetry raster (host, row-major [ny][nx], dtype SWDG_PIX_F32
 * or SWDG_PIX_F64, depth positive down) with pixel (i, j) covering
 * [xo + i dx, xo + (i+1) dx] x [yo + j dy, yo + (j+1) dy].  Requires the mesh.
 * Mode S requires every cell to cover a whole number P <= 32 of pixels in
 * both directions, aligned to pixel edges (at most 4 distinct P per mesh);
 * the raster is re-tiled per cell.
 * Mode P needs nx, ny >= 2.  Errors: SWDG_EINVAL, SWDG_ESTATE. */
int swdg_upload_bathymetry(swdg_ctx* ctx, const void* raster, int dtype, int64_t nx, int64_t ny,
                           double xo, double yo, double dx, double dy);

/* Boundary condition of tag (0..15): SWDG_BC_WALL or SWDG_BC_TIDE. */
int swdg_set_boundary(swdg_ctx* ctx, int tag, int kind, double amp, double period, double phase);

/* Per-cell Manning coefficient n (Eq. manning), [n] float64; NULL sets 0. */
int swdg_set_manning(swdg_ctx* ctx, const double* n_per_cell, int where);

/* Tracer numerical diffusion (Eq. numdiff): with a diffusivity nu_c [n] per
 * cell (>= 0; host or device per where), the term -sum_K int_K nu_c h grad c
 * . grad psi_i joins the tracer residual R (volume points, h the sub-grid
 * depth); the paper sets nu_c = C |K| r^-2 S with a case-dependent strain
 * rate S, which the caller computes.  NULL turns it off (the default).  It
 * moves no tracer mass and is dissipative. */
int swdg_set_tracer_diffusivity(swdg_ctx* ctx, const double* nu, int where);

/* Set the state (zeta, qx, qy, c), each [n][(r+1)^2] float64.  Resets the
 * per-cell degree flags to r. */
int swdg_set_state(swdg_ctx* ctx, const double* zeta, const double* qx, const double* qy,
                   const double* c, int where);
int swdg_get_state(swdg_ctx* ctx, double* zeta, double* qx, double* qy, double* c, int where);

/* Residual of the current state at time t: F, Gx, Gy, R, Lx, Ly (Eqs.
 * mass_rhs, discharge_rhs, r_concentration, discharge_rhs_implicit), each
 * [n][(r+1)^2] float64, so that M d(state)/dt = residual.  Any output may be
 * NULL.  Sets every member's clock to t. */
int swdg_residual(swdg_ctx* ctx, double t, double* F, double* Gx, double* Gy, double* R,
                  double* Lx, double* Ly, int where);

/* cfl * min over all face points of J_K / (lambda l_Gamma) for the current
 * state at time t (Eq. deltat_fe); on an ensemble, the smallest member step.
 * Sets every member's clock to t. */
int swdg_cfl_dt(swdg_ctx* ctx, double t, double* dt);

/* Advance n_steps time steps.  dt_or_neg >= 0: fixed step; < 0: the CFL step
 * of every step is computed on the device.  t_inout (may be NULL) is the
 * start time on entry and the end time on return.  Each step: degree switch
 * (Eq. criteria_p) with mass-exact remap, then the stages and final
 * combination of the tableau.  Returns SWDG_ENAN if the state became
 * non-finite.  On an ensemble (swdg_set_members) every member takes its own
 * CFL step and keeps its own clock: t_inout must be NULL (SWDG_EINVAL
 * otherwise) and the clocks are read with swdg_member_times.  The kernels of
 * a step are launched once for the whole ensemble and captured in one CUDA
 * graph. */
int swdg_step(swdg_ctx* ctx, int n_steps, double dt_or_neg, double* t_inout);

/* Profiling variant of swdg_step: runs n_steps with the kernels launched one
 * by one (no graph), a CUDA event pair around each launch on the context's
 * stream.  ms_out[SWDG_PROF_SLOTS] receives the summed time per kernel slot:
 * 0 step start (degree switch + H(zeta^n)), 1..4 residual of stage 1..4
 * (the cell kernel), 5..7 stage update 2..4, 8 final combination, 9..12 the
 * face points of stage 1..4 (the face kernel of that residual).  Unused
 * slots are 0.  Same numerics and status handling as swdg_step. */
#define SWDG_PROF_SLOTS 13
int swdg_step_profile(swdg_ctx* ctx, int n_steps, double dt_or_neg, double* t_inout,
                      double* ms_out);

/* Apply the degree switch of Eq. criteria_p (and its remap) to the current
 * state, as at the start of a step; flags_out [n] uint8 (host) may be NULL. */
int swdg_degree_switch(swdg_ctx* ctx, uint8_t* flags_out);

/* Zeta at n gauge points xy [n][2] (host), written to zeta_out [n] (host);
 * NaN for a point outside the mesh.  On an ensemble the first cell (in cell
 * order) containing the point answers; see swdg_gather_gauges_member. */
int swdg_gather_gauges(swdg_ctx* ctx, int n, const double* xy, double* zeta_out);

/* Transpose of swdg_gather_gauges, for losses over gauge time series (the
 * paper has no counterpart): adds gbar[g] times the derivative of the gauge
 * value zeta(xy[g]) with respect to each nodal zeta value of its cell to
 * zeta_b [n_cells][(r+1)^2] (host or device per where; xy [n][2] and gbar [n]
 * are host arrays).  A constant (r_K = 0) cell is differentiated as its
 * polynomial; a point outside the mesh adds nothing.  Both gauge calls locate
 * the points on the host once and reuse the cells while the points and the
 * mesh stay the same. */
int swdg_gauges_vjp(swdg_ctx* ctx, int n, const double* xy, const double* gbar, double* zeta_b,
                    int where);

/* out[8] = total mass sum_K Hbar_K (Eq. positivity-7), tracer mass, min wet
 * depth over mass points, number of r_K = r cells, max Newton iterations of
 * the last step, positivity violations (cumulative), last dt, t.  On an
 * ensemble the first four are over all members and dt, t are member 0's. */
int swdg_diagnostics(swdg_ctx* ctx, double out[8]);

/* Discrete adjoint of the residual (Sec. 3.2): the vector-Jacobian product
 * of (F, Gx, Gy, R, Lx, Ly) at the current state and time t.  Inputs: the
 * cotangents F_b .. Ly_b [n][(r+1)^2] (any may be NULL = 0).  Outputs (any
 * may be NULL): zeta_b, qx_b, qy_b, c_b [n][(r+1)^2] = sum over every
 * residual entry of its cotangent times its derivative with respect to each
 * nodal value; manning_b [n] the same with respect to each cell's Manning
 * coefficient; delta_b [n] with respect to a bathymetry offset of each cell
 * (every pixel depth of cell K, or in mode P every sampled depth, deepened by
 * delta_K), at delta = 0.  Kinks: max(x, 0) in the sub-grid integrals has
 * derivative [x > 0] (Eq. mask); the reconstruction's min and the wave-speed
 * max follow the side whose residual is differentiated at ties; |x| and
 * sqrt(x) have derivative 0 at 0.  Always FP64 (also in an FP32-bulk
 * context).  The paper states the forward operator only. */
int swdg_residual_vjp(swdg_ctx* ctx, double t, const double* F_b, const double* Gx_b,
                      const double* Gy_b, const double* R_b, const double* Lx_b,
                      const double* Ly_b, double* zeta_b, double* qx_b, double* qy_b,
                      double* c_b, double* manning_b, double* delta_b, int where);

/* Discrete adjoint of one time step (the paper states the forward scheme only).
 * swdg_step_record advances one step of fixed size dt (> 0) like swdg_step
 * (t_inout may be NULL: the context's clock) and keeps what the adjoint needs:
 * the start state, the state after the degree switch, the stage states and
 * the degree flags after every stage update.  swdg_step_vjp then pulls the
 * cotangent of the state after that step (zeta_b .. c_b, [n][(r+1)^2], NULL =
 * 0) back to the state before it (zeta_b_out .. c_b_out), to the Manning
 * coefficients (manning_b [n]) and to per-cell bathymetry offsets (delta_b
 * [n], every depth of cell K deepened by delta_K, at delta = 0); any output
 * may be NULL.  The derivative is taken along the path the forward took:
 * the time step and every discrete decision (degree flags, r_K = 0 fallbacks,
 * the tracer's dry guard) are held fixed, each converged nonlinear solve is
 * differentiated by the implicit function theorem (the continuity Newton
 * solve by M(zeta^(l))^-1, M symmetric), the remap of an r_K = 0 cell and a
 * constant field are differentiated as their formulas, and the kinks follow
 * swdg_residual_vjp.  A multi-step adjoint records and pulls back the steps
 * in reverse order, re-running each step from a stored (checkpointed) start
 * state.  FP64 contexts with one member only (SWDG_EINVAL otherwise);
 * swdg_step_vjp without a recorded step returns SWDG_ESTATE. */
int swdg_step_record(swdg_ctx* ctx, double dt, double* t_inout);
/* Record slots, so that a block of steps is run forward once and then pulled
 * back from its records: swdg_adjoint_slots reserves n_slots records (each
 * (s + 2) states of [4][n][(r+1)^2] float64 plus 2 (s + 1) n bytes, s the
 * stages of the tableau); swdg_step_record_slot / swdg_step_vjp_slot are
 * swdg_step_record / swdg_step_vjp on slot `slot` (the plain calls use slot
 * 0).  SWDG_EINVAL for a slot out of range, SWDG_ESTATE for an empty one. */
int swdg_adjoint_slots(swdg_ctx* ctx, int n_slots);
int swdg_step_record_slot(swdg_ctx* ctx, int slot, double dt, double* t_inout);
int swdg_step_vjp_slot(swdg_ctx* ctx, int slot, const double* zeta_b, const double* qx_b,
                       const double* qy_b, const double* c_b, double* zeta_b_out,
                       double* qx_b_out, double* qy_b_out, double* c_b_out, double* manning_b,
                       double* delta_b, int where);
/* Per-cell bathymetry offsets delta [n] (host or device per where; NULL = 0):
 * every depth of cell K (its pixels in mode S -- rounded to the raster's
 * precision --, its sampled depths in mode P) becomes the uploaded depth +
 * delta_K, the parameter whose cotangent swdg_step_vjp returns.  Offsets are
 * absolute (relative to the uploaded bathymetry), not cumulative. */
int swdg_set_bathymetry_offset(swdg_ctx* ctx, const double* delta, int where);
int swdg_step_vjp(swdg_ctx* ctx, const double* zeta_b, const double* qx_b, const double* qy_b,
                  const double* c_b, double* zeta_b_out, double* qx_b_out, double* qy_b_out,
                  double* c_b_out, double* manning_b, double* delta_b, int where);

/* ---- ensembles (the paper has no counterpart: many independent problems,
 * e.g. a parameter sweep of tides, friction and bathymetry, advanced by the
 * same kernel launches) ----
 *
 * The mesh uploaded with swdg_upload_mesh is the disjoint union of the
 * members' meshes: member m owns cells [first_cell[m], first_cell[m+1]),
 * first_cell [n_members + 1] (host) running from 0 to n_cells, and no face
 * may join cells of two members (SWDG_EINVAL).  Members may overlap in
 * space.  Each member has its own CFL step, clock and boundary table (all
 * initialised from the context's: every boundary set so far, clock 0); state,
 * Manning coefficients and diagnostics stay per cell.  Re-uploading the mesh
 * ends the ensemble.  n_members = 1 turns a context back into a plain one. */
#define SWDG_MAX_MEMBERS 65536
int swdg_set_members(swdg_ctx* ctx, int n_members, const int64_t* first_cell);

/* Bathymetry of an ensemble: member m's cells take their pixels (or point
 * samples) from rasters[m] (host, dtype SWDG_PIX_*, [ny][nx] row-major) of
 * size nxny[2m], nxny[2m+1] and geometry geo[4m..4m+3] = x_origin, y_origin,
 * dx, dy -- the rules of swdg_upload_bathymetry apply per member, and at most
 * 4 distinct pixel counts per cell over the whole ensemble.  Each raster is
 * on the device only while its member is re-tiled. */
int swdg_upload_bathymetry_members(swdg_ctx* ctx, const void* const* rasters, int dtype,
                                   const int64_t* nxny, const double* geo);

/* Boundary tag of one member (as swdg_set_boundary, which sets the tag of
 * every member). */
int swdg_set_boundary_member(swdg_ctx* ctx, int member, int tag, int kind, double amp,
                             double period, double phase);

/* The members' clocks: set != 0 writes t [n_members] (host) as every
 * member's time; set == 0 reads t and dt_last [n_members] (host, either may be
 * NULL). */
int swdg_member_times(swdg_ctx* ctx, double* t, double* dt_last, int set);

/* out [n_members][8]: swdg_diagnostics per member (mass, tracer mass and min
 * depth over the member's cells, its r_K = r cell count, the context-wide
 * Newton maximum and violation count, its last dt and t). */
int swdg_member_diagnostics(swdg_ctx* ctx, double* out);

/* swdg_gather_gauges over the cells of one member. */
int swdg_gather_gauges_member(swdg_ctx* ctx, int member, int n, const double* xy,
                              double* zeta_out);

/* ---- dynamic h-adaptation (Sec. 3.4) ----
 * A forest of quadtrees over an nx0 x ny0 grid of coarse cells (origin x0,
 * y0; size hx0 x hy0); leaf (l, i, j) is the cell [x0 + i hx0 / 2^l, ...] x
 * [y0 + j hy0 / 2^l, ...] at level l = 0..max_level (the paper's mesh level
 * n_K = l + 1).  Domain faces carry tags[4] (W, E, S, N) unless periodic.
 * Leaves are listed along the Morton curve of their lower-left corners on the
 * level-max_level grid. */
typedef struct {
    int nx0, ny0;
    double x0, y0, hx0, hy0;
    int max_level;
    double h_min;   /* H_min: a cell with max(hx, hy) <= h_min is not refined */
    int tags[4];
    int periodic[2];
} swdg_forest;

/* Criteria of Sec. 3.4 (host, no GPU): with eta_max = max eta, flags[k] = 1
 * (refine) if eta_k > theta_r eta_max, l < max_level and max(hx, hy) > h_min;
 * else -1 (coarsen) if eta_k < theta_c eta_max and l > 0; else 0.
 * lij [n][3] = (l, i, j) of each leaf. */
int swdg_forest_flags(const swdg_forest* f, int64_t n, const int32_t* lij, const double* eta,
                      double theta_r, double theta_c, int8_t* flags);
/* Adapted leaf set (host, no GPU): refine the leaves flagged 1, merge four
 * sibling leaves that are all flagged -1 into their parent, then split leaves
 * until every face joins leaves at most one level apart (the smallest such
 * set).  Writes *n_out, and the ordered leaves to lij_out if n_out <= cap
 * (SWDG_EINVAL otherwise). */
int swdg_forest_adapt(const swdg_forest* f, int64_t n, const int32_t* lij, const int8_t* flags,
                      int64_t cap, int32_t* lij_out, int64_t* n_out);
/* Mesh of a 2:1-balanced ordered leaf set (host, no GPU): x0y0, hxhy [n][2],
 * nbr [n][4][2] in the layout of swdg_upload_mesh. */
int swdg_forest_mesh(const swdg_forest* f, int64_t n, const int32_t* lij, double* x0y0,
                     double* hxhy, int32_t* nbr);

/* Adaptation of a context's mesh (one member, FP64 or FP32-bulk).
 * swdg_amr_setup declares the forest the current mesh belongs to (every cell
 * must be one of its leaves; SWDG_EINVAL otherwise).
 * swdg_amr_indicator writes eta [n] (host): kind 0 = max over the volume
 * Gauss points of |curl u| (Sec. 4.4; u = f(h) q with f the desingularised
 * factor of Eq. velocity and grad h = A grad zeta), kind 1 = max of |grad c|
 * (Sec. 5).
 * swdg_amr_adapt flags the leaves by the criteria (eta from the caller, host
 * [n], or NULL for indicator `kind`), adapts the forest, remaps the state
 * (a kept cell keeps its values, a child takes its parent's polynomial, a
 * parent the L2 projection of its children -- conservative for every field),
 * rebuilds mesh and bathymetry (from the uploaded raster; every new cell must
 * span whole pixels) and carries the per-cell Manning and diffusivity values
 * over (children inherit, a parent takes the children's mean).  report [9]
 * (may be NULL): cells before, cells after, leaves refined, parents formed,
 * Q^n = the change of the total wet mass sum_K Hbar_K across the adaptation
 * (Eq. mass-loss: with a conservative remap, the bathymetry-integral term),
 * the change of the tracer mass, and the milliseconds spent on the
 * indicator, on the forest (host) and on the remap and rebuild.  Launch
 * shapes return to their defaults
 * and a bathymetry offset is dropped.  Not for ensembles. */
int swdg_amr_setup(swdg_ctx* ctx, const swdg_forest* f);
int swdg_amr_indicator(swdg_ctx* ctx, int kind, double* eta);
int swdg_amr_adapt(swdg_ctx* ctx, const double* eta, int kind, double theta_r, double theta_c,
                   double* report);
/* (l, i, j) of the current leaves, lij [n][3] (host). */
int swdg_amr_leaves(const swdg_ctx* ctx, int32_t* lij);

/* ---- launch shapes (the paper has no counterpart) ----
 * Each kernel kind runs one warp per cell, grid-stride over all cells: kind
 * SWDG_KIND_BEGIN (degree switch and H, C~), SWDG_KIND_RESIDUAL,
 * SWDG_KIND_STAGE (stage update and final combination), SWDG_KIND_AUX (masks,
 * diagnostics).  A shape is (grid blocks, warps per block 1..8); the default
 * is 4 warps per block and one block per 4 cells (at most 9728 blocks).
 * Shapes change speed only: every cell's arithmetic is the same, so results
 * are bitwise identical under any shape. */
#define SWDG_KIND_BEGIN 0
#define SWDG_KIND_RESIDUAL 1
#define SWDG_KIND_STAGE 2
#define SWDG_KIND_AUX 3
int swdg_set_shape(swdg_ctx* ctx, int kind, int grid, int warps_per_block);
/* out [4][2] = grid, warps per block of each kind. */
int swdg_get_shapes(const swdg_ctx* ctx, int* out);

/* Autotuner: times every candidate shape of the begin, residual and stage
 * kernels on the context's own mesh and state (warps per block 1, 2, 4, 8;
 * grid = SMs x resident blocks, i.e. a persistent launch, or one block per
 * wpb cells), `repeats` eager steps each after one warm-up step, and keeps the
 * fastest per kind.  The state, masks, counters and clocks are restored
 * afterwards, so the tuning steps leave no trace.  report [3][3] (may be
 * NULL): grid, warps per block and ms per step of the chosen shape of each
 * kind.  Requires a state; call it outside stream capture. */
int swdg_autotune(swdg_ctx* ctx, int repeats, double* report);

/* Measurement helper (the paper has no counterpart): the arithmetic peak of
 * the current device for one precision, measured by independent FMA chains
 * in registers (8 chains per thread, 256 threads per block, SMs x resident
 * blocks; no memory traffic), best of three timed launches after one warm-up
 * on the legacy stream.  dtype SWDG_PIX_F64 or SWDG_PIX_F32; tflops [1] and
 * ms [1] (host, either may be NULL) receive 2 x FMAs / time and the launch
 * time.  Allocates 8 bytes of device memory for the duration of the call.
 * Returns SWDG_EINVAL for another dtype, SWDG_ECUDA on a CUDA error. */
int swdg_probe_fma(int dtype, double* tflops, double* ms);

/* Test helper (the paper has no counterpart): the kernels' own root of the
 * Manning term, z = h^(-1/3) (an FP32 reciprocal cube root refined by two
 * Newton-Raphson steps for z^-3 = h in FP64; 1 / cbrt(h) outside the FP32
 * range), and z^3, the 1/h the residual takes at wet points with friction,
 * evaluated on the device for n host values h [n] > 0 into z [n] and
 * rcp [n] (host).  1 <= n <= 2^24.  Allocates 24 n bytes of device memory for
 * the duration of the call.  Returns SWDG_EINVAL for bad sizes or pointers,
 * SWDG_ECUDA on a CUDA error. */
int swdg_probe_roots(const double* h, int64_t n, double* z, double* rcp);

/* Allocation-free residual (the paper has no counterpart; this exists for
 * callers that cannot allocate device memory -- for example code running
 * inside a memory pool that forbids new allocations, or a host that has
 * already reserved every byte of the device).  It evaluates exactly what
 * swdg_residual evaluates, plus the CFL step of swdg_cfl_dt, without a
 * context: the caller passes every input and output as device buffers, and
 * the only scratch (the step scalars, the pixel-overlap table and one
 * constant-field byte per cell, about 1.01 MiB in all) lives in a fixed array
 * inside the library, held on each GPU where the library's device code is
 * loaded until the process exits.  It calls no cudaMalloc/cudaFree.  CUDA
 * loads device code lazily by default: the array and this degree's kernels
 * are placed on a device at the first call there (for that degree), which
 * itself needs about 1 MiB plus the kernels' code of free device memory.  So
 * make one warm-up call per degree while memory is still free, or run the
 * process with CUDA_MODULE_LOADING=EAGER, which places everything when the
 * library is loaded.
 *   cfg: degree 1..3, subgrid_mode 0 (pixel sub-cells), precision 0 (FP64;
 *        anything else is SWDG_EINVAL), g, eps_vel, cfl and stream are used
 *        (stream NULL: the legacy stream);
 *   n_cells <= SWDG_NOALLOC_MAX_CELLS, else SWDG_EINVAL;
 *   hxhy [n][2], nbr [n][4][2] (conforming faces only),
 *   tiles [n][P][P] depth pixels of each cell (P <= 32, dtype SWDG_PIX_*),
 *   manning [n] (zeros for no friction), state [4][n][(r+1)^2]
 *   (zeta, qx, qy, c): device pointers, read only;
 *   bc_kind/amp/period/phase: host arrays of 16 entries, or NULL for walls;
 *   residual [6][n][(r+1)^2] (F, Gx, Gy, R, Lx, Ly) and dt_out [1] (may be
 *   NULL): device outputs;  err (may be NULL): message on failure.
 * The first call on a device looks up the scratch array's address for that
 * device and keeps it for the life of the process; after cudaDeviceReset()
 * on that device the kept address is stale, so do not call this entry point
 * on a device again after resetting it.  Every call shares the one scratch
 * array (it is re-initialised at each call); calls that overlap on the GPU
 * (other streams, other threads) race on it.  Each call reads a status word
 * back and synchronises the stream before returning, so no call may be made
 * inside stream capture. */
#define SWDG_NOALLOC_MAX_CELLS 1048576
int swdg_residual_noalloc(const swdg_config* cfg, int64_t n_cells, const double* hxhy,
                          const int32_t* nbr, const void* tiles, int pixels_per_side, int pix_dtype,
                          const double* manning, const int32_t* bc_kind, const double* bc_amp,
                          const double* bc_period, const double* bc_phase, const double* state,
                          double t, double* residual, double* dt_out, char* err, int err_len);

const char* swdg_last_error(const swdg_ctx* ctx);
void swdg_destroy(swdg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
