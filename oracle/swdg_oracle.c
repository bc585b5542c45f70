/*
 * swdg_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Written from arXiv 2505.18743, Sections 2-3 and Appendix A.  Each
 * function names the passage it restates.  No code is shared with the CUDA
 * library: quadrature rules come from Newton iteration on Legendre
 * polynomials, sub-grid integrals from explicit rectangle/pixel overlaps in
 * physical coordinates, and every linear system is assembled densely and
 * solved by Gaussian elimination with partial pivoting.
 *
 * Readings of the paper taken where it is silent or ambiguous:
 *  - mode S: the point p of a tensor rule owns the sub-cell given by its
 *    cumulative weights; V_p(eta) = sum_k w_k max(eta + z_k, 0) and
 *    A_p(eta) = sum_k w_k [eta + z_k > 0] over the pixel area fractions w_k;
 *  - hydrostatic reconstruction in mode S: h*- = min(V-(zeta-), V+(zeta-)),
 *    which is Eq. hydro_rec_vars when each side is a point sample (mode P);
 *  - wall: mirrored ghost; tidal boundary: imposed elevation, q+ = q-;
 *  - a field whose nodal values on a cell are all equal is evaluated as that
 *    constant (exact dry and at-rest cells);
 *  - the degree switch of Eq. criteria_p happens once per step from zeta^n,
 *    with a mass-exact remap to r_K = 0;
 *  - a continuity Newton solve on an r_K = r cell that meets a completely dry
 *    mass sub-cell switches that cell to r_K = 0 for the rest of the step;
 *  - Newton stops when the cell's l1 increment is below
 *    newton_tol * sum_i (1 + |zeta_i| + max|z_b|) or after newton_max steps.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "swdg_oracle.h"

#define MAXP 6   /* max points per direction in any rule used here */
#define MAXND 16 /* (r+1)^2 for r <= 3 */
#define MAXTAG 16

static char g_err[256];
static void set_err(const char* m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char* ora_error(void) { return g_err; }

/* ------------------------------------------------------------------ */
/* Legendre polynomials and the Gauss rules of Table tab:quadrature     */
/* ------------------------------------------------------------------ */

/* P_n(x), P_n'(x), P_n''(x) on [-1,1] by the three-term recurrence */
static void legendre(int n, double x, double* p, double* dp, double* ddp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; *ddp = 0.0; return; }
    for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    /* derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n), valid off +-1 */
    *dp = n * (p0 - x * p1) / (1.0 - x * x);
    /* (1 - x^2) P_n'' = 2 x P_n' - n (n + 1) P_n */
    *ddp = (2.0 * x * (*dp) - n * (n + 1.0) * p1) / (1.0 - x * x);
}

/* kind 0: n-point Gauss-Legendre, kind 1: n-point Gauss-Legendre-Lobatto,
 * both mapped to [0,1] with weights summing to 1, nodes ascending */
int ora_rule(int kind, int n, double* nodes, double* weights) {
    if (n < 1 || n > 12 || (kind == 1 && n < 2)) { set_err("bad rule size"); return -1; }
    double x[16], w[16];
    if (kind == 0) {
        for (int k = 0; k < n; k++) {
            double xi = cos(M_PI * (k + 0.75) / (n + 0.5));
            for (int it = 0; it < 100; it++) {
                double p, dp, ddp;
                legendre(n, xi, &p, &dp, &ddp);
                double d = p / dp;
                xi -= d;
                if (fabs(d) < 1e-17) break;
            }
            double p, dp, ddp;
            legendre(n, xi, &p, &dp, &ddp);
            x[k] = xi;
            w[k] = 2.0 / ((1.0 - xi * xi) * dp * dp);
        }
    } else {
        x[0] = -1.0;
        x[n - 1] = 1.0;
        w[0] = w[n - 1] = 2.0 / (n * (n - 1.0));
        for (int k = 1; k < n - 1; k++) {
            /* interior nodes: roots of P'_{n-1} */
            double xi = -cos(M_PI * k / (n - 1.0));
            for (int it = 0; it < 100; it++) {
                double p, dp, ddp;
                legendre(n - 1, xi, &p, &dp, &ddp);
                double d = dp / ddp;
                xi -= d;
                if (fabs(d) < 1e-17) break;
            }
            double p, dp, ddp;
            legendre(n - 1, xi, &p, &dp, &ddp);
            x[k] = xi;
            w[k] = 2.0 / (n * (n - 1.0) * p * p);
        }
    }
    /* ascending order */
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (x[j] < x[i]) {
                double t = x[i]; x[i] = x[j]; x[j] = t;
                t = w[i]; w[i] = w[j]; w[j] = t;
            }
    for (int k = 0; k < n; k++) {
        nodes[k] = 0.5 * (1.0 + x[k]);
        weights[k] = 0.5 * w[k];
    }
    if (kind == 1) { nodes[0] = 0.0; nodes[n - 1] = 1.0; }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Time integrators of Appendix A                                       */
/* ------------------------------------------------------------------ */
int ora_tableau(int tab, int* s, double* a, double* at, double* b, double* bt, double* c) {
    /* a, at: 4x4 row-major; b, bt, c: 4 */
    memset(a, 0, 16 * sizeof(double));
    memset(at, 0, 16 * sizeof(double));
    memset(b, 0, 4 * sizeof(double));
    memset(bt, 0, 4 * sizeof(double));
    memset(c, 0, 4 * sizeof(double));
    if (tab == 0) {
        /* Table tab:imex_rk2_butch: RK32 explicit part, TR-BDF2 implicit part */
        double chi = 1.0 - sqrt(2.0) / 2.0, a32 = 0.5;
        double b2 = (1.0 - 2.0 * chi) / (4.0 * chi), b1 = 1.0 - b2 - chi, b3 = chi;
        *s = 3;
        a[1 * 4 + 0] = 2.0 * chi;
        a[2 * 4 + 0] = 1.0 - a32;
        a[2 * 4 + 1] = a32;
        at[1 * 4 + 0] = chi;
        at[1 * 4 + 1] = chi;
        at[2 * 4 + 0] = b1;
        at[2 * 4 + 1] = b2;
        at[2 * 4 + 2] = b3;
        b[0] = bt[0] = b1;
        b[1] = bt[1] = b2;
        b[2] = bt[2] = b3;
        c[0] = 0.0;
        c[1] = 2.0 * chi;
        c[2] = 1.0;
        return 0;
    }
    if (tab == 1) { /* Table tab:rk3 (SSP33); friction taken explicitly */
        *s = 3;
        a[1 * 4 + 0] = 1.0;
        a[2 * 4 + 0] = 0.25;
        a[2 * 4 + 1] = 0.25;
        b[0] = 1.0 / 6.0; b[1] = 1.0 / 6.0; b[2] = 2.0 / 3.0;
        c[0] = 0.0; c[1] = 1.0; c[2] = 0.5;
    } else if (tab == 2) { /* Table tab:rk4 (RK44) */
        *s = 4;
        a[1 * 4 + 0] = 0.5;
        a[2 * 4 + 1] = 0.5;
        a[3 * 4 + 2] = 1.0;
        b[0] = 1.0 / 6.0; b[1] = 2.0 / 6.0; b[2] = 2.0 / 6.0; b[3] = 1.0 / 6.0;
        c[0] = 0.0; c[1] = 0.5; c[2] = 0.5; c[3] = 1.0;
    } else if (tab == 3) { /* forward Euler, Eq. algebraic_elevation_forwardeuler */
        *s = 1;
        b[0] = 1.0;
    } else {
        set_err("bad tableau");
        return -1;
    }
    memcpy(at, a, 16 * sizeof(double));
    memcpy(bt, b, 4 * sizeof(double));
    return 0;
}

/* ------------------------------------------------------------------ */
/* oracle state                                                         */
/* ------------------------------------------------------------------ */
struct ora {
    ora_config cfg;
    int r, nd1, nd, nv, nm, ng;
    double xs[MAXP];                 /* Gauss-Lobatto support nodes of Q_r (Sec. 3.2) */
    double xv[MAXP], wv[MAXP], sv[MAXP + 1]; /* volume GL, floor(3r/2)+1 points */
    double xm[MAXP], wm[MAXP], sm[MAXP + 1]; /* face / mass GLL, r+2 points */
    double xg[MAXP], wg[MAXP], sg[MAXP + 1]; /* momentum mass GL, r+1 points */
    int64_t n;
    double *x0, *y0, *hx, *hy;
    int32_t* nbr;
    double* ras;
    int64_t nx, ny;
    double xo, yo, dx, dy;
    int bc_kind[MAXTAG];
    double bc_amp[MAXTAG], bc_per[MAXTAG], bc_ph[MAXTAG];
    double* manning;
    double* nu_c; /* tracer numerical diffusivity per cell (Eq. numdiff), NULL: none */
    double* u[4]; /* zeta, qx, qy, c: [n][nd] */
    uint8_t* flag;
    double* zmax; /* per cell: dry-start level (Eq. initial_guess) */
    double* zabs; /* per cell: max |z_b| (Newton tolerance scale) */
    int tab_s;
    double ta[16], tat[16], tb[4], tbt[4], tc[4];
    int last_newton;
    int64_t pos_viol, fallbacks;
    double last_dt, t;
};

/* Lagrange polynomial l_a on the support nodes, and its derivative (Sec. 3.2) */
static double lag(const ora* o, int a, double x) {
    double v = 1.0;
    for (int b = 0; b < o->nd1; b++)
        if (b != a) v *= (x - o->xs[b]) / (o->xs[a] - o->xs[b]);
    return v;
}
static double dlag(const ora* o, int a, double x) {
    double s = 0.0;
    for (int k = 0; k < o->nd1; k++) {
        if (k == a) continue;
        double v = 1.0 / (o->xs[a] - o->xs[k]);
        for (int b = 0; b < o->nd1; b++)
            if (b != a && b != k) v *= (x - o->xs[b]) / (o->xs[a] - o->xs[b]);
        s += v;
    }
    return s;
}
static double psi(const ora* o, int i, double xi, double eta) {
    return lag(o, i % o->nd1, xi) * lag(o, i / o->nd1, eta);
}

static int is_const(const double* u, int nd) {
    for (int i = 1; i < nd; i++)
        if (u[i] != u[0]) return 0;
    return 1;
}

/* value and reference gradient of one field of one cell at (xi, eta):
 * zeta ~ sum_j zeta_j psi_j (Sec. 3.2); a constant field is returned exactly */
static void field_at(const ora* o, const double* u, double xi, double eta, double* v,
                     double* dxi, double* deta) {
    if (is_const(u, o->nd)) {
        *v = u[0];
        if (dxi) *dxi = 0.0;
        if (deta) *deta = 0.0;
        return;
    }
    double s = 0.0, sx = 0.0, sy = 0.0;
    for (int b = 0; b < o->nd1; b++)
        for (int a = 0; a < o->nd1; a++) {
            double ua = u[a + o->nd1 * b];
            s += ua * lag(o, a, xi) * lag(o, b, eta);
            if (dxi) sx += ua * dlag(o, a, xi) * lag(o, b, eta);
            if (deta) sy += ua * lag(o, a, xi) * dlag(o, b, eta);
        }
    *v = s;
    if (dxi) *dxi = sx;
    if (deta) *deta = sy;
}

/* ------------------------------------------------------------------ */
/* sub-grid bathymetry (Sec. 3.3, Eqs. depth_rhs, mask; R1 reading)     */
/* ------------------------------------------------------------------ */
typedef struct {
    double X0, X1, Y0, Y1; /* sub-cell rectangle (mode S) */
    double px, py;         /* sampling point (mode P) */
} site;

static double snap(double v) {
    double r = floor(v + 0.5);
    return fabs(v - r) < 1e-9 ? r : v;
}

/* V = sum_k w_k max(eta + z_k, 0), A = sum_k w_k [eta + z_k > 0] over the
 * pixels k overlapping the rectangle, w_k = overlap area / rectangle area */
int ora_subgrid_rect(const ora* o, double X0, double X1, double Y0, double Y1, double eta,
                     double* V, double* A) {
    double a0 = snap((X0 - o->xo) / o->dx), a1 = snap((X1 - o->xo) / o->dx);
    double b0 = snap((Y0 - o->yo) / o->dy), b1 = snap((Y1 - o->yo) / o->dy);
    double area = (a1 - a0) * (b1 - b0);
    int64_t i0 = (int64_t)floor(a0), i1 = (int64_t)ceil(a1) - 1;
    int64_t j0 = (int64_t)floor(b0), j1 = (int64_t)ceil(b1) - 1;
    if (i0 < 0) i0 = 0;
    if (j0 < 0) j0 = 0;
    if (i1 > o->nx - 1) i1 = o->nx - 1;
    if (j1 > o->ny - 1) j1 = o->ny - 1;
    double v = 0.0, w = 0.0;
    for (int64_t j = j0; j <= j1; j++) {
        double oy = fmin(b1, (double)(j + 1)) - fmax(b0, (double)j);
        if (oy <= 0.0) continue;
        for (int64_t i = i0; i <= i1; i++) {
            double ox = fmin(a1, (double)(i + 1)) - fmax(a0, (double)i);
            if (ox <= 0.0) continue;
            double wk = ox * oy / area;
            double d = eta + o->ras[j * o->nx + i];
            if (d > 0.0) {
                v += wk * d;
                w += wk;
            }
        }
    }
    *V = v;
    *A = w;
    return 0;
}

/* bathymetry depth at a point: bilinear interpolation of pixel-centre values,
 * clamped at the raster edge (mode P; "linear interpolation within each pixel",
 * Sec. 5) */
double ora_zb_point(const ora* o, double x, double y) {
    double fi = (x - o->xo) / o->dx - 0.5, fj = (y - o->yo) / o->dy - 0.5;
    if (fi < 0.0) fi = 0.0;
    if (fj < 0.0) fj = 0.0;
    if (fi > o->nx - 1.0) fi = o->nx - 1.0;
    if (fj > o->ny - 1.0) fj = o->ny - 1.0;
    int64_t i0 = (int64_t)floor(fi), j0 = (int64_t)floor(fj);
    if (i0 > o->nx - 2) i0 = o->nx - 2;
    if (j0 > o->ny - 2) j0 = o->ny - 2;
    double t = fi - i0, s = fj - j0;
    const double* z = o->ras;
    int64_t nx = o->nx;
    return (1.0 - t) * (1.0 - s) * z[j0 * nx + i0] + t * (1.0 - s) * z[j0 * nx + i0 + 1] +
           (1.0 - t) * s * z[(j0 + 1) * nx + i0] + t * s * z[(j0 + 1) * nx + i0 + 1];
}

static void site_VA(const ora* o, const site* s, double eta, double* V, double* A) {
    if (o->cfg.subgrid_mode == 1) {
        double d = eta + ora_zb_point(o, s->px, s->py);
        if (d > 0.0) { *V = d; *A = 1.0; }
        else { *V = 0.0; *A = 0.0; }
        return;
    }
    ora_subgrid_rect(o, s->X0, s->X1, s->Y0, s->Y1, eta, V, A);
}
static double site_V(const ora* o, const site* s, double eta) {
    double V, A;
    site_VA(o, s, eta, &V, &A);
    return V;
}

/* sub-cell of point (ia, ib) of a tensor rule with breakpoints sb and nodes xq */
static site cell_site(const ora* o, int64_t K, const double* sb, const double* xq, int ia, int ib) {
    site s;
    s.X0 = o->x0[K] + sb[ia] * o->hx[K];
    s.X1 = o->x0[K] + sb[ia + 1] * o->hx[K];
    s.Y0 = o->y0[K] + sb[ib] * o->hy[K];
    s.Y1 = o->y0[K] + sb[ib + 1] * o->hy[K];
    s.px = o->x0[K] + xq[ia] * o->hx[K];
    s.py = o->y0[K] + xq[ib] * o->hy[K];
    return s;
}

int ora_subgrid_point(const ora* o, int64_t K, int set, int p, double eta, double* V, double* A) {
    const double *sb, *xq;
    int n;
    if (set == 0) { sb = o->sv; xq = o->xv; n = o->nv; }
    else if (set == 1) { sb = o->sm; xq = o->xm; n = o->nm; }
    else { sb = o->sg; xq = o->xg; n = o->ng; }
    if (K < 0 || K >= o->n || p < 0 || p >= n * n) { set_err("bad point"); return -1; }
    site s = cell_site(o, K, sb, xq, p % n, p / n);
    site_VA(o, &s, eta, V, A);
    return 0;
}

/* face strip of cell K on face f: the rectangle between the face and the first
 * Gauss-Lobatto breakpoint inside K (normal extent w_1 H), tangentially the
 * alpha-th GLL sub-interval of the (sub)face [t0, t0 + L] */
static site face_site(const ora* o, int64_t K, int f, double t0, double L, int al) {
    site s;
    double lo = t0 + o->sm[al] * L, hi = t0 + o->sm[al + 1] * L, tp = t0 + o->xm[al] * L;
    double x0 = o->x0[K], y0 = o->y0[K], hx = o->hx[K], hy = o->hy[K];
    int nm = o->nm;
    if (f == 0 || f == 1) {
        if (f == 0) { s.X0 = x0; s.X1 = x0 + o->sm[1] * hx; s.px = x0; }
        else { s.X0 = x0 + o->sm[nm - 1] * hx; s.X1 = x0 + hx; s.px = x0 + hx; }
        s.Y0 = lo; s.Y1 = hi; s.py = tp;
    } else {
        if (f == 2) { s.Y0 = y0; s.Y1 = y0 + o->sm[1] * hy; s.py = y0; }
        else { s.Y0 = y0 + o->sm[nm - 1] * hy; s.Y1 = y0 + hy; s.py = y0 + hy; }
        s.X0 = lo; s.X1 = hi; s.px = tp;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* pointwise physics                                                    */
/* ------------------------------------------------------------------ */
/* desingularised velocity, Eq. velocity */
static void velocity(const ora* o, double h, double qx, double qy, double* ux, double* uy) {
    double e = o->cfg.eps_vel, h4 = h * h * h * h, e4 = e * e * e * e;
    double f = sqrt(2.0) * h / sqrt(fmax(h4, e4) + h4);
    if (h <= 0.0) f = 0.0;
    *ux = f * qx;
    *uy = f * qy;
}
/* Manning coefficient gamma = g n^2 |q| / h_des^(7/3), Eqs. manning and
 * discharge_rhs_implicit, with h_des the desingularised depth of Eq. velocity */
static double gamma_manning(const ora* o, double n, double h, double qx, double qy) {
    if (n == 0.0 || h <= 0.0) return 0.0;
    double e = o->cfg.eps_vel, h4 = h * h * h * h, e4 = e * e * e * e;
    double hdes = sqrt(fmax(h4, e4) + h4) / (sqrt(2.0) * h);
    return o->cfg.g * n * n * sqrt(qx * qx + qy * qy) / pow(hdes, 7.0 / 3.0);
}

/* ------------------------------------------------------------------ */
/* create                                                               */
/* ------------------------------------------------------------------ */
static void breakpoints(const double* w, int n, double* sb) {
    sb[0] = 0.0;
    for (int k = 0; k < n; k++) sb[k + 1] = sb[k] + w[k];
    sb[n] = 1.0;
}

ora* ora_create(const ora_config* cfg, int64_t n_cells, const double* x0y0, const double* hxhy,
                const int32_t* nbr, const double* raster, int64_t nx, int64_t ny, double xo,
                double yo, double dx, double dy) {
    if (!cfg || cfg->degree < 1 || cfg->degree > 3 || n_cells < 1 || nx < 2 || ny < 2 ||
        !(dx > 0) || !(dy > 0) || cfg->newton_max < 1) {
        set_err("ora_create: invalid arguments");
        return NULL;
    }
    for (int64_t k = 0; k < n_cells * 8; k++) {
        int32_t v = nbr[k];
        int slot = (int)(k & 1);
        if (v >= n_cells || (slot == 0 && v < -MAXTAG) || (slot == 1 && v < -1)) {
            set_err("ora_create: bad neighbour table");
            return NULL;
        }
    }
    ora* o = (ora*)calloc(1, sizeof(ora));
    o->cfg = *cfg;
    o->r = cfg->degree;
    o->nd1 = o->r + 1;
    o->nd = o->nd1 * o->nd1;
    o->nv = (3 * o->r) / 2 + 1;
    o->nm = o->r + 2;
    o->ng = o->r + 1;
    double w[MAXP];
    ora_rule(1, o->nd1, o->xs, w);
    ora_rule(0, o->nv, o->xv, o->wv);
    ora_rule(1, o->nm, o->xm, o->wm);
    ora_rule(0, o->ng, o->xg, o->wg);
    breakpoints(o->wv, o->nv, o->sv);
    breakpoints(o->wm, o->nm, o->sm);
    breakpoints(o->wg, o->ng, o->sg);
    o->n = n_cells;
    o->x0 = malloc(n_cells * sizeof(double));
    o->y0 = malloc(n_cells * sizeof(double));
    o->hx = malloc(n_cells * sizeof(double));
    o->hy = malloc(n_cells * sizeof(double));
    for (int64_t k = 0; k < n_cells; k++) {
        o->x0[k] = x0y0[2 * k];
        o->y0[k] = x0y0[2 * k + 1];
        o->hx[k] = hxhy[2 * k];
        o->hy[k] = hxhy[2 * k + 1];
    }
    o->nbr = malloc(n_cells * 8 * sizeof(int32_t));
    memcpy(o->nbr, nbr, n_cells * 8 * sizeof(int32_t));
    o->ras = malloc(nx * ny * sizeof(double));
    memcpy(o->ras, raster, nx * ny * sizeof(double));
    o->nx = nx; o->ny = ny; o->xo = xo; o->yo = yo; o->dx = dx; o->dy = dy;
    o->manning = calloc(n_cells, sizeof(double));
    for (int f = 0; f < 4; f++) o->u[f] = calloc(n_cells * o->nd, sizeof(double));
    o->flag = malloc(n_cells);
    memset(o->flag, o->r, n_cells);
    o->zmax = malloc(n_cells * sizeof(double));
    o->zabs = malloc(n_cells * sizeof(double));
    for (int64_t K = 0; K < n_cells; K++) {
        double zm = -INFINITY, za = 0.0;
        if (cfg->subgrid_mode == 1) {
            /* max over the Gauss-Lobatto mass points (Eq. initial_guess) */
            for (int p = 0; p < o->nm * o->nm; p++) {
                site s = cell_site(o, K, o->sm, o->xm, p % o->nm, p / o->nm);
                double z = ora_zb_point(o, s.px, s.py);
                zm = fmax(zm, z);
                za = fmax(za, fabs(z));
            }
        } else {
            /* max over the pixels inside the cell (R13 reading) */
            double a0 = snap((o->x0[K] - xo) / dx), a1 = snap((o->x0[K] + o->hx[K] - xo) / dx);
            double b0 = snap((o->y0[K] - yo) / dy), b1 = snap((o->y0[K] + o->hy[K] - yo) / dy);
            int64_t i0 = (int64_t)floor(a0), i1 = (int64_t)ceil(a1) - 1;
            int64_t j0 = (int64_t)floor(b0), j1 = (int64_t)ceil(b1) - 1;
            if (i0 < 0 || j0 < 0 || i1 >= nx || j1 >= ny) {
                set_err("ora_create: raster does not cover the mesh");
                ora_destroy(o);
                return NULL;
            }
            for (int64_t j = j0; j <= j1; j++)
                for (int64_t i = i0; i <= i1; i++) {
                    zm = fmax(zm, raster[j * nx + i]);
                    za = fmax(za, fabs(raster[j * nx + i]));
                }
        }
        o->zmax[K] = zm;
        o->zabs[K] = za;
    }
    for (int k = 0; k < MAXTAG; k++) o->bc_kind[k] = 0;
    if (ora_tableau(cfg->tableau, &o->tab_s, o->ta, o->tat, o->tb, o->tbt, o->tc)) {
        ora_destroy(o);
        return NULL;
    }
    return o;
}

void ora_destroy(ora* o) {
    if (!o) return;
    free(o->x0); free(o->y0); free(o->hx); free(o->hy); free(o->nbr); free(o->ras);
    free(o->manning);
    free(o->nu_c);
    for (int f = 0; f < 4; f++) free(o->u[f]);
    free(o->flag); free(o->zmax); free(o->zabs);
    free(o);
}

int ora_set_boundary(ora* o, int tag, int kind, double amp, double period, double phase) {
    if (tag < 0 || tag >= MAXTAG || kind < 0 || kind > 1 || (kind == 1 && !(period > 0))) {
        set_err("bad boundary");
        return -1;
    }
    o->bc_kind[tag] = kind;
    o->bc_amp[tag] = amp;
    o->bc_per[tag] = period;
    o->bc_ph[tag] = phase;
    return 0;
}
int ora_set_tracer_diffusivity(ora* o, const double* nu) {
    free(o->nu_c);
    o->nu_c = NULL;
    if (!nu) return 0;
    o->nu_c = malloc(o->n * sizeof(double));
    for (int64_t k = 0; k < o->n; k++) o->nu_c[k] = nu[k];
    return 0;
}

int ora_set_manning(ora* o, const double* n) {
    for (int64_t k = 0; k < o->n; k++) o->manning[k] = n ? n[k] : 0.0;
    return 0;
}
int ora_set_state(ora* o, const double* z, const double* qx, const double* qy, const double* c) {
    const double* src[4] = {z, qx, qy, c};
    for (int f = 0; f < 4; f++) memcpy(o->u[f], src[f], o->n * o->nd * sizeof(double));
    memset(o->flag, o->r, o->n);
    return 0;
}
int ora_get_state(const ora* o, double* z, double* qx, double* qy, double* c) {
    double* dst[4] = {z, qx, qy, c};
    for (int f = 0; f < 4; f++)
        if (dst[f]) memcpy(dst[f], o->u[f], o->n * o->nd * sizeof(double));
    return 0;
}
int ora_get_flags(const ora* o, uint8_t* flags) {
    memcpy(flags, o->flag, o->n);
    return 0;
}

/* ------------------------------------------------------------------ */
/* residual: Eqs. mass_rhs, discharge_rhs, discharge_rhs_implicit,      */
/* r_concentration with the Rusanov flux (Eq. lxf_parameter) and the    */
/* hydrostatic reconstruction (Eqs. hydro_rec, hydro_rec_vars)          */
/* ------------------------------------------------------------------ */
typedef struct {
    double z, qx, qy, c; /* trace values */
} trace;

/* numerical fluxes at one face point, seen from the "-" side with outward
 * normal (nx, ny); h-, h+ from each side's own sub-grid operator (R3) and
 * h*+- = min of both operators at that side's elevation (R2).  Returns
 * {F, Gx, Gy, R} and lambda. */
static void face_point_flux(const ora* o, const trace* m, const trace* p, double hm, double hp,
                            double hsm, double hsp, double nx, double ny, double out[4],
                            double* lam) {
    double g = o->cfg.g;
    double umx, umy, upx, upy;
    velocity(o, hm, m->qx, m->qy, &umx, &umy);
    velocity(o, hp, p->qx, p->qy, &upx, &upy);
    double unm = umx * nx + umy * ny, unp = upx * nx + upy * ny;
    double l = fmax(fabs(unm) + sqrt(g * hm), fabs(unp) + sqrt(g * hp));
    double qsmx = hsm * umx, qsmy = hsm * umy, qspx = hsp * upx, qspy = hsp * upy;
    /* continuity: ({{q*}} + lambda/2 [[zeta*]]) . n-, [[zeta*]].n- = h*- - h*+ */
    out[0] = 0.5 * ((qsmx + qspx) * nx + (qsmy + qspy) * ny) + 0.5 * l * (hsm - hsp);
    /* momentum: ({{q* (x) u}} + lambda/2 <<q*>>) : (phi (x) n-), minus the
     * non-conservative pressure term g {{h*}} {{phi}} . [[zeta*]] (Eq. pressure_tumolo) */
    double pres = g * 0.5 * (hsm + hsp) * 0.5 * (hsm - hsp);
    out[1] = 0.5 * (qsmx * unm + qspx * unp) + 0.5 * l * (qsmx - qspx) - pres * nx;
    out[2] = 0.5 * (qsmy * unm + qspy * unp) + 0.5 * l * (qsmy - qspy) - pres * ny;
    /* tracer: ({{q* c}} + lambda/2 [[h* c]]) . n- */
    out[3] = 0.5 * ((qsmx * m->c + qspx * p->c) * nx + (qsmy * m->c + qspy * p->c) * ny) +
             0.5 * l * (hsm * m->c - hsp * p->c);
    *lam = l;
}

int ora_face_flux_p(const ora* o, const double in[12], double out[7]) {
    trace m = {in[0], in[1], in[2], in[3]}, p = {in[5], in[6], in[7], in[8]};
    double zbm = in[4], zbp = in[9];
    double hm = fmax(m.z + zbm, 0.0), hp = fmax(p.z + zbp, 0.0);
    double hsm = fmin(fmax(m.z + zbm, 0.0), fmax(m.z + zbp, 0.0));
    double hsp = fmin(fmax(p.z + zbp, 0.0), fmax(p.z + zbm, 0.0));
    double f[4], l;
    face_point_flux(o, &m, &p, hm, hp, hsm, hsp, in[10], in[11], f, &l);
    for (int k = 0; k < 4; k++) out[k] = f[k];
    out[4] = l;
    out[5] = hsm;
    out[6] = hsp;
    return 0;
}

static const double NRM[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

static void trace_at(const ora* o, int64_t K, double xi, double eta, trace* tr) {
    int nd = o->nd;
    field_at(o, o->u[0] + K * nd, xi, eta, &tr->z, NULL, NULL);
    field_at(o, o->u[1] + K * nd, xi, eta, &tr->qx, NULL, NULL);
    field_at(o, o->u[2] + K * nd, xi, eta, &tr->qy, NULL, NULL);
    field_at(o, o->u[3] + K * nd, xi, eta, &tr->c, NULL, NULL);
}

/* reference coordinates of the physical face point (tangential coordinate t)
 * seen from cell K through its face f */
static void face_ref(const ora* o, int64_t K, int f, double t, double* xi, double* eta) {
    if (f == 0 || f == 1) {
        *xi = (f == 0) ? 0.0 : 1.0;
        *eta = (t - o->y0[K]) / o->hy[K];
    } else {
        *eta = (f == 2) ? 0.0 : 1.0;
        *xi = (t - o->x0[K]) / o->hx[K];
    }
}

/* one (sub)face [t0, t0+L] of cell K, face f, with neighbour nb (or boundary) */
static void subface(const ora* o, int64_t K, int f, int64_t nb, int tag, double t0, double L,
                    double t, double* F, double* Gx, double* Gy, double* R, double* dtmin) {
    double nx = NRM[f][0], ny = NRM[f][1];
    int fo = f ^ 1; /* opposite face of the neighbour */
    double J = o->hx[K] * o->hy[K];
    for (int al = 0; al < o->nm; al++) {
        double tp = t0 + o->xm[al] * L;
        double xi, eta;
        face_ref(o, K, f, tp, &xi, &eta);
        trace m, p;
        trace_at(o, K, xi, eta, &m);
        site sm_ = face_site(o, K, f, t0, L, al), sp_;
        if (nb >= 0) {
            double xn, en;
            face_ref(o, nb, fo, tp, &xn, &en);
            trace_at(o, nb, xn, en, &p);
            sp_ = face_site(o, nb, fo, t0, L, al);
        } else {
            sp_ = sm_;
            if (o->bc_kind[tag] == 1) {
                p = m;
                p.z = o->bc_amp[tag] * sin(2.0 * M_PI * t / o->bc_per[tag] + o->bc_ph[tag]);
            } else {
                double qn = m.qx * nx + m.qy * ny;
                p = m;
                p.qx = m.qx - 2.0 * qn * nx;
                p.qy = m.qy - 2.0 * qn * ny;
            }
        }
        double hm = site_V(o, &sm_, m.z), hp = site_V(o, &sp_, p.z);
        double hsm = fmin(hm, site_V(o, &sp_, m.z));
        double hsp = fmin(hp, site_V(o, &sm_, p.z));
        double fl[4], lam;
        face_point_flux(o, &m, &p, hm, hp, hsm, hsp, nx, ny, fl, &lam);
        double wl = L * o->wm[al];
        for (int i = 0; i < o->nd; i++) {
            double ps = psi(o, i, xi, eta);
            F[i] -= wl * fl[0] * ps;
            Gx[i] -= wl * fl[1] * ps;
            Gy[i] -= wl * fl[2] * ps;
            R[i] -= wl * fl[3] * ps;
        }
        /* positivity time step, Eq. deltat_fe: J_K / (lambda l_Gamma) */
        double d = J / (fmax(lam, 1e-12) * L);
        if (d < *dtmin) *dtmin = d;
    }
}

static void cell_residual(const ora* o, int64_t K, double t, double* F, double* Gx, double* Gy,
                          double* R, double* Lx, double* Ly, double* dtmin) {
    int nd = o->nd;
    double g = o->cfg.g, hx = o->hx[K], hy = o->hy[K], J = hx * hy;
    for (int i = 0; i < nd; i++) F[i] = Gx[i] = Gy[i] = R[i] = Lx[i] = Ly[i] = 0.0;
    /* volume terms on the (floor(3r/2)+1)^2 Gauss-Legendre points */
    for (int ib = 0; ib < o->nv; ib++)
        for (int ia = 0; ia < o->nv; ia++) {
            double xi = o->xv[ia], eta = o->xv[ib], w = o->wv[ia] * o->wv[ib];
            double z, zx, zy, qx, qy, c, cx, cy;
            field_at(o, o->u[0] + K * nd, xi, eta, &z, &zx, &zy);
            field_at(o, o->u[1] + K * nd, xi, eta, &qx, NULL, NULL);
            field_at(o, o->u[2] + K * nd, xi, eta, &qy, NULL, NULL);
            field_at(o, o->u[3] + K * nd, xi, eta, &c, &cx, &cy);
            zx /= hx;
            zy /= hy;
            cx /= hx;
            cy /= hy;
            /* tracer numerical diffusion nu_c h grad c (Eq. numdiff) */
            double nuh = o->nu_c ? o->nu_c[K] : 0.0;
            site s = cell_site(o, K, o->sv, o->xv, ia, ib);
            double h = site_V(o, &s, z);
            double ux, uy;
            velocity(o, h, qx, qy, &ux, &uy);
            double gam = gamma_manning(o, o->manning[K], h, qx, qy);
            for (int i = 0; i < nd; i++) {
                int a = i % o->nd1, b = i / o->nd1;
                double ps = lag(o, a, xi) * lag(o, b, eta);
                double px = dlag(o, a, xi) * lag(o, b, eta) / hx;
                double py = lag(o, a, xi) * dlag(o, b, eta) / hy;
                F[i] += J * w * (qx * px + qy * py);
                Gx[i] += J * w * (qx * ux * px + qx * uy * py - g * h * zx * ps);
                Gy[i] += J * w * (qy * ux * px + qy * uy * py - g * h * zy * ps);
                R[i] += J * w * c * (qx * px + qy * py);
                if (nuh != 0.0) R[i] -= J * w * nuh * h * (cx * px + cy * py);
                Lx[i] -= J * w * gam * qx * ps;
                Ly[i] -= J * w * gam * qy * ps;
            }
        }
    /* face terms on r+2 Gauss-Lobatto points per (sub)face */
    for (int f = 0; f < 4; f++) {
        int32_t s0 = o->nbr[K * 8 + f * 2], s1 = o->nbr[K * 8 + f * 2 + 1];
        int tang_x = (f >= 2); /* tangential axis x for S/N faces */
        double own_t0 = tang_x ? o->x0[K] : o->y0[K], own_L = tang_x ? hx : hy;
        if (s0 < 0) {
            subface(o, K, f, -1, -1 - s0, own_t0, own_L, t, F, Gx, Gy, R, dtmin);
        } else if (s1 >= 0) {
            /* coarse side of a 2:1 hanging face: integrate over both fine subfaces */
            for (int k = 0; k < 2; k++) {
                int64_t nb = k == 0 ? s0 : s1;
                double t0 = tang_x ? o->x0[nb] : o->y0[nb], L = tang_x ? o->hx[nb] : o->hy[nb];
                subface(o, K, f, nb, 0, t0, L, t, F, Gx, Gy, R, dtmin);
            }
        } else {
            subface(o, K, f, s0, 0, own_t0, own_L, t, F, Gx, Gy, R, dtmin);
        }
    }
}

int ora_residual(ora* o, double t, int64_t n_sel, const int64_t* cells, double* F, double* Gx,
                 double* Gy, double* R, double* Lx, double* Ly) {
    int64_t n = cells ? n_sel : o->n;
    int nd = o->nd;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; k++) {
        int64_t K = cells ? cells[k] : k;
        double dtm = INFINITY;
        cell_residual(o, K, t, F + k * nd, Gx + k * nd, Gy + k * nd, R + k * nd, Lx + k * nd,
                      Ly + k * nd, &dtm);
    }
    return 0;
}

/* minimum over the mesh of J_K / (lambda l_Gamma), Eq. deltat_fe */
static double dt_scan(const ora* o, double t) {
    double best = INFINITY;
    int nd = o->nd;
#pragma omp parallel
    {
        double F[MAXND], Gx[MAXND], Gy[MAXND], R[MAXND], loc = INFINITY;
#pragma omp for schedule(dynamic, 16)
        for (int64_t K = 0; K < o->n; K++) {
            for (int f = 0; f < 4; f++) {
                int32_t s0 = o->nbr[K * 8 + f * 2], s1 = o->nbr[K * 8 + f * 2 + 1];
                int tx = (f >= 2);
                double t0 = tx ? o->x0[K] : o->y0[K], L = tx ? o->hx[K] : o->hy[K];
                for (int i = 0; i < nd; i++) F[i] = Gx[i] = Gy[i] = R[i] = 0.0;
                if (s0 < 0) subface(o, K, f, -1, -1 - s0, t0, L, t, F, Gx, Gy, R, &loc);
                else if (s1 >= 0) {
                    for (int k = 0; k < 2; k++) {
                        int64_t nb = k == 0 ? s0 : s1;
                        subface(o, K, f, nb, 0, tx ? o->x0[nb] : o->y0[nb],
                                tx ? o->hx[nb] : o->hy[nb], t, F, Gx, Gy, R, &loc);
                    }
                } else subface(o, K, f, s0, 0, t0, L, t, F, Gx, Gy, R, &loc);
            }
        }
#pragma omp critical
        if (loc < best) best = loc;
    }
    return best;
}

int ora_cfl_dt(ora* o, double t, double* dt) {
    *dt = o->cfg.cfl * dt_scan(o, t);
    return 0;
}

/* ------------------------------------------------------------------ */
/* dense linear algebra                                                 */
/* ------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting: A x = b, A n x n row-major
 * (destroyed), b overwritten by x.  Returns -1 on a zero pivot. */
static int gauss_solve(int n, double* A, double* b) {
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; i++) {
            double m = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; j++) A[i * n + j] -= m * A[k * n + j];
            b[i] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < n; j++) s -= A[k * n + j] * b[j];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* mass-type operators (Eqs. depth_rhs, mass_matrix, mass_matrix_      */
/* concentration, concentration_rhs) on the (r+2)^2 GLL points           */
/* ------------------------------------------------------------------ */
/* H_i(zeta) and, if M != NULL, M_ij = dH_i/dzeta_j; returns the number of
 * completely dry mass sub-cells (A_p == 0) */
static int mass_ops(const ora* o, int64_t K, const double* z, double* H, double* M, double* Vp) {
    int nd = o->nd, ndry = 0;
    double J = o->hx[K] * o->hy[K];
    for (int i = 0; i < nd; i++) {
        H[i] = 0.0;
        if (M)
            for (int j = 0; j < nd; j++) M[i * nd + j] = 0.0;
    }
    for (int ib = 0; ib < o->nm; ib++)
        for (int ia = 0; ia < o->nm; ia++) {
            double xi = o->xm[ia], eta = o->xm[ib], w = J * o->wm[ia] * o->wm[ib];
            double e;
            field_at(o, z, xi, eta, &e, NULL, NULL);
            site s = cell_site(o, K, o->sm, o->xm, ia, ib);
            double V, A;
            site_VA(o, &s, e, &V, &A);
            if (A == 0.0) ndry++;
            if (Vp) Vp[ia + o->nm * ib] = V;
            for (int i = 0; i < nd; i++) {
                double pi = psi(o, i, xi, eta);
                H[i] += w * pi * V;
                if (M)
                    for (int j = 0; j < nd; j++) M[i * nd + j] += w * pi * psi(o, j, xi, eta) * A;
            }
        }
    return ndry;
}

/* scalar (r_K = 0) wet mass and wet area at a constant elevation */
static void mass_scalar(const ora* o, int64_t K, double e, double* H, double* A) {
    double J = o->hx[K] * o->hy[K], h = 0.0, a = 0.0;
    for (int ib = 0; ib < o->nm; ib++)
        for (int ia = 0; ia < o->nm; ia++) {
            site s = cell_site(o, K, o->sm, o->xm, ia, ib);
            double V, Ap;
            site_VA(o, &s, e, &V, &Ap);
            double w = J * o->wm[ia] * o->wm[ib];
            h += w * V;
            a += w * Ap;
        }
    *H = h;
    *A = a;
}

/* wet mass Hbar_K = int_K max(zeta + z_b, 0) (Eq. positivity-7) */
static double cell_mass(const ora* o, int64_t K, const double* z, const double* c, double* tracer,
                        double* hmin) {
    double J = o->hx[K] * o->hy[K], m = 0.0, tm = 0.0, hm = INFINITY;
    for (int ib = 0; ib < o->nm; ib++)
        for (int ia = 0; ia < o->nm; ia++) {
            double xi = o->xm[ia], eta = o->xm[ib], w = J * o->wm[ia] * o->wm[ib];
            double e, cc = 0.0;
            field_at(o, z, xi, eta, &e, NULL, NULL);
            if (c) field_at(o, c, xi, eta, &cc, NULL, NULL);
            site s = cell_site(o, K, o->sm, o->xm, ia, ib);
            double V = site_V(o, &s, e);
            m += w * V;
            tm += w * V * cc;
            if (V < hm) hm = V;
        }
    if (tracer) *tracer = tm;
    if (hmin) *hmin = hm;
    return m;
}

int ora_cell_mass(const ora* o, double* hbar) {
    for (int64_t K = 0; K < o->n; K++)
        hbar[K] = cell_mass(o, K, o->u[0] + K * o->nd, NULL, NULL, NULL);
    return 0;
}

/* ------------------------------------------------------------------ */
/* degree adaptation (Eq. criteria_p) with a mass-exact remap           */
/* ------------------------------------------------------------------ */
static int newton_done(const ora* o, int64_t K, double inc_l1, const double* z, int nd) {
    double s = 0.0;
    for (int i = 0; i < nd; i++) s += 1.0 + fabs(z[i]) + o->zabs[K];
    return inc_l1 <= o->cfg.newton_tol * s;
}

/* scalar Newton for Hbar(e) = target from e0 (Eqs. newton, initial_guess);
 * returns iterations */
static int scalar_newton(const ora* o, int64_t K, double target, double* e) {
    int nd = o->nd, it = 0;
    double H, A;
    mass_scalar(o, K, *e, &H, &A);
    if (A == 0.0) *e = -o->zmax[K] + o->cfg.eps0;
    for (int k = 0; k < o->cfg.newton_max; k++) {
        mass_scalar(o, K, *e, &H, &A);
        if (A == 0.0) break; /* converged to a dry state: skip the division */
        double d = (H - target) / A;
        *e -= d;
        it++;
        double zz = *e;
        double inc = nd * fabs(d);
        double s = nd * (1.0 + fabs(zz) + o->zabs[K]);
        if (inc <= o->cfg.newton_tol * s) break;
    }
    return it;
}

static void remap_cell(ora* o, int64_t K) {
    int nd = o->nd;
    double J = o->hx[K] * o->hy[K];
    double *z = o->u[0] + K * nd, *qx = o->u[1] + K * nd, *qy = o->u[2] + K * nd,
           *c = o->u[3] + K * nd;
    double tracer, m = cell_mass(o, K, z, c, &tracer, NULL);
    /* q and c: Gauss-Legendre (r+1)^2 means */
    double mq[3] = {0, 0, 0};
    double* fl[3] = {qx, qy, c};
    for (int ib = 0; ib < o->ng; ib++)
        for (int ia = 0; ia < o->ng; ia++)
            for (int f = 0; f < 3; f++) {
                double v;
                field_at(o, fl[f], o->xg[ia], o->xg[ib], &v, NULL, NULL);
                mq[f] += o->wg[ia] * o->wg[ib] * v;
            }
    double cnew = (m > 1e-14 * J * o->cfg.h_lim) ? tracer / m : mq[2];
    if (!is_const(c, nd))
        for (int i = 0; i < nd; i++) c[i] = cnew;
    for (int f = 0; f < 2; f++)
        if (!is_const(fl[f], nd))
            for (int i = 0; i < nd; i++) fl[f][i] = mq[f];
    if (!is_const(z, nd)) {
        double e;
        if (m <= 0.0) {
            e = -o->zmax[K];
        } else {
            /* start above the root: the largest point value of zeta */
            e = -INFINITY;
            for (int ib = 0; ib < o->nm; ib++)
                for (int ia = 0; ia < o->nm; ia++) {
                    double v;
                    field_at(o, z, o->xm[ia], o->xm[ib], &v, NULL, NULL);
                    if (v > e) e = v;
                }
            scalar_newton(o, K, m, &e);
        }
        for (int i = 0; i < nd; i++) z[i] = e;
    }
}

int ora_degree_switch(ora* o) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t K = 0; K < o->n; K++) {
        double hmin;
        cell_mass(o, K, o->u[0] + K * o->nd, NULL, NULL, &hmin);
        o->flag[K] = (hmin > o->cfg.h_lim) ? (uint8_t)o->r : 0;
        if (o->flag[K] == 0) remap_cell(o, K);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* stage solve (Eqs. algebraic_elevation, newton, algebraic_discharge,  */
/* algebraic_concentration) for one cell                                */
/* ------------------------------------------------------------------ */
typedef struct {
    double* u[4];  /* stage states v^(1..s) are separate buffers */
} stbuf;

typedef struct {
    const double *F, *Gx, *Gy, *R, *Lx, *Ly; /* one stage's residual, [n][nd] */
} resbuf;

/* the friction term a stage with an implicit diagonal actually solved:
 * Llin_i = -sum_p J w_p gamma(v^(l-1))(x_p) q^(l)(x_p) . phi_i(x_p) on the
 * (r+1)^2 Gauss-Legendre points of Eq. mass_matrix_discharge.  The final
 * combination uses it for the last stage, so that it reproduces that stage's
 * implicit solve (TR-BDF2 is stiffly accurate) and stays L-stable; earlier
 * stages enter with L(v^(m)) as in Eq. imex_shw. */
static void linearised_friction(const ora* o, int64_t K, int active, double* const* uprev,
                                double* const* ucur, double* const* llin) {
    int nd = o->nd;
    int64_t off = K * nd;
    double J = o->hx[K] * o->hy[K];
    for (int i = 0; i < nd; i++) llin[0][off + i] = llin[1][off + i] = 0.0;
    if (!active || o->manning[K] == 0.0) return;
    for (int ib = 0; ib < o->ng; ib++)
        for (int ia = 0; ia < o->ng; ia++) {
            double xi = o->xg[ia], eta = o->xg[ib], w = J * o->wg[ia] * o->wg[ib];
            double ze, qx, qy, V, A, q[2];
            field_at(o, uprev[0] + off, xi, eta, &ze, NULL, NULL);
            field_at(o, uprev[1] + off, xi, eta, &qx, NULL, NULL);
            field_at(o, uprev[2] + off, xi, eta, &qy, NULL, NULL);
            site s = cell_site(o, K, o->sg, o->xg, ia, ib);
            site_VA(o, &s, ze, &V, &A);
            double gam = gamma_manning(o, o->manning[K], V, qx, qy);
            field_at(o, ucur[1] + off, xi, eta, &q[0], NULL, NULL);
            field_at(o, ucur[2] + off, xi, eta, &q[1], NULL, NULL);
            for (int i = 0; i < nd; i++) {
                double pi = psi(o, i, xi, eta);
                llin[0][off + i] -= w * gam * q[0] * pi;
                llin[1][off + i] -= w * gam * q[1] * pi;
            }
        }
}

/* solve the stage with explicit weights wa[m], implicit weights wat[m] for the
 * m < nres previous residuals and implicit diagonal add; state v^n in un,
 * previous stage (for gamma) in uprev, result into uout */
static int stage_cell(ora* o, int64_t K, double dt, const double* wa, const double* wat, double add,
                      int nres, const resbuf* rs, double* const* un, double* const* uprev,
                      double* const* uout, const double* HN, double HNbar, const double* CN,
                      double CNbar, double* const* llin, int* newton_its) {
    int nd = o->nd, nm = o->nm;
    int64_t off = K * nd;
    double J = o->hx[K] * o->hy[K];
    double T[MAXND], rq[2][MAXND], rc[MAXND];
    double Tbar = 0.0;
    for (int i = 0; i < nd; i++) {
        double sf = 0.0, sgx = 0.0, sgy = 0.0, sr = 0.0;
        for (int m = 0; m < nres; m++) {
            sf += wa[m] * rs[m].F[off + i];
            sgx += wa[m] * rs[m].Gx[off + i] + wat[m] * rs[m].Lx[off + i];
            sgy += wa[m] * rs[m].Gy[off + i] + wat[m] * rs[m].Ly[off + i];
            sr += wa[m] * rs[m].R[off + i];
        }
        T[i] = HN[i] + dt * sf;
        Tbar += dt * sf;
        rq[0][i] = dt * sgx;
        rq[1][i] = dt * sgy;
        rc[i] = CN[i] + dt * sr;
    }
    Tbar += HNbar;
    int viol = (Tbar < 0.0);
    int scalar = (o->flag[K] == 0);
    double znew[MAXND];
    int its = 0;
    if (!scalar) {
        double M[MAXND * MAXND], H[MAXND], d[MAXND];
        memcpy(znew, un[0] + off, nd * sizeof(double));
        for (int k = 0; k < o->cfg.newton_max; k++) {
            int ndry = mass_ops(o, K, znew, H, M, NULL);
            if (ndry) { scalar = 1; break; }
            for (int i = 0; i < nd; i++) d[i] = H[i] - T[i];
            if (gauss_solve(nd, M, d)) { scalar = 1; break; }
            double inc = 0.0;
            for (int i = 0; i < nd; i++) {
                znew[i] -= d[i];
                inc += fabs(d[i]);
            }
            its++;
            if (newton_done(o, K, inc, znew, nd)) break;
        }
        if (!scalar && mass_ops(o, K, znew, H, NULL, NULL)) scalar = 1;
        if (scalar) {
            o->flag[K] = 0;
#pragma omp atomic
            o->fallbacks++;
        }
    }
    if (scalar) {
        /* r_K = 0: one unknown per field, test function 1 (Sec. 3.4) */
        const double* z0 = un[0] + off;
        double e;
        if (is_const(z0, nd)) e = z0[0];
        else {
            e = 0.0;
            for (int ib = 0; ib < nm; ib++)
                for (int ia = 0; ia < nm; ia++) {
                    double v;
                    field_at(o, z0, o->xm[ia], o->xm[ib], &v, NULL, NULL);
                    e += o->wm[ia] * o->wm[ib] * v;
                }
        }
        its = scalar_newton(o, K, Tbar, &e);
        for (int i = 0; i < nd; i++) znew[i] = e;
        /* momentum: sum of rows of the friction-modified mass matrix */
        double den = 0.0, num[2] = {0, 0};
        for (int ib = 0; ib < o->ng; ib++)
            for (int ia = 0; ia < o->ng; ia++) {
                double xi = o->xg[ia], eta = o->xg[ib], w = J * o->wg[ia] * o->wg[ib];
                double gam = 0.0;
                if (add != 0.0) {
                    double ze, qx, qy, V, A;
                    field_at(o, uprev[0] + off, xi, eta, &ze, NULL, NULL);
                    field_at(o, uprev[1] + off, xi, eta, &qx, NULL, NULL);
                    field_at(o, uprev[2] + off, xi, eta, &qy, NULL, NULL);
                    site s = cell_site(o, K, o->sg, o->xg, ia, ib);
                    site_VA(o, &s, ze, &V, &A);
                    gam = gamma_manning(o, o->manning[K], V, qx, qy);
                }
                den += w * (1.0 + add * dt * gam);
                for (int f = 0; f < 2; f++) {
                    double qn;
                    field_at(o, un[1 + f] + off, xi, eta, &qn, NULL, NULL);
                    num[f] += w * qn;
                }
            }
        for (int f = 0; f < 2; f++) {
            double s = num[f];
            for (int i = 0; i < nd; i++) s += rq[f][i];
            double v = s / den;
            for (int i = 0; i < nd; i++) uout[1 + f][off + i] = v;
        }
        if (llin) linearised_friction(o, K, add != 0.0, uprev, uout, llin);
        /* tracer: H(zeta^(l)) C = sum_i (C~_i + dt sum a R_i) */
        double Hs, As;
        mass_scalar(o, K, e, &Hs, &As);
        double rsum = CNbar;
        for (int i = 0; i < nd; i++) rsum += rc[i] - CN[i];
        if (Hs > 1e-14 * J * o->cfg.h_lim) {
            double v = rsum / Hs;
            for (int i = 0; i < nd; i++) uout[3][off + i] = v;
        } else {
            memcpy(uout[3] + off, un[3] + off, nd * sizeof(double));
        }
        memcpy(uout[0] + off, znew, nd * sizeof(double));
    } else {
        memcpy(uout[0] + off, znew, nd * sizeof(double));
        /* momentum: A^(l) Q = Q~^n + dt sum (a G + a~ L), Eq. mass_matrix_discharge
         * on (r+1)^2 Gauss-Legendre points */
        double A[MAXND * MAXND], b[2][MAXND];
        for (int i = 0; i < nd; i++) {
            b[0][i] = rq[0][i];
            b[1][i] = rq[1][i];
            for (int j = 0; j < nd; j++) A[i * nd + j] = 0.0;
        }
        for (int ib = 0; ib < o->ng; ib++)
            for (int ia = 0; ia < o->ng; ia++) {
                double xi = o->xg[ia], eta = o->xg[ib], w = J * o->wg[ia] * o->wg[ib];
                double gam = 0.0;
                if (add != 0.0) {
                    double ze, qx, qy, V, Ap;
                    field_at(o, uprev[0] + off, xi, eta, &ze, NULL, NULL);
                    field_at(o, uprev[1] + off, xi, eta, &qx, NULL, NULL);
                    field_at(o, uprev[2] + off, xi, eta, &qy, NULL, NULL);
                    site s = cell_site(o, K, o->sg, o->xg, ia, ib);
                    site_VA(o, &s, ze, &V, &Ap);
                    gam = gamma_manning(o, o->manning[K], V, qx, qy);
                }
                double qn[2];
                field_at(o, un[1] + off, xi, eta, &qn[0], NULL, NULL);
                field_at(o, un[2] + off, xi, eta, &qn[1], NULL, NULL);
                for (int i = 0; i < nd; i++) {
                    double pi = psi(o, i, xi, eta);
                    b[0][i] += w * qn[0] * pi;
                    b[1][i] += w * qn[1] * pi;
                    for (int j = 0; j < nd; j++)
                        A[i * nd + j] += w * (1.0 + add * dt * gam) * pi * psi(o, j, xi, eta);
                }
            }
        for (int f = 0; f < 2; f++) {
            double Ac[MAXND * MAXND];
            memcpy(Ac, A, sizeof(double) * nd * nd);
            gauss_solve(nd, Ac, b[f]);
            memcpy(uout[1 + f] + off, b[f], nd * sizeof(double));
        }
        if (llin) linearised_friction(o, K, add != 0.0, uprev, uout, llin);
        /* tracer: dense depth-weighted mass matrix (Eq. mass_matrix_concentration) */
        double Hc[MAXND * MAXND], Vp[64], Hd[MAXND];
        mass_ops(o, K, znew, Hd, NULL, Vp);
        for (int i = 0; i < nd * nd; i++) Hc[i] = 0.0;
        for (int ib = 0; ib < nm; ib++)
            for (int ia = 0; ia < nm; ia++) {
                double xi = o->xm[ia], eta = o->xm[ib], w = J * o->wm[ia] * o->wm[ib];
                double V = Vp[ia + nm * ib];
                for (int i = 0; i < nd; i++) {
                    double pi = psi(o, i, xi, eta);
                    for (int j = 0; j < nd; j++) Hc[i * nd + j] += w * V * pi * psi(o, j, xi, eta);
                }
            }
        gauss_solve(nd, Hc, rc);
        memcpy(uout[3] + off, rc, nd * sizeof(double));
    }
    *newton_its = its;
    return viol;
}

/* H_i(zeta^n) and C~_i^n of one cell (Eqs. depth_rhs, concentration_rhs) */
static void step_start_cell(const ora* o, int64_t K, double* HN, double* HNbar, double* CN,
                            double* CNbar) {
    int nd = o->nd, nm = o->nm;
    double J = o->hx[K] * o->hy[K];
    const double *z = o->u[0] + K * nd, *c = o->u[3] + K * nd;
    for (int i = 0; i < nd; i++) HN[i] = CN[i] = 0.0;
    double hb = 0.0, cb = 0.0;
    for (int ib = 0; ib < nm; ib++)
        for (int ia = 0; ia < nm; ia++) {
            double xi = o->xm[ia], eta = o->xm[ib], w = J * o->wm[ia] * o->wm[ib];
            double e, cc;
            field_at(o, z, xi, eta, &e, NULL, NULL);
            field_at(o, c, xi, eta, &cc, NULL, NULL);
            site s = cell_site(o, K, o->sm, o->xm, ia, ib);
            double V = site_V(o, &s, e);
            hb += w * V;
            cb += w * V * cc;
            for (int i = 0; i < nd; i++) {
                double pi = psi(o, i, xi, eta);
                HN[i] += w * pi * V;
                CN[i] += w * pi * V * cc;
            }
        }
    *HNbar = hb;
    *CNbar = cb;
}

int ora_step(ora* o, int n_steps, double dt_in, double* t_inout) {
    int64_t n = o->n;
    int nd = o->nd, s = o->tab_s;
    size_t sz = (size_t)n * nd;
    double *stage[4][4], *res[4][6], *llin[4][2];
    for (int l = 0; l < s; l++) {
        for (int f = 0; f < 4; f++) stage[l][f] = malloc(sz * sizeof(double));
        for (int f = 0; f < 6; f++) res[l][f] = malloc(sz * sizeof(double));
        for (int f = 0; f < 2; f++) llin[l][f] = calloc(sz, sizeof(double));
    }
    double *HN = malloc(sz * sizeof(double)), *CN = malloc(sz * sizeof(double));
    double *HNb = malloc(n * sizeof(double)), *CNb = malloc(n * sizeof(double));
    double* un[4] = {o->u[0], o->u[1], o->u[2], o->u[3]};
    double t = t_inout ? *t_inout : o->t;
    for (int step = 0; step < n_steps; step++) {
        ora_degree_switch(o);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t K = 0; K < n; K++)
            step_start_cell(o, K, HN + K * nd, HNb + K, CN + K * nd, CNb + K);
        double dt = dt_in;
        int maxits = 0;
        int64_t viol = 0;
        for (int l = 0; l < s; l++) {
            double* cur[4];
            if (l == 0) {
                for (int f = 0; f < 4; f++) {
                    memcpy(stage[0][f], un[f], sz * sizeof(double));
                    cur[f] = stage[0][f];
                }
                if (dt < 0.0) dt = o->cfg.cfl * dt_scan(o, t);
            } else {
                resbuf rs[4];
                for (int m = 0; m < l; m++) {
                    rs[m].F = res[m][0]; rs[m].Gx = res[m][1]; rs[m].Gy = res[m][2];
                    rs[m].R = res[m][3]; rs[m].Lx = res[m][4]; rs[m].Ly = res[m][5];
                }
                double wa[4], wat[4];
                for (int m = 0; m < l; m++) {
                    wa[m] = o->ta[l * 4 + m];
                    wat[m] = o->tat[l * 4 + m];
                }
                double add = o->tat[l * 4 + l];
                for (int f = 0; f < 4; f++) cur[f] = stage[l][f];
                double* const* prev = stage[l - 1];
#pragma omp parallel for schedule(dynamic, 16) reduction(max : maxits) reduction(+ : viol)
                for (int64_t K = 0; K < n; K++) {
                    int its;
                    viol += stage_cell(o, K, dt, wa, wat, add, l, rs, un, prev, cur, HN + K * nd,
                                       HNb[K], CN + K * nd, CNb[K], llin[l], &its);
                    if (its > maxits) maxits = its;
                }
            }
            /* residual of this stage at t + c_l dt */
            double* sv[4] = {o->u[0], o->u[1], o->u[2], o->u[3]};
            for (int f = 0; f < 4; f++) o->u[f] = cur[f];
            ora_residual(o, t + o->tc[l] * dt, 0, NULL, res[l][0], res[l][1], res[l][2],
                         res[l][3], res[l][4], res[l][5]);
            for (int f = 0; f < 4; f++) o->u[f] = sv[f];
        }
        /* final combination with b, b~ (no implicit diagonal) */
        {
            resbuf rs[4];
            for (int m = 0; m < s; m++) {
                /* last stage: the linearised friction it solved (R8 reading) */
                int imp = (m == s - 1) && (o->tat[m * 4 + m] != 0.0);
                rs[m].F = res[m][0]; rs[m].Gx = res[m][1]; rs[m].Gy = res[m][2];
                rs[m].R = res[m][3];
                rs[m].Lx = imp ? llin[m][0] : res[m][4];
                rs[m].Ly = imp ? llin[m][1] : res[m][5];
            }
            double* outp[4];
            double* tmp[4];
            for (int f = 0; f < 4; f++) {
                tmp[f] = malloc(sz * sizeof(double));
                outp[f] = tmp[f];
            }
            double* const* prev = stage[s - 1];
#pragma omp parallel for schedule(dynamic, 16) reduction(max : maxits) reduction(+ : viol)
            for (int64_t K = 0; K < n; K++) {
                int its;
                viol += stage_cell(o, K, dt, o->tb, o->tbt, 0.0, s, rs, un, prev, outp,
                                   HN + K * nd, HNb[K], CN + K * nd, CNb[K], NULL, &its);
                if (its > maxits) maxits = its;
            }
            for (int f = 0; f < 4; f++) {
                memcpy(o->u[f], tmp[f], sz * sizeof(double));
                free(tmp[f]);
            }
        }
        t += dt;
        o->last_dt = dt;
        o->last_newton = maxits;
        o->pos_viol += viol;
    }
    o->t = t;
    if (t_inout) *t_inout = t;
    for (int l = 0; l < s; l++) {
        for (int f = 0; f < 4; f++) free(stage[l][f]);
        for (int f = 0; f < 6; f++) free(res[l][f]);
        for (int f = 0; f < 2; f++) free(llin[l][f]);
    }
    free(HN); free(CN); free(HNb); free(CNb);
    return 0;
}

int ora_diagnostics(ora* o, double out[8]) {
    double m = 0.0, tm = 0.0, hmin = INFINITY;
    int64_t rc = 0;
    for (int64_t K = 0; K < o->n; K++) {
        double tr, hm;
        m += cell_mass(o, K, o->u[0] + K * o->nd, o->u[3] + K * o->nd, &tr, &hm);
        tm += tr;
        if (hm < hmin) hmin = hm;
        rc += (o->flag[K] != 0);
    }
    out[0] = m;
    out[1] = tm;
    out[2] = hmin;
    out[3] = (double)rc;
    out[4] = o->last_newton;
    out[5] = (double)o->pos_viol;
    out[6] = o->last_dt;
    out[7] = o->t;
    return 0;
}

int ora_gauges(const ora* o, int n, const double* xy, double* out) {
    for (int k = 0; k < n; k++) {
        double x = xy[2 * k], y = xy[2 * k + 1];
        out[k] = NAN;
        for (int64_t K = 0; K < o->n; K++) {
            if (x >= o->x0[K] && x <= o->x0[K] + o->hx[K] && y >= o->y0[K] &&
                y <= o->y0[K] + o->hy[K]) {
                double v;
                field_at(o, o->u[0] + K * o->nd, (x - o->x0[K]) / o->hx[K],
                         (y - o->y0[K]) / o->hy[K], &v, NULL, NULL);
                out[k] = v;
                break;
            }
        }
    }
    return 0;
}

/* Definition 3.1: zeta = zeta0 where some mass point is wet at zeta0, else the
 * dry level -max z_b of the cell */
int ora_lake_at_rest(const ora* o, double zeta0, double* zeta_out) {
    for (int64_t K = 0; K < o->n; K++) {
        int wet = 0;
        for (int p = 0; p < o->nm * o->nm && !wet; p++) {
            site s = cell_site(o, K, o->sm, o->xm, p % o->nm, p / o->nm);
            double V, A;
            site_VA(o, &s, zeta0, &V, &A);
            if (A > 0.0) wet = 1;
        }
        for (int i = 0; i < o->nd; i++) zeta_out[K * o->nd + i] = wet ? zeta0 : -o->zmax[K];
    }
    return 0;
}
