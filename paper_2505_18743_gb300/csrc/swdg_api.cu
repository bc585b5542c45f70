// swdg_api.cu -- C-ABI of the sub-grid DG shallow-water hot path (see
// include/swdg.h): context, validation, uploads, per-degree tables, the step
// driver (one captured CUDA graph per time step) and setup kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/swdg.h"
#include "swdg_adjoint.cuh"
#include "swdg_kernels.cuh"
#include "swdg_launch.h"
#include "swdg_forest.h"
#include "swdg_amr.cuh"

using namespace swdg;

namespace swdg {
bool get_launch(int degree, int mode, int pix, int prec, Launch* out) {
    switch (degree) {
    case 1: return get_launch_r1(mode, pix, prec, out);
    case 2: return get_launch_r2(mode, pix, prec, out);
    case 3: return get_launch_r3(mode, pix, prec, out);
    default: return false;
    }
}
} // namespace swdg

struct swdg_ctx {
    swdg_config cfg;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int R = 1, nd = 4;
    int64_t n = 0;
    int mode = 0, pix = 1;
    bool has_mesh = false, has_bathy = false, has_state = false;
    Launch L{};
    Tables tb{};
    Dev d{};
    int nsm = 152;           // SMs of the context's device
    Shape shp[KK_N] = {};    // launch shape per kernel kind (default or autotuned)
    bool tuned = false;
    // ensemble members: cells [first[m], first[m+1]) form member m
    int nmemb = 1;
    std::vector<int64_t> first;
    int32_t* memb = nullptr;
    Member* mb = nullptr;
    Bc* bcd = nullptr;
    int64_t* first_d = nullptr; // [nmemb + 1]
    double* adj = nullptr;      // adjoint scratch: 6 + 4 fields of [n][nd], then 2 [n]
    // step adjoint workspace (swdg_step_record / swdg_step_vjp)
    struct AdjWs {
        // per record slot: v^n, v~^n, the stage states 1..s-1 and v^{n+1} ([s+2][4][n][nd]),
        // the masks of v~^n, the stages and v^{n+1} ([s+1][n]), the flags after the degree
        // switch, each stage and the final combination ([s+1][n])
        int nslots = 0;
        double* rec_u = nullptr;
        uint8_t *rec_cm = nullptr, *rec_flags = nullptr;
        std::vector<double> t0, dt;
        std::vector<char> valid;
        // adjoint scratch
        double *ubs = nullptr, *rbar = nullptr, *llb = nullptr, *HNb = nullptr, *CNb = nullptr,
               *nbar = nullptr, *dbar = nullptr, *vb = nullptr, *ubpre = nullptr;
    } ws;
    double* mdiag = nullptr;    // [nmemb][4]
    std::vector<Bc> bch;
    // device allocations
    double* nu_c = nullptr; // tracer numerical diffusivity per cell
    // dynamic h-adaptation: the forest, the leaf of every cell, the uploaded raster
    // gauges: the cells of the last gauge set (located on the host once) and a
    // device scratch for its points, values and cells
    std::vector<double> gxy;
    int64_t gk0 = 0, gk1 = 0;
    double* gdev = nullptr;
    int32_t* gcell = nullptr;
    int gcap = 0;
    // face points of the residual, each evaluated once (k_faces): the job
    // list and the per-cell flux slots
    int64_t* fjobs = nullptr;
    double* fflux = nullptr;
    int64_t njobs = 0;
    bool amr = false;
    swdg_forest forest{};
    std::vector<Leaf> leaves;
    std::vector<uint8_t> ras_h;
    // with adaptation set up, the raster also stays on the device for the
    // re-tiling of every rebuild (reuse_raster: this upload is such a rebuild)
    bool keep_raster = false, reuse_raster = false;
    void* ras_dev = nullptr;
    size_t ras_dev_bytes = 0;
    int ras_dtype = 0;
    int64_t ras_nx = 0, ras_ny = 0;
    double ras_geo[4] = {0, 0, 1, 1};
    double *x0y0 = nullptr, *hxhy = nullptr, *ihxhy = nullptr, *manning = nullptr, *U = nullptr, *res = nullptr,
           *llin = nullptr, *HN = nullptr, *CN = nullptr, *HNbar = nullptr, *CNbar = nullptr,
           *zpts = nullptr, *zmax = nullptr, *zmin = nullptr, *zabs = nullptr, *diag = nullptr;
    float2* zsb = nullptr; // sub-cell depth bounds (mode S)
    float* uF = nullptr;   // FP32 copy of U (FP32-bulk)
    int32_t* nbr = nullptr;
    uint8_t *cmask = nullptr, *flag = nullptr, *wet0 = nullptr, *finfo = nullptr, *pcls = nullptr;
    double* qpts = nullptr; // q^n at the momentum points (step start -> stage updates)
    int64_t* tile_off = nullptr;
    OvTab* ov = nullptr;
    double* zhang = nullptr;
    void* tiles = nullptr;
    // the uploaded depth data, kept once an offset is applied (swdg_set_bathymetry_offset)
    void* tiles0 = nullptr;
    double* zpts0 = nullptr;
    int64_t npix = 0;
    Scalars* sc = nullptr;
    Scalars* sc_host = nullptr; // pinned staging
    double* pin = nullptr;      // pinned staging for small reads
    cudaGraphExec_t graph = nullptr;
    double graph_dt = -2.0;
    std::vector<double> x0y0_h, hxhy_h;
    std::vector<int32_t> nbr_h;
    std::vector<uint8_t> finfo_h;
    std::string err;
};

static int fail(swdg_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, SWDG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
    } while (0)

// ---------------------------------------------------------------------------
// 1D rules in closed form (Table tab:quadrature), mapped to [0, 1]
// ---------------------------------------------------------------------------
static bool gauss_legendre(int n, double* x, double* w) {
    double t[5], v[5];
    switch (n) {
    case 1: t[0] = 0; v[0] = 2; break;
    case 2: t[0] = -1 / std::sqrt(3.0); t[1] = -t[0]; v[0] = v[1] = 1; break;
    case 3:
        t[0] = -std::sqrt(0.6); t[1] = 0; t[2] = -t[0];
        v[0] = v[2] = 5.0 / 9.0; v[1] = 8.0 / 9.0;
        break;
    case 4: {
        double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
        double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
        t[0] = -b; t[1] = -a; t[2] = a; t[3] = b;
        v[1] = v[2] = (18.0 + std::sqrt(30.0)) / 36.0;
        v[0] = v[3] = (18.0 - std::sqrt(30.0)) / 36.0;
        break;
    }
    case 5: {
        double a = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        double b = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        t[0] = -b; t[1] = -a; t[2] = 0; t[3] = a; t[4] = b;
        v[2] = 128.0 / 225.0;
        v[1] = v[3] = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0;
        v[0] = v[4] = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
        break;
    }
    default: return false;
    }
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (1.0 + t[i]);
        w[i] = 0.5 * v[i];
    }
    return true;
}

static bool gauss_lobatto(int n, double* x, double* w) {
    double t[5], v[5];
    switch (n) {
    case 2: t[0] = -1; t[1] = 1; v[0] = v[1] = 1; break;
    case 3: t[0] = -1; t[1] = 0; t[2] = 1; v[0] = v[2] = 1.0 / 3.0; v[1] = 4.0 / 3.0; break;
    case 4:
        t[0] = -1; t[1] = -1 / std::sqrt(5.0); t[2] = -t[1]; t[3] = 1;
        v[0] = v[3] = 1.0 / 6.0; v[1] = v[2] = 5.0 / 6.0;
        break;
    case 5:
        t[0] = -1; t[1] = -std::sqrt(3.0 / 7.0); t[2] = 0; t[3] = -t[1]; t[4] = 1;
        v[0] = v[4] = 0.1; v[1] = v[3] = 49.0 / 90.0; v[2] = 32.0 / 45.0;
        break;
    default: return false;
    }
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (1.0 + t[i]);
        w[i] = 0.5 * v[i];
    }
    x[0] = 0.0;
    x[n - 1] = 1.0;
    return true;
}

// Lagrange basis on the support nodes xs[0..m): value and derivative at x
static void lagrange(const double* xs, int m, int a, double x, double* v, double* dv) {
    double p = 1.0;
    for (int b = 0; b < m; ++b)
        if (b != a) p *= (x - xs[b]) / (xs[a] - xs[b]);
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == a) continue;
        double q = 1.0 / (xs[a] - xs[k]);
        for (int b = 0; b < m; ++b)
            if (b != a && b != k) q *= (x - xs[b]) / (xs[a] - xs[b]);
        s += q;
    }
    *v = p;
    *dv = s;
}

// inverse of a small dense matrix by Gauss-Jordan with partial pivoting
static bool invert(int m, const double* A, double* Ainv) {
    double W[8][16];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < 2 * m; ++j) W[i][j] = j < m ? A[i * m + j] : (j - m == i ? 1.0 : 0.0);
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int i = k + 1; i < m; ++i)
            if (std::fabs(W[i][k]) > std::fabs(W[p][k])) p = i;
        if (W[p][k] == 0.0) return false;
        for (int j = 0; j < 2 * m; ++j) std::swap(W[k][j], W[p][j]);
        double piv = W[k][k];
        for (int j = 0; j < 2 * m; ++j) W[k][j] /= piv;
        for (int i = 0; i < m; ++i) {
            if (i == k) continue;
            double f = W[i][k];
            for (int j = 0; j < 2 * m; ++j) W[i][j] -= f * W[k][j];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Ainv[i * m + j] = W[i][m + j];
    return true;
}

// pixel-overlap fractions of the sub-intervals [sb[a], sb[a+1]] (reference
// units of the cell) with P pixels per cell side
static void overlap_set(const double* sb_in, int n, int P, OvTab& ov, int set) {
    double sb[MXI + 1];
    for (int a = 0; a <= n; ++a) {
        double u = sb_in[a] * P, r = std::floor(u + 0.5);
        sb[a] = std::fabs(u - r) < 1e-9 ? r / P : sb_in[a];
    }
    for (int a = 0; a < n; ++a) {
        int lo = std::max(0, (int)std::floor(sb[a] * P));
        int hi = std::min(P - 1, (int)std::ceil(sb[a + 1] * P) - 1);
        ov.lo[set][a] = lo;
        ov.cnt[set][a] = hi - lo + 1;
        double width = sb[a + 1] - sb[a];
        for (int k = lo; k <= hi; ++k) {
            double o = std::min(sb[a + 1], (k + 1.0) / P) - std::max(sb[a], (double)k / P);
            ov.frac[set][a][k - lo] = o > 0.0 ? o / width : 0.0;
        }
    }
}

static void breakpoints(const double* w, int n, double* sb) {
    sb[0] = 0.0;
    for (int a = 0; a < n; ++a) sb[a + 1] = sb[a] + w[a];
    sb[n] = 1.0;
}

static bool build_tables(int R, Tables& tb) {
    const int nd1 = R + 1, nv = (3 * R) / 2 + 1, nm = R + 2, ng = R + 1;
    double w[MXP];
    memset(&tb, 0, sizeof tb);
    if (!gauss_lobatto(nd1, tb.xs, w)) return false;
    double xv[MXP], wv[MXP], xm[MXP], wm[MXP], xg[MXP], wg[MXP];
    if (!gauss_legendre(nv, xv, wv) || !gauss_lobatto(nm, xm, wm) || !gauss_legendre(ng, xg, wg))
        return false;
    for (int q = 0; q < nv; ++q) {
        tb.wv[q] = wv[q];
        tb.xq[SET_VOL][q] = xv[q];
        for (int a = 0; a < nd1; ++a) lagrange(tb.xs, nd1, a, xv[q], &tb.Bv[q][a], &tb.Dv[q][a]);
    }
    for (int q = 0; q < nm; ++q) {
        tb.wm[q] = wm[q];
        tb.xq[SET_MASS][q] = xm[q];
        double dv;
        for (int a = 0; a < nd1; ++a) {
            lagrange(tb.xs, nd1, a, xm[q], &tb.Bm[q][a], &dv);
            // the fine-face GLL point q of half h in the coarse face's coordinate
            for (int h = 0; h < 2; ++h) lagrange(tb.xs, nd1, a, 0.5 * (h + xm[q]), &tb.BmH[h][q][a], &dv);
        }
    }
    double Bg[MXN * MXN], Bgi[MXN * MXN];
    for (int q = 0; q < ng; ++q) {
        tb.wg[q] = wg[q];
        tb.xq[SET_MOM][q] = xg[q];
        double dv;
        for (int a = 0; a < nd1; ++a) {
            lagrange(tb.xs, nd1, a, xg[q], &tb.Bg[q][a], &dv);
            Bg[q * nd1 + a] = tb.Bg[q][a];
        }
    }
    if (!invert(nd1, Bg, Bgi)) return false;
    for (int a = 0; a < nd1; ++a)
        for (int q = 0; q < ng; ++q) tb.Bginv[a][q] = Bgi[a * nd1 + q];
    // 1D Gauss-Lobatto mass matrix (exact for degree 2r) and its inverse
    double M1[MXN * MXN], M1i[MXN * MXN];
    for (int a = 0; a < nd1; ++a)
        for (int c = 0; c < nd1; ++c) {
            double s = 0.0;
            for (int q = 0; q < nm; ++q) s += wm[q] * tb.Bm[q][a] * tb.Bm[q][c];
            M1[a * nd1 + c] = s;
        }
    if (!invert(nd1, M1, M1i)) return false;
    for (int a = 0; a < nd1; ++a)
        for (int c = 0; c < nd1; ++c) tb.M1inv[a][c] = M1i[a * nd1 + c];
    for (int q = 0; q < MXP; ++q)
        for (int a = 0; a < MXN; ++a) {
            tb.BvF[q][a] = (float)tb.Bv[q][a];
            tb.DvF[q][a] = (float)tb.Dv[q][a];
            tb.BmF[q][a] = (float)tb.Bm[q][a];
            tb.BgF[q][a] = (float)tb.Bg[q][a];
            tb.BmHF[0][q][a] = (float)tb.BmH[0][q][a];
            tb.BmHF[1][q][a] = (float)tb.BmH[1][q][a];
            tb.BginvF[a][q] = (float)tb.Bginv[a][q];
        }
    for (int q = 0; q < MXP; ++q) {
        tb.wvF[q] = (float)tb.wv[q];
        tb.wgF[q] = (float)tb.wg[q];
    }
    return true;
}

// overlap tables of the four point sets for P pixels per cell side
static bool build_overlaps(int R, int P, const Tables& tb, OvTab& ov) {
    const int nv = (3 * R) / 2 + 1, nm = R + 2, ng = R + 1;
    if (P < 1 || P > MXPIX) return false;
    memset(&ov, 0, sizeof ov);
    ov.P = P;
    double sb[MXI + 1];
    breakpoints(tb.wv, nv, sb);
    overlap_set(sb, nv, P, ov, SET_VOL);
    breakpoints(tb.wm, nm, sb);
    overlap_set(sb, nm, P, ov, SET_MASS);
    double sm[MXP + 1];
    memcpy(sm, sb, sizeof sm);
    breakpoints(tb.wg, ng, sb);
    overlap_set(sb, ng, P, ov, SET_MOM);
    // the GLL sub-intervals of the two fine halves of a face, in coarse units:
    // interval h nm + a is [(h + sm[a]) / 2, (h + sm[a+1]) / 2]
    for (int h = 0; h < 2; ++h) {
        double hb[MXP + 1];
        for (int a = 0; a <= nm; ++a) hb[a] = 0.5 * (h + sm[a]);
        OvTab tmp;
        memset(&tmp, 0, sizeof tmp);
        overlap_set(hb, nm, P, tmp, SET_HALF);
        for (int a = 0; a < nm; ++a) {
            ov.lo[SET_HALF][h * nm + a] = tmp.lo[SET_HALF][a];
            ov.cnt[SET_HALF][h * nm + a] = tmp.cnt[SET_HALF][a];
            memcpy(ov.frac[SET_HALF][h * nm + a], tmp.frac[SET_HALF][a], sizeof(ov.frac[0][0]));
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// setup kernels (S0: re-tile the raster, point samples, per-cell depth bounds)
// ---------------------------------------------------------------------------
// one warp per cell: the cell's P x P pixels to its tile
template <typename Pix>
__global__ void k_retile(const Pix* __restrict__ ras, int64_t nx, const int32_t* col0,
                         const int32_t* row0, const int64_t* off, const uint8_t* pcls,
                         const OvTab* ov, Pix* tiles, int64_t n) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < n; k += nw) {
        const int P = ov[pcls[k]].P;
        for (int i = lane; i < P * P; i += 32)
            tiles[off[k] + i] = ras[(int64_t)(row0[k] + i / P) * nx + col0[k] + i % P];
    }
}

// per-cell min / max / max |.| of the pixel depths
template <typename Pix>
__global__ void k_tile_bounds(const Pix* __restrict__ tiles, const int64_t* off,
                              const uint8_t* pcls, const OvTab* ov, int64_t n, double* zmax,
                              double* zmin, double* zabs) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < n; k += nw) {
        const int P = ov[pcls[k]].P;
        double m = -INFINITY, mn = INFINITY, a = 0.0;
        for (int i = lane; i < P * P; i += 32) {
            const double z = (double)tiles[off[k] + i];
            m = fmax(m, z);
            mn = fmin(mn, z);
            a = fmax(a, fabs(z));
        }
        m = warp_max(m);
        mn = warp_min(mn);
        a = warp_max(a);
        if (lane == 0) {
            zmax[k] = m;
            zmin[k] = mn;
            zabs[k] = a;
        }
    }
}

// mean depth sum_k w_k z_k of a sub-cell (sets setx / sety, intervals ia / ib)
template <typename Pix>
__device__ double subcell_mean(const Pix* tile, const OvTab& o, int setx, int ia, int sety, int ib) {
    double s = 0.0;
    for (int j = 0; j < o.cnt[sety][ib]; ++j) {
        double r = 0.0;
        for (int a = 0; a < o.cnt[setx][ia]; ++a)
            r += o.frac[setx][ia][a] *
                 (double)tile[(size_t)(o.lo[sety][ib] + j) * o.P + o.lo[setx][ia] + a];
        s += o.frac[sety][ib][j] * r;
    }
    return s;
}

// the smallest and largest depth of the pixels a sub-cell overlaps
template <typename Pix>
__device__ float2 subcell_bounds(const Pix* tile, const OvTab& o, int setx, int ia, int sety,
                                 int ib) {
    double lo = INFINITY, hi = -INFINITY;
    for (int j = 0; j < o.cnt[sety][ib]; ++j)
        for (int a = 0; a < o.cnt[setx][ia]; ++a) {
            const double z = (double)tile[(size_t)(o.lo[sety][ib] + j) * o.P + o.lo[setx][ia] + a];
            lo = fmin(lo, z);
            hi = fmax(hi, z);
        }
    // rounded outwards: looser bounds only make the sub-grid shortcut rarer
    return make_float2(__double2float_rd(lo), __double2float_ru(hi));
}

// one warp per cell: mean depth (and depth bounds, zsb non-null) of every
// sub-cell of the three point sets and of the coarse-side strips of its 2:1
// faces (mode S)
template <typename Pix>
__global__ void k_subcell_means(const Pix* __restrict__ tiles, const int64_t* off,
                                const uint8_t* pcls, const OvTab* ov, const uint8_t* finfo, int nv,
                                int nm, int ng, double* zpts, double* zhang, float2* zsb, int64_t n) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nzp = nv * nv + nm * nm + ng * ng;
    for (int64_t k = warp; k < n; k += nw) {
        const OvTab& o = ov[pcls[k]];
        const Pix* tile = tiles + off[k];
        for (int i = lane; i < nzp + 8 * nm; i += 32) {
            if (i < nzp) {
                int p = i, set = SET_VOL, q = nv;
                if (p >= nv * nv) {
                    p -= nv * nv;
                    set = SET_MASS;
                    q = nm;
                    if (p >= nm * nm) {
                        p -= nm * nm;
                        set = SET_MOM;
                        q = ng;
                    }
                }
                zpts[k * nzp + i] = subcell_mean(tile, o, set, p % q, set, p / q);
                if (zsb) zsb[k * nzp + i] = subcell_bounds(tile, o, set, p % q, set, p / q);
            } else {
                const int r = i - nzp, f = r / (2 * nm), h = (r / nm) % 2, al = r % nm;
                double v = 0.0;
                if ((finfo[k * 4 + f] & 3) == FI_COARSE) {
                    const int m = (f == 0 || f == 2) ? 0 : nm - 1;
                    v = f < 2 ? subcell_mean(tile, o, SET_MASS, m, SET_HALF, h * nm + al)
                              : subcell_mean(tile, o, SET_HALF, h * nm + al, SET_MASS, m);
                }
                zhang[((k * 4 + f) * 2 + h) * nm + al] = v;
            }
        }
    }
}

// bilinear interpolation of pixel-centre values, clamped at the raster edge
template <typename Pix>
__device__ double bilinear(const Pix* __restrict__ ras, int64_t nx, int64_t ny, double xo,
                           double yo, double dx, double dy, double x, double y) {
    double fi = (x - xo) / dx - 0.5, fj = (y - yo) / dy - 0.5;
    fi = fmin(fmax(fi, 0.0), (double)(nx - 1));
    fj = fmin(fmax(fj, 0.0), (double)(ny - 1));
    int64_t i0 = (int64_t)floor(fi), j0 = (int64_t)floor(fj);
    if (i0 > nx - 2) i0 = nx - 2;
    if (j0 > ny - 2) j0 = ny - 2;
    const double t = fi - i0, s = fj - j0;
    const double z00 = ras[j0 * nx + i0], z10 = ras[j0 * nx + i0 + 1];
    const double z01 = ras[(j0 + 1) * nx + i0], z11 = ras[(j0 + 1) * nx + i0 + 1];
    return (1.0 - t) * (1.0 - s) * z00 + t * (1.0 - s) * z10 + (1.0 - t) * s * z01 + t * s * z11;
}

// mode P: z_b at every point of the three point sets and at the fine-face
// points of 2:1 faces seen from the coarse side
template <typename Pix>
__global__ void k_point_samples(const Pix* __restrict__ ras, int64_t nx, int64_t ny, double xo,
                                double yo, double dx, double dy, const double* x0y0,
                                const double* hxhy, const uint8_t* finfo,
                                const __grid_constant__ Tables tb, int nv, int nm, int ng,
                                double* zpts, double* zhang, double* zmax, double* zmin,
                                double* zabs, int64_t n) {
    const int nzp = nv * nv + nm * nm + ng * ng;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double x0 = x0y0[2 * k], y0 = x0y0[2 * k + 1], hx = hxhy[2 * k], hy = hxhy[2 * k + 1];
        int off = 0;
        double m = -INFINITY, mn = INFINITY, a = 0.0;
        for (int s = 0; s < 3; ++s) {
            const int q = s == 0 ? nv : (s == 1 ? nm : ng);
            for (int p = 0; p < q * q; ++p) {
                const double x = x0 + tb.xq[s][p % q] * hx, y = y0 + tb.xq[s][p / q] * hy;
                const double z = bilinear<Pix>(ras, nx, ny, xo, yo, dx, dy, x, y);
                zpts[k * nzp + off + p] = z;
                if (s == 1) {
                    m = fmax(m, z);
                    mn = fmin(mn, z);
                    a = fmax(a, fabs(z));
                }
            }
            off += q * q;
        }
        for (int f = 0; f < 4; ++f)
            for (int h = 0; h < 2; ++h)
                for (int al = 0; al < nm; ++al) {
                    double z = 0.0;
                    if ((finfo[k * 4 + f] & 3) == FI_COARSE) {
                        const double tq = 0.5 * (h + tb.xq[SET_MASS][al]);
                        const double x = f == 0 ? x0 : f == 1 ? x0 + hx : x0 + tq * hx;
                        const double y = f == 2 ? y0 : f == 3 ? y0 + hy : y0 + tq * hy;
                        z = bilinear<Pix>(ras, nx, ny, xo, yo, dx, dy, x, y);
                    }
                    zhang[((k * 4 + f) * 2 + h) * nm + al] = z;
                }
        zmax[k] = m;
        zmin[k] = mn;
        zabs[k] = a;
    }
}

// deterministic reduction of the per-cell diagnostics (one block)
// block i reduces cells [first[i], first[i+1]) to out[4 i ..] (first == null:
// one block over [k0, k1))
__global__ void k_diag_reduce(const double* part, const int64_t* first, int64_t k0, int64_t k1,
                              double* out) {
    __shared__ double s[4][256];
    if (first) {
        k0 = first[blockIdx.x];
        k1 = first[blockIdx.x + 1];
        out += 4 * blockIdx.x;
    }
    const int64_t n = k1 - k0;
    part += 4 * k0;
    double m = 0.0, tm = 0.0, hmin = INFINITY, rc = 0.0;
    const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * chunk, e = min(n, b + chunk);
    for (int64_t k = b; k < e; ++k) {
        m += part[4 * k];
        tm += part[4 * k + 1];
        hmin = fmin(hmin, part[4 * k + 2]);
        rc += part[4 * k + 3];
    }
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = tm;
    s[2][threadIdx.x] = hmin;
    s[3][threadIdx.x] = rc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] += s[3][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) out[i] = s[i][0];
}

// ---------------------------------------------------------------------------
// tableaux of Appendix A (the same numbers as the paper's Butcher tables)
// ---------------------------------------------------------------------------
static bool set_tableau(int tab, Dev& d) {
    memset(d.a, 0, sizeof d.a);
    memset(d.at, 0, sizeof d.at);
    memset(d.b, 0, sizeof d.b);
    memset(d.bt, 0, sizeof d.bt);
    memset(d.c, 0, sizeof d.c);
    if (tab == 0) {
        const double chi = 1.0 - std::sqrt(2.0) / 2.0, a32 = 0.5;
        const double b2 = (1.0 - 2.0 * chi) / (4.0 * chi), b1 = 1.0 - b2 - chi, b3 = chi;
        d.s = 3;
        d.a[1][0] = 2.0 * chi;
        d.a[2][0] = 1.0 - a32;
        d.a[2][1] = a32;
        d.at[1][0] = chi;
        d.at[1][1] = chi;
        d.at[2][0] = b1;
        d.at[2][1] = b2;
        d.at[2][2] = b3;
        d.b[0] = d.bt[0] = b1;
        d.b[1] = d.bt[1] = b2;
        d.b[2] = d.bt[2] = b3;
        d.c[1] = 2.0 * chi;
        d.c[2] = 1.0;
        return true;
    }
    if (tab == 1) {
        d.s = 3;
        d.a[1][0] = 1.0;
        d.a[2][0] = 0.25;
        d.a[2][1] = 0.25;
        d.b[0] = 1.0 / 6.0; d.b[1] = 1.0 / 6.0; d.b[2] = 2.0 / 3.0;
        d.c[1] = 1.0; d.c[2] = 0.5;
    } else if (tab == 2) {
        d.s = 4;
        d.a[1][0] = 0.5;
        d.a[2][1] = 0.5;
        d.a[3][2] = 1.0;
        d.b[0] = 1.0 / 6.0; d.b[1] = 1.0 / 3.0; d.b[2] = 1.0 / 3.0; d.b[3] = 1.0 / 6.0;
        d.c[1] = 0.5; d.c[2] = 0.5; d.c[3] = 1.0;
    } else if (tab == 3) {
        d.s = 1;
        d.b[0] = 1.0;
    } else {
        return false;
    }
    memcpy(d.at, d.a, sizeof d.a);
    memcpy(d.bt, d.b, sizeof d.b);
    return true;
}

static void invalidate_graph(swdg_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
}

static int grid_for(int64_t n, int wpb = WPB) {
    int64_t b = (n + wpb - 1) / wpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152LL * 64));
}

// default shapes: WPB warps per block, one block per WPB cells (grid-stride
// beyond 152 x 64 blocks); the stage update (two cells per warp) 2 warps per
// block, which its shared memory per cell favours
static void default_shapes(swdg_ctx* c) {
    for (int i = 0; i < KK_N; ++i) c->shp[i] = Shape{grid_for(c->n), WPB};
    c->shp[KK_STAGE] = Shape{grid_for(c->n, 4), 2};
    c->tuned = false;
}

static void free_members(swdg_ctx* c) {
    cudaFree(c->memb); cudaFree(c->mb); cudaFree(c->bcd); cudaFree(c->first_d); cudaFree(c->mdiag);
    c->memb = nullptr;
    c->mb = nullptr;
    c->bcd = nullptr;
    c->first_d = nullptr;
    c->mdiag = nullptr;
    c->nmemb = 1;
    c->first.assign({0, c->n});
    c->bch.clear();
    c->d.memb = nullptr;
    c->d.mbc = nullptr;
    c->d.mb = &c->sc->m0;
    c->d.nmemb = 1;
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

int swdg_create(const swdg_config* cfg, swdg_ctx** out) {
    swdg_ctx* ctx = nullptr;
    if (!cfg || !out) return SWDG_EINVAL;
    *out = nullptr;
    if (cfg->degree < 1 || cfg->degree > 3 || cfg->precision < 0 || cfg->precision > 1 ||
        cfg->subgrid_mode < 0 ||
        cfg->subgrid_mode > 1 || cfg->tableau < 0 || cfg->tableau > 3 || !(cfg->g > 0) ||
        !(cfg->eps_vel > 0) || !(cfg->h_lim >= 0) || !(cfg->eps0 > 0) || !(cfg->cfl > 0) ||
        cfg->newton_max < 1 || !(cfg->newton_tol >= 0))
        return SWDG_EINVAL;
    ctx = new swdg_ctx();
    ctx->cfg = *cfg;
    ctx->st = (cudaStream_t)cfg->stream;
    if (!ctx->st) {
        // a private blocking stream: ordered with the legacy default stream and
        // capturable into a CUDA graph
        if (cudaStreamCreate(&ctx->st) != cudaSuccess) {
            delete ctx;
            return SWDG_ECUDA;
        }
        ctx->own_stream = true;
    }
    ctx->R = cfg->degree;
    ctx->nd = (cfg->degree + 1) * (cfg->degree + 1);
    ctx->mode = cfg->subgrid_mode;
    if (!build_tables(ctx->R, ctx->tb)) {
        delete ctx;
        return SWDG_EINVAL;
    }
    Dev& d = ctx->d;
    d.mode = ctx->mode;
    d.g = cfg->g;
    d.eps = cfg->eps_vel;
    d.hlim = cfg->h_lim;
    d.eps0 = cfg->eps0;
    d.cfl = cfg->cfl;
    d.newton_tol = cfg->newton_tol;
    d.newton_max = cfg->newton_max;
    set_tableau(cfg->tableau, d);
    for (int i = 0; i < MXTAG; ++i) {
        d.bc_kind[i] = SWDG_BC_WALL;
        d.bc_amp[i] = 0.0;
        d.bc_per[i] = 1.0;
        d.bc_ph[i] = 0.0;
    }
    cudaError_t e = cudaMalloc(&ctx->sc, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->sc_host, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->pin, 64 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->sc, 0, sizeof(Scalars), ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) {
        swdg_destroy(ctx);
        return SWDG_ECUDA;
    }
    d.sc = ctx->sc;
    d.mb = &ctx->sc->m0;
    d.nmemb = 1;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
    *out = ctx;
    return SWDG_OK;
}

static void free_mesh(swdg_ctx* c) {
    cudaFree(c->x0y0); cudaFree(c->hxhy); cudaFree(c->ihxhy); cudaFree(c->manning); cudaFree(c->U); cudaFree(c->res);
    cudaFree(c->llin); cudaFree(c->HN); cudaFree(c->CN); cudaFree(c->HNbar); cudaFree(c->CNbar);
    cudaFree(c->nbr); cudaFree(c->cmask); cudaFree(c->flag); cudaFree(c->wet0); cudaFree(c->diag);
    cudaFree(c->finfo);
    cudaFree(c->uF);
    c->uF = nullptr;
    cudaFree(c->qpts);
    c->qpts = nullptr;
    cudaFree(c->adj);
    c->adj = nullptr;
    cudaFree(c->gdev);
    cudaFree(c->gcell);
    c->gdev = nullptr;
    c->gcell = nullptr;
    c->gcap = 0;
    c->gxy.clear();
    cudaFree(c->fjobs);
    cudaFree(c->fflux);
    c->fjobs = nullptr;
    c->fflux = nullptr;
    c->njobs = 0;
    c->d.fjobs = nullptr;
    c->d.fflux = nullptr;
    c->d.njobs = 0;
    cudaFree(c->nu_c);
    c->nu_c = nullptr;
    c->d.nu_c = nullptr;
    for (double* p : {c->ws.rec_u, c->ws.ubs, c->ws.rbar, c->ws.llb, c->ws.HNb, c->ws.CNb,
                      c->ws.nbar, c->ws.dbar, c->ws.vb, c->ws.ubpre})
        cudaFree(p);
    cudaFree(c->ws.rec_cm);
    cudaFree(c->ws.rec_flags);
    c->ws = swdg_ctx::AdjWs{};
    c->x0y0 = c->hxhy = c->ihxhy = c->manning = c->U = c->res = c->llin = c->HN = c->CN = c->HNbar =
        c->CNbar = c->diag = nullptr;
    c->nbr = nullptr;
    c->cmask = c->flag = c->wet0 = c->finfo = nullptr;
}
static void free_bathy(swdg_ctx* c) {
    cudaFree(c->tiles); cudaFree(c->zpts); cudaFree(c->zmax); cudaFree(c->zmin); cudaFree(c->zabs);
    cudaFree(c->zsb);
    c->zsb = nullptr;
    cudaFree(c->zhang); cudaFree(c->tile_off); cudaFree(c->pcls); cudaFree(c->ov);
    cudaFree(c->tiles0); cudaFree(c->zpts0);
    c->tiles0 = nullptr;
    c->zpts0 = nullptr;
    c->tiles = nullptr;
    c->zpts = c->zmax = c->zmin = c->zabs = c->zhang = nullptr;
    c->tile_off = nullptr;
    c->pcls = nullptr;
    c->ov = nullptr;
}

void swdg_destroy(swdg_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    invalidate_graph(c);
    free_mesh(c);
    free_bathy(c);
    cudaFree(c->ras_dev);
    cudaFree(c->memb); cudaFree(c->mb); cudaFree(c->bcd); cudaFree(c->first_d); cudaFree(c->mdiag);
    cudaFree(c->sc);
    if (c->sc_host) cudaFreeHost(c->sc_host);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
}

const char* swdg_last_error(const swdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

// face info of every cell face (FI_*), validating conforming and 2:1 faces
static int classify_faces(swdg_ctx* ctx, int64_t n, const double* x0y0, const double* hxhy,
                          const int32_t* nbr, std::vector<uint8_t>& fi) {
    fi.assign(4 * n, 0);
    auto tang = [&](int64_t k, int f, double& t0, double& L) {
        t0 = f < 2 ? x0y0[2 * k + 1] : x0y0[2 * k];
        L = f < 2 ? hxhy[2 * k + 1] : hxhy[2 * k];
    };
    for (int64_t k = 0; k < n; ++k) {
        if (!(hxhy[2 * k] > 0) || !(hxhy[2 * k + 1] > 0) || !std::isfinite(x0y0[2 * k]) ||
            !std::isfinite(x0y0[2 * k + 1]))
            return fail(ctx, SWDG_EINVAL, "upload_mesh: cell %lld has a bad size or origin",
                        (long long)k);
        for (int f = 0; f < 4; ++f) {
            const int32_t s0 = nbr[k * 8 + 2 * f], s1 = nbr[k * 8 + 2 * f + 1];
            const int fo = f ^ 1;
            if (s0 >= n || s1 >= n || s0 < -MXTAG || s1 < -1 || (s0 < 0 && s1 != -1))
                return fail(ctx, SWDG_EINVAL, "upload_mesh: cell %lld face %d: bad neighbour slots",
                            (long long)k, f);
            if (s0 < 0) continue;
            double tk0, Lk;
            tang(k, f, tk0, Lk);
            if (s1 >= 0) {
                // coarse side: two fine neighbours covering the lower and upper halves
                for (int h = 0; h < 2; ++h) {
                    const int64_t q = h ? s1 : s0;
                    double tq0, Lq;
                    tang(q, fo, tq0, Lq);
                    if (nbr[q * 8 + 2 * fo] != (int32_t)k || nbr[q * 8 + 2 * fo + 1] != -1 ||
                        std::fabs(2.0 * Lq - Lk) > 1e-9 * Lk ||
                        std::fabs(tq0 - (tk0 + 0.5 * h * Lk)) > 1e-9 * Lk)
                        return fail(ctx, SWDG_EINVAL,
                                    "upload_mesh: cell %lld face %d: inconsistent 2:1 face",
                                    (long long)k, f);
                }
                fi[4 * k + f] = FI_COARSE;
                continue;
            }
            const int32_t b0 = nbr[(int64_t)s0 * 8 + 2 * fo], b1 = nbr[(int64_t)s0 * 8 + 2 * fo + 1];
            double tn0, Ln;
            tang(s0, fo, tn0, Ln);
            if (b0 == (int32_t)k && b1 == -1) {
                if (std::fabs(Ln - Lk) > 1e-9 * Lk)
                    return fail(ctx, SWDG_EINVAL,
                                "upload_mesh: cell %lld face %d is non-conforming without a 2:1 "
                                "neighbour list",
                                (long long)k, f);
            } else if (b1 >= 0 && (b0 == (int32_t)k || b1 == (int32_t)k)) {
                const int h = b1 == (int32_t)k ? 1 : 0;
                if (std::fabs(2.0 * Lk - Ln) > 1e-9 * Ln ||
                    std::fabs(tk0 - (tn0 + 0.5 * h * Ln)) > 1e-9 * Ln)
                    return fail(ctx, SWDG_EINVAL, "upload_mesh: cell %lld face %d: bad 2:1 geometry",
                                (long long)k, f);
                fi[4 * k + f] = (uint8_t)(FI_FINE | (h << 2));
            } else {
                return fail(ctx, SWDG_EINVAL,
                            "upload_mesh: cell %lld face %d and cell %d are not mutual neighbours",
                            (long long)k, f, s0);
            }
        }
    }
    return SWDG_OK;
}

int swdg_upload_mesh(swdg_ctx* ctx, int64_t n, const double* x0y0, const double* hxhy,
                     const int32_t* nbr) {
    if (!ctx) return SWDG_EINVAL;
    if (n < 1 || !x0y0 || !hxhy || !nbr) return fail(ctx, SWDG_EINVAL, "upload_mesh: bad arguments");
    std::vector<uint8_t> fi;
    int rc = classify_faces(ctx, n, x0y0, hxhy, nbr, fi);
    if (rc) return rc;
    invalidate_graph(ctx);
    free_mesh(ctx);
    free_bathy(ctx);
    ctx->has_bathy = ctx->has_state = false;
    ctx->n = n;
    ctx->amr = false; // a new mesh leaves the forest (swdg_amr_adapt sets it again)
    free_members(ctx);
    const size_t nd = ctx->nd;
    CK(cudaMalloc(&ctx->x0y0, 2 * n * sizeof(double)));
    CK(cudaMalloc(&ctx->hxhy, 2 * n * sizeof(double)));
    CK(cudaMalloc(&ctx->ihxhy, 2 * n * sizeof(double)));
    CK(cudaMalloc(&ctx->nbr, 8 * n * sizeof(int32_t)));
    CK(cudaMalloc(&ctx->finfo, 4 * n));
    CK(cudaMalloc(&ctx->manning, n * sizeof(double)));
    CK(cudaMalloc(&ctx->U, (size_t)NBUF * 4 * n * nd * sizeof(double)));
    if (ctx->cfg.precision == 1) CK(cudaMalloc(&ctx->uF, (size_t)NBUF * 4 * n * nd * sizeof(float)));
    CK(cudaMalloc(&ctx->res, (size_t)MXS * 6 * n * nd * sizeof(double)));
    CK(cudaMalloc(&ctx->llin, 2 * n * nd * sizeof(double)));
    CK(cudaMalloc(&ctx->HN, n * nd * sizeof(double)));
    CK(cudaMalloc(&ctx->CN, n * nd * sizeof(double)));
    CK(cudaMalloc(&ctx->HNbar, n * sizeof(double)));
    CK(cudaMalloc(&ctx->CNbar, n * sizeof(double)));
    CK(cudaMalloc(&ctx->cmask, (size_t)NBUF * n));
    CK(cudaMalloc(&ctx->flag, n));
    CK(cudaMalloc(&ctx->wet0, n));
    // FP64 contexts only: the FP32-bulk momentum block interpolates FP32
    // nodal values itself, so the step start's extra write would not pay
    if (ctx->cfg.precision == 0) CK(cudaMalloc(&ctx->qpts, 2 * (size_t)n * nd * sizeof(double)));
    CK(cudaMalloc(&ctx->diag, 4 * n * sizeof(double) + 8 * sizeof(double)));
    CK(cudaMemcpyAsync(ctx->x0y0, x0y0, 2 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->hxhy, hxhy, 2 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->nbr, nbr, 8 * n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->finfo, fi.data(), 4 * n, cudaMemcpyHostToDevice, ctx->st));
    std::vector<double> inv(2 * n);
    for (int64_t i = 0; i < 2 * n; ++i) inv[i] = 1.0 / hxhy[i];
    CK(cudaMemcpyAsync(ctx->ihxhy, inv.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaMemsetAsync(ctx->manning, 0, n * sizeof(double), ctx->st));
    CK(cudaMemsetAsync(ctx->llin, 0, 2 * n * nd * sizeof(double), ctx->st));
    CK(cudaMemsetAsync(ctx->flag, ctx->R, n, ctx->st));
    CK(cudaMemsetAsync(ctx->wet0, 0, n, ctx->st));
    CK(cudaMemsetAsync(ctx->cmask, 0, (size_t)NBUF * n, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->x0y0_h.assign(x0y0, x0y0 + 2 * n);
    ctx->hxhy_h.assign(hxhy, hxhy + 2 * n);
    ctx->finfo_h = fi;
    ctx->nbr_h.assign(nbr, nbr + 8 * n);
    {
        // face jobs: every (cell, face, half, GLL point) whose cell is the lower
        // index of the face, or whose face is on the boundary (or is its own
        // neighbour), in cell order
        const int NM = ctx->R + 2;
        std::vector<int64_t> jobs;
        jobs.reserve((size_t)n * 2 * NM + 64);
        for (int64_t k = 0; k < n; ++k)
            for (int f = 0; f < 4; ++f) {
                const bool coarse = (fi[k * 4 + f] & 3) == FI_COARSE;
                for (int h = 0; h < (coarse ? 2 : 1); ++h) {
                    const int32_t s0 = nbr[k * 8 + f * 2];
                    const int64_t nb = s0 < 0 ? -1 : (coarse && h ? nbr[k * 8 + f * 2 + 1] : s0);
                    if (nb >= 0 && nb < k) continue;
                    for (int al = 0; al < NM; ++al)
                        jobs.push_back((k << 8) | (int64_t)f | ((int64_t)h << 2) | ((int64_t)al << 3));
                }
            }
        ctx->njobs = (int64_t)jobs.size();
        CK(cudaMalloc(&ctx->fjobs, jobs.size() * sizeof(int64_t)));
        CK(cudaMalloc(&ctx->fflux, (size_t)n * 32 * NM * sizeof(double)));
        CK(cudaMemcpyAsync(ctx->fjobs, jobs.data(), jobs.size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemsetAsync(ctx->fflux, 0, (size_t)n * 32 * NM * sizeof(double), ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    Dev& d = ctx->d;
    d.n = n;
    d.x0y0 = ctx->x0y0;
    d.hxhy = ctx->hxhy;
    d.ihxhy = ctx->ihxhy;
    d.nbr = ctx->nbr;
    d.finfo = ctx->finfo;
    d.fflux = ctx->fflux;
    d.fjobs = ctx->fjobs;
    d.njobs = ctx->njobs;
    d.manning = ctx->manning;
    d.U = ctx->U;
    d.uF = ctx->uF;
    d.cmask = ctx->cmask;
    d.res = ctx->res;
    d.llin = ctx->llin;
    d.HN = ctx->HN;
    d.CN = ctx->CN;
    d.HNbar = ctx->HNbar;
    d.CNbar = ctx->CNbar;
    d.flag = ctx->flag;
    d.wet0 = ctx->wet0;
    d.qpts = ctx->qpts;
    d.any_friction = 0;
    default_shapes(ctx);
    ctx->has_mesh = true;
    return SWDG_OK;
}

// bathymetry of every cell from nseg rasters: cells [first[i], first[i+1])
// take their pixels (mode S) or point samples (mode P) from raster i, whose
// geometry is geo[4 i ..] = (x_origin, y_origin, dx, dy) and size nxny[2 i ..]
static int upload_bathy(swdg_ctx* ctx, int nseg, const void* const* rasters, int dtype,
                        const int64_t* nxny, const double* geo, const int64_t* first) {
    const char* who = "upload_bathymetry";
    if (!ctx->has_mesh) return fail(ctx, SWDG_ESTATE, "%s: no mesh", who);
    if (dtype != SWDG_PIX_F32 && dtype != SWDG_PIX_F64)
        return fail(ctx, SWDG_EINVAL, "%s: bad pixel dtype", who);
    for (int i = 0; i < nseg; ++i)
        if (!rasters[i] || nxny[2 * i] < 2 || nxny[2 * i + 1] < 2 || !(geo[4 * i + 2] > 0) ||
            !(geo[4 * i + 3] > 0) || !std::isfinite(geo[4 * i]) || !std::isfinite(geo[4 * i + 1]))
            return fail(ctx, SWDG_EINVAL, "%s: bad raster %d", who, i);
    const int64_t n = ctx->n;
    const size_t es = dtype == SWDG_PIX_F32 ? 4 : 8;
    const int R_ = ctx->R, nv_ = (3 * R_) / 2 + 1, nm_ = R_ + 2, ng_ = R_ + 1;
    const int nzp_ = nv_ * nv_ + nm_ * nm_ + ng_ * ng_;
    std::vector<int32_t> col0, row0;
    std::vector<int64_t> toff;
    std::vector<uint8_t> cls;
    std::vector<int> Ps;
    int64_t npix = 0;
    if (ctx->mode == 0) {
        col0.resize(n);
        row0.resize(n);
        toff.resize(n);
        cls.resize(n);
        for (int sg = 0; sg < nseg; ++sg) {
            const double xo = geo[4 * sg], yo = geo[4 * sg + 1], dx = geo[4 * sg + 2],
                         dy = geo[4 * sg + 3];
            const int64_t nx = nxny[2 * sg], ny = nxny[2 * sg + 1];
            for (int64_t k = first[sg]; k < first[sg + 1]; ++k) {
                const double cx = (ctx->x0y0_h[2 * k] - xo) / dx,
                             cy = (ctx->x0y0_h[2 * k + 1] - yo) / dy;
                const double px = ctx->hxhy_h[2 * k] / dx, py = ctx->hxhy_h[2 * k + 1] / dy;
                const double rcx = std::floor(cx + 0.5), rcy = std::floor(cy + 0.5);
                const double rpx = std::floor(px + 0.5), rpy = std::floor(py + 0.5);
                if (std::fabs(cx - rcx) > 1e-6 || std::fabs(cy - rcy) > 1e-6 ||
                    std::fabs(px - rpx) > 1e-6 || std::fabs(py - rpy) > 1e-6 || rpx != rpy)
                    return fail(ctx, SWDG_EINVAL,
                                "%s: cell %lld does not span the same whole number of pixels in x "
                                "and y, aligned to pixel edges",
                                who, (long long)k);
                const int P = (int)rpx;
                if (P < 1 || P > MXPIX)
                    return fail(ctx, SWDG_EINVAL, "%s: %d pixels per cell side (max %d)", who, P,
                                MXPIX);
                if (rcx < 0 || rcy < 0 || rcx + P > nx || rcy + P > ny)
                    return fail(ctx, SWDG_EINVAL, "%s: raster %d does not cover cell %lld", who, sg,
                                (long long)k);
                int c = -1;
                for (size_t i = 0; i < Ps.size(); ++i)
                    if (Ps[i] == P) c = (int)i;
                if (c < 0) {
                    if ((int)Ps.size() == MXCLS)
                        return fail(ctx, SWDG_EINVAL,
                                    "%s: more than %d distinct pixel counts per cell", who, MXCLS);
                    Ps.push_back(P);
                    c = (int)Ps.size() - 1;
                }
                col0[k] = (int32_t)rcx;
                row0[k] = (int32_t)rcy;
                cls[k] = (uint8_t)c;
                toff[k] = npix;
                npix += (int64_t)P * P;
            }
        }
    }
    invalidate_graph(ctx);
    free_bathy(ctx);
    ctx->has_bathy = false;
    CK(cudaMalloc(&ctx->zmax, n * sizeof(double)));
    CK(cudaMalloc(&ctx->zmin, n * sizeof(double)));
    CK(cudaMalloc(&ctx->zabs, n * sizeof(double)));
    CK(cudaMalloc(&ctx->zpts, (size_t)n * nzp_ * sizeof(double)));
    if (ctx->mode == 0) CK(cudaMalloc(&ctx->zsb, (size_t)n * nzp_ * sizeof(float2)));
    CK(cudaMalloc(&ctx->zhang, (size_t)n * 8 * nm_ * sizeof(double)));
    // one raster on the device at a time; a single raster of an adaptive
    // context stays there (and a rebuild re-tiles from it)
    const bool keep = nseg == 1 && ctx->keep_raster;
    auto put_raster = [&](int sg, void** ras) -> int {
        const size_t bytes = (size_t)nxny[2 * sg] * nxny[2 * sg + 1] * es;
        if (keep && ctx->ras_dev && ctx->ras_dev_bytes == bytes) {
            *ras = ctx->ras_dev;
            if (ctx->reuse_raster) return SWDG_OK;
        } else {
            if (keep) {
                cudaFree(ctx->ras_dev);
                ctx->ras_dev = nullptr;
                ctx->ras_dev_bytes = 0;
            }
            CK(cudaMalloc(ras, bytes));
            if (keep) {
                ctx->ras_dev = *ras;
                ctx->ras_dev_bytes = bytes;
            }
        }
        CK(cudaMemcpyAsync(*ras, rasters[sg], bytes, cudaMemcpyHostToDevice, ctx->st));
        return SWDG_OK;
    };
    if (ctx->mode == 0) {
        std::vector<OvTab> ovh(Ps.size());
        for (size_t i = 0; i < Ps.size(); ++i)
            if (!build_overlaps(ctx->R, Ps[i], ctx->tb, ovh[i]))
                return fail(ctx, SWDG_EINVAL, "%s: bad pixel count", who);
        int32_t *c0 = nullptr, *r0 = nullptr;
        CK(cudaMalloc(&c0, n * sizeof(int32_t)));
        CK(cudaMalloc(&r0, n * sizeof(int32_t)));
        CK(cudaMalloc(&ctx->tile_off, n * sizeof(int64_t)));
        CK(cudaMalloc(&ctx->pcls, n));
        CK(cudaMalloc(&ctx->ov, Ps.size() * sizeof(OvTab)));
        CK(cudaMemcpyAsync(c0, col0.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(r0, row0.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(ctx->tile_off, toff.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice,
                           ctx->st));
        CK(cudaMemcpyAsync(ctx->pcls, cls.data(), n, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(ctx->ov, ovh.data(), Ps.size() * sizeof(OvTab), cudaMemcpyHostToDevice,
                           ctx->st));
        CK(cudaMalloc(&ctx->tiles, (size_t)npix * es));
        for (int sg = 0; sg < nseg; ++sg) {
            const int64_t k0 = first[sg], nk = first[sg + 1] - first[sg];
            if (nk == 0) continue;
            void* ras = nullptr;
            int rc = put_raster(sg, &ras);
            if (rc) return rc;
            const int gw = (int)std::min<int64_t>(152 * 32, (nk * 32 + 255) / 256 + 1);
            if (dtype == SWDG_PIX_F32)
                k_retile<float><<<gw, 256, 0, ctx->st>>>((const float*)ras, nxny[2 * sg], c0 + k0,
                                                        r0 + k0, ctx->tile_off + k0, ctx->pcls + k0,
                                                        ctx->ov, (float*)ctx->tiles, nk);
            else
                k_retile<double><<<gw, 256, 0, ctx->st>>>((const double*)ras, nxny[2 * sg], c0 + k0,
                                                         r0 + k0, ctx->tile_off + k0,
                                                         ctx->pcls + k0, ctx->ov,
                                                         (double*)ctx->tiles, nk);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(ctx->st));
            if (!keep) cudaFree(ras);
        }
        const int gw = (int)std::min<int64_t>(152 * 32, (n * 32 + 255) / 256 + 1); // warp per cell
        if (dtype == SWDG_PIX_F32) {
            k_tile_bounds<float><<<gw, 256, 0, ctx->st>>>((const float*)ctx->tiles, ctx->tile_off,
                                                         ctx->pcls, ctx->ov, n, ctx->zmax, ctx->zmin,
                                                         ctx->zabs);
            k_subcell_means<float><<<gw, 256, 0, ctx->st>>>(
                (const float*)ctx->tiles, ctx->tile_off, ctx->pcls, ctx->ov, ctx->finfo, nv_, nm_, ng_,
                ctx->zpts, ctx->zhang, ctx->zsb, n);
        } else {
            k_tile_bounds<double><<<gw, 256, 0, ctx->st>>>((const double*)ctx->tiles, ctx->tile_off,
                                                          ctx->pcls, ctx->ov, n, ctx->zmax,
                                                          ctx->zmin, ctx->zabs);
            k_subcell_means<double><<<gw, 256, 0, ctx->st>>>(
                (const double*)ctx->tiles, ctx->tile_off, ctx->pcls, ctx->ov, ctx->finfo, nv_, nm_,
                ng_, ctx->zpts, ctx->zhang, ctx->zsb, n);
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->st));
        cudaFree(c0);
        cudaFree(r0);
    } else {
        for (int sg = 0; sg < nseg; ++sg) {
            const int64_t k0 = first[sg], nk = first[sg + 1] - first[sg];
            if (nk == 0) continue;
            void* ras = nullptr;
            int rc = put_raster(sg, &ras);
            if (rc) return rc;
            const double xo = geo[4 * sg], yo = geo[4 * sg + 1], dx = geo[4 * sg + 2],
                         dy = geo[4 * sg + 3];
            const int64_t nx = nxny[2 * sg], ny = nxny[2 * sg + 1];
            const int g2 = (int)std::min<int64_t>(152 * 16, (nk + 127) / 128);
            if (dtype == SWDG_PIX_F32)
                k_point_samples<float><<<g2, 128, 0, ctx->st>>>(
                    (const float*)ras, nx, ny, xo, yo, dx, dy, ctx->x0y0 + 2 * k0,
                    ctx->hxhy + 2 * k0, ctx->finfo + 4 * k0, ctx->tb, nv_, nm_, ng_,
                    ctx->zpts + k0 * nzp_, ctx->zhang + k0 * 8 * nm_, ctx->zmax + k0,
                    ctx->zmin + k0, ctx->zabs + k0, nk);
            else
                k_point_samples<double><<<g2, 128, 0, ctx->st>>>(
                    (const double*)ras, nx, ny, xo, yo, dx, dy, ctx->x0y0 + 2 * k0,
                    ctx->hxhy + 2 * k0, ctx->finfo + 4 * k0, ctx->tb, nv_, nm_, ng_,
                    ctx->zpts + k0 * nzp_, ctx->zhang + k0 * 8 * nm_, ctx->zmax + k0,
                    ctx->zmin + k0, ctx->zabs + k0, nk);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(ctx->st));
            if (!keep) cudaFree(ras);
        }
    }
    ctx->pix = dtype == SWDG_PIX_F32 ? 0 : 1;
    if (!get_launch(ctx->R, ctx->mode, ctx->pix, ctx->cfg.precision, &ctx->L))
        return fail(ctx, SWDG_EINVAL, "%s: no kernels for this configuration", who);
    if (!ctx->L.prepare())
        return fail(ctx, SWDG_ECUDA, "%s: shared-memory opt-in of the kernels failed", who);
    Dev& d = ctx->d;
    d.tiles = ctx->tiles;
    d.tile_off = ctx->tile_off;
    d.pcls = ctx->pcls;
    d.ov = ctx->ov;
    d.zhang = ctx->zhang;
    d.zpts = ctx->zpts;
    d.zsb = ctx->mode == 0 ? ctx->zsb : nullptr;
    d.zmax = ctx->zmax;
    d.zmin = ctx->zmin;
    d.zabs = ctx->zabs;
    ctx->npix = npix;
    ctx->has_bathy = true;
    return SWDG_OK;
}

int swdg_upload_bathymetry(swdg_ctx* ctx, const void* raster, int dtype, int64_t nx, int64_t ny,
                           double xo, double yo, double dx, double dy) {
    if (!ctx) return SWDG_EINVAL;
    if (!raster) return fail(ctx, SWDG_EINVAL, "upload_bathymetry: bad arguments");
    const void* r[1] = {raster};
    const int64_t nxny[2] = {nx, ny};
    const double geo[4] = {xo, yo, dx, dy};
    const int64_t first[2] = {0, ctx->n};
    int rc = upload_bathy(ctx, 1, r, dtype, nxny, geo, first);
    if (rc) return rc;
    // a host copy for re-tiling after an adaptation of the mesh
    if (ctx->ras_h.data() != (const uint8_t*)raster) {
        const size_t bytes = (size_t)nx * ny * (dtype == SWDG_PIX_F32 ? 4 : 8);
        ctx->ras_h.assign((const uint8_t*)raster, (const uint8_t*)raster + bytes);
    }
    ctx->ras_dtype = dtype;
    ctx->ras_nx = nx;
    ctx->ras_ny = ny;
    ctx->ras_geo[0] = xo;
    ctx->ras_geo[1] = yo;
    ctx->ras_geo[2] = dx;
    ctx->ras_geo[3] = dy;
    return SWDG_OK;
}

int swdg_upload_bathymetry_members(swdg_ctx* ctx, const void* const* rasters, int dtype,
                                   const int64_t* nxny, const double* geo) {
    if (!ctx) return SWDG_EINVAL;
    if (!rasters || !nxny || !geo)
        return fail(ctx, SWDG_EINVAL, "upload_bathymetry_members: bad arguments");
    return upload_bathy(ctx, ctx->nmemb, rasters, dtype, nxny, geo, ctx->first.data());
}

int swdg_set_boundary(swdg_ctx* ctx, int tag, int kind, double amp, double period, double phase) {
    if (!ctx) return SWDG_EINVAL;
    if (tag < 0 || tag >= MXTAG || (kind != SWDG_BC_WALL && kind != SWDG_BC_TIDE) ||
        (kind == SWDG_BC_TIDE && !(period > 0)) || !std::isfinite(amp) || !std::isfinite(phase))
        return fail(ctx, SWDG_EINVAL, "set_boundary: bad arguments");
    ctx->d.bc_kind[tag] = kind;
    ctx->d.bc_amp[tag] = amp;
    ctx->d.bc_per[tag] = period;
    ctx->d.bc_ph[tag] = phase;
    invalidate_graph(ctx);
    if (ctx->nmemb > 1) {
        // an ensemble: the same boundary for every member
        for (Bc& b : ctx->bch) {
            b.kind[tag] = kind;
            b.amp[tag] = amp;
            b.per[tag] = period;
            b.ph[tag] = phase;
        }
        CK(cudaMemcpyAsync(ctx->bcd, ctx->bch.data(), ctx->bch.size() * sizeof(Bc),
                           cudaMemcpyHostToDevice, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return SWDG_OK;
}

int swdg_set_tracer_diffusivity(swdg_ctx* ctx, const double* nu, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_mesh) return fail(ctx, SWDG_ESTATE, "set_tracer_diffusivity: no mesh");
    const int64_t n = ctx->n;
    if (!nu) {
        cudaFree(ctx->nu_c);
        ctx->nu_c = nullptr;
        ctx->d.nu_c = nullptr;
        invalidate_graph(ctx);
        return SWDG_OK;
    }
    if (where == SWDG_HOST)
        for (int64_t k = 0; k < n; ++k)
            if (!(nu[k] >= 0) || !std::isfinite(nu[k]))
                return fail(ctx, SWDG_EINVAL, "set_tracer_diffusivity: bad value at cell %lld",
                            (long long)k);
    if (!ctx->nu_c) CK(cudaMalloc(&ctx->nu_c, n * sizeof(double)));
    CK(cudaMemcpyAsync(ctx->nu_c, nu, n * sizeof(double),
                       where == SWDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->d.nu_c = ctx->nu_c;
    invalidate_graph(ctx);
    return SWDG_OK;
}

int swdg_set_manning(swdg_ctx* ctx, const double* nman, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_mesh) return fail(ctx, SWDG_ESTATE, "set_manning: no mesh");
    const int64_t n = ctx->n;
    if (!nman) {
        CK(cudaMemsetAsync(ctx->manning, 0, n * sizeof(double), ctx->st));
    } else if (where == SWDG_HOST) {
        for (int64_t k = 0; k < n; ++k)
            if (!(nman[k] >= 0) || !std::isfinite(nman[k]))
                return fail(ctx, SWDG_EINVAL, "set_manning: bad value at cell %lld", (long long)k);
        CK(cudaMemcpyAsync(ctx->manning, nman, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    } else {
        CK(cudaMemcpyAsync(ctx->manning, nman, n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_set_state(swdg_ctx* ctx, const double* z, const double* qx, const double* qy,
                   const double* c, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_mesh || !ctx->has_bathy)
        return fail(ctx, SWDG_ESTATE, "set_state: upload the mesh and bathymetry first");
    if (!z || !qx || !qy || !c || (where != SWDG_HOST && where != SWDG_DEVICE))
        return fail(ctx, SWDG_EINVAL, "set_state: bad arguments");
    const size_t sz = (size_t)ctx->n * ctx->nd * sizeof(double);
    const double* src[4] = {z, qx, qy, c};
    for (int f = 0; f < 4; ++f)
        CK(cudaMemcpyAsync(ctx->U + (size_t)f * ctx->n * ctx->nd, src[f], sz,
                           where == SWDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           ctx->st));
    CK(cudaMemsetAsync(ctx->flag, ctx->R, ctx->n, ctx->st));
    ctx->L.masks(ctx->d, 0, ctx->shp[KK_AUX], ctx->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->st));
    ctx->has_state = true;
    return SWDG_OK;
}

int swdg_get_state(swdg_ctx* ctx, double* z, double* qx, double* qy, double* c, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "get_state: no state");
    const size_t sz = (size_t)ctx->n * ctx->nd * sizeof(double);
    double* dst[4] = {z, qx, qy, c};
    for (int f = 0; f < 4; ++f)
        if (dst[f])
            CK(cudaMemcpyAsync(dst[f], ctx->U + (size_t)f * ctx->n * ctx->nd, sz,
                               where == SWDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                               ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

__global__ void k_set_clocks(Member* mb, int nm, double t, int reset_rmax) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
        mb[i].t = t;
        if (reset_rmax) mb[i].rmax = 0ull;
    }
}

// every member's clock to t (reset_rmax: also the CFL maximum)
static int put_clocks(swdg_ctx* ctx, double t, int reset_rmax) {
    k_set_clocks<<<(ctx->d.nmemb + 255) / 256, 256, 0, ctx->st>>>(ctx->d.mb, ctx->d.nmemb, t,
                                                                 reset_rmax);
    CK(cudaGetLastError());
    return SWDG_OK;
}

static int put_fixed_dt(swdg_ctx* ctx, double fixed_dt) {
    ctx->pin[1] = fixed_dt;
    CK(cudaMemcpyAsync(&ctx->sc->fixed_dt, &ctx->pin[1], sizeof(double), cudaMemcpyHostToDevice,
                       ctx->st));
    return SWDG_OK;
}

static int put_time(swdg_ctx* ctx, double t, double fixed_dt) {
    int rc = put_clocks(ctx, t, 0);
    return rc ? rc : put_fixed_dt(ctx, fixed_dt);
}

// the member clocks on the host
static int read_clocks(swdg_ctx* ctx, std::vector<Member>& out) {
    out.resize(ctx->d.nmemb);
    CK(cudaMemcpyAsync(out.data(), ctx->d.mb, out.size() * sizeof(Member), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_residual(swdg_ctx* ctx, double t, double* F, double* Gx, double* Gy, double* R, double* Lx,
                  double* Ly, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "residual: no state");
    int rc = put_time(ctx, t, -1.0);
    if (rc) return rc;
    if (ctx->d.fflux) ctx->L.faces(ctx->d, ctx->tb, 0, 0.0, 0, ctx->st);
    ctx->L.residual(ctx->d, ctx->tb, 0, 0, 0.0, 0, ctx->shp[KK_RESIDUAL], ctx->st);
    CK(cudaGetLastError());
    double* dst[6] = {F, Gx, Gy, R, Lx, Ly};
    const size_t sz = (size_t)ctx->n * ctx->nd * sizeof(double);
    for (int f = 0; f < 6; ++f)
        if (dst[f])
            CK(cudaMemcpyAsync(dst[f], ctx->res + (size_t)f * ctx->n * ctx->nd, sz,
                               where == SWDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                               ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_cfl_dt(swdg_ctx* ctx, double t, double* dt) {
    if (!ctx || !dt) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "cfl_dt: no state");
    int rc = put_clocks(ctx, t, 1);
    if (!rc) rc = put_fixed_dt(ctx, -1.0);
    if (rc) return rc;
    if (ctx->d.fflux) ctx->L.faces(ctx->d, ctx->tb, 0, 0.0, 1, ctx->st);
    ctx->L.residual(ctx->d, ctx->tb, 0, 0, 0.0, 1, ctx->shp[KK_RESIDUAL], ctx->st);
    CK(cudaGetLastError());
    std::vector<Member> mh;
    rc = read_clocks(ctx, mh);
    if (rc) return rc;
    // the smallest member step: cfl / max over members of max lambda l / J
    double rmax = 0.0;
    for (const Member& m : mh) {
        double r;
        memcpy(&r, &m.rmax, sizeof r);
        rmax = std::max(rmax, r);
    }
    *dt = ctx->cfg.cfl / rmax;
    return SWDG_OK;
}

// the kernels of one time step, in stream order; with ev != nullptr an event
// pair brackets every launch (slot layout of swdg_step_profile)
// views of record slot `slot` (see AdjWs): state k = 0 v^n, 1 v~^n, 1 + l stage l, s + 1 v^{n+1};
// masks / flags k = 0 v~^n (degree switch), l stage l, s final
static double* rec_state(swdg_ctx* c, int slot, int k) {
    const size_t f4 = 4 * (size_t)c->n * c->nd;
    return c->ws.rec_u + ((size_t)slot * (c->d.s + 2) + k) * f4;
}
static uint8_t* rec_mask(swdg_ctx* c, int slot, int k) {
    return c->ws.rec_cm + ((size_t)slot * (c->d.s + 1) + k) * (size_t)c->n;
}
static uint8_t* rec_flag(swdg_ctx* c, int slot, int k) {
    return c->ws.rec_flags + ((size_t)slot * (c->d.s + 1) + k) * (size_t)c->n;
}

static int enqueue_step(swdg_ctx* ctx, cudaEvent_t (*ev)[2] = nullptr, int rec_slot = -1) {
    const Dev& d = ctx->d;
    const int s = d.s;
    const int64_t n = ctx->n;
    const size_t ub = 4 * (size_t)n * ctx->nd * sizeof(double);
    const bool rec = rec_slot >= 0;
    auto mark = [&](int slot, int which) {
        if (ev) cudaEventRecord(ev[slot][which], ctx->st);
    };
    // recording for the adjoint: v^n, v~^n and its masks, the flags after the
    // degree switch and after every stage update
    // keep the state of buffer `buf` as record state k with its masks (mask slot km)
    auto keep = [&](int buf, int k, int km) {
        if (!rec) return;
        cudaMemcpyAsync(rec_state(ctx, rec_slot, k), ctx->U + (size_t)buf * 4 * n * ctx->nd, ub,
                        cudaMemcpyDeviceToDevice, ctx->st);
        if (km >= 0)
            cudaMemcpyAsync(rec_mask(ctx, rec_slot, km), ctx->cmask + (size_t)buf * n, n,
                            cudaMemcpyDeviceToDevice, ctx->st);
    };
    auto keep_flags = [&](int k) {
        if (rec) cudaMemcpyAsync(rec_flag(ctx, rec_slot, k), ctx->flag, n, cudaMemcpyDeviceToDevice,
                                 ctx->st);
    };
    keep(0, 0, -1);
    mark(0, 0);
    ctx->L.step_begin(d, ctx->tb, 1, ctx->shp[KK_BEGIN], ctx->st);
    mark(0, 1);
    keep(0, 1, 0);
    keep_flags(0);
    for (int l = 0; l < s; ++l) {
        if (l > 0) {
            StageArgs sa{};
            sa.out_buf = l;
            sa.prev_buf = l - 1;
            sa.nres = l;
            for (int m = 0; m < l; ++m) {
                sa.wa[m] = d.a[l][m];
                sa.wat[m] = d.at[l][m];
            }
            sa.add = d.at[l][l];
            sa.use_llin = 0;
            sa.make_llin = (l == s - 1 && d.at[l][l] != 0.0) ? 1 : 0;
            sa.final_ = 0;
            mark(4 + l, 0);
            ctx->L.stage(d, ctx->tb, sa, ctx->shp[KK_STAGE], ctx->st);
            mark(4 + l, 1);
            keep(l, 1 + l, l);
            keep_flags(l);
        }
        mark(9 + l, 0);
        if (d.fflux) ctx->L.faces(d, ctx->tb, l, d.c[l], l == 0 ? 1 : 0, ctx->st);
        mark(9 + l, 1);
        mark(1 + l, 0);
        ctx->L.residual(d, ctx->tb, l, l, d.c[l], l == 0 ? 1 : 0, ctx->shp[KK_RESIDUAL], ctx->st);
        mark(1 + l, 1);
    }
    StageArgs sa{};
    sa.out_buf = 0;
    sa.prev_buf = s - 1;
    sa.nres = s;
    for (int m = 0; m < s; ++m) {
        sa.wa[m] = d.b[m];
        sa.wat[m] = d.bt[m];
    }
    sa.add = 0.0;
    sa.use_llin = (d.at[s - 1][s - 1] != 0.0) ? 1 : 0;
    sa.make_llin = 0;
    sa.final_ = 1;
    mark(8, 0);
    ctx->L.stage(d, ctx->tb, sa, ctx->shp[KK_STAGE], ctx->st);
    mark(8, 1);
    keep(0, s + 1, s);
    keep_flags(s);
    CK(cudaGetLastError());
    return SWDG_OK;
}

static int ensure_graph(swdg_ctx* ctx) {
    if (ctx->graph) return SWDG_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(ctx);
    cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, SWDG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return fail(ctx, SWDG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return SWDG_OK;
}

int swdg_step(swdg_ctx* ctx, int n_steps, double dt, double* t_inout) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "step: no state");
    if (n_steps < 0 || !std::isfinite(dt)) return fail(ctx, SWDG_EINVAL, "step: bad arguments");
    if (t_inout && ctx->nmemb > 1)
        return fail(ctx, SWDG_EINVAL,
                    "step: an ensemble keeps one clock per member; pass t_inout = NULL and use "
                    "swdg_member_times");
    {
        int rc0 = t_inout ? put_time(ctx, *t_inout, dt >= 0.0 ? dt : -1.0)
                          : put_fixed_dt(ctx, dt >= 0.0 ? dt : -1.0);
        if (rc0) return rc0;
    }
    int rc = ensure_graph(ctx);
    if (rc) return rc;
    for (int i = 0; i < n_steps; ++i) {
        if (ctx->graph) CK(cudaGraphLaunch(ctx->graph, ctx->st));
        else {
            rc = enqueue_step(ctx);
            if (rc) return rc;
        }
    }
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (t_inout) *t_inout = ctx->sc_host->m0.t;
    if (ctx->sc_host->status & ST_NAN) return fail(ctx, SWDG_ENAN, "step: non-finite state");
    return SWDG_OK;
}

int swdg_step_profile(swdg_ctx* ctx, int n_steps, double dt, double* t_inout, double* ms_out) {
    if (!ctx || !ms_out) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "step_profile: no state");
    if (n_steps < 0 || !std::isfinite(dt)) return fail(ctx, SWDG_EINVAL, "step_profile: bad arguments");
    if (t_inout && ctx->nmemb > 1)
        return fail(ctx, SWDG_EINVAL, "step_profile: pass t_inout = NULL for an ensemble");
    int rc = t_inout ? put_time(ctx, *t_inout, dt >= 0.0 ? dt : -1.0)
                     : put_fixed_dt(ctx, dt >= 0.0 ? dt : -1.0);
    if (rc) return rc;
    cudaEvent_t ev[SWDG_PROF_SLOTS][2];
    for (int i = 0; i < SWDG_PROF_SLOTS; ++i) {
        ms_out[i] = 0.0;
        CK(cudaEventCreate(&ev[i][0]));
        CK(cudaEventCreate(&ev[i][1]));
    }
    bool used[SWDG_PROF_SLOTS] = {};
    used[0] = used[8] = true;
    for (int l = 0; l < ctx->d.s; ++l) {
        used[1 + l] = true;
        used[9 + l] = ctx->d.fflux != nullptr;
        if (l > 0) used[4 + l] = true;
    }
    for (int i = 0; i < n_steps; ++i) {
        rc = enqueue_step(ctx, ev);
        if (rc) return rc;
        CK(cudaStreamSynchronize(ctx->st));
        for (int k = 0; k < SWDG_PROF_SLOTS; ++k) {
            if (!used[k]) continue;
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ev[k][0], ev[k][1]));
            ms_out[k] += ms;
        }
    }
    for (int i = 0; i < SWDG_PROF_SLOTS; ++i) {
        cudaEventDestroy(ev[i][0]);
        cudaEventDestroy(ev[i][1]);
    }
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (t_inout) *t_inout = ctx->sc_host->m0.t;
    if (ctx->sc_host->status & ST_NAN) return fail(ctx, SWDG_ENAN, "step_profile: non-finite state");
    return SWDG_OK;
}

int swdg_degree_switch(swdg_ctx* ctx, uint8_t* flags_out) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "degree_switch: no state");
    ctx->L.step_begin(ctx->d, ctx->tb, 1, ctx->shp[KK_BEGIN], ctx->st);
    CK(cudaGetLastError());
    if (flags_out)
        CK(cudaMemcpyAsync(flags_out, ctx->flag, ctx->n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

// device copies of the gauge points xy [n][2] and of the cell holding each
// (the first containing cell of [k0, k1), -1 outside); the points are located
// again only when they or the range change
static int gauges_prepare(swdg_ctx* ctx, int n, const double* xy, int64_t k0, int64_t k1) {
    if (n > ctx->gcap) {
        cudaFree(ctx->gdev);
        cudaFree(ctx->gcell);
        ctx->gdev = nullptr;
        ctx->gcell = nullptr;
        ctx->gcap = 0;
        ctx->gxy.clear();
        CK(cudaMalloc(&ctx->gdev, 3 * (size_t)n * sizeof(double)));
        CK(cudaMalloc(&ctx->gcell, (size_t)n * sizeof(int32_t)));
        ctx->gcap = n;
    }
    if ((int64_t)ctx->gxy.size() == 2 * (int64_t)n && ctx->gk0 == k0 && ctx->gk1 == k1 &&
        memcmp(ctx->gxy.data(), xy, 2 * (size_t)n * sizeof(double)) == 0)
        return SWDG_OK;
    std::vector<int32_t> cell(n, -1);
    for (int g = 0; g < n; ++g) {
        const double x = xy[2 * g], y = xy[2 * g + 1];
        for (int64_t k = k0; k < k1; ++k) {
            const double x0 = ctx->x0y0_h[2 * k], y0 = ctx->x0y0_h[2 * k + 1];
            if (x >= x0 && x <= x0 + ctx->hxhy_h[2 * k] && y >= y0 &&
                y <= y0 + ctx->hxhy_h[2 * k + 1]) {
                cell[g] = (int32_t)k;
                break;
            }
        }
    }
    CK(cudaMemcpyAsync(ctx->gdev, xy, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaMemcpyAsync(ctx->gcell, cell.data(), (size_t)n * sizeof(int32_t),
                       cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->gxy.assign(xy, xy + 2 * (size_t)n);
    ctx->gk0 = k0;
    ctx->gk1 = k1;
    return SWDG_OK;
}

int swdg_gather_gauges(swdg_ctx* ctx, int n, const double* xy, double* out) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "gather_gauges: no state");
    if (n < 0 || (n > 0 && (!xy || !out))) return fail(ctx, SWDG_EINVAL, "gather_gauges: bad arguments");
    if (n == 0) return SWDG_OK;
    int rc = gauges_prepare(ctx, n, xy, 0, ctx->n);
    if (rc) return rc;
    ctx->L.gauges(ctx->d, ctx->tb, n, ctx->gdev, ctx->gdev + 2 * n, 0, ctx->n, ctx->gcell, ctx->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, ctx->gdev + 2 * n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_gauges_vjp(swdg_ctx* ctx, int n, const double* xy, const double* gbar, double* zeta_b,
                    int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "gauges_vjp: no state");
    if (n < 0 || (n > 0 && (!xy || !gbar || !zeta_b)) || (where != SWDG_HOST && where != SWDG_DEVICE))
        return fail(ctx, SWDG_EINVAL, "gauges_vjp: bad arguments");
    if (n == 0) return SWDG_OK;
    const size_t fb = (size_t)ctx->n * ctx->nd * sizeof(double);
    int rc = gauges_prepare(ctx, n, xy, 0, ctx->n);
    if (rc) return rc;
    double* gb = ctx->gdev + 2 * n;
    CK(cudaMemcpyAsync(gb, gbar, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    double* zb = zeta_b;
    double* tmp = nullptr;
    if (where == SWDG_HOST) {
        CK(cudaMalloc(&tmp, fb));
        zb = tmp;
        CK(cudaMemcpyAsync(zb, zeta_b, fb, cudaMemcpyHostToDevice, ctx->st));
    }
    ctx->L.gauges_vjp(ctx->d, ctx->tb, n, ctx->gdev, gb, zb, ctx->gcell, ctx->st);
    CK(cudaGetLastError());
    if (where == SWDG_HOST) CK(cudaMemcpyAsync(zeta_b, zb, fb, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    cudaFree(tmp);
    return SWDG_OK;
}

int swdg_diagnostics(swdg_ctx* ctx, double out[8]) {
    if (!ctx || !out) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "diagnostics: no state");
    ctx->L.cell_diag(ctx->d, ctx->tb, ctx->diag, ctx->shp[KK_AUX], ctx->st);
    k_diag_reduce<<<1, 256, 0, ctx->st>>>(ctx->diag, nullptr, 0, ctx->n, ctx->diag + 4 * ctx->n);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->pin, ctx->diag + 4 * ctx->n, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    out[0] = ctx->pin[0];
    out[1] = ctx->pin[1];
    out[2] = ctx->pin[2];
    out[3] = ctx->pin[3];
    out[4] = ctx->sc_host->maxits;
    out[5] = ctx->sc_host->viol;
    std::vector<Member> mh;
    int rc = read_clocks(ctx, mh);
    if (rc) return rc;
    out[6] = mh[0].dt_last; // member 0 of an ensemble
    out[7] = mh[0].t;
    return SWDG_OK;
}

// ---------------------------------------------------------------------------
// discrete adjoint of the residual
// ---------------------------------------------------------------------------
int swdg_residual_vjp(swdg_ctx* ctx, double t, const double* Fb, const double* Gxb,
                      const double* Gyb, const double* Rb, const double* Lxb, const double* Lyb,
                      double* zeta_b, double* qx_b, double* qy_b, double* c_b, double* manning_b,
                      double* delta_b, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "residual_vjp: no state");
    if (where != SWDG_HOST && where != SWDG_DEVICE)
        return fail(ctx, SWDG_EINVAL, "residual_vjp: bad where");
    const int64_t n = ctx->n;
    const size_t f = (size_t)n * ctx->nd, fb = f * sizeof(double);
    if (!ctx->adj) CK(cudaMalloc(&ctx->adj, (10 * f + 2 * (size_t)n) * sizeof(double)));
    const cudaMemcpyKind in = where == SWDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = where == SWDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const double* src[6] = {Fb, Gxb, Gyb, Rb, Lxb, Lyb};
    for (int i = 0; i < 6; ++i) {
        if (src[i]) CK(cudaMemcpyAsync(ctx->adj + i * f, src[i], fb, in, ctx->st));
        else CK(cudaMemsetAsync(ctx->adj + i * f, 0, fb, ctx->st));
    }
    int rc = put_clocks(ctx, t, 0);
    if (rc) return rc;
    double* ub = ctx->adj + 6 * f;
    double* nb = ctx->adj + 10 * f;
    double* db = nb + n;
    ctx->L.residual_vjp(ctx->d, ctx->tb, ctx->U, ctx->cmask, ctx->adj, ub, nb, db, 0,
                        Shape{grid_for(n), WPB}, ctx->st);
    CK(cudaGetLastError());
    double* dst[4] = {zeta_b, qx_b, qy_b, c_b};
    for (int i = 0; i < 4; ++i)
        if (dst[i]) CK(cudaMemcpyAsync(dst[i], ub + i * f, fb, out, ctx->st));
    if (manning_b) CK(cudaMemcpyAsync(manning_b, nb, n * sizeof(double), out, ctx->st));
    if (delta_b) CK(cudaMemcpyAsync(delta_b, db, n * sizeof(double), out, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

// ---------------------------------------------------------------------------
// discrete adjoint of a time step
// ---------------------------------------------------------------------------
static int adjoint_ready(swdg_ctx* ctx, const char* who) {
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "%s: no state", who);
    if (ctx->cfg.precision != 0)
        return fail(ctx, SWDG_EINVAL, "%s: the step adjoint differentiates the FP64 path", who);
    if (ctx->nmemb != 1) return fail(ctx, SWDG_EINVAL, "%s: not for an ensemble", who);
    return SWDG_OK;
}

static int alloc_scratch(swdg_ctx* ctx) {
    auto& w = ctx->ws;
    if (w.ubs) return SWDG_OK;
    const int64_t n = ctx->n;
    const size_t f = (size_t)n * ctx->nd;
    CK(cudaMalloc(&w.ubs, (size_t)MXS * 4 * f * sizeof(double)));
    CK(cudaMalloc(&w.rbar, (size_t)MXS * 6 * f * sizeof(double)));
    CK(cudaMalloc(&w.llb, 2 * f * sizeof(double)));
    CK(cudaMalloc(&w.HNb, f * sizeof(double)));
    CK(cudaMalloc(&w.CNb, f * sizeof(double)));
    CK(cudaMalloc(&w.nbar, n * sizeof(double)));
    CK(cudaMalloc(&w.dbar, n * sizeof(double)));
    CK(cudaMalloc(&w.vb, 4 * f * sizeof(double)));
    CK(cudaMalloc(&w.ubpre, 4 * f * sizeof(double)));
    return SWDG_OK;
}

int swdg_adjoint_slots(swdg_ctx* ctx, int nslots) {
    if (!ctx) return SWDG_EINVAL;
    int rc = adjoint_ready(ctx, "adjoint_slots");
    if (rc) return rc;
    if (nslots < 1 || nslots > 4096) return fail(ctx, SWDG_EINVAL, "adjoint_slots: 1..4096 slots");
    auto& w = ctx->ws;
    if (nslots == w.nslots) return SWDG_OK;
    cudaFree(w.rec_u);
    cudaFree(w.rec_cm);
    cudaFree(w.rec_flags);
    w.rec_u = nullptr;
    w.rec_cm = w.rec_flags = nullptr;
    w.nslots = 0;
    const int s = ctx->d.s;
    const size_t f4 = 4 * (size_t)ctx->n * ctx->nd;
    CK(cudaMalloc(&w.rec_u, (size_t)nslots * (s + 2) * f4 * sizeof(double)));
    CK(cudaMalloc(&w.rec_cm, (size_t)nslots * (s + 1) * ctx->n));
    CK(cudaMalloc(&w.rec_flags, (size_t)nslots * (s + 1) * ctx->n));
    w.nslots = nslots;
    w.t0.assign(nslots, 0.0);
    w.dt.assign(nslots, 0.0);
    w.valid.assign(nslots, 0);
    return alloc_scratch(ctx);
}

int swdg_step_record_slot(swdg_ctx* ctx, int slot, double dt, double* t_inout) {
    if (!ctx) return SWDG_EINVAL;
    int rc = adjoint_ready(ctx, "step_record");
    if (rc) return rc;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, SWDG_EINVAL, "step_record: dt > 0 required");
    auto& w = ctx->ws;
    if (slot < 0 || slot >= w.nslots) return fail(ctx, SWDG_EINVAL, "step_record: bad slot %d", slot);
    std::vector<Member> mh;
    rc = read_clocks(ctx, mh);
    if (rc) return rc;
    const double t0 = t_inout ? *t_inout : mh[0].t;
    rc = put_time(ctx, t0, dt);
    if (rc) return rc;
    rc = enqueue_step(ctx, nullptr, slot);
    if (rc) return rc;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    w.t0[slot] = t0;
    w.dt[slot] = dt;
    w.valid[slot] = 1;
    if (t_inout) *t_inout = ctx->sc_host->m0.t;
    if (ctx->sc_host->status & ST_NAN) return fail(ctx, SWDG_ENAN, "step_record: non-finite state");
    return SWDG_OK;
}

int swdg_step_record(swdg_ctx* ctx, double dt, double* t_inout) {
    if (!ctx) return SWDG_EINVAL;
    if (ctx->ws.nslots < 1) {
        int rc = swdg_adjoint_slots(ctx, 1);
        if (rc) return rc;
    }
    return swdg_step_record_slot(ctx, 0, dt, t_inout);
}

int swdg_step_vjp_slot(swdg_ctx* ctx, int slot, const double* zeta_b, const double* qx_b,
                       const double* qy_b, const double* c_b, double* zeta_b_out, double* qx_b_out,
                       double* qy_b_out, double* c_b_out, double* manning_b, double* delta_b,
                       int where) {
    if (!ctx) return SWDG_EINVAL;
    int rc = adjoint_ready(ctx, "step_vjp");
    if (rc) return rc;
    auto& w = ctx->ws;
    if (slot < 0 || slot >= w.nslots || !w.valid[slot])
        return fail(ctx, SWDG_ESTATE, "step_vjp: no recorded step in slot %d (swdg_step_record)", slot);
    if (where != SWDG_HOST && where != SWDG_DEVICE) return fail(ctx, SWDG_EINVAL, "step_vjp: bad where");
    const Dev& d = ctx->d;
    const int64_t n = ctx->n;
    const int s = d.s;
    const size_t f = (size_t)n * ctx->nd, fb = f * sizeof(double);
    const double t0 = w.t0[slot], dt = w.dt[slot];
    const cudaMemcpyKind in = where == SWDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out = where == SWDG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const double* src[4] = {zeta_b, qx_b, qy_b, c_b};
    for (int i = 0; i < 4; ++i) {
        if (src[i]) CK(cudaMemcpyAsync(w.vb + i * f, src[i], fb, in, ctx->st));
        else CK(cudaMemsetAsync(w.vb + i * f, 0, fb, ctx->st));
    }
    CK(cudaMemsetAsync(w.ubs, 0, (size_t)s * 4 * fb, ctx->st));
    CK(cudaMemsetAsync(w.rbar, 0, (size_t)s * 6 * fb, ctx->st));
    CK(cudaMemsetAsync(w.llb, 0, 2 * fb, ctx->st));
    CK(cudaMemsetAsync(w.HNb, 0, fb, ctx->st));
    CK(cudaMemsetAsync(w.CNb, 0, fb, ctx->st));
    CK(cudaMemsetAsync(w.nbar, 0, n * sizeof(double), ctx->st));
    CK(cudaMemsetAsync(w.dbar, 0, n * sizeof(double), ctx->st));
    const Shape shp{grid_for(n), WPB};
    // stage l state and masks of the recorded step (l = 0: v~^n)
    auto ust = [&](int l) { return rec_state(ctx, slot, 1 + l); };
    auto cst = [&](int l) { return rec_mask(ctx, slot, l); };
    const double* vtil = ust(0);
    const uint8_t* cmtil = cst(0);
    const bool imp = d.at[s - 1][s - 1] != 0.0;
    // final combination (weights b, b~, no implicit diagonal)
    StageVjpArgs a{};
    a.un = vtil;
    a.cmn = cmtil;
    a.rbar = w.rbar;
    a.HNb = w.HNb;
    a.CNb = w.CNb;
    a.ubn = w.ubs;
    a.nbar = w.nbar;
    a.dbar = w.dbar;
    a.dt = dt;
    a.uo = rec_state(ctx, slot, s + 1);
    a.cmo = rec_mask(ctx, slot, s);
    a.up = ust(s - 1);
    a.cmp = cst(s - 1);
    a.flag = rec_flag(ctx, slot, s);
    a.vb = w.vb;
    a.llb_in = nullptr;
    a.llb_out = w.llb;
    a.ubp = w.ubs + (size_t)(s - 1) * 4 * f;
    for (int m = 0; m < s; ++m) {
        a.wa[m] = d.b[m];
        a.wat[m] = d.bt[m];
    }
    a.add = 0.0;
    a.nres = s;
    a.make_llin = 0;
    a.use_llin = imp ? 1 : 0;
    ctx->L.stage_vjp(d, ctx->tb, a, shp, ctx->st);
    CK(cudaGetLastError());
    for (int l = s - 1; l >= 0; --l) {
        // residual of stage l at t^n + c_l dt
        rc = put_clocks(ctx, t0 + d.c[l] * dt, 0);
        if (rc) return rc;
        ctx->L.residual_vjp(d, ctx->tb, ust(l), cst(l), w.rbar + (size_t)l * 6 * f,
                            w.ubs + (size_t)l * 4 * f, w.nbar, w.dbar, 1, shp, ctx->st);
        CK(cudaGetLastError());
        if (l == 0) break;
        StageVjpArgs b = a;
        b.uo = ust(l);
        b.cmo = cst(l);
        b.up = ust(l - 1);
        b.cmp = cst(l - 1);
        b.flag = rec_flag(ctx, slot, l);
        b.vb = w.ubs + (size_t)l * 4 * f;
        b.make_llin = (l == s - 1 && d.at[l][l] != 0.0) ? 1 : 0;
        b.llb_in = b.make_llin ? w.llb : nullptr;
        b.llb_out = nullptr;
        b.use_llin = 0;
        b.ubp = w.ubs + (size_t)(l - 1) * 4 * f;
        for (int m = 0; m < MXS; ++m) {
            b.wa[m] = m < l ? d.a[l][m] : 0.0;
            b.wat[m] = m < l ? d.at[l][m] : 0.0;
        }
        b.add = d.at[l][l];
        b.nres = l;
        ctx->L.stage_vjp(d, ctx->tb, b, shp, ctx->st);
        CK(cudaGetLastError());
    }
    BeginVjpArgs bg{};
    bg.upre = rec_state(ctx, slot, 0);
    bg.un = vtil;
    bg.cmn = cmtil;
    bg.flag0 = rec_flag(ctx, slot, 0);
    bg.HNb = w.HNb;
    bg.CNb = w.CNb;
    bg.ubn = w.ubs;
    bg.ubpre = w.ubpre;
    bg.dbar = w.dbar;
    ctx->L.begin_vjp(d, ctx->tb, bg, shp, ctx->st);
    CK(cudaGetLastError());
    rc = put_clocks(ctx, t0 + dt, 0);
    if (rc) return rc;
    double* dst[4] = {zeta_b_out, qx_b_out, qy_b_out, c_b_out};
    for (int i = 0; i < 4; ++i)
        if (dst[i]) CK(cudaMemcpyAsync(dst[i], w.ubpre + i * f, fb, out, ctx->st));
    if (manning_b) CK(cudaMemcpyAsync(manning_b, w.nbar, n * sizeof(double), out, ctx->st));
    if (delta_b) CK(cudaMemcpyAsync(delta_b, w.dbar, n * sizeof(double), out, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_step_vjp(swdg_ctx* ctx, const double* zeta_b, const double* qx_b, const double* qy_b,
                  const double* c_b, double* zeta_b_out, double* qx_b_out, double* qy_b_out,
                  double* c_b_out, double* manning_b, double* delta_b, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (ctx->ws.nslots < 1) return fail(ctx, SWDG_ESTATE, "step_vjp: no recorded step (swdg_step_record)");
    return swdg_step_vjp_slot(ctx, 0, zeta_b, qx_b, qy_b, c_b, zeta_b_out, qx_b_out, qy_b_out,
                              c_b_out, manning_b, delta_b, where);
}

// ---------------------------------------------------------------------------
// per-cell bathymetry offsets (the parameter of the step adjoint)
// ---------------------------------------------------------------------------
} // extern "C"

template <typename Pix>
__global__ void k_offset_tiles(const Pix* __restrict__ base, Pix* tiles, const int64_t* off,
                               const uint8_t* pcls, const OvTab* ov, const double* delta,
                               int64_t n) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < n; k += nw) {
        const int P = ov[pcls[k]].P;
        const double dk = delta ? delta[k] : 0.0;
        for (int i = lane; i < P * P; i += 32)
            tiles[off[k] + i] = (Pix)((double)base[off[k] + i] + dk);
    }
}

// mode P: every sampled depth of cell k moves by delta_k; bounds from the mass points
__global__ void k_offset_points(const double* __restrict__ base, double* zpts, double* zhang,
                                double* zmax, double* zmin, double* zabs, const double* delta,
                                int nzp, int nv2, int nm2, int zh, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double dk = delta ? delta[k] : 0.0;
        double m = -INFINITY, mn = INFINITY, a = 0.0;
        for (int p = 0; p < nzp; ++p) {
            const double z = base[k * nzp + p] + dk;
            zpts[k * nzp + p] = z;
            if (p >= nv2 && p < nv2 + nm2) {
                m = fmax(m, z);
                mn = fmin(mn, z);
                a = fmax(a, fabs(z));
            }
        }
        for (int i = 0; i < zh; ++i) zhang[k * zh + i] = base[n * nzp + k * zh + i] + dk;
        zmax[k] = m;
        zmin[k] = mn;
        zabs[k] = a;
    }
}

extern "C" {

int swdg_set_bathymetry_offset(swdg_ctx* ctx, const double* delta, int where) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_bathy) return fail(ctx, SWDG_ESTATE, "set_bathymetry_offset: no bathymetry");
    if (where != SWDG_HOST && where != SWDG_DEVICE)
        return fail(ctx, SWDG_EINVAL, "set_bathymetry_offset: bad where");
    const int64_t n = ctx->n;
    const int R_ = ctx->R, nv_ = (3 * R_) / 2 + 1, nm_ = R_ + 2, ng_ = R_ + 1;
    const int nzp_ = nv_ * nv_ + nm_ * nm_ + ng_ * ng_, zh = 8 * nm_;
    const size_t es = ctx->pix == 0 ? 4 : 8;
    double* dd = nullptr;
    if (delta) {
        if (where == SWDG_HOST) {
            for (int64_t k = 0; k < n; ++k)
                if (!std::isfinite(delta[k]))
                    return fail(ctx, SWDG_EINVAL, "set_bathymetry_offset: bad value at cell %lld",
                                (long long)k);
        }
        CK(cudaMalloc(&dd, n * sizeof(double)));
        CK(cudaMemcpyAsync(dd, delta, n * sizeof(double),
                           where == SWDG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           ctx->st));
    }
    const int gw = (int)std::min<int64_t>(152 * 32, (n * 32 + 255) / 256 + 1);
    if (ctx->mode == 0) {
        if (!ctx->tiles0) { // keep the uploaded pixels
            CK(cudaMalloc(&ctx->tiles0, (size_t)ctx->npix * es));
            CK(cudaMemcpyAsync(ctx->tiles0, ctx->tiles, (size_t)ctx->npix * es,
                               cudaMemcpyDeviceToDevice, ctx->st));
        }
        if (ctx->pix == 0)
            k_offset_tiles<float><<<gw, 256, 0, ctx->st>>>((const float*)ctx->tiles0,
                                                          (float*)ctx->tiles, ctx->tile_off,
                                                          ctx->pcls, ctx->ov, dd, n);
        else
            k_offset_tiles<double><<<gw, 256, 0, ctx->st>>>((const double*)ctx->tiles0,
                                                           (double*)ctx->tiles, ctx->tile_off,
                                                           ctx->pcls, ctx->ov, dd, n);
        // bounds, sub-cell means and coarse-side strips of the moved pixels
        if (ctx->pix == 0) {
            k_tile_bounds<float><<<gw, 256, 0, ctx->st>>>((const float*)ctx->tiles, ctx->tile_off,
                                                         ctx->pcls, ctx->ov, n, ctx->zmax, ctx->zmin,
                                                         ctx->zabs);
            k_subcell_means<float><<<gw, 256, 0, ctx->st>>>(
                (const float*)ctx->tiles, ctx->tile_off, ctx->pcls, ctx->ov, ctx->finfo, nv_, nm_, ng_,
                ctx->zpts, ctx->zhang, ctx->zsb, n);
        } else {
            k_tile_bounds<double><<<gw, 256, 0, ctx->st>>>((const double*)ctx->tiles, ctx->tile_off,
                                                          ctx->pcls, ctx->ov, n, ctx->zmax,
                                                          ctx->zmin, ctx->zabs);
            k_subcell_means<double><<<gw, 256, 0, ctx->st>>>(
                (const double*)ctx->tiles, ctx->tile_off, ctx->pcls, ctx->ov, ctx->finfo, nv_, nm_,
                ng_, ctx->zpts, ctx->zhang, ctx->zsb, n);
        }
    } else {
        if (!ctx->zpts0) { // keep the uploaded samples: [n][nzp] then [n][8 nm]
            CK(cudaMalloc(&ctx->zpts0, (size_t)n * (nzp_ + zh) * sizeof(double)));
            CK(cudaMemcpyAsync(ctx->zpts0, ctx->zpts, (size_t)n * nzp_ * sizeof(double),
                               cudaMemcpyDeviceToDevice, ctx->st));
            CK(cudaMemcpyAsync(ctx->zpts0 + (size_t)n * nzp_, ctx->zhang, (size_t)n * zh * sizeof(double),
                               cudaMemcpyDeviceToDevice, ctx->st));
        }
        k_offset_points<<<(int)std::min<int64_t>(152 * 16, (n + 127) / 128), 128, 0, ctx->st>>>(
            ctx->zpts0, ctx->zpts, ctx->zhang, ctx->zmax, ctx->zmin, ctx->zabs, dd, nzp_,
            nv_ * nv_, nm_ * nm_, zh, n);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->st));
    cudaFree(dd);
    return SWDG_OK;
}

// ---------------------------------------------------------------------------
// dynamic h-adaptation (Sec. 3.4)
// ---------------------------------------------------------------------------
int swdg_amr_setup(swdg_ctx* ctx, const swdg_forest* f) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_mesh) return fail(ctx, SWDG_ESTATE, "amr_setup: no mesh");
    if (ctx->nmemb != 1) return fail(ctx, SWDG_EINVAL, "amr_setup: not for an ensemble");
    if (!forest_valid(f)) return fail(ctx, SWDG_EINVAL, "amr_setup: bad forest");
    Forest F{*f};
    std::vector<Leaf> lv;
    if (!F.leaves_of(ctx->n, ctx->x0y0_h.data(), ctx->hxhy_h.data(), lv))
        return fail(ctx, SWDG_EINVAL, "amr_setup: a cell is not a leaf of the forest");
    std::vector<double> x(2 * ctx->n), h(2 * ctx->n);
    std::vector<int32_t> nb(8 * ctx->n);
    try {
        F.mesh(lv, x.data(), h.data(), nb.data());
    } catch (...) {
        return fail(ctx, SWDG_EINVAL, "amr_setup: the cells are not a 2:1-balanced leaf set");
    }
    if (nb != ctx->nbr_h)
        return fail(ctx, SWDG_EINVAL,
                    "amr_setup: the mesh's neighbours differ from the forest's (tags, periodicity)");
    ctx->forest = *f;
    ctx->leaves = lv;
    ctx->amr = true;
    ctx->keep_raster = true;
    return SWDG_OK;
}

int swdg_amr_leaves(const swdg_ctx* ctx, int32_t* lij) {
    if (!ctx || !lij || !ctx->amr) return SWDG_EINVAL;
    for (size_t k = 0; k < ctx->leaves.size(); ++k) {
        lij[3 * k] = ctx->leaves[k].l;
        lij[3 * k + 1] = ctx->leaves[k].i;
        lij[3 * k + 2] = ctx->leaves[k].j;
    }
    return SWDG_OK;
}

int swdg_amr_indicator(swdg_ctx* ctx, int kind, double* eta) {
    if (!ctx || !eta) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "amr_indicator: no state");
    if (kind != 0 && kind != 1) return fail(ctx, SWDG_EINVAL, "amr_indicator: kind 0 or 1");
    double* buf = nullptr;
    CK(cudaMalloc(&buf, ctx->n * sizeof(double)));
    ctx->L.indicator(ctx->d, ctx->tb, kind, buf, Shape{grid_for(ctx->n), WPB}, ctx->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(eta, buf, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    cudaFree(buf);
    return SWDG_OK;
}

int swdg_amr_adapt(swdg_ctx* ctx, const double* eta_in, int kind, double theta_r, double theta_c,
                   double* report) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->amr) return fail(ctx, SWDG_ESTATE, "amr_adapt: no forest (swdg_amr_setup)");
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "amr_adapt: no state");
    if (ctx->ras_h.empty()) return fail(ctx, SWDG_ESTATE, "amr_adapt: no raster to re-tile");
    if (!std::isfinite(theta_r) || !std::isfinite(theta_c))
        return fail(ctx, SWDG_EINVAL, "amr_adapt: bad thresholds");
    const int64_t n = ctx->n;
    const int nd = ctx->nd;
    using clk = std::chrono::steady_clock;
    auto ms = [](clk::time_point a, clk::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    const clk::time_point c0 = clk::now();
    std::vector<double> eta(n);
    if (eta_in) {
        for (int64_t k = 0; k < n; ++k) {
            if (!std::isfinite(eta_in[k]) || eta_in[k] < 0.0)
                return fail(ctx, SWDG_EINVAL, "amr_adapt: bad indicator at cell %lld", (long long)k);
            eta[k] = eta_in[k];
        }
    } else {
        int rc = swdg_amr_indicator(ctx, kind, eta.data());
        if (rc) return rc;
    }
    const clk::time_point c1 = clk::now();
    Forest F{ctx->forest};
    std::vector<int8_t> fl(n);
    F.flags(ctx->leaves, eta.data(), theta_r, theta_c, fl.data());
    std::vector<Leaf> nl = F.adapt(ctx->leaves, fl.data());
    const int64_t n2 = (int64_t)nl.size();
    // the plan of every new cell
    CellIndex old(ctx->forest);
    for (int64_t k = 0; k < n; ++k)
        old.set(ctx->leaves[k].l, ctx->leaves[k].i, ctx->leaves[k].j, (int32_t)k);
    std::vector<int8_t> type(n2);
    std::vector<int32_t> src(4 * n2, 0);
    std::vector<double> rel(3 * n2, 0.0);
    int64_t nref = 0, npar = 0;
    bool same = n2 == n;
    for (int64_t k = 0; k < n2; ++k) {
        const Leaf c = nl[k];
        int32_t v = old.get(c.l, c.i, c.j);
        if (v >= 0) {
            type[k] = 0;
            src[4 * k] = v;
            if (v != k) same = false;
            continue;
        }
        same = false;
        int la = c.l - 1;
        int64_t ia = c.i >> 1, ja = c.j >> 1;
        for (; la >= 0; --la, ia >>= 1, ja >>= 1) {
            v = old.get(la, ia, ja);
            if (v >= 0) break;
        }
        if (la >= 0) {
            type[k] = 1;
            src[4 * k] = v;
            const double s_ = 1.0 / (double)(1 << (c.l - la));
            rel[3 * k] = s_;
            rel[3 * k + 1] = c.i * s_ - (double)ia;
            rel[3 * k + 2] = c.j * s_ - (double)ja;
            continue;
        }
        type[k] = 2;
        ++npar;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int32_t ch = c.l + 1 <= ctx->forest.max_level
                                       ? old.get(c.l + 1, 2 * (int64_t)c.i + a, 2 * (int64_t)c.j + b)
                                       : -1;
                if (ch < 0)
                    return fail(ctx, SWDG_EINVAL, "amr_adapt: internal: a new parent without its children");
                src[4 * k + a + 2 * b] = ch;
            }
    }
    for (int64_t k = 0; k < n; ++k)
        if (fl[k] == 1) ++nref;
    double d0[8], d1[8];
    int rc = swdg_diagnostics(ctx, d0);
    if (rc) return rc;
    if (same) {
        if (report) {
            const double rr[9] = {(double)n, (double)n, 0.0, 0.0, 0.0, 0.0, ms(c0, c1),
                                  ms(c1, clk::now()), 0.0};
            memcpy(report, rr, sizeof rr);
        }
        return SWDG_OK;
    }
    // every new cell must span whole, aligned pixels (mode S)
    std::vector<double> x(2 * n2), h(2 * n2);
    std::vector<int32_t> nb(8 * n2);
    F.mesh(nl, x.data(), h.data(), nb.data());
    if (ctx->mode == 0) {
        const double dx = ctx->ras_geo[2], dy = ctx->ras_geo[3];
        for (int64_t k = 0; k < n2; ++k) {
            const double px = h[2 * k] / dx, py = h[2 * k + 1] / dy;
            const double cx = (x[2 * k] - ctx->ras_geo[0]) / dx, cy = (x[2 * k + 1] - ctx->ras_geo[1]) / dy;
            if (std::fabs(px - std::round(px)) > 1e-6 || std::fabs(py - std::round(py)) > 1e-6 ||
                std::round(px) < 1 || std::round(px) > MXPIX || std::round(px) != std::round(py) ||
                std::fabs(cx - std::round(cx)) > 1e-6 || std::fabs(cy - std::round(cy)) > 1e-6)
                return fail(ctx, SWDG_EINVAL,
                            "amr_adapt: new cell %lld would not span whole pixels (raise h_min)",
                            (long long)k);
        }
    }
    const clk::time_point c2 = clk::now();
    // remap the state on the device
    int8_t* dtype_ = nullptr;
    int32_t* dsrc = nullptr;
    double *drel = nullptr, *unew = nullptr;
    CK(cudaMalloc(&dtype_, n2));
    CK(cudaMalloc(&dsrc, 4 * n2 * sizeof(int32_t)));
    CK(cudaMalloc(&drel, 3 * n2 * sizeof(double)));
    CK(cudaMalloc(&unew, 4 * (size_t)n2 * nd * sizeof(double)));
    CK(cudaMemcpyAsync(dtype_, type.data(), n2, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(dsrc, src.data(), 4 * n2 * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(drel, rel.data(), 3 * n2 * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
    RemapArgs ra{ctx->U, n, dtype_, dsrc, drel, unew, n2};
    ctx->L.remap(ctx->tb, ra, Shape{grid_for(n2), WPB}, ctx->st);
    CK(cudaGetLastError());
    // per-cell coefficients: children inherit, a parent takes its children's mean
    std::vector<double> man(n), nu;
    CK(cudaMemcpyAsync(man.data(), ctx->manning, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (ctx->nu_c) {
        nu.resize(n);
        CK(cudaMemcpyAsync(nu.data(), ctx->nu_c, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    }
    CK(cudaStreamSynchronize(ctx->st));
    auto carry = [&](const std::vector<double>& a) {
        std::vector<double> b(n2);
        for (int64_t k = 0; k < n2; ++k) {
            if (type[k] == 2)
                b[k] = 0.25 * (a[src[4 * k]] + a[src[4 * k + 1]] + a[src[4 * k + 2]] + a[src[4 * k + 3]]);
            else
                b[k] = a[src[4 * k]];
        }
        return b;
    };
    const std::vector<double> man2 = carry(man);
    const std::vector<double> nu2 = nu.empty() ? std::vector<double>() : carry(nu);
    // the new mesh, bathymetry, coefficients and state
    rc = swdg_upload_mesh(ctx, n2, x.data(), h.data(), nb.data());
    // the kept raster (its host copy is the same data: nothing is copied)
    ctx->reuse_raster = true;
    if (!rc) rc = swdg_upload_bathymetry(ctx, ctx->ras_h.data(), ctx->ras_dtype, ctx->ras_nx,
                                        ctx->ras_ny, ctx->ras_geo[0], ctx->ras_geo[1],
                                        ctx->ras_geo[2], ctx->ras_geo[3]);
    ctx->reuse_raster = false;
    if (!rc) rc = swdg_set_manning(ctx, man2.data(), SWDG_HOST);
    if (!rc && !nu2.empty()) rc = swdg_set_tracer_diffusivity(ctx, nu2.data(), SWDG_HOST);
    const size_t fb = (size_t)n2 * nd;
    if (!rc) rc = swdg_set_state(ctx, unew, unew + fb, unew + 2 * fb, unew + 3 * fb, SWDG_DEVICE);
    cudaFree(dtype_);
    cudaFree(dsrc);
    cudaFree(drel);
    cudaFree(unew);
    if (rc) return rc;
    ctx->leaves = nl;
    ctx->amr = true;
    rc = swdg_diagnostics(ctx, d1);
    if (rc) return rc;
    if (report) {
        const double rr[9] = {(double)n, (double)n2, (double)nref, (double)npar, d1[0] - d0[0],
                              d1[1] - d0[1], ms(c0, c1), ms(c1, c2), ms(c2, clk::now())};
        memcpy(report, rr, sizeof rr);
    }
    return SWDG_OK;
}

// ---------------------------------------------------------------------------
// ensembles: independent members stepped by the same launches
// ---------------------------------------------------------------------------
int swdg_set_members(swdg_ctx* ctx, int n_members, const int64_t* first_cell) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_mesh) return fail(ctx, SWDG_ESTATE, "set_members: no mesh");
    if (n_members < 1 || n_members > SWDG_MAX_MEMBERS || !first_cell)
        return fail(ctx, SWDG_EINVAL, "set_members: 1..%d members and first_cell required",
                    SWDG_MAX_MEMBERS);
    const int64_t n = ctx->n;
    if (first_cell[0] != 0 || first_cell[n_members] != n)
        return fail(ctx, SWDG_EINVAL, "set_members: first_cell must run from 0 to n_cells");
    for (int m = 0; m < n_members; ++m)
        if (first_cell[m + 1] <= first_cell[m])
            return fail(ctx, SWDG_EINVAL, "set_members: member %d has no cells", m);
    // members are independent problems: no face may join two of them
    std::vector<int32_t> mh(n);
    for (int m = 0; m < n_members; ++m)
        for (int64_t k = first_cell[m]; k < first_cell[m + 1]; ++k) mh[k] = m;
    for (int64_t k = 0; k < n; ++k)
        for (int j = 0; j < 8; ++j) {
            const int32_t nb = ctx->nbr_h[8 * k + j];
            if (nb >= 0 && mh[nb] != mh[k])
                return fail(ctx, SWDG_EINVAL,
                            "set_members: cell %lld (member %d) neighbours cell %d of member %d",
                            (long long)k, mh[k], nb, mh[nb]);
        }
    invalidate_graph(ctx);
    free_members(ctx);
    if (n_members == 1) return SWDG_OK;
    ctx->nmemb = n_members;
    ctx->first.assign(first_cell, first_cell + n_members + 1);
    Bc b0{};
    for (int i = 0; i < MXTAG; ++i) {
        b0.kind[i] = ctx->d.bc_kind[i];
        b0.amp[i] = ctx->d.bc_amp[i];
        b0.per[i] = ctx->d.bc_per[i];
        b0.ph[i] = ctx->d.bc_ph[i];
    }
    ctx->bch.assign(n_members, b0);
    CK(cudaMalloc(&ctx->memb, n * sizeof(int32_t)));
    CK(cudaMalloc(&ctx->mb, n_members * sizeof(Member)));
    CK(cudaMalloc(&ctx->bcd, n_members * sizeof(Bc)));
    CK(cudaMalloc(&ctx->first_d, (n_members + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&ctx->mdiag, 4 * (size_t)n_members * sizeof(double)));
    CK(cudaMemcpyAsync(ctx->memb, mh.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->mb, 0, n_members * sizeof(Member), ctx->st));
    CK(cudaMemcpyAsync(ctx->bcd, ctx->bch.data(), n_members * sizeof(Bc), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaMemcpyAsync(ctx->first_d, first_cell, (n_members + 1) * sizeof(int64_t),
                       cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->d.memb = ctx->memb;
    ctx->d.mb = ctx->mb;
    ctx->d.mbc = ctx->bcd;
    ctx->d.nmemb = n_members;
    return SWDG_OK;
}

int swdg_set_boundary_member(swdg_ctx* ctx, int member, int tag, int kind, double amp,
                             double period, double phase) {
    if (!ctx) return SWDG_EINVAL;
    if (ctx->nmemb == 1 && member == 0) return swdg_set_boundary(ctx, tag, kind, amp, period, phase);
    if (member < 0 || member >= ctx->nmemb || tag < 0 || tag >= MXTAG ||
        (kind != SWDG_BC_WALL && kind != SWDG_BC_TIDE) || (kind == SWDG_BC_TIDE && !(period > 0)) ||
        !std::isfinite(amp) || !std::isfinite(phase))
        return fail(ctx, SWDG_EINVAL, "set_boundary_member: bad arguments");
    Bc& b = ctx->bch[member];
    b.kind[tag] = kind;
    b.amp[tag] = amp;
    b.per[tag] = period;
    b.ph[tag] = phase;
    CK(cudaMemcpyAsync(ctx->bcd + member, &b, sizeof(Bc), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

int swdg_member_times(swdg_ctx* ctx, double* t, double* dt_last, int set) {
    if (!ctx) return SWDG_EINVAL;
    const int M = ctx->d.nmemb;
    std::vector<Member> mh;
    int rc = read_clocks(ctx, mh);
    if (rc) return rc;
    if (set) {
        if (!t) return fail(ctx, SWDG_EINVAL, "member_times: t required to set");
        for (int m = 0; m < M; ++m)
            if (!std::isfinite(t[m]))
                return fail(ctx, SWDG_EINVAL, "member_times: t[%d] is not finite", m);
        for (int m = 0; m < M; ++m) mh[m].t = t[m];
        CK(cudaMemcpyAsync(ctx->d.mb, mh.data(), M * sizeof(Member), cudaMemcpyHostToDevice,
                           ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        return SWDG_OK;
    }
    for (int m = 0; m < M; ++m) {
        if (t) t[m] = mh[m].t;
        if (dt_last) dt_last[m] = mh[m].dt_last;
    }
    return SWDG_OK;
}

int swdg_member_diagnostics(swdg_ctx* ctx, double* out) {
    if (!ctx || !out) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "member_diagnostics: no state");
    if (ctx->nmemb == 1) return swdg_diagnostics(ctx, out);
    const int M = ctx->nmemb;
    ctx->L.cell_diag(ctx->d, ctx->tb, ctx->diag, ctx->shp[KK_AUX], ctx->st);
    k_diag_reduce<<<M, 256, 0, ctx->st>>>(ctx->diag, ctx->first_d, 0, 0, ctx->mdiag);
    CK(cudaGetLastError());
    std::vector<double> part(4 * (size_t)M);
    CK(cudaMemcpyAsync(part.data(), ctx->mdiag, part.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    std::vector<Member> mh;
    int rc = read_clocks(ctx, mh);
    if (rc) return rc;
    for (int m = 0; m < M; ++m) {
        double* o = out + 8 * (size_t)m;
        for (int i = 0; i < 4; ++i) o[i] = part[4 * m + i];
        o[4] = ctx->sc_host->maxits; // context-wide counters
        o[5] = ctx->sc_host->viol;
        o[6] = mh[m].dt_last;
        o[7] = mh[m].t;
    }
    return SWDG_OK;
}

int swdg_gather_gauges_member(swdg_ctx* ctx, int member, int n, const double* xy, double* out) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "gather_gauges_member: no state");
    if (member < 0 || member >= ctx->nmemb || n < 0 || (n > 0 && (!xy || !out)))
        return fail(ctx, SWDG_EINVAL, "gather_gauges_member: bad arguments");
    if (n == 0) return SWDG_OK;
    int rc = gauges_prepare(ctx, n, xy, ctx->first[member], ctx->first[member + 1]);
    if (rc) return rc;
    ctx->L.gauges(ctx->d, ctx->tb, n, ctx->gdev, ctx->gdev + 2 * n, ctx->first[member],
                  ctx->first[member + 1], ctx->gcell, ctx->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, ctx->gdev + 2 * n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return SWDG_OK;
}

// ---------------------------------------------------------------------------
// launch shapes and their autotuner
// ---------------------------------------------------------------------------
int swdg_set_shape(swdg_ctx* ctx, int kind, int grid, int warps_per_block) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_bathy) return fail(ctx, SWDG_ESTATE, "set_shape: upload the bathymetry first");
    if (kind < 0 || kind >= KK_N || warps_per_block < 1 || warps_per_block > MAXWPB || grid < 1 ||
        ctx->L.occupancy(kind, warps_per_block) < 1)
        return fail(ctx, SWDG_EINVAL, "set_shape: bad kind, grid or warps per block");
    ctx->shp[kind] = Shape{grid, warps_per_block};
    invalidate_graph(ctx);
    return SWDG_OK;
}

int swdg_get_shapes(const swdg_ctx* ctx, int* out) {
    if (!ctx || !out) return SWDG_EINVAL;
    for (int i = 0; i < KK_N; ++i) {
        out[2 * i] = ctx->shp[i].grid;
        out[2 * i + 1] = ctx->shp[i].wpb;
    }
    return SWDG_OK;
}

// candidate c of kind k: warps per block and grid (persistent: SMs x resident
// blocks; full: one block per wpb cells)
static bool candidate(swdg_ctx* ctx, int kind, int c, Shape& s) {
    static const int wpbs[4] = {1, 2, 4, 8};
    if (c < 0 || c >= 8) return false;
    const int wpb = wpbs[c / 2];
    const int occ = ctx->L.occupancy(kind, wpb);
    if (occ < 1) return false;
    const int64_t cover = (ctx->n + wpb - 1) / wpb;
    const int64_t pers = (int64_t)ctx->nsm * occ;
    int64_t g = (c % 2 == 0) ? std::min(pers, cover) : std::min<int64_t>(cover, 152LL * 64 * 4 / wpb);
    s = Shape{(int)std::max<int64_t>(1, g), wpb};
    return true;
}

int swdg_autotune(swdg_ctx* ctx, int repeats, double* report) {
    if (!ctx) return SWDG_EINVAL;
    if (!ctx->has_state) return fail(ctx, SWDG_ESTATE, "autotune: no state");
    if (repeats < 1) repeats = 1;
    const int64_t n = ctx->n;
    const size_t ubytes = 4 * (size_t)n * ctx->nd * sizeof(double);
    // snapshot: state buffer 0, its masks, the counters and every member clock
    double* usave = nullptr;
    uint8_t* msave = nullptr;
    CK(cudaMalloc(&usave, ubytes));
    CK(cudaMalloc(&msave, n));
    std::vector<Member> clocks;
    int rc = read_clocks(ctx, clocks);
    if (rc) return rc;
    Scalars sc0;
    CK(cudaMemcpyAsync(&sc0, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(usave, ctx->U, ubytes, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(msave, ctx->cmask, n, cudaMemcpyDeviceToDevice, ctx->st));
    rc = put_fixed_dt(ctx, -1.0); // tuning steps take the CFL step
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->st));
    const Shape keep[KK_N] = {ctx->shp[0], ctx->shp[1], ctx->shp[2], ctx->shp[3]};
    double best[KK_N];
    Shape pick[KK_N];
    for (int k = 0; k < KK_N; ++k) {
        best[k] = INFINITY;
        pick[k] = keep[k];
    }
    cudaEvent_t ev[SWDG_PROF_SLOTS][2];
    for (int i = 0; i < SWDG_PROF_SLOTS; ++i) {
        cudaEventCreate(&ev[i][0]);
        cudaEventCreate(&ev[i][1]);
    }
    bool used[SWDG_PROF_SLOTS] = {};
    used[0] = used[8] = true;
    for (int l = 0; l < ctx->d.s; ++l) {
        used[1 + l] = true;
        if (l > 0) used[4 + l] = true;
    }
    for (int c = 0; c < 8 && !rc; ++c) {
        Shape cs[KK_N];
        bool ok[KK_N];
        for (int k = 0; k < KK_N; ++k) {
            ok[k] = candidate(ctx, k, c, cs[k]);
            ctx->shp[k] = ok[k] ? cs[k] : keep[k];
        }
        double tk[KK_N] = {0, 0, 0, 0};
        for (int r = 0; r < repeats + 1 && !rc; ++r) { // first pass: warm-up
            rc = enqueue_step(ctx, ev);
            if (rc) break;
            if (cudaStreamSynchronize(ctx->st) != cudaSuccess) {
                rc = fail(ctx, SWDG_ECUDA, "autotune: step failed");
                break;
            }
            if (r == 0) continue;
            for (int sl = 0; sl < SWDG_PROF_SLOTS; ++sl) {
                if (!used[sl]) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, ev[sl][0], ev[sl][1]);
                const int k = sl == 0 ? KK_BEGIN : (sl <= 4 ? KK_RESIDUAL : KK_STAGE);
                tk[k] += ms;
            }
        }
        for (int k = 0; k < 3 && !rc; ++k)
            if (ok[k] && tk[k] < best[k]) {
                best[k] = tk[k];
                pick[k] = cs[k];
            }
    }
    for (int i = 0; i < SWDG_PROF_SLOTS; ++i) {
        cudaEventDestroy(ev[i][0]);
        cudaEventDestroy(ev[i][1]);
    }
    // restore the state, masks, counters and clocks the tuning steps advanced
    cudaMemcpyAsync(ctx->U, usave, ubytes, cudaMemcpyDeviceToDevice, ctx->st);
    cudaMemcpyAsync(ctx->cmask, msave, n, cudaMemcpyDeviceToDevice, ctx->st);
    // the FP32 copy of buffer 0 follows the restored state (the masks it
    // recomputes are the restored ones: a function of the state)
    if (ctx->uF) ctx->L.masks(ctx->d, 0, ctx->shp[KK_AUX], ctx->st);
    cudaMemcpyAsync(ctx->sc, &sc0, sizeof(Scalars), cudaMemcpyHostToDevice, ctx->st);
    cudaMemcpyAsync(ctx->d.mb, clocks.data(), clocks.size() * sizeof(Member),
                    cudaMemcpyHostToDevice, ctx->st);
    cudaError_t e = cudaStreamSynchronize(ctx->st);
    cudaFree(usave);
    cudaFree(msave);
    if (rc) {
        for (int k = 0; k < KK_N; ++k) ctx->shp[k] = keep[k];
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, SWDG_ECUDA, "autotune: restore failed");
    for (int k = 0; k < 3; ++k) ctx->shp[k] = pick[k];
    ctx->shp[KK_AUX] = keep[KK_AUX];
    ctx->tuned = true;
    invalidate_graph(ctx);
    if (report)
        for (int k = 0; k < 3; ++k) {
            report[3 * k] = pick[k].grid;
            report[3 * k + 1] = pick[k].wpb;
            report[3 * k + 2] = best[k] / repeats;
        }
    return SWDG_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// arithmetic peak probe: independent FMA chains in registers, no memory
// traffic; the measured FP64 (or FP32) rate is the roofline of the kernels
// that are bound by that pipe
// ---------------------------------------------------------------------------
template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_chains(T b, T c, int iters, T* sink) {
    T a[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) a[j] = (T)(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < CH; ++j) a[j] = fma(a[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < CH; ++j) s += a[j];
    if (s == T(-1.2345e-7)) *sink = s; // never true: keeps the chains alive
}

template <typename T>
static int probe_fma_run(int iters, double* tflops, double* ms_out) {
    constexpr int CH = 8, TPB = 256;
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_chains<T, CH>, TPB, 0) !=
            cudaSuccess ||
        occ < 1)
        return SWDG_ECUDA;
    const int grid = nsm * occ;
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(T));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) { // the first launch warms up
        cudaEventRecord(e0, 0);
        k_fma_chains<T, CH><<<grid, TPB>>>((T)0.999999, (T)1e-3, iters, sink);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || !(best > 0.0f)) return SWDG_ECUDA;
    const double flops = 2.0 * CH * (double)iters * grid * TPB;
    if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return SWDG_OK;
}

extern "C" int swdg_probe_fma(int dtype, double* tflops, double* ms) {
    if (dtype == SWDG_PIX_F64) return probe_fma_run<double>(4096, tflops, ms);
    if (dtype == SWDG_PIX_F32) return probe_fma_run<float>(65536, tflops, ms);
    return SWDG_EINVAL;
}

// z = h^(-1/3) and z^3 as the kernels form them (inv_cbrt), one value per thread
__global__ void k_probe_roots(const double* h, int64_t n, double* z, double* rcp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double zi = inv_cbrt(h[i]);
        z[i] = zi;
        rcp[i] = zi * zi * zi;
    }
}

extern "C" int swdg_probe_roots(const double* h, int64_t n, double* z, double* rcp) {
    if (!h || !z || !rcp || n < 1 || n > (int64_t(1) << 24)) return SWDG_EINVAL;
    double* dv = nullptr;
    const size_t b = (size_t)n * sizeof(double);
    if (cudaMalloc(&dv, 3 * b) != cudaSuccess) return SWDG_ECUDA;
    bool ok = cudaMemcpy(dv, h, b, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
        const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
        k_probe_roots<<<grid, 256>>>(dv, n, dv + n, dv + 2 * n);
        ok = cudaGetLastError() == cudaSuccess && cudaMemcpy(z, dv + n, b, cudaMemcpyDeviceToHost) ==
                                                     cudaSuccess &&
             cudaMemcpy(rcp, dv + 2 * n, b, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    cudaFree(dv);
    return ok ? SWDG_OK : SWDG_ECUDA;
}

// ---------------------------------------------------------------------------
// allocation-free residual: its only scratch is this file-scope array (step
// scalars in the first 256 bytes, then the pixel-overlap table, then one
// constant-field mask byte per cell), held on every GPU where the library's
// device code is loaded (lazily, at the first call, unless the process loads
// modules eagerly)
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_OV_BYTES = ((sizeof(OvTab) + 255) / 256) * 256;
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[256 + NOALLOC_OV_BYTES + SWDG_NOALLOC_MAX_CELLS];
static void* g_noalloc_addr[256];   // device address of the array, per device ordinal
static bool g_noalloc_ready[256];

__global__ void k_noalloc_begin(Scalars* sc, double t) {
    sc->m0.t = t;
    sc->fixed_dt = -1.0;
    sc->m0.dt_last = 0.0;
    sc->m0.rmax = 0ull;
    sc->maxits = 0;
    sc->viol = 0;
    sc->fallback = 0;
    sc->status = 0;
}

// the mesh checks of swdg_upload_mesh, on the device: bit 1 of status on failure
__global__ void k_noalloc_check_mesh(const double* hxhy, const int32_t* nbr, int64_t n,
                                     Scalars* sc) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        bool ok = hxhy[2 * k] > 0.0 && hxhy[2 * k + 1] > 0.0;
        for (int f = 0; f < 4 && ok; ++f) {
            const int32_t s0 = nbr[k * 8 + 2 * f], s1 = nbr[k * 8 + 2 * f + 1];
            if (s1 != -1 || s0 >= n || s0 < -MXTAG) ok = false;
            else if (s0 >= 0) {
                const int fo = f ^ 1;
                const double tk = f < 2 ? hxhy[2 * k + 1] : hxhy[2 * k];
                const double tn = f < 2 ? hxhy[2 * (int64_t)s0 + 1] : hxhy[2 * (int64_t)s0];
                if (nbr[(int64_t)s0 * 8 + 2 * fo] != (int32_t)k || fabs(tk - tn) > 1e-9 * tk)
                    ok = false;
            }
        }
        if (!ok) atomicOr(&sc->status, 2);
    }
}

__global__ void k_noalloc_end(const Scalars* sc, double cfl, double* dt_out) {
    *dt_out = cfl / __longlong_as_double(sc->m0.rmax);
}

static int noalloc_fail(char* err, int err_len, int code, const char* msg) {
    if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg);
    return code;
}

extern "C" int swdg_residual_noalloc(const swdg_config* cfg, int64_t n, const double* hxhy,
                                     const int32_t* nbr, const void* tiles, int P, int pix_dtype,
                                     const double* manning, const int32_t* bc_kind,
                                     const double* bc_amp, const double* bc_period,
                                     const double* bc_phase, const double* state, double t,
                                     double* residual, double* dt_out, char* err, int err_len) {
    if (!cfg || cfg->degree < 1 || cfg->degree > 3 || cfg->subgrid_mode != 0 ||
        cfg->precision != 0 || !(cfg->g > 0) || !(cfg->eps_vel > 0) || !(cfg->cfl > 0))
        return noalloc_fail(err, err_len, SWDG_EINVAL,
                            "residual_noalloc: degree 1..3, subgrid_mode 0, precision 0 (FP64), "
                            "g, eps_vel, cfl > 0");
    if (n < 1 || n > SWDG_NOALLOC_MAX_CELLS)
        return noalloc_fail(err, err_len, SWDG_EINVAL,
                            "residual_noalloc: n_cells must be in 1..SWDG_NOALLOC_MAX_CELLS "
                            "(1048576)");
    if (P < 1 || P > MXPIX || (pix_dtype != SWDG_PIX_F32 && pix_dtype != SWDG_PIX_F64))
        return noalloc_fail(err, err_len, SWDG_EINVAL,
                            "residual_noalloc: pixels_per_side in 1..32, pix_dtype F32 or F64");
    if (!hxhy || !nbr || !tiles || !manning || !state || !residual)
        return noalloc_fail(err, err_len, SWDG_EINVAL, "residual_noalloc: null device buffer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return noalloc_fail(err, err_len, SWDG_ECUDA, "residual_noalloc: no current device");
    if (!g_noalloc_ready[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(err, err_len, SWDG_ECUDA,
                                "residual_noalloc: cudaGetSymbolAddress of the scratch failed");
        g_noalloc_addr[dev] = p;
        g_noalloc_ready[dev] = true;
    }
    unsigned char* scratch = (unsigned char*)g_noalloc_addr[dev];
    Scalars* sc = (Scalars*)scratch;
    OvTab* ovd = (OvTab*)(scratch + 256);
    uint8_t* cmask = (uint8_t*)(scratch + 256 + NOALLOC_OV_BYTES);
    cudaStream_t st = (cudaStream_t)cfg->stream;

    Tables tb;
    static OvTab ovh; // host copy, reused by every call (not thread-safe, like the scratch)
    if (!build_tables(cfg->degree, tb) || !build_overlaps(cfg->degree, P, tb, ovh))
        return noalloc_fail(err, err_len, SWDG_EINVAL, "residual_noalloc: table construction failed");
    Launch L{};
    if (!get_launch(cfg->degree, 0, pix_dtype == SWDG_PIX_F32 ? 0 : 1, 0, &L))
        return noalloc_fail(err, err_len, SWDG_EINVAL, "residual_noalloc: no kernels for this case");
    Dev d{};
    d.n = n;
    d.hxhy = hxhy;
    d.nbr = nbr;
    d.tiles = tiles;
    d.ov = ovd; // one pixel count; tile k starts at k P^2; conforming faces only
    d.manning = manning;
    d.U = const_cast<double*>(state); // read only: buffer 0 of the kernels' state layout
    d.cmask = cmask;
    d.res = residual;
    d.sc = sc;
    d.mb = &sc->m0;
    d.nmemb = 1;
    d.mode = 0;
    d.g = cfg->g;
    d.eps = cfg->eps_vel;
    d.cfl = cfg->cfl;
    for (int i = 0; i < MXTAG; ++i) {
        d.bc_kind[i] = bc_kind ? bc_kind[i] : SWDG_BC_WALL;
        d.bc_amp[i] = bc_amp ? bc_amp[i] : 0.0;
        d.bc_per[i] = bc_period ? bc_period[i] : 1.0;
        d.bc_ph[i] = bc_phase ? bc_phase[i] : 0.0;
        if (d.bc_kind[i] != SWDG_BC_WALL && d.bc_kind[i] != SWDG_BC_TIDE)
            return noalloc_fail(err, err_len, SWDG_EINVAL, "residual_noalloc: bad boundary kind");
        if (d.bc_kind[i] == SWDG_BC_TIDE && !(d.bc_per[i] > 0))
            return noalloc_fail(err, err_len, SWDG_EINVAL, "residual_noalloc: tide period <= 0");
    }
    cudaError_t ec = cudaMemcpyAsync(ovd, &ovh, sizeof(OvTab), cudaMemcpyHostToDevice, st);
    if (ec != cudaSuccess) return noalloc_fail(err, err_len, SWDG_ECUDA, cudaGetErrorString(ec));
    k_noalloc_begin<<<1, 1, 0, st>>>(sc, t);
    k_noalloc_check_mesh<<<(int)std::min<int64_t>(152 * 8, (n + 255) / 256), 256, 0, st>>>(hxhy, nbr,
                                                                                        n, sc);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(err, err_len, SWDG_ECUDA, cudaGetErrorString(e));
    if (status)
        return noalloc_fail(err, err_len, SWDG_EINVAL,
                            "residual_noalloc: bad mesh (sizes, neighbour indices, tags or a "
                            "non-conforming face)");
    const Shape shp{grid_for(n), WPB};
    L.masks(d, 0, shp, st);
    L.residual(d, tb, 0, 0, 0.0, 1, shp, st);
    if (dt_out) k_noalloc_end<<<1, 1, 0, st>>>(sc, cfg->cfl, dt_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(err, err_len, SWDG_ECUDA, cudaGetErrorString(e));
    return SWDG_OK;
}
