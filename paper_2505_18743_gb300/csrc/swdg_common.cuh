// swdg_common.cuh -- device data structures and warp helpers of the sm_103a
// sub-grid DG shallow-water hot path (arXiv 2505.18743).
//
// Layout in HBM (one context):
//   state   U[buf][field][cell][(r+1)^2]  float64, field = zeta, qx, qy, c
//   cmask   [buf][cell] uint8: bit f set when field f is constant on the cell
//           (such a field is evaluated as that constant, exactly)
//   resid   R[stage][6][cell][(r+1)^2] float64, 6 = F, Gx, Gy, R, Lx, Ly
//   tiles   [cell][P][P] float32|float64 bathymetry depth (mode S)
//   zpts    [cell][NV^2 + NM^2 + NG^2] float64: point samples (mode P) or
//           sub-cell mean depths sum_k w_k z_k (mode S)
// Small per-degree tables (1D interpolation matrices, quadrature weights,
// pixel-overlap fractions) travel as a __grid_constant__ kernel parameter.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace swdg {

constexpr int MXP = 6;    // max quadrature points per direction (GL 5 for r = 3)
constexpr int MXN = 4;    // max nodes per direction (r + 1)
constexpr int MXPIX = 32; // max pixels per cell side in mode S
constexpr int MXTAG = 16;
constexpr int MXS = 4;    // max RK stages
constexpr int NBUF = 4;   // state buffers: v^n plus stages 2..4

// point sets
constexpr int SET_VOL = 0;  // volume Gauss-Legendre, floor(3r/2)+1 per direction
constexpr int SET_MASS = 1; // face / mass Gauss-Lobatto, r+2 per direction
constexpr int SET_MOM = 2;  // momentum mass Gauss-Legendre, r+1 per direction
constexpr int SET_HALF = 3; // coarse side of a 2:1 face: the GLL sub-intervals of each
                            // fine half face, h NM + al, in coarse coordinates
constexpr int NSET = 4;
constexpr int MXI = 2 * MXP; // max sub-intervals per set
constexpr int MXCLS = 4;     // max distinct pixel counts per cell side

// face info byte of a cell's face: FI_COARSE = this cell is the coarse side of
// a 2:1 face (two fine neighbours); FI_FINE | half << 2 = this cell is one of
// the two fine cells (half 0: lower tangential half of the coarse face)
constexpr int FI_COARSE = 1;
constexpr int FI_FINE = 2;

// pixel-overlap fractions of the sub-intervals of the four point sets for
// one pixel count P per cell side
struct OvTab {
    int P;
    int lo[NSET][MXI], cnt[NSET][MXI];
    double frac[NSET][MXI][MXPIX + 1];
};

// status bits
constexpr int ST_NAN = 1;

template <int R>
struct Sz {
    static constexpr int ND1 = R + 1, ND = ND1 * ND1;
    static constexpr int NV = (3 * R) / 2 + 1, NVP = NV * NV;
    static constexpr int NM = R + 2, NMP = NM * NM;
    static constexpr int NG = R + 1, NGP = NG * NG;
    static constexpr int NZP = NVP + NMP + NGP; // mode P samples per cell
};

struct Tables {
    double Bv[MXP][MXN], Dv[MXP][MXN], wv[MXP]; // nodal -> volume GL (value, d/dxi)
    double Bm[MXP][MXN], wm[MXP];               // nodal -> mass / face GLL
    double Bg[MXP][MXN], wg[MXP];               // nodal -> momentum GL (square)
    double Bginv[MXN][MXP];                     // inverse of Bg
    double M1inv[MXN][MXN];                     // inverse of the 1D GLL mass matrix
    double BmH[2][MXP][MXN];                    // nodal -> fine-face GLL points of half h
    // FP32 copies for the FP32-bulk kernels
    float BvF[MXP][MXN], DvF[MXP][MXN], BmF[MXP][MXN], BmHF[2][MXP][MXN], BgF[MXP][MXN];
    float BginvF[MXN][MXP];
    float wvF[MXP];                             // volume GL weights (FP32-bulk residual)
    float wgF[MXP];                             // momentum GL weights (FP32-bulk stage update)
    double xs[MXN];                             // support nodes on [0, 1]
    double xq[3][MXP];                          // nodes of the three point sets on [0, 1]
};

// clock of one ensemble member (a plain context is an ensemble of one)
struct Member {
    double t;                 // time at the start of the current step
    double dt_last;
    unsigned long long rmax;  // bits of max lambda l_Gamma / J_K over the member (non-negative double)
    double pad_;
};

// boundary table of one member: kind (SWDG_BC_*) and tide of every tag
struct Bc {
    int kind[MXTAG];
    double amp[MXTAG], per[MXTAG], ph[MXTAG];
};

struct Scalars {
    Member m0;                // the clock of a single-member context
    double fixed_dt;          // >= 0: fixed step, < 0: CFL
    int maxits, viol, fallback, status;
};

struct Dev {
    int64_t n;
    const double* x0y0;
    const double* hxhy;
    const double* ihxhy; // 1/hx, 1/hy per cell (null: computed in the kernel)
    const int32_t* nbr;
    const void* tiles;
    const int64_t* tile_off; // first pixel of each cell's tile (null: k P^2)
    const uint8_t* pcls;     // pixel-count class of each cell (null: class 0)
    const OvTab* ov;         // overlap tables per class
    const uint8_t* finfo;    // [cell][4] face info (null: all conforming)
    const double* zhang;     // [cell][4][2][NM]: coarse-side strip means / samples
    const double* zpts;
    const double* zmax; // dry-start level of Eq. initial_guess (max z_b of the cell)
    const double* zmin; // min z_b of the cell: every pixel is wet when eta > -zmin
    const double* zabs; // max |z_b| of the cell (Newton tolerance scale)
    // [cell][NZP] (min, max) of the pixel depths of each sub-cell of the three
    // point sets (mode S; min rounded down, max up); null: the cell's bounds
    const float2* zsb;
    const double* manning;
    const double* nu_c; // tracer numerical diffusivity per cell (Eq. numdiff); null: none
    double* U;
    // FP32 copy of U in the same layout (FP32-bulk contexts; null otherwise),
    // written wherever U and its masks are written (k_masks, the step start,
    // the stage update), read by the FP32 face and residual arithmetic
    float* uF;
    uint8_t* cmask;
    double* res;
    double* llin;
    double* HN;
    double* CN;
    double* HNbar;
    double* CNbar;
    uint8_t* flag;
    // 1 where every mass point of the cell was fully wet at zeta^n (written by
    // the step start with H(zeta^n); null: unknown)
    uint8_t* wet0;
    // [cell][2][(r+1)^2]: qx, qy of v^n at the momentum points, written by the
    // step start (the same for every stage of the step; FP64 contexts); null:
    // interpolated by the stage update itself
    double* qpts;
    Scalars* sc;
    Member* mb;            // member clocks [nmemb] (a single member: &sc->m0)
    const int32_t* memb;   // member of each cell (null: every cell in member 0)
    const Bc* mbc;         // per-member boundary tables (null: the tables below)
    int nmemb;
    int mode; // 0 S, 1 P
    int s;    // stages
    double g, eps, hlim, eps0, cfl, newton_tol;
    int newton_max;
    int any_friction;
    int bc_kind[MXTAG];
    double bc_amp[MXTAG], bc_per[MXTAG], bc_ph[MXTAG];
    double a[MXS][MXS], at[MXS][MXS], b[MXS], bt[MXS], c[MXS];
    // face points evaluated once by k_faces (null fflux: the residual
    // integrates its faces itself)
    double* fflux;        // [cell][4 fields][4 faces][2 halves][NM]
    const int64_t* fjobs; // k << 8 | f | h << 2 | al << 3, k the lower index of the face
    int64_t njobs;
};

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// sums over a team of TL lanes (the whole warp, or one of its two halves;
// tm = the team's lanes); for TL = 32 the same order as warp_sum
template <int TL>
__device__ __forceinline__ double team_sum(double v, unsigned tm) {
#pragma unroll
    for (int o = TL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(tm, v, o);
    return v;
}
// two team sums at once, each bit for bit the team_sum of its value: the first
// level of the butterfly sums a on the team's lower half and b on its upper
// half (one addition per lane for both), the other levels run on both halves
// together, and a last exchange gives every lane both results.  Each level
// adds the same pairs as team_sum (addition commutes), so the tree is the
// same; the FP64 additions halve.  Teams are aligned groups of TL lanes.
template <int TL>
__device__ __forceinline__ void team_sum2(double& a, double& b, unsigned tm) {
    const bool hi = (threadIdx.x & (TL / 2)) != 0;
    double v = (hi ? b : a) + __shfl_xor_sync(tm, hi ? a : b, TL / 2);
#pragma unroll
    for (int o = TL / 4; o > 0; o >>= 1) v += __shfl_xor_sync(tm, v, o);
    const double w = __shfl_xor_sync(tm, v, TL / 2);
    a = hi ? w : v;
    b = hi ? v : w;
}
// maxima of non-negative values (no NaN) over the team's lanes tm by their bit
// patterns, which order like the values: integer reductions, off the FP64 pipe
__device__ __forceinline__ float team_max_nonneg(float v, unsigned tm) {
    return __uint_as_float(__reduce_max_sync(tm, __float_as_uint(v)));
}
__device__ __forceinline__ double team_max_nonneg(double v, unsigned tm) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned mh = __reduce_max_sync(tm, hi);
    const unsigned ml = __reduce_max_sync(tm, hi == mh ? lo : 0u);
    return __longlong_as_double((long long)(((unsigned long long)mh << 32) | ml));
}
// equality and finiteness of doubles tested on their bit patterns, on the
// integer pipe (FP64 compares take the FP64 pipe).  same_bits differs from ==
// only for +0 against -0 and for NaN: a constant-field mask may treat those
// either way, since a field marked non-constant takes the general path.
__device__ __forceinline__ bool same_bits(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool finite_bits(double v) {
    constexpr long long EXP = 0x7ff0000000000000ll;
    return (__double_as_longlong(v) & EXP) != EXP;
}
// v == 0.0 (either sign) on the bit pattern
__device__ __forceinline__ bool zero_bits(double v) {
    return (__double_as_longlong(v) << 1) == 0;
}
// Order-preserving integer key of a double that is not NaN: a > b exactly when
// okey(a) > okey(b), except that -0 keys below +0 (negative doubles have their
// non-sign bits flipped, so they order as negative integers).
__device__ __forceinline__ long long okey(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
// the key of -z for a threshold -z, with -0 taken as +0, so that
// okey(eta) > nkey_neg(z) is exactly eta > -z for every eta that is not NaN
// (for eta = +-0 and -z = -0 both are false)
__device__ __forceinline__ long long nkey_neg(double z) {
    long long b = __double_as_longlong(z) ^ (long long)0x8000000000000000ull;
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ bool nan_bits(double v) {
    return (__double_as_longlong(v) & 0x7fffffffffffffffll) > 0x7ff0000000000000ll;
}
__device__ __forceinline__ double* ufield(const Dev& d, int buf, int f, int nd) {
    return d.U + ((size_t)buf * 4 + f) * (size_t)d.n * nd;
}
__device__ __forceinline__ float* ufieldF(const Dev& d, int buf, int f, int nd) {
    return d.uF + ((size_t)buf * 4 + f) * (size_t)d.n * nd;
}
__device__ __forceinline__ double* rfield(const Dev& d, int stage, int f, int nd) {
    return d.res + ((size_t)stage * 6 + f) * (size_t)d.n * nd;
}

__device__ __forceinline__ int member_of(const Dev& d, int64_t k) {
    return d.memb ? d.memb[k] : 0;
}

__device__ __forceinline__ double get_dt(const Dev& d, int m) {
    // dt = cfl min J/(lambda l) = cfl / max(lambda l / J) over the member's
    // cells, Eq. deltat_fe
    return d.sc->fixed_dt >= 0.0 ? d.sc->fixed_dt : d.cfl / __longlong_as_double(d.mb[m].rmax);
}

// x^(-1/3) of a positive double: an FP32 reciprocal-cube-root seed refined by
// two Newton-Raphson steps for z^-3 = x in FP64, z <- z + z (1 - x z^3) / 3
// (quadratic convergence, no division: ~1e-7 -> ~1e-14 -> rounding).  Values
// outside the FP32 seed's comfortable range take 1 / cbrt(x).
__device__ __forceinline__ double inv_cbrt(double x) {
    const float xf = (float)x;
    if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / cbrt(x);
    double z = (double)rcbrtf(xf);
    constexpr double third = 1.0 / 3.0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-x, z * z * z, 1.0);
        z = fma(z * third, e, z);
    }
    return z;
}

// desingularised velocity factor u = f q, Eq. velocity (T = double or float)
template <typename T>
__device__ __forceinline__ T vel_factor(T h, T eps) {
    if (h <= T(0)) return T(0);
    if (h >= eps) return T(1) / h; // max(h^4, eps^4) = h^4: sqrt(2) h / sqrt(2 h^4) = 1/h
    T h4 = (h * h) * (h * h), e4 = (eps * eps) * (eps * eps);
    return sqrt(T(2)) * h / sqrt(e4 + h4);
}
// Manning coefficient gamma = g n^2 |q| / h_des^(7/3), Eqs. manning, discharge_rhs_implicit
template <typename T>
__device__ __forceinline__ T gamma_manning(T n, T h, T qx, T qy, T g, T eps) {
    if (n == T(0) || h <= T(0)) return T(0);
    T hdes = h; // h_des = h when h >= eps
    if (h < eps) {
        T h4 = (h * h) * (h * h), e4 = (eps * eps) * (eps * eps);
        hdes = sqrt(e4 + h4) / (sqrt(T(2)) * h);
    }
    if constexpr (std::is_same<T, double>::value) {
        // h_des^(-7/3) = z^7 with z = h_des^(-1/3): no division, no cbrt
        const double z = inv_cbrt(hdes), z3 = z * z * z;
        return g * n * n * sqrt(qx * qx + qy * qy) * (z3 * z3 * z);
    } else {
        return g * n * n * sqrt(qx * qx + qy * qy) / (hdes * hdes * cbrt(hdes));
    }
}

// the velocity factor and the Manning coefficient of one point together: on
// the wet branch (h >= eps, where h_des = h) both come from one root, in FP64
// z = h^(-1/3) with 1/h = z^3 and h^(-7/3) = z^7 (1/h by division where
// there is no friction), otherwise from 1/h with h^(-7/3) = (1/h)^2
// cbrt(1/h); below eps as vel_factor and gamma_manning
template <typename T>
__device__ __forceinline__ void vel_gamma(T n, T h, T qx, T qy, T g, T eps, T& fv, T& gam) {
    if (h >= eps && h > T(0)) {
        if constexpr (std::is_same<T, double>::value) {
            if (n == 0.0) {
                fv = 1.0 / h;
                gam = 0.0;
            } else {
                // with friction, 1/h = z^3 from z = h^(-1/3) (a few ulp from the
                // rounded quotient, no FP64 division); gamma ~ z^7
                const double z = inv_cbrt(h), rh = z * z * z;
                fv = rh;
                gam = g * n * n * sqrt(qx * qx + qy * qy) * (rh * rh) * z;
            }
            return;
        }
        const T rh = T(1) / h;
        fv = rh;
        const T c3 = cbrt(rh); // h^(-1/3)
        gam = (n == T(0)) ? T(0) : g * n * n * sqrt(qx * qx + qy * qy) * (rh * rh) * c3;
    } else {
        fv = vel_factor<T>(h, eps);
        gam = gamma_manning<T>(n, h, qx, qy, g, eps);
    }
}

// sub-grid wet depth V and wet area A of sub-cell (ia, ib) of point set `set`
// (mode S): V = sum_k w_k max(eta + z_k, 0), A = sum_k w_k [eta + z_k > 0]
template <typename Pix>
__device__ __forceinline__ void subgrid_S(const Pix* __restrict__ tile, const OvTab& ov, int setx,
                                          int ia, int sety, int ib, double eta, double& V,
                                          double& A, bool& full) {
    const int P = ov.P;
    const int lox = ov.lo[setx][ia], cx = ov.cnt[setx][ia];
    const int loy = ov.lo[sety][ib], cy = ov.cnt[sety][ib];
    double v = 0.0, a = 0.0;
    bool f = true;
    for (int j = 0; j < cy; ++j) {
        const Pix* row = tile + (size_t)(loy + j) * P + lox;
        double vr = 0.0, ar = 0.0;
        for (int i = 0; i < cx; ++i) {
            double dd = eta + (double)row[i];
            if (dd > 0.0) {
                double fx = ov.frac[setx][ia][i];
                vr += fx * dd;
                ar += fx;
            } else {
                f = false;
            }
        }
        double fy = ov.frac[sety][ib][j];
        v += fy * vr;
        a += fy * ar;
    }
    V = v;
    A = a;
    full = f;
}

__device__ __forceinline__ void subgrid_P(double z, double eta, double& V, double& A) {
    double dd = eta + z;
    if (dd > 0.0) { V = dd; A = 1.0; }
    else { V = 0.0; A = 0.0; }
}

} // namespace swdg
