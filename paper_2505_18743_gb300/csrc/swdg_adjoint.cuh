// swdg_adjoint.cuh -- discrete adjoint of the residual (Sec. 3.2): the
// vector-Jacobian product of (F, G, R, L) with respect to the nodal state,
// the Manning coefficient n_K and a bathymetry offset delta_K per cell (every
// depth of cell K shifted by delta_K), at delta = 0.
//
// Gather form, one warp per cell, no atomics: a cell's cotangent collects
// every residual entry that depends on its own data -- its volume terms, and
// on each of its (sub)face points both its own face term and its
// neighbour's (the neighbour's residual cotangent is read there).  The linear
// parts are the transposes of the forward contractions (interpolation <->
// test integration, trace <-> lift); the pointwise parts (velocity, friction,
// reconstruction, Rusanov flux) are differentiated by forward-mode dual
// numbers through the same templates the forward residual runs, every input
// direction of a point carried in one evaluation.  The sub-grid operator enters through V and its exact
// derivative A = dV/d(eta) = dV/d(delta).
//
// Derivative conventions at the kinks: max(x, 0) -> [x > 0] (Eq. mask); the
// reconstruction's min follows its first argument at ties, the first argument
// being the side whose residual is differentiated; the wave-speed max takes
// the symmetric subgradient (half of each side's derivative) at exact ties,
// so the derivative does not depend on the order of the face's two cells;
// |x| and sqrt(x) have derivative 0 at 0; a constant field is differentiated
// as its polynomial.
#pragma once
#include "swdg_kernels.cuh"

namespace swdg {
namespace ad {

// value and one directional derivative
struct D1 {
    double v, d;
    __device__ __forceinline__ D1() : v(0.0), d(0.0) {}
    __device__ __forceinline__ D1(double x) : v(x), d(0.0) {}
    __device__ __forceinline__ D1(double x, double dx) : v(x), d(dx) {}
};
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return D1(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return D1(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ D1 operator-(D1 a) { return D1(-a.v, -a.d); }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return D1(a.v * b.v, a.d * b.v + a.v * b.d); }
// a / b through one reciprocal of b (the value is a.v (1/b.v), within an ulp
// of the forward's quotient; only derivatives are taken from dual values)
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
    const double ib = 1.0 / b.v;
    const double q = a.v * ib;
    return D1(q, (a.d - q * b.d) * ib);
}
__device__ __forceinline__ D1& operator+=(D1& a, D1 b) { return a = a + b; }
__device__ __forceinline__ D1& operator*=(D1& a, D1 b) { return a = a * b; }
__device__ __forceinline__ bool operator<(D1 a, D1 b) { return a.v < b.v; }
__device__ __forceinline__ bool operator<=(D1 a, D1 b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>(D1 a, D1 b) { return a.v > b.v; }
__device__ __forceinline__ bool operator>=(D1 a, D1 b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(D1 a, D1 b) { return a.v == b.v; }
__device__ __forceinline__ D1 sqrt(D1 a) {
    const double s = ::sqrt(a.v);
    return D1(s, a.v > 0.0 ? 0.5 * a.d / s : 0.0);
}
__device__ __forceinline__ D1 cbrt(D1 a) {
    const double s = ::cbrt(a.v);
    return D1(s, a.v != 0.0 ? a.d / (3.0 * s * s) : 0.0);
}
__device__ __forceinline__ D1 fabs(D1 a) {
    return D1(::fabs(a.v), a.v > 0.0 ? a.d : (a.v < 0.0 ? -a.d : 0.0));
}
__device__ __forceinline__ D1 fmax(D1 a, D1 b) { return a.v >= b.v ? a : b; }
// the wave-speed bound: the symmetric subgradient at an exact tie
__device__ __forceinline__ D1 wave_speed_max(D1 a, D1 b) {
    return a.v > b.v ? a : (a.v < b.v ? b : D1(a.v, 0.5 * (a.d + b.d)));
}
__device__ __forceinline__ D1 fmin(D1 a, D1 b) { return a.v <= b.v ? a : b; }

// value and W directional derivatives (all directions in one evaluation)
template <int W>
struct DN {
    double v, d[W];
    __device__ __forceinline__ DN() : v(0.0) {
#pragma unroll
        for (int i = 0; i < W; ++i) d[i] = 0.0;
    }
    __device__ __forceinline__ DN(double x) : v(x) {
#pragma unroll
        for (int i = 0; i < W; ++i) d[i] = 0.0;
    }
    // x with unit derivative along direction dir (none when dir is outside [0, W))
    __device__ __forceinline__ static DN seed(double x, int dir) {
        DN r(x);
#pragma unroll
        for (int i = 0; i < W; ++i) r.d[i] = (i == dir) ? 1.0 : 0.0;
        return r;
    }
    // derivative v along direction dir, if dir is one of this value's
    __device__ __forceinline__ void set(int dir, double v) {
#pragma unroll
        for (int i = 0; i < W; ++i)
            if (i == dir) d[i] = v;
    }
};
template <int W>
__device__ __forceinline__ DN<W> operator+(const DN<W>& a, const DN<W>& b) {
    DN<W> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int W>
__device__ __forceinline__ DN<W> operator-(const DN<W>& a, const DN<W>& b) {
    DN<W> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int W>
__device__ __forceinline__ DN<W> operator-(const DN<W>& a) {
    DN<W> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int W>
__device__ __forceinline__ DN<W> operator*(const DN<W>& a, const DN<W>& b) {
    DN<W> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
// a / b through one reciprocal of b, as for D1
template <int W>
__device__ __forceinline__ DN<W> operator/(const DN<W>& a, const DN<W>& b) {
    DN<W> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int W>
__device__ __forceinline__ DN<W>& operator+=(DN<W>& a, const DN<W>& b) { return a = a + b; }
template <int W>
__device__ __forceinline__ bool operator<(const DN<W>& a, const DN<W>& b) { return a.v < b.v; }
template <int W>
__device__ __forceinline__ bool operator<=(const DN<W>& a, const DN<W>& b) { return a.v <= b.v; }
template <int W>
__device__ __forceinline__ bool operator>(const DN<W>& a, const DN<W>& b) { return a.v > b.v; }
template <int W>
__device__ __forceinline__ bool operator>=(const DN<W>& a, const DN<W>& b) { return a.v >= b.v; }
template <int W>
__device__ __forceinline__ bool operator==(const DN<W>& a, const DN<W>& b) { return a.v == b.v; }
template <int W>
__device__ __forceinline__ DN<W> scale_d(double v, const DN<W>& a, double f) {
    DN<W> r(v);
#pragma unroll
    for (int i = 0; i < W; ++i) r.d[i] = a.d[i] * f;
    return r;
}
template <int W>
__device__ __forceinline__ DN<W> sqrt(const DN<W>& a) {
    const double s = ::sqrt(a.v);
    return scale_d(s, a, a.v > 0.0 ? 0.5 / s : 0.0);
}
template <int W>
__device__ __forceinline__ DN<W> cbrt(const DN<W>& a) {
    const double s = ::cbrt(a.v);
    return scale_d(s, a, a.v != 0.0 ? 1.0 / (3.0 * s * s) : 0.0);
}
template <int W>
__device__ __forceinline__ DN<W> fabs(const DN<W>& a) {
    return scale_d(::fabs(a.v), a, a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0));
}
template <int W>
__device__ __forceinline__ DN<W> fmax(const DN<W>& a, const DN<W>& b) { return a.v >= b.v ? a : b; }
template <int W>
__device__ __forceinline__ DN<W> wave_speed_max(const DN<W>& a, const DN<W>& b) {
    // selects only (no branch over the whole value): a, b, or at a tie the mean
    const bool gt = a.v > b.v, lt = a.v < b.v;
    DN<W> m;
    m.v = gt ? a.v : b.v;
#pragma unroll
    for (int i = 0; i < W; ++i) m.d[i] = gt ? a.d[i] : (lt ? b.d[i] : 0.5 * (a.d[i] + b.d[i]));
    return m;
}
template <int W>
__device__ __forceinline__ DN<W> fmin(const DN<W>& a, const DN<W>& b) { return a.v <= b.v ? a : b; }

} // namespace ad

template <int R>
constexpr int vjp_smem() {
    // su [4 ND] state, rb [6 ND] own cotangents, tz [2 ND1 NV], tq [3 ND1 NV],
    // tc [12 ND1 NV] cotangent x-contractions, xv [8 NVP] point cotangents,
    // xf [4 * 4 * 2 NM] face-point cotangents, tt [3 NV ND1] transposes,
    // tcd [ND1 NV] d/dxi x-contraction of c (tracer diffusion)
    using S = Sz<R>;
    return 4 * S::ND + 6 * S::ND + 2 * S::ND1 * S::NV + 3 * S::ND1 * S::NV +
           12 * S::ND1 * S::NV + 8 * S::NVP + 32 * S::NM + 3 * S::NV * S::ND1 + S::ND1 * S::NV;
}

// the face fluxes of one face point seen from side A (outward normal n_A):
// {F, Gx, Gy, R} of side A's residual including its pressure term
template <typename T, bool DC = false>
__device__ __forceinline__ void side_flux(T qxA, T qyA, T cA, T hA, T hsA, T qxB, T qyB, T cB,
                                          T hB, T hsB, double nx, double ny, double g, double eps,
                                          T out[4], T* dc = nullptr) {
    T pres, lam;
    rusanov<T, DC>(qxA, qyA, cA, hA, hsA, qxB, qyB, cB, hB, hsB, hsA - hsB, T(nx), T(ny), T(g),
                   T(eps), out, pres, lam, dc);
    out[1] = out[1] - pres * T(nx);
    out[2] = out[2] - pres * T(ny);
}

// register cap: 160 keeps 12 warps resident per SM at r <= 2 (no spills at
// r = 2); r = 3 carries all six directions per lane and keeps more
template <int R, typename Pix, int MODE>
__global__ void __maxnreg__(R == 3 ? 232 : 160)
    k_residual_vjp(const __grid_constant__ Dev d, const __grid_constant__ Tables tb_g,
                   const double* __restrict__ u, const uint8_t* __restrict__ cmask,
                   const double* __restrict__ rbar, double* __restrict__ ubar,
                   double* __restrict__ nbar, double* __restrict__ dbar, int accumulate) {
    // the basis tables in shared memory, as in the forward residual (lane-indexed reads)
    __shared__ Tables s_tb;
    {
        const unsigned* src = (const unsigned*)&tb_g;
        unsigned* dst = (unsigned*)&s_tb;
        for (int i = threadIdx.x; i < (int)(sizeof(Tables) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    const Tables& tb = s_tb;
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NV = S::NV, NVP = S::NVP, NM = S::NM;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* su = smem + warp * vjp_smem<R>();
    double* rb = su + 4 * ND;          // [6][ND] F, Gx, Gy, R, Lx, Ly bars of the cell
    double* tz = rb + 6 * ND;          // [2][ND1][NV] zeta: x-value, x-derivative
    double* tq = tz + 2 * ND1 * NV;    // [3][ND1][NV] qx, qy, c: x-value
    double* tc = tq + 3 * ND1 * NV;    // [6 fields][2: value, d/dxi][ND1][NV]
    double* xv = tc + 12 * ND1 * NV;   // [8][NVP]: bars of z, z_xi, z_eta, qx, qy, c, c_xi, c_eta
    double* xf = xv + 8 * NVP;         // [4 fields][4 faces][2 halves][NM]
    double* tt = xf + 32 * NM;         // [3][NV][ND1]
    double* tcd = tt + 3 * NV * ND1;   // [ND1][NV] c: x-derivative
    const double g = d.g, eps = d.eps;
    const int64_t n = d.n;
    const size_t fs = (size_t)n * ND;  // field stride of the state and cotangent arrays

    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = u[(i / ND) * fs + k * ND + (i % ND)];
        for (int i = lane; i < 6 * ND; i += 32) rb[i] = rbar[(i / ND) * fs + k * ND + (i % ND)];
        const unsigned cm = cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double ihx = 1.0 / hx, ihy = 1.0 / hy;
        const double man = d.manning[k];
        const double nu = d.nu_c ? d.nu_c[k] : 0.0;
        __syncwarp();
        if (nu != 0.0)
            for (int i = lane; i < ND1 * NV; i += 32) {
                const int b = i / NV, al = i % NV;
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += tb.Dv[al][a] * su[3 * ND + ND1 * b + a];
                tcd[i] = s;
            }
        // x-contractions of the state (values at points) and of the cotangents
        // (value and d/dxi: the transposed test functions)
        for (int i = lane; i < 2 * ND1 * NV; i += 32) {
            const int f = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < ND1; ++a) s += (f ? tb.Dv[al][a] : tb.Bv[al][a]) * su[ND1 * b + a];
            tz[i] = s;
        }
        for (int i = lane; i < 3 * ND1 * NV; i += 32) {
            const int f = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < ND1; ++a) s += tb.Bv[al][a] * su[(1 + f) * ND + ND1 * b + a];
            tq[i] = s;
        }
        for (int i = lane; i < 12 * ND1 * NV; i += 32) {
            const int fd = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
            const int fl = fd >> 1, der = fd & 1;
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < ND1; ++a)
                s += (der ? tb.Dv[al][a] : tb.Bv[al][a]) * rb[fl * ND + ND1 * b + a];
            tc[i] = s;
        }
        __syncwarp();
        // volume points: one per lane.  Of the 8 input directions of a point
        // (z, z_xi, z_eta, qx, qy, c, delta, n) the dual numbers carry the first
        // six: z and delta enter only through h = V(z + delta), so their
        // derivatives are equal, and n only through gamma, which is
        // proportional to n^2 (d gamma / dn = 2 gamma / n).  When the points
        // fit in half a warp the two halves take the same point, each with
        // three of the six directions (lane + 16 hands its three to lane), so
        // the dual arithmetic runs on all 32 lanes
        constexpr bool VSPLIT = NVP <= 16;
        constexpr int VW = VSPLIT ? 3 : 6;         // directions per lane
        const int vb0 = VSPLIT ? (lane >> 4) * VW : 0; // first direction of this lane
        constexpr int VSTEP = VSPLIT ? 16 : 32;
        double dsum = 0.0, nsum = 0.0;
        for (int p0 = 0; p0 < NVP; p0 += VSTEP) {
            const int pl = p0 + (VSPLIT ? (lane & 15) : lane);
            const bool pv = pl < NVP;    // a lane past the last point computes point 0, unused
            const int p = pv ? pl : 0;
            const int al = p % NV, be = p / NV;
            double z = 0.0, zxd = 0.0, zyd = 0.0, qx = 0.0, qy = 0.0, c = 0.0;
            // cotangent interpolations: [field][0: (Bv x, Bv y), 1: (Dv x, Bv y), 2: (Bv x, Dv y)]
            double cb[6][3];
#pragma unroll
            for (int fl = 0; fl < 6; ++fl) cb[fl][0] = cb[fl][1] = cb[fl][2] = 0.0;
#pragma unroll
            for (int b = 0; b < ND1; ++b) {
                const double Bb = tb.Bv[be][b], Db = tb.Dv[be][b];
                z += Bb * tz[b * NV + al];
                zxd += Bb * tz[(ND1 + b) * NV + al];
                zyd += Db * tz[b * NV + al];
                qx += Bb * tq[(0 * ND1 + b) * NV + al];
                qy += Bb * tq[(1 * ND1 + b) * NV + al];
                c += Bb * tq[(2 * ND1 + b) * NV + al];
#pragma unroll
                for (int fl = 0; fl < 6; ++fl) {
                    const double v0 = tc[((2 * fl) * ND1 + b) * NV + al];
                    const double v1 = tc[((2 * fl + 1) * ND1 + b) * NV + al];
                    cb[fl][0] += Bb * v0;
                    cb[fl][1] += Bb * v1;
                    cb[fl][2] += Db * v0;
                }
            }
            // forward values as the forward residual takes them (constant fields exact)
            if (cm & 1u) { z = su[0]; zxd = 0.0; zyd = 0.0; }
            if (cm & 2u) qx = su[ND];
            if (cm & 4u) qy = su[2 * ND];
            if (cm & 8u) c = su[3 * ND];
            double V, A;
            ST::VA(d, tb, k, SET_VOL, al, be, z, V, A);
            const double w = J * tb.wv[al] * tb.wv[be];
            // cotangents of the 12 point outputs of the forward (see k_residual)
            const double Xb[12] = {cb[0][1], cb[0][2], cb[3][1], cb[3][2],     // F x,y; R x,y
                                   cb[1][1], cb[1][2], cb[1][0],               // Gx x, y, v
                                   cb[2][1], cb[2][2], cb[2][0],               // Gy x, y, v
                                   cb[4][0], cb[5][0]};                        // Lx, Ly
            double xb[8];
            {
                // dual directions: 0 z, 1 z_xi, 2 z_eta, 3 qx, 4 qy, 5 c
                // (this lane: vb0 .. vb0 + VW - 1); 6 delta = 0 and 7 n follow
                using DV = ad::DN<VW>;
                const DV zx = DV::seed(zxd, 1 - vb0) * DV(ihx);
                const DV zy = DV::seed(zyd, 2 - vb0) * DV(ihy);
                const DV vqx = DV::seed(qx, 3 - vb0), vqy = DV::seed(qy, 4 - vb0);
                const DV vc = DV::seed(c, 5 - vb0);
                DV h(V);
                h.set(0 - vb0, A);
                const DV nn(man);
                const DV fv = vel_factor<DV>(h, DV(eps));
                const DV ux = fv * vqx, uy = fv * vqy;
                const DV gam = gamma_manning<DV>(nn, h, vqx, vqy, DV(g), DV(eps));
                const DV W(w), wx(w * ihx), wy(w * ihy), gg(g);
                const DV X[12] = {wx * vqx, wy * vqy, wx * vc * vqx, wy * vc * vqy,
                                  wx * vqx * ux, wy * vqx * uy, -(W * gg * h * zx),
                                  wx * vqy * ux, wy * vqy * uy, -(W * gg * h * zy),
                                  -(W * gam * vqx), -(W * gam * vqy)};
#pragma unroll
                for (int dir = 0; dir < VW; ++dir) {
                    double s_ = 0.0;
#pragma unroll
                    for (int o = 0; o < 12; ++o) s_ += Xb[o] * X[o].d[dir];
                    xb[dir] = s_;
                }
                if constexpr (VSPLIT) {
#pragma unroll
                    for (int dir = 0; dir < VW; ++dir)
                        xb[VW + dir] = __shfl_down_sync(0xffffffffu, xb[dir], 16);
                }
                xb[6] = xb[0]; // delta: as z, through h = V(z + delta)
                // n: X_10 = -w gamma qx, X_11 = -w gamma qy with gamma ~ n^2
                const double dgdn = man != 0.0 ? 2.0 * gam.v / man : 0.0;
                xb[7] = -(Xb[10] * w * dgdn * qx + Xb[11] * w * dgdn * qy);
            }
            // tracer numerical diffusion (Eq. numdiff): X_2 -= w nu h c_xi / hx^2,
            // X_3 -= w nu h c_eta / hy^2 (linear in grad c; h = V(z + delta))
            double xcx = 0.0, xcy = 0.0;
            if (nu != 0.0) {
                double cxd = 0.0, cyd = 0.0;
#pragma unroll
                for (int b = 0; b < ND1; ++b) {
                    cxd += tb.Bv[be][b] * tcd[b * NV + al];
                    cyd += tb.Dv[be][b] * tq[(2 * ND1 + b) * NV + al];
                }
                const double kx = w * nu * ihx * ihx, ky = w * nu * ihy * ihy;
                xcx = -Xb[2] * kx * V;
                xcy = -Xb[3] * ky * V;
                const double xh = -(Xb[2] * kx * cxd + Xb[3] * ky * cyd);
                xb[0] += A * xh;
                xb[6] += A * xh;
            }
            if (pv && (!VSPLIT || lane < 16)) {
                for (int q = 0; q < 6; ++q) xv[q * NVP + p] = xb[q];
                xv[6 * NVP + p] = xcx;
                xv[7 * NVP + p] = xcy;
                dsum += xb[6];
                nsum += xb[7];
            }
        }
        __syncwarp();
        // faces: one (sub)face point per lane, as the forward
        unsigned fi[4]; // indexed by constants only (registers)
#pragma unroll
        for (int f = 0; f < 4; ++f) fi[f] = d.finfo ? d.finfo[k * 4 + f] : 0;
        // the face points of faces 0..3 start at 0, b1, b2, b3 (2 NM points on
        // a coarse 2:1 face, else NM)
        auto npts = [&](unsigned inf) { return (((inf & 3) == FI_COARSE) ? 2 : 1) * NM; };
        const int b1 = npts(fi[0]), b2 = b1 + npts(fi[1]), b3 = b2 + npts(fi[2]),
                  b4 = b3 + npts(fi[3]);
        // the own side's directions at a face point: zeta, qx, qy and delta
        // are carried by dual numbers; the tracer flux is linear in the
        // concentrations, so the c direction is its partial derivative dc
        // (from the same flux evaluation).  As for the volume points: with at
        // most 16 face points per conforming cell the two halves share a
        // point, directions 0-1 and 2-3
        constexpr bool FSPLIT = 4 * NM <= 16;
        constexpr int FW = FSPLIT ? 2 : 4;
        const int fb0 = FSPLIT ? (lane >> 4) * FW : 0;
        constexpr int FSTEP = FSPLIT ? 16 : 32;
        for (int it0 = 0; it0 < b4; it0 += FSTEP) {
            const int il = it0 + (FSPLIT ? (lane & 15) : lane);
            const bool iv = il < b4; // a lane past the last point computes point 0, unused
            const int it = iv ? il : 0;
            const int f = (it >= b1) + (it >= b2) + (it >= b3);
            const int r_ = it - (f == 0 ? 0 : f == 1 ? b1 : f == 2 ? b2 : b3), h = r_ / NM,
                      al = r_ % NM;
            const unsigned info = f == 0 ? fi[0] : f == 1 ? fi[1] : f == 2 ? fi[2] : fi[3];
            const bool coarse = (info & 3) == FI_COARSE, fine = (info & 3) == FI_FINE;
            const int half = (int)(info >> 2);
            const double nx = (f == 0) ? -1.0 : (f == 1) ? 1.0 : 0.0;
            const double ny = (f == 2) ? -1.0 : (f == 3) ? 1.0 : 0.0;
            const double L = ((f < 2) ? hy : hx) * (coarse ? 0.5 : 1.0);
            const double wl = L * tb.wm[al];
            const double(*Bown)[MXN] = coarse ? tb.BmH[h] : tb.Bm;
            double tm[4], ym[4];
            face_trace<ND1>(su, ND, cm, f, Bown, al, tm);
            face_trace<ND1>(rb, ND, 0u, f, Bown, al, ym); // own residual cotangent at the point
#pragma unroll
            for (int cf = 0; cf < 4; ++cf) ym[cf] *= -wl;
            int ia, ib;
            face_site_index<NM>(f, al, ia, ib);
            auto own_VA = [&](double eta, double& V, double& A) {
                if (coarse) ST::VA_half(d, k, f, h, al, eta, V, A);
                else ST::VA(d, tb, k, SET_MASS, ia, ib, eta, V, A);
            };
            const int32_t s0 = d.nbr[k * 8 + f * 2];
            double hm, Am;
            own_VA(tm[0], hm, Am);
            double xb[5], xl[FW], xc = 0.0; // xc: the c direction
            if (s0 >= 0) {
                const int64_t nb = coarse ? (int64_t)(h ? d.nbr[k * 8 + f * 2 + 1] : s0) : (int64_t)s0;
                const int fo = f ^ 1;
                const double(*Bnb)[MXN] = fine ? tb.BmH[half] : tb.Bm;
                double tp[4], yp[4];
                face_trace<ND1>(u + nb * ND, fs, cmask[nb], fo, Bnb, al, tp);
                face_trace<ND1>(rbar + nb * ND, fs, 0u, fo, Bnb, al, yp);
#pragma unroll
                for (int cf = 0; cf < 4; ++cf) yp[cf] *= -wl;
                int ja, jb;
                face_site_index<NM>(fo, al, ja, jb);
                auto nb_VA = [&](double eta, double& V, double& A) {
                    if (fine) ST::VA_half(d, nb, fo, half, al, eta, V, A);
                    else ST::VA(d, tb, nb, SET_MASS, ja, jb, eta, V, A);
                };
                double hp, Ap, Vnm, Anm, Vop, Aop;
                nb_VA(tp[0], hp, Ap);
                nb_VA(tm[0], Vnm, Anm);
                own_VA(tp[0], Vop, Aop);
                {
                    // dual directions of the own side: 0 zeta, 1 qx, 2 qy, 3 delta
                    // (this lane: fb0 .. fb0 + FW - 1)
                    using DF = ad::DN<FW>;
                    const DF qxm = DF::seed(tm[1], 1 - fb0), qym = DF::seed(tm[2], 2 - fb0);
                    const DF cmv(tm[3]);
                    DF hmD(hm), vnmD(Vnm), vopD(Vop);
                    hmD.set(0 - fb0, Am);   // own operator at own zeta
                    hmD.set(3 - fb0, Am);
                    vnmD.set(0 - fb0, Anm); // neighbour's operator at own zeta
                    vopD.set(3 - fb0, Aop); // own operator at neighbour's zeta
                    const DF hpD(hp);
                    const DF hsm = ad::fmin(hmD, vnmD), hsp = ad::fmin(hpD, vopD);
                    const DF qxp(tp[1]), qyp(tp[2]), cpv(tp[3]);
                    // the face is evaluated once, the lower cell index as side A
                    // (as the forward does); the flux of each side follows from it:
                    // F_side = s raw - pres n_A (momentum), s = +1 for side A, -1 for B
                    // (one call with the sides selected, so the warp does not split)
                    const bool own_low = k < nb;
                    const DF aqx = own_low ? qxm : qxp, aqy = own_low ? qym : qyp;
                    const DF ac = own_low ? cmv : cpv, ah = own_low ? hmD : hpD;
                    const DF ahs = own_low ? hsm : hsp;
                    const DF bqx = own_low ? qxp : qxm, bqy = own_low ? qyp : qym;
                    const DF bc = own_low ? cpv : cmv, bh = own_low ? hpD : hmD;
                    const DF bhs = own_low ? hsp : hsm;
                    const double nAx = own_low ? nx : -nx, nAy = own_low ? ny : -ny;
                    DF raw[4], pres, lam, dcs[2];
                    rusanov<DF, true>(aqx, aqy, ac, ah, ahs, bqx, bqy, bc, bh, bhs, ahs - bhs,
                                      DF(nAx), DF(nAy), DF(g), DF(eps), raw, pres, lam, dcs);
                    const DF pnx = pres * DF(nAx), pny = pres * DF(nAy);
                    const DF so(own_low ? 1.0 : -1.0), sn(own_low ? -1.0 : 1.0);
                    DF oo[4], on[4]; // own side's flux, the neighbour's (its own normal)
                    oo[0] = so * raw[0];
                    oo[1] = so * raw[1] - pnx;
                    oo[2] = so * raw[2] - pny;
                    oo[3] = so * raw[3];
                    on[0] = sn * raw[0];
                    on[1] = sn * raw[1] - pnx;
                    on[2] = sn * raw[2] - pny;
                    on[3] = sn * raw[3];
#pragma unroll
                    for (int dir = 0; dir < FW; ++dir) {
                        double s_ = 0.0;
#pragma unroll
                        for (int cf = 0; cf < 4; ++cf) s_ += ym[cf] * oo[cf].d[dir] + yp[cf] * on[cf].d[dir];
                        xl[dir] = s_;
                    }
                    // c of the own side: only the tracer flux, R_own = so raw3,
                    // R_nb = sn raw3
                    xc = (ym[3] * so.v + yp[3] * sn.v) * (own_low ? dcs[0].v : dcs[1].v);
                }
            } else {
                const int tag = -1 - s0;
                const int mem = member_of(d, k);
                const double t = d.mb[mem].t;
                const bool tide = d.mbc ? d.mbc[mem].kind[tag] == 1 : d.bc_kind[tag] == 1;
                double zt = 0.0, Vt = 0.0, At = 0.0;
                if (tide) {
                    const double amp = d.mbc ? d.mbc[mem].amp[tag] : d.bc_amp[tag];
                    const double per = d.mbc ? d.mbc[mem].per[tag] : d.bc_per[tag];
                    const double ph = d.mbc ? d.mbc[mem].ph[tag] : d.bc_ph[tag];
                    zt = amp * sin(2.0 * M_PI * t / per + ph);
                    own_VA(zt, Vt, At);
                }
                {
                    using DF = ad::DN<FW>;
                    const DF qxm = DF::seed(tm[1], 1 - fb0), qym = DF::seed(tm[2], 2 - fb0);
                    const DF cmv(tm[3]);
                    DF hmD(hm);
                    hmD.set(0 - fb0, Am);
                    hmD.set(3 - fb0, Am);
                    DF qxp = qxm, qyp = qym, hpD = hmD;
                    if (tide) {
                        hpD = DF(Vt); // ghost elevation fixed, same operator
                        hpD.set(3 - fb0, At);
                    } else {
                        const DF qn = qxm * DF(nx) + qym * DF(ny);
                        qxp = qxm - DF(2.0) * qn * DF(nx);
                        qyp = qym - DF(2.0) * qn * DF(ny);
                    }
                    DF oo[4], dcs[2];
                    side_flux<DF, true>(qxm, qym, cmv, hmD, hmD, qxp, qyp, cmv, hpD, hpD, nx, ny, g,
                                        eps, oo, dcs);
#pragma unroll
                    for (int dir = 0; dir < FW; ++dir) {
                        double s_ = 0.0;
#pragma unroll
                        for (int cf = 0; cf < 4; ++cf) s_ += ym[cf] * oo[cf].d[dir];
                        xl[dir] = s_;
                    }
                    // the ghost carries the own concentration: both partials
                    xc = ym[3] * (dcs[0].v + dcs[1].v);
                }
            }
            // all lanes (the branches have joined): gather the five directions
            // xb = {zeta, qx, qy, c, delta}
            if constexpr (FSPLIT) {
                xb[0] = xl[0];
                xb[1] = xl[1];
                xb[2] = __shfl_down_sync(0xffffffffu, xl[0], 16);
                xb[4] = __shfl_down_sync(0xffffffffu, xl[1], 16);
            } else {
                xb[0] = xl[0];
                xb[1] = xl[1];
                xb[2] = xl[2];
                xb[4] = xl[3];
            }
            xb[3] = xc;
            if (iv && (!FSPLIT || lane < 16)) {
#pragma unroll
                for (int cf = 0; cf < 4; ++cf) xf[((cf * 4 + f) * 2 + h) * NM + al] = xb[cf];
                dsum += xb[4];
            }
        }
        __syncwarp();
        // transposed interpolation of the volume-point cotangents, every field
        // in one uniform pass per direction.  y: segments of NV ND1 jobs --
        // 0 zeta (Bv z + Dv z_eta), 1 zeta (Bv z_xi), 2 qx, 3 qy (Bv), 4 c
        // (Bv c + Dv c_eta), 5 c (Bv c_xi); the diffusion rows c_xi, c_eta are
        // zero without diffusion.  x: per field, Bv on the first segment plus
        // Dv on the second (zeta: 0, 1; c: 4, 5; qx, qy: none).  The
        // cotangent x-contractions tc are consumed by now and hold ty.
        {
            constexpr int NY = NV * ND1;
            double* ty = tc; // [6][NV][ND1]
            const int nseg = nu != 0.0 ? 6 : 5;
            for (int i = lane; i < nseg * NY; i += 32) {
                const int seg = i / NY, r_ = i % NY, al = r_ / ND1, b = r_ % ND1;
                const int src1 = seg == 0 ? 0 : seg == 1 ? 1 : seg == 5 ? 6 : seg + 1;
                const double* x1 = xv + src1 * NVP + al;
                const double* x2 = xv + (seg == 0 ? 2 : 7) * NVP + al;
                const double m2 = (seg == 0 || seg == 4) ? 1.0 : 0.0;
                double s_ = 0.0;
#pragma unroll
                for (int be = 0; be < NV; ++be)
                    s_ += tb.Bv[be][b] * x1[NV * be] + m2 * (tb.Dv[be][b] * x2[NV * be]);
                ty[i] = s_;
            }
            __syncwarp();
            double* uacc = xv; // [4][ND]: the point cotangents are consumed by now
            for (int i = lane; i < 4 * ND; i += 32) {
                const int fl = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
                // (without diffusion the c_xi segment is not formed: t2 = t1, times 0)
                const int sa = fl == 0 ? 0 : fl + 1, sb = fl == 0 ? 1 : (nu != 0.0 ? 5 : sa);
                const double m2 = (fl == 0 || (fl == 3 && nu != 0.0)) ? 1.0 : 0.0;
                const double* t1 = ty + sa * NY + b;
                const double* t2 = ty + sb * NY + b;
                double s_ = 0.0;
#pragma unroll
                for (int al = 0; al < NV; ++al)
                    s_ += tb.Bv[al][a] * t1[al * ND1] + m2 * (tb.Dv[al][a] * t2[al * ND1]);
                uacc[i] = s_;
            }
        }
        // lift the face-point cotangents onto the face nodes, then write.  The
        // faces are added in two uniform passes, the x faces (node columns
        // a = 0, ND1 - 1) and then the y faces (rows b = 0, ND1 - 1), one item
        // per field, face and node along it, as in the forward residual
        double* uacc = xv;
        __syncwarp();
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = lane; i < 4 * 2 * ND1; i += 32) {
                const int cf = i / (2 * ND1), r_ = i % (2 * ND1), f = 2 * pass + r_ / ND1;
                const int tn = r_ % ND1; // node index along the face
                const unsigned inf = f == 0 ? fi[0] : f == 1 ? fi[1] : f == 2 ? fi[2] : fi[3];
                const double* fp = xf + (cf * 4 + f) * 2 * NM;
                double s = 0.0;
                if ((inf & 3) == FI_COARSE) {
#pragma unroll
                    for (int al = 0; al < NM; ++al)
                        s += tb.BmH[0][al][tn] * fp[al] + tb.BmH[1][al][tn] * fp[NM + al];
                } else {
#pragma unroll
                    for (int al = 0; al < NM; ++al) s += tb.Bm[al][tn] * fp[al];
                }
                uacc[cf * ND + face_node<ND1>(f, tn)] += s;
            }
            __syncwarp();
        }
        for (int i = lane; i < 4 * ND; i += 32) {
            const int cf = i / ND, j = i % ND;
            if (accumulate) ubar[cf * fs + k * ND + j] += uacc[i];
            else ubar[cf * fs + k * ND + j] = uacc[i];
        }
        const double ds = warp_sum(dsum), ns = warp_sum(nsum);
        if (lane == 0) {
            dbar[k] = accumulate ? dbar[k] + ds : ds;
            nbar[k] = accumulate ? nbar[k] + ns : ns;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// adjoint of one stage update (or of the final combination), Sec. 3.1: the
// cotangent of the stage output v^(l) pulled back to the residuals of the
// earlier stages, to H(zeta^n) and C~^n, to v~^n (the start state after the
// degree switch) through Q~^n, to the previous stage v^(l-1) through the
// friction coefficient, and to n_K, delta_K.  Each converged solve is
// differentiated by the implicit function theorem: the continuity solve
// H(zeta^(l)) = T by M(zeta^(l))^-1 (M symmetric), the tracer solve by
// H_c(zeta^(l))^-1 and dH_c/dzeta, the momentum solve by A^-1 = S^-1 D^-1 S^-T.
// Cell-local: every output is accumulated by the cell's own warp.
// ---------------------------------------------------------------------------
struct StageVjpArgs {
    const double* un;     // v~^n [4][n][nd]
    const uint8_t* cmn;   // its constant-field masks
    const double* uo;     // stage output v^(l) [4][n][nd]
    const uint8_t* cmo;
    const double* up;     // previous stage v^(l-1) [4][n][nd] (friction coefficient)
    const uint8_t* cmp;
    const uint8_t* flag;  // degree flags after this stage (0: the r_K = 0 path)
    const double* vb;     // cotangent of v^(l) [4][n][nd]
    const double* llb_in; // cotangent of the linearised friction this stage formed [2][n][nd]
    double* rbar;         // [stage][6][n][nd] (+=, stages m < nres)
    double* llb_out;      // (+=) cotangent of the linearised friction standing for L of stage nres-1
    double* HNb;          // [n][nd] (+=)
    double* CNb;          // [n][nd] (+=)
    double* ubn;          // cotangent of v~^n [4][n][nd] (+=)
    double* ubp;          // cotangent of v^(l-1) [4][n][nd] (+=)
    double* nbar;         // [n] (+=)
    double* dbar;         // [n] (+=)
    double wa[MXS], wat[MXS], add, dt;
    int nres, make_llin, use_llin;
};

template <int R>
constexpr int stage_vjp_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 5 * S::NMP + S::ND * S::ND + S::ND1 * S::ND1 * S::NM + S::ND +
           2 * S::NM * S::NM + 3 * S::ND + 9 * S::NGP;
}

template <int R, typename Pix, int MODE>
__global__ void __maxnreg__(128)
    k_stage_vjp(const __grid_constant__ Dev d, const __grid_constant__ Tables tb_g,
                const __grid_constant__ StageVjpArgs a) {
    __shared__ Tables s_tb; // basis tables in shared memory (lane-indexed reads)
    {
        const unsigned* src = (const unsigned*)&tb_g;
        unsigned* dst = (unsigned*)&s_tb;
        for (int i = threadIdx.x; i < (int)(sizeof(Tables) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    const Tables& tb = s_tb;
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    // two cells per warp, one per team of 16 lanes (at r <= 2 a cell's loops
    // run over at most 16 nodes and points): "warp" is the team within the
    // block, "lane" the lane within the team, wpb the teams per block
    constexpr int TL = 16;
    const int warp = threadIdx.x / TL, lane = threadIdx.x % TL, wpb = blockDim.x / TL;
    const unsigned tm = 0xFFFFu << (threadIdx.x & 16); // the team's lanes
    double* vb = smem + warp * stage_vjp_smem<R>(); // [4][ND] cotangent of v^(l)
    double* pz = vb + 4 * ND;          // [NMP] zeta^(l) at the mass points
    double* pc = pz + NMP;             // [NMP] c^(l)
    double* pV = pc + NMP;             // [NMP] J w V
    double* pA = pV + NMP;             // [NMP] J w A
    double* pw = pA + NMP;             // [NMP] scratch
    double* M = pw + NMP;              // [ND][ND]
    double* Y = M + ND * ND;           // [ND1 ND1 NM]
    double* inv = Y + ND1 * ND1 * NM;  // [ND]
    double* tmp = inv + ND;            // [2 NM NM]
    double* rcb = tmp + 2 * NM * NM;   // [ND] cotangent of the tracer right-hand side
    double* Tb = rcb + ND;             // [ND] cotangent of T
    double* x = Tb + ND;               // [ND] scratch
    double* gam = x + ND;              // [NGP] friction coefficient of v^(l-1)
    double* gb = gam + NGP;            // [NGP] its cotangent
    double* g3 = gb + NGP;             // [3][NGP] v^(l-1) at the momentum points
    double* Xb = g3 + 3 * NGP;         // [2][NGP]
    double* SQ = Xb + 2 * NGP;         // [2][NGP]
    const int64_t n = d.n;
    const size_t fs = (size_t)n * ND;
    const double g = d.g, eps = d.eps, dt = a.dt;

    // the right-hand-side cotangents spread to the residuals of stages m < nres
    auto to_res = [&](int field, int i, int64_t k, double v, bool implicit) {
        for (int m = 0; m < a.nres; ++m) {
            const double w = implicit ? a.wat[m] : a.wa[m];
            if (w == 0.0) continue;
            const int fld = implicit ? field + 3 : field; // L_x, L_y sit 3 after G_x, G_y
            if (implicit && a.use_llin && m == a.nres - 1)
                a.llb_out[(size_t)(field - 1) * fs + k * ND + i] += dt * w * v;
            else
                a.rbar[((size_t)m * 6 + fld) * fs + k * ND + i] += dt * w * v;
        }
    };

    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += TL) vb[i] = a.vb[(i / ND) * fs + k * ND + (i % ND)];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double man = d.manning[k];
        const bool scalar = a.flag[k] == 0;
        const bool need_gam = (a.add != 0.0 || a.make_llin) && man != 0.0;
        double dsum = 0.0, nsum = 0.0;
        __syncwarp(tm);
        // friction coefficient of v^(l-1) on the momentum points (forward values)
        if (need_gam) {
            const unsigned cmp = a.cmp[k];
            for (int f = 0; f < 3; ++f) {
                tens_interp<ND1, NG, double, TL>(tb.Bg, a.up + f * fs + k * ND, tmp, g3 + f * NGP, lane, tm);
                if (cmp & (1u << f))
                    for (int p = lane; p < NGP; p += TL) g3[f * NGP + p] = a.up[f * fs + k * ND];
                __syncwarp(tm);
            }
            for (int p = lane; p < NGP; p += TL) {
                double V, A;
                ST::VA(d, tb, k, SET_MOM, p % NG, p / NG, g3[p], V, A);
                gam[p] = gamma_manning<double>(man, V, g3[NGP + p], g3[2 * NGP + p], g, eps);
            }
        } else {
            for (int p = lane; p < NGP; p += TL) gam[p] = 0.0;
        }
        for (int p = lane; p < NGP; p += TL) gb[p] = 0.0;
        __syncwarp(tm);
        if (!scalar) {
            // linearised friction Llin_f = -S^T (D0 gamma S Q_f) formed by this stage
            if (a.make_llin && a.llb_in && need_gam) {
                for (int f = 0; f < 2; ++f) {
                    tens_interp<ND1, NG, double, TL>(tb.Bg, a.uo + (1 + f) * fs + k * ND, tmp, SQ + f * NGP, lane, tm);
                    tens_interp<ND1, NG, double, TL>(tb.Bg, a.llb_in + f * fs + k * ND, tmp, Xb + f * NGP, lane, tm);
                }
                for (int p = lane; p < NGP; p += TL) {
                    const double D0 = J * tb.wg[p % NG] * tb.wg[p / NG];
                    gb[p] -= D0 * (SQ[p] * Xb[p] + SQ[NGP + p] * Xb[NGP + p]);
                    Xb[p] *= -D0 * gam[p];
                    Xb[NGP + p] *= -D0 * gam[p];
                }
                __syncwarp(tm);
                for (int f = 0; f < 2; ++f) {
                    tens_test<ND1, NG, double, TL>(tb.Bg, Xb + f * NGP, tmp, x, lane, tm);
                    for (int i = lane; i < ND; i += TL) vb[(1 + f) * ND + i] += x[i];
                    __syncwarp(tm);
                }
            }
            // tracer: rcb = H_c^-1 c_bar, H_c = B^T diag(J w V(zeta^(l))) B
            const unsigned cmo = a.cmo[k];
            tens_interp<ND1, NM, double, TL>(tb.Bm, a.uo + k * ND, tmp, pz, lane, tm);
            tens_interp<ND1, NM, double, TL>(tb.Bm, a.uo + 3 * fs + k * ND, tmp, pc, lane, tm);
            bool allfull = true; // every pixel of every mass sub-cell wet at zeta^(l)
            for (int p = lane; p < NMP; p += TL) {
                if (cmo & 1u) pz[p] = a.uo[k * ND];
                if (cmo & 8u) pc[p] = a.uo[3 * fs + k * ND];
                double V, A;
                bool full;
                ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pz[p], V, A, full);
                const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
                pV[p] = w * V;
                pA[p] = w * A;
                allfull = allfull && full && !zero_bits(A);
            }
            allfull = __all_sync(tm, allfull);
            __syncwarp(tm);
            // the forward's mixed-precision solve (FP32 factor, FP64 refinement to
            // 1e-15, FP64 Cholesky fallback); its FP32 arrays overlay M and Y, its
            // iterate and residual take x and Tb, its points pw (all idle here)
            for (int i = lane; i < ND; i += TL) rcb[i] = vb[3 * ND + i];
            __syncwarp(tm);
            solve_mass_mixed<ND1, NM, TL>(tb, pV, rcb, (float*)M, (float*)Y, x, Tb, pw, tmp, M, Y,
                                          inv, lane, tm);
            // dH_c/dzeta: zeta_bar(p) -= J w A rcb(p) c(p); the same for delta
            tens_interp<ND1, NM, double, TL>(tb.Bm, rcb, tmp, pw, lane, tm);
            for (int p = lane; p < NMP; p += TL) {
                pw[p] = -pA[p] * pw[p] * pc[p];
                dsum += pw[p];
            }
            __syncwarp(tm);
            tens_test<ND1, NM, double, TL>(tb.Bm, pw, tmp, x, lane, tm);
            for (int i = lane; i < ND; i += TL) {
                vb[i] += x[i];
                a.CNb[k * ND + i] += rcb[i];
                to_res(3, i, k, rcb[i], false);
            }
            __syncwarp(tm);
            // momentum: X_bar = S^-T Q_bar; rq_bar = S^-1 (X_bar / D); q^n part D0 X_bar / D;
            // D_bar = -X_bar (S Q) / D -> gamma_bar
            for (int f = 0; f < 2; ++f) {
                kron_apply<ND1, true, MXP, double, TL>(tb.Bginv, vb + (1 + f) * ND, tmp, Xb + f * NGP, 1.0, lane, tm);
                tens_interp<ND1, NG, double, TL>(tb.Bg, a.uo + (1 + f) * fs + k * ND, tmp, SQ + f * NGP, lane, tm);
            }
            for (int p = lane; p < NGP; p += TL) {
                const double D0 = J * tb.wg[p % NG] * tb.wg[p / NG];
                const double D = D0 * (1.0 + a.add * dt * gam[p]);
                gb[p] -= (Xb[p] * SQ[p] + Xb[NGP + p] * SQ[NGP + p]) / D * D0 * a.add * dt;
                Xb[p] /= D;
                Xb[NGP + p] /= D;
                SQ[p] = Xb[p] * D0;           // q^n cotangent at the points
                SQ[NGP + p] = Xb[NGP + p] * D0;
            }
            __syncwarp(tm);
            for (int f = 0; f < 2; ++f) {
                kron_apply<ND1, false, MXP, double, TL>(tb.Bginv, Xb + f * NGP, tmp, x, 1.0, lane, tm);
                for (int i = lane; i < ND; i += TL) {
                    to_res(1 + f, i, k, x[i], false);
                    to_res(1 + f, i, k, x[i], true);
                }
                __syncwarp(tm);
                tens_test<ND1, NG, double, TL>(tb.Bg, SQ + f * NGP, tmp, x, lane, tm);
                for (int i = lane; i < ND; i += TL) a.ubn[(1 + f) * fs + k * ND + i] += x[i];
                __syncwarp(tm);
            }
            // continuity: T_bar = M(zeta^(l))^-1 zeta_bar, M = B^T diag(J w A) B; the
            // offset moves H(zeta^(l)) by J w A: delta_bar -= sum J w A T_bar(p)
            if (allfull) {
                // wholly wet: M = J (M1 x M1), inverted by its tensor factors (as the
                // forward's Newton step there)
                kron_apply<ND1, false, MXN, double, TL>(tb.M1inv, vb, tmp, Tb, 1.0 / J, lane, tm);
            } else {
                assemble_mass<ND1, NM, TL>(tb, pA, Y, M, lane, tm);
                for (int i = lane; i < ND; i += TL) Tb[i] = vb[i];
                __syncwarp(tm);
                chol_solve<ND, TL>(M, Tb, inv, lane, tm);
            }
            tens_interp<ND1, NM, double, TL>(tb.Bm, Tb, tmp, pw, lane, tm);
            for (int p = lane; p < NMP; p += TL) dsum -= pA[p] * pw[p];
            for (int i = lane; i < ND; i += TL) {
                a.HNb[k * ND + i] += Tb[i];
                to_res(0, i, k, Tb[i], false);
            }
            __syncwarp(tm);
        } else {
            // the r_K = 0 path: one value per field, test function 1
            const double e = a.uo[k * ND], cl = a.uo[3 * fs + k * ND];
            const double vq[2] = {a.uo[fs + k * ND], a.uo[2 * fs + k * ND]};
            double ez = 0.0, qs[2] = {0.0, 0.0}, cs = 0.0;
            for (int i = lane; i < ND; i += TL) {
                ez += vb[i];
                qs[0] += vb[ND + i];
                qs[1] += vb[2 * ND + i];
                cs += vb[3 * ND + i];
            }
            ez = team_sum<TL>(ez, tm);
            qs[0] = team_sum<TL>(qs[0], tm);
            qs[1] = team_sum<TL>(qs[1], tm);
            cs = team_sum<TL>(cs, tm);
            if (a.make_llin && a.llb_in && need_gam) {
                for (int f = 0; f < 2; ++f)
                    tens_interp<ND1, NG, double, TL>(tb.Bg, a.llb_in + f * fs + k * ND, tmp, Xb + f * NGP, lane, tm);
                double s0 = 0.0, s1 = 0.0;
                for (int p = lane; p < NGP; p += TL) {
                    const double D0 = J * tb.wg[p % NG] * tb.wg[p / NG];
                    gb[p] -= D0 * (vq[0] * Xb[p] + vq[1] * Xb[NGP + p]);
                    s0 -= D0 * gam[p] * Xb[p];
                    s1 -= D0 * gam[p] * Xb[NGP + p];
                }
                qs[0] += team_sum<TL>(s0, tm);
                qs[1] += team_sum<TL>(s1, tm);
            }
            double Hs, As;
            mass_scalar_pixels<R, Pix, MODE, TL>(d, tb, k, J, e, lane, Hs, As, tm);
            // tracer: c = (CNbar + dt sum a sum_i R_i) / Hbar(e), or c^n in a dry cell
            if (Hs > 1e-14 * J * d.hlim) {
                const double rsb = cs / Hs, Hsb = -cs * cl / Hs;
                ez += Hsb * As;
                if (lane == 0) dsum += Hsb * As;
                for (int i = lane; i < ND; i += TL) {
                    a.CNb[k * ND + i] += rsb;
                    to_res(3, i, k, rsb, false);
                }
            } else {
                for (int i = lane; i < ND; i += TL) a.ubn[3 * fs + k * ND + i] += vb[3 * ND + i];
            }
            // momentum: q = (sum_p D0 q^n(p) + sum_i rq_i) / sum_p D
            double den = 0.0;
            for (int p = lane; p < NGP; p += TL) {
                const double D0 = J * tb.wg[p % NG] * tb.wg[p / NG];
                den += D0 * (1.0 + a.add * dt * gam[p]);
            }
            den = team_sum<TL>(den, tm);
            const double denb = -(qs[0] * vq[0] + qs[1] * vq[1]) / den;
            for (int p = lane; p < NGP; p += TL) {
                const double D0 = J * tb.wg[p % NG] * tb.wg[p / NG];
                gb[p] += denb * D0 * a.add * dt;
                Xb[p] = D0 * qs[0] / den;
                Xb[NGP + p] = D0 * qs[1] / den;
            }
            __syncwarp(tm);
            for (int f = 0; f < 2; ++f) {
                tens_test<ND1, NG, double, TL>(tb.Bg, Xb + f * NGP, tmp, x, lane, tm);
                for (int i = lane; i < ND; i += TL) {
                    a.ubn[(1 + f) * fs + k * ND + i] += x[i];
                    to_res(1 + f, i, k, qs[f] / den, false);
                    to_res(1 + f, i, k, qs[f] / den, true);
                }
                __syncwarp(tm);
            }
            // continuity: Hbar(e) = HNbar + dt sum a sum_i F_i (the offset moves Hbar by A)
            if (As > 0.0) {
                const double tsb = ez / As;
                if (lane == 0) dsum -= ez;
                for (int i = lane; i < ND; i += TL) {
                    a.HNb[k * ND + i] += tsb;
                    to_res(0, i, k, tsb, false);
                }
            }
            __syncwarp(tm);
        }
        // friction coefficient of v^(l-1): gamma(n, V(zeta), qx, qy) at each point
        if (need_gam) {
            for (int p = lane; p < NGP; p += TL) {
                double V, A;
                ST::VA(d, tb, k, SET_MOM, p % NG, p / NG, g3[p], V, A);
                const double qx = g3[NGP + p], qy = g3[2 * NGP + p], gbp = gb[p];
                // directions: 0 h, 1 qx, 2 qy, 3 n
                using DG = ad::DN<4>;
                const DG r = gamma_manning<DG>(DG::seed(man, 3), DG::seed(V, 0), DG::seed(qx, 1),
                                               DG::seed(qy, 2), DG(g), DG(eps));
                const double* dg = r.d;
                g3[p] = gbp * dg[0] * A;
                g3[NGP + p] = gbp * dg[1];
                g3[2 * NGP + p] = gbp * dg[2];
                dsum += gbp * dg[0] * A;
                nsum += gbp * dg[3];
            }
            __syncwarp(tm);
            for (int f = 0; f < 3; ++f) {
                tens_test<ND1, NG, double, TL>(tb.Bg, g3 + f * NGP, tmp, x, lane, tm);
                for (int i = lane; i < ND; i += TL) a.ubp[f * fs + k * ND + i] += x[i];
                __syncwarp(tm);
            }
        }
        const double ds = team_sum<TL>(dsum, tm), ns = team_sum<TL>(nsum, tm);
        if (lane == 0) {
            a.dbar[k] += ds;
            a.nbar[k] += ns;
        }
        __syncwarp(tm);
    }
}

// ---------------------------------------------------------------------------
// adjoint of the step start: H(zeta~^n), C~^n (Eqs. depth_rhs,
// concentration_rhs) and the degree switch's mass-exact remap of r_K = 0
// cells (zeta: Hbar(e) = Hbar(zeta^n); q: Gauss-Legendre means; c: tracer
// mass / mass, or the mean in a dry cell; a completely dry cell sits at
// -max(z_b + delta))
// ---------------------------------------------------------------------------
struct BeginVjpArgs {
    const double* upre;   // v^n before the degree switch [4][n][nd]
    const double* un;     // v~^n [4][n][nd]
    const uint8_t* cmn;
    const uint8_t* flag0; // flags of the degree switch
    const double* HNb;
    const double* CNb;
    const double* ubn;    // cotangent of v~^n (all but the H, C~ parts)
    double* ubpre;        // out: cotangent of v^n [4][n][nd]
    double* dbar;         // (+=)
};

template <int R>
constexpr int begin_vjp_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 6 * S::NMP + 2 * S::NM * S::NM + S::ND + S::NGP;
}

template <int R, typename Pix, int MODE>
__global__ void __maxnreg__(96)
    k_begin_vjp(const __grid_constant__ Dev d, const __grid_constant__ Tables tb_g,
                const __grid_constant__ BeginVjpArgs a) {
    __shared__ Tables s_tb; // basis tables in shared memory (lane-indexed reads)
    {
        const unsigned* src = (const unsigned*)&tb_g;
        unsigned* dst = (unsigned*)&s_tb;
        for (int i = threadIdx.x; i < (int)(sizeof(Tables) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    const Tables& tb = s_tb;
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* ub = smem + warp * begin_vjp_smem<R>(); // [4][ND]
    double* pz = ub + 4 * ND;   // [NMP]
    double* pc = pz + NMP;
    double* h1 = pc + NMP;      // [NMP] H_bar at the points, then zeta~ cotangent
    double* c1 = h1 + NMP;      // [NMP] C~_bar at the points, then c~ cotangent
    double* pV = c1 + NMP;      // [NMP]
    double* pA = pV + NMP;      // [NMP]
    double* tmp = pA + NMP;     // [2 NM NM]
    double* x = tmp + 2 * NM * NM; // [ND]
    double* pg = x + ND;        // [NGP]
    const int64_t n = d.n;
    const size_t fs = (size_t)n * ND;
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += 32) ub[i] = a.ubn[(i / ND) * fs + k * ND + (i % ND)];
        const double J = d.hxhy[2 * k] * d.hxhy[2 * k + 1];
        const unsigned cm = a.cmn[k];
        double dsum = 0.0;
        __syncwarp();
        // H_i = sum_p J w V(zeta~) psi_i, C~_i = sum_p J w V c~ psi_i
        tens_interp<ND1, NM>(tb.Bm, a.un + k * ND, tmp, pz, lane);
        tens_interp<ND1, NM>(tb.Bm, a.un + 3 * fs + k * ND, tmp, pc, lane);
        tens_interp<ND1, NM>(tb.Bm, a.HNb + k * ND, tmp, h1, lane);
        tens_interp<ND1, NM>(tb.Bm, a.CNb + k * ND, tmp, c1, lane);
        for (int p = lane; p < NMP; p += 32) {
            if (cm & 1u) pz[p] = a.un[k * ND];
            if (cm & 8u) pc[p] = a.un[3 * fs + k * ND];
            double V, A;
            ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pz[p], V, A);
            const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
            const double zt = w * A * (h1[p] + pc[p] * c1[p]);
            c1[p] = w * V * c1[p];
            h1[p] = zt;
            dsum += zt;
        }
        __syncwarp();
        tens_test<ND1, NM>(tb.Bm, h1, tmp, x, lane);
        for (int i = lane; i < ND; i += 32) ub[i] += x[i];
        __syncwarp();
        tens_test<ND1, NM>(tb.Bm, c1, tmp, x, lane);
        for (int i = lane; i < ND; i += 32) ub[3 * ND + i] += x[i];
        __syncwarp();
        if (a.flag0[k] != 0) {
            for (int i = lane; i < 4 * ND; i += 32) a.ubpre[(i / ND) * fs + k * ND + (i % ND)] = ub[i];
        } else {
            // remap of v^n to one value per field
            tens_interp<ND1, NM>(tb.Bm, a.upre + k * ND, tmp, pz, lane);
            tens_interp<ND1, NM>(tb.Bm, a.upre + 3 * fs + k * ND, tmp, pc, lane);
            double m = 0.0, tr = 0.0, Am = 0.0;
            for (int p = lane; p < NMP; p += 32) {
                double V, A;
                ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pz[p], V, A);
                const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
                pV[p] = w * V;
                pA[p] = w * A;
                m += w * V;
                tr += w * V * pc[p];
                Am += w * A;
            }
            m = warp_sum(m);
            tr = warp_sum(tr);
            Am = warp_sum(Am);
            double ez = 0.0, qs[2] = {0.0, 0.0}, cs = 0.0;
            for (int i = lane; i < ND; i += 32) {
                ez += ub[i];
                qs[0] += ub[ND + i];
                qs[1] += ub[2 * ND + i];
                cs += ub[3 * ND + i];
            }
            ez = warp_sum(ez);
            qs[0] = warp_sum(qs[0]);
            qs[1] = warp_sum(qs[1]);
            cs = warp_sum(cs);
            // q~ = sum_p w_p q(p) on the Gauss-Legendre points
            for (int f = 0; f < 2; ++f) {
                for (int p = lane; p < NGP; p += 32) pg[p] = tb.wg[p % NG] * tb.wg[p / NG] * qs[f];
                __syncwarp();
                tens_test<ND1, NG>(tb.Bg, pg, tmp, x, lane);
                for (int i = lane; i < ND; i += 32) a.ubpre[(1 + f) * fs + k * ND + i] = x[i];
                __syncwarp();
            }
            double mb = 0.0;
            for (int p = lane; p < NMP; p += 32) h1[p] = 0.0;
            if (m > 1e-14 * J * d.hlim) { // c~ = tracer / m
                const double tb_ = cs / m;
                mb -= cs * (tr / m) / m;
                for (int p = lane; p < NMP; p += 32) {
                    c1[p] = tb_ * pV[p];
                    h1[p] += tb_ * pA[p] * pc[p];
                    dsum += tb_ * pA[p] * pc[p];
                }
                __syncwarp();
                tens_test<ND1, NM>(tb.Bm, c1, tmp, x, lane);
            } else {                       // c~ = Gauss-Legendre mean
                for (int p = lane; p < NGP; p += 32) pg[p] = tb.wg[p % NG] * tb.wg[p / NG] * cs;
                __syncwarp();
                tens_test<ND1, NG>(tb.Bg, pg, tmp, x, lane);
            }
            for (int i = lane; i < ND; i += 32) a.ubpre[3 * fs + k * ND + i] = x[i];
            __syncwarp();
            // zeta~ = e with Hbar(e, delta) = m(zeta^n, delta); dry: e = -max(z_b + delta)
            if (m > 0.0) {
                double Hs, As;
                mass_scalar_pixels<R, Pix, MODE>(d, tb, k, J, a.un[k * ND], lane, Hs, As);
                if (As > 0.0) mb += ez / As;
            }
            if (lane == 0) dsum -= ez;
            for (int p = lane; p < NMP; p += 32) {
                h1[p] += mb * pA[p];
                dsum += mb * pA[p];
            }
            __syncwarp();
            tens_test<ND1, NM>(tb.Bm, h1, tmp, x, lane);
            for (int i = lane; i < ND; i += 32) a.ubpre[k * ND + i] = x[i];
            __syncwarp();
        }
        const double ds = warp_sum(dsum);
        if (lane == 0) a.dbar[k] += ds;
        __syncwarp();
    }
}

} // namespace swdg
