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
// numbers through the same templates the forward residual runs, one input
// direction per pass.  The sub-grid operator enters through V and its exact
// derivative A = dV/d(eta) = dV/d(delta).
//
// Derivative conventions at the kinks: max(x, 0) -> [x > 0] (Eq. mask); the
// reconstruction's min and the wave-speed max follow their first argument at
// ties, the first argument being the side whose residual is differentiated;
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
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
    const double q = a.v / b.v;
    return D1(q, (a.d - q * b.d) / b.v);
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
__device__ __forceinline__ D1 fmin(D1 a, D1 b) { return a.v <= b.v ? a : b; }

} // namespace ad

template <int R>
constexpr int vjp_smem() {
    // su [4 ND] state, rb [6 ND] own cotangents, tz [2 ND1 NV], tq [3 ND1 NV],
    // tc [12 ND1 NV] cotangent x-contractions, xv [6 NVP] point cotangents,
    // xf [4 * 4 * 2 NM] face-point cotangents, tt [3 NV ND1] transposes
    using S = Sz<R>;
    return 4 * S::ND + 6 * S::ND + 2 * S::ND1 * S::NV + 3 * S::ND1 * S::NV +
           12 * S::ND1 * S::NV + 6 * S::NVP + 32 * S::NM + 3 * S::NV * S::ND1;
}

// the face fluxes of one face point seen from side A (outward normal n_A):
// {F, Gx, Gy, R} of side A's residual including its pressure term
template <typename T>
__device__ __forceinline__ void side_flux(T qxA, T qyA, T cA, T hA, T hsA, T qxB, T qyB, T cB,
                                          T hB, T hsB, double nx, double ny, double g, double eps,
                                          T out[4]) {
    T pres, lam;
    rusanov<T>(qxA, qyA, cA, hA, hsA, qxB, qyB, cB, hB, hsB, hsA - hsB, T(nx), T(ny), T(g), T(eps),
               out, pres, lam);
    out[1] = out[1] - pres * T(nx);
    out[2] = out[2] - pres * T(ny);
}

template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(32 * MAXWPB)
    k_residual_vjp(const __grid_constant__ Dev d, const __grid_constant__ Tables tb,
                   const double* __restrict__ rbar, double* __restrict__ ubar,
                   double* __restrict__ nbar, double* __restrict__ dbar) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    using ad::D1;
    constexpr int ND1 = S::ND1, ND = S::ND, NV = S::NV, NVP = S::NVP, NM = S::NM;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* su = smem + warp * vjp_smem<R>();
    double* rb = su + 4 * ND;          // [6][ND] F, Gx, Gy, R, Lx, Ly bars of the cell
    double* tz = rb + 6 * ND;          // [2][ND1][NV] zeta: x-value, x-derivative
    double* tq = tz + 2 * ND1 * NV;    // [3][ND1][NV] qx, qy, c: x-value
    double* tc = tq + 3 * ND1 * NV;    // [6 fields][2: value, d/dxi][ND1][NV]
    double* xv = tc + 12 * ND1 * NV;   // [6][NVP]: bars of z, z_xi, z_eta, qx, qy, c at points
    double* xf = xv + 6 * NVP;         // [4 fields][4 faces][2 halves][NM]
    double* tt = xf + 32 * NM;         // [3][NV][ND1]
    const double g = d.g, eps = d.eps;
    const int64_t n = d.n;
    const size_t fs = (size_t)n * ND;  // field stride of the state and cotangent arrays

    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        for (int i = lane; i < 6 * ND; i += 32) rb[i] = rbar[(i / ND) * fs + k * ND + (i % ND)];
        const unsigned cm = d.cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double ihx = 1.0 / hx, ihy = 1.0 / hy;
        const double man = d.manning[k];
        __syncwarp();
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
        // volume points: one per lane
        double dsum = 0.0, nsum = 0.0;
        for (int p = lane; p < NVP; p += 32) {
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
            // input directions: 0 z, 1 z_xi, 2 z_eta, 3 qx, 4 qy, 5 c, 6 delta, 7 n
#pragma unroll 1
            for (int dir = 0; dir < 8; ++dir) {
                const D1 zz(z, dir == 0 ? 1.0 : 0.0);
                const D1 zx = D1(zxd, dir == 1 ? 1.0 : 0.0) * D1(ihx);
                const D1 zy = D1(zyd, dir == 2 ? 1.0 : 0.0) * D1(ihy);
                const D1 vqx(qx, dir == 3 ? 1.0 : 0.0), vqy(qy, dir == 4 ? 1.0 : 0.0);
                const D1 vc(c, dir == 5 ? 1.0 : 0.0);
                const D1 h(V, A * (zz.d + (dir == 6 ? 1.0 : 0.0)));
                const D1 nn(man, dir == 7 ? 1.0 : 0.0);
                const D1 fv = vel_factor<D1>(h, D1(eps));
                const D1 ux = fv * vqx, uy = fv * vqy;
                const D1 gam = gamma_manning<D1>(nn, h, vqx, vqy, D1(g), D1(eps));
                const D1 W(w), wx(w * ihx), wy(w * ihy), gg(g);
                const D1 X[12] = {wx * vqx, wy * vqy, wx * vc * vqx, wy * vc * vqy,
                                  wx * vqx * ux, wy * vqx * uy, -(W * gg * h * zx),
                                  wx * vqy * ux, wy * vqy * uy, -(W * gg * h * zy),
                                  -(W * gam * vqx), -(W * gam * vqy)};
                double s = 0.0;
#pragma unroll
                for (int o = 0; o < 12; ++o) s += Xb[o] * X[o].d;
                xb[dir] = s;
            }
            for (int q = 0; q < 6; ++q) xv[q * NVP + p] = xb[q];
            dsum += xb[6];
            nsum += xb[7];
        }
        __syncwarp();
        // faces: one (sub)face point per lane, as the forward
        unsigned char fi[4];
        int base[5];
        base[0] = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            fi[f] = d.finfo ? d.finfo[k * 4 + f] : 0;
            base[f + 1] = base[f] + (((fi[f] & 3) == FI_COARSE) ? 2 : 1) * NM;
        }
        for (int it = lane; it < base[4]; it += 32) {
            const int f = (it >= base[1]) + (it >= base[2]) + (it >= base[3]);
            const int r_ = it - base[f], h = r_ / NM, al = r_ % NM;
            const unsigned info = fi[f];
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
            double xb[5];
            if (s0 >= 0) {
                const int64_t nb = coarse ? (int64_t)(h ? d.nbr[k * 8 + f * 2 + 1] : s0) : (int64_t)s0;
                const int fo = f ^ 1;
                const double(*Bnb)[MXN] = fine ? tb.BmH[half] : tb.Bm;
                double tp[4], yp[4];
                face_trace<ND1>(ufield(d, 0, 0, ND) + nb * ND, fs, d.cmask[nb], fo, Bnb, al, tp);
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
#pragma unroll 1
                for (int dir = 0; dir < 5; ++dir) {
                    // directions of the own side: 0 zeta, 1 qx, 2 qy, 3 c, 4 delta
                    const double dz = dir == 0 ? 1.0 : 0.0, dd = dir == 4 ? 1.0 : 0.0;
                    const D1 qxm(tm[1], dir == 1 ? 1.0 : 0.0), qym(tm[2], dir == 2 ? 1.0 : 0.0);
                    const D1 cmv(tm[3], dir == 3 ? 1.0 : 0.0);
                    const D1 hmD(hm, Am * (dz + dd));         // own operator at own zeta
                    const D1 vnmD(Vnm, Anm * dz);              // neighbour's operator at own zeta
                    const D1 vopD(Vop, Aop * dd);              // own operator at neighbour's zeta
                    const D1 hpD(hp);
                    const D1 hsm = ad::fmin(hmD, vnmD), hsp = ad::fmin(hpD, vopD);
                    const D1 qxp(tp[1]), qyp(tp[2]), cpv(tp[3]);
                    D1 oo[4], on[4];
                    side_flux<D1>(qxm, qym, cmv, hmD, hsm, qxp, qyp, cpv, hpD, hsp, nx, ny, g, eps, oo);
                    side_flux<D1>(qxp, qyp, cpv, hpD, hsp, qxm, qym, cmv, hmD, hsm, -nx, -ny, g, eps, on);
                    double s = 0.0;
#pragma unroll
                    for (int cf = 0; cf < 4; ++cf) s += ym[cf] * oo[cf].d + yp[cf] * on[cf].d;
                    xb[dir] = s;
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
#pragma unroll 1
                for (int dir = 0; dir < 5; ++dir) {
                    const double dz = dir == 0 ? 1.0 : 0.0, dd = dir == 4 ? 1.0 : 0.0;
                    const D1 qxm(tm[1], dir == 1 ? 1.0 : 0.0), qym(tm[2], dir == 2 ? 1.0 : 0.0);
                    const D1 cmv(tm[3], dir == 3 ? 1.0 : 0.0);
                    const D1 hmD(hm, Am * (dz + dd));
                    D1 qxp = qxm, qyp = qym, hpD = hmD;
                    if (tide) {
                        hpD = D1(Vt, At * dd); // ghost elevation fixed, same operator
                    } else {
                        const D1 qn = qxm * D1(nx) + qym * D1(ny);
                        qxp = qxm - D1(2.0) * qn * D1(nx);
                        qyp = qym - D1(2.0) * qn * D1(ny);
                    }
                    D1 oo[4];
                    side_flux<D1>(qxm, qym, cmv, hmD, hmD, qxp, qyp, cmv, hpD, hpD, nx, ny, g, eps, oo);
                    double s = 0.0;
#pragma unroll
                    for (int cf = 0; cf < 4; ++cf) s += ym[cf] * oo[cf].d;
                    xb[dir] = s;
                }
            }
#pragma unroll
            for (int cf = 0; cf < 4; ++cf) xf[((cf * 4 + f) * 2 + h) * NM + al] = xb[cf];
            dsum += xb[4];
        }
        __syncwarp();
        // transposed interpolation of the volume-point cotangents: y, then x
        // zeta: q = 0 holds the (Bv, Bv) z and (Bv, Dv) z_eta parts, q = 1 the
        // (Dv, Bv) z_xi part, both after the y-contraction
        for (int i = lane; i < 2 * NV * ND1; i += 32) {
            const int q = i / (NV * ND1), r_ = i % (NV * ND1), al = r_ / ND1, b = r_ % ND1;
            double s = 0.0;
            if (q == 0) {
#pragma unroll
                for (int be = 0; be < NV; ++be)
                    s += tb.Bv[be][b] * xv[0 * NVP + al + NV * be] +
                         tb.Dv[be][b] * xv[2 * NVP + al + NV * be];
            } else {
#pragma unroll
                for (int be = 0; be < NV; ++be) s += tb.Bv[be][b] * xv[1 * NVP + al + NV * be];
            }
            tt[i] = s;
        }
        __syncwarp();
        constexpr int NC = (ND + 31) / 32; // nodes per lane
        double ub[4 * NC];
        for (int i = lane, c_ = 0; i < ND; i += 32, ++c_) {
            const int a = i % ND1, b = i / ND1;
            double s = 0.0;
#pragma unroll
            for (int al = 0; al < NV; ++al)
                s += tb.Bv[al][a] * tt[(0 * NV + al) * ND1 + b] +
                     tb.Dv[al][a] * tt[(1 * NV + al) * ND1 + b];
            ub[c_] = s;
        }
        __syncwarp();
        // qx, qy, c: (Bv, Bv) transposes
        for (int fl = 0; fl < 3; ++fl) {
            for (int i = lane; i < NV * ND1; i += 32) {
                const int al = i / ND1, b = i % ND1;
                double s = 0.0;
#pragma unroll
                for (int be = 0; be < NV; ++be) s += tb.Bv[be][b] * xv[(3 + fl) * NVP + al + NV * be];
                tt[i] = s;
            }
            __syncwarp();
            for (int i = lane, c_ = 0; i < ND; i += 32, ++c_) {
                const int a = i % ND1, b = i / ND1;
                double s = 0.0;
#pragma unroll
                for (int al = 0; al < NV; ++al) s += tb.Bv[al][a] * tt[al * ND1 + b];
                ub[(1 + fl) * NC + c_] = s;
            }
            __syncwarp();
        }
        // lift the face-point cotangents onto the face nodes, then write
        for (int i = lane, c_ = 0; i < ND; i += 32, ++c_) {
            const int a = i % ND1, b = i / ND1;
#pragma unroll
            for (int cf = 0; cf < 4; ++cf) {
                double s = ub[cf * NC + c_];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const bool on = (f == 0 && a == 0) || (f == 1 && a == ND1 - 1) ||
                                    (f == 2 && b == 0) || (f == 3 && b == ND1 - 1);
                    if (!on) continue;
                    const int tn = f < 2 ? b : a;
                    const double* fp = xf + (cf * 4 + f) * 2 * NM;
                    if ((fi[f] & 3) == FI_COARSE) {
                        for (int al = 0; al < NM; ++al)
                            s += tb.BmH[0][al][tn] * fp[al] + tb.BmH[1][al][tn] * fp[NM + al];
                    } else {
                        for (int al = 0; al < NM; ++al) s += tb.Bm[al][tn] * fp[al];
                    }
                }
                ubar[cf * fs + k * ND + i] = s;
            }
        }
        const double ds = warp_sum(dsum), ns = warp_sum(nsum);
        if (lane == 0) {
            dbar[k] = ds;
            nbar[k] = ns;
        }
        __syncwarp();
    }
}

} // namespace swdg
