// swdg_kernels.cuh -- sm_103a kernels of the sub-grid DG shallow-water hot
// path (arXiv 2505.18743): residual (Sec. 3.2), degree switch (Eq.
// criteria_p), stage update (Sec. 3.1) and auxiliary reductions.
//
// Mapping: one warp per cell, four warps per block, grid-stride over cells.
// Each warp stages its cell in shared memory and evaluates the tensor-product
// operators by sum factorisation (1D contractions), one quadrature point,
// degree of freedom or face point per lane.
#pragma once
#include "swdg_common.cuh"

namespace swdg {

constexpr int WPB = 4; // warps per block
constexpr int TPB = 32 * WPB;

// ---------------------------------------------------------------------------
// small tensor contractions on a warp (all arrays in shared memory, x fastest)
// ---------------------------------------------------------------------------
// out[q1 NO + q0] = sum_b B[q1][b] sum_a B[q0][a] in[b NI + a]
template <int NI, int NO>
__device__ __forceinline__ void tens_interp(const double (*B)[MXN], const double* in, double* tmp,
                                            double* out, int lane) {
    for (int i = lane; i < NI * NO; i += 32) {
        int b = i / NO, q0 = i % NO;
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < NI; ++a) s += B[q0][a] * in[b * NI + a];
        tmp[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < NO * NO; i += 32) {
        int q1 = i / NO, q0 = i % NO;
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < NI; ++b) s += B[q1][b] * tmp[b * NO + q0];
        out[i] = s;
    }
    __syncwarp();
}

// out[b NI + a] = sum_q1 B[q1][b] sum_q0 B[q0][a] in[q1 NO + q0]   (transpose)
template <int NI, int NO>
__device__ __forceinline__ void tens_test(const double (*B)[MXN], const double* in, double* tmp,
                                          double* out, int lane) {
    for (int i = lane; i < NO * NI; i += 32) {
        int q1 = i / NI, a = i % NI;
        double s = 0.0;
#pragma unroll
        for (int q0 = 0; q0 < NO; ++q0) s += B[q0][a] * in[q1 * NO + q0];
        tmp[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < NI * NI; i += 32) {
        int b = i / NI, a = i % NI;
        double s = 0.0;
#pragma unroll
        for (int q1 = 0; q1 < NO; ++q1) s += B[q1][b] * tmp[q1 * NI + a];
        out[i] = s;
    }
    __syncwarp();
}

// out[b N + a] = scale * sum_d C(b,d) sum_c C(a,c) in[d N + c], C(i,j) = T ? M[j][i] : M[i][j]
template <int N, bool T, int LD>
__device__ __forceinline__ void kron_apply(const double (*M)[LD], const double* in, double* tmp,
                                           double* out, double scale, int lane) {
    for (int i = lane; i < N * N; i += 32) {
        int d = i / N, a = i % N;
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) s += (T ? M[c][a] : M[a][c]) * in[d * N + c];
        tmp[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < N * N; i += 32) {
        int b = i / N, a = i % N;
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < N; ++d) s += (T ? M[d][b] : M[b][d]) * tmp[d * N + a];
        out[i] = scale * s;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// bathymetry sampling sites
// ---------------------------------------------------------------------------
template <int R, typename Pix, int MODE>
struct Site {
    using S = Sz<R>;
    static __device__ __forceinline__ int offset(int set) {
        return set == SET_VOL ? 0 : (set == SET_MASS ? S::NVP : S::NVP + S::NMP);
    }
    static __device__ __forceinline__ int count(int set) {
        return set == SET_VOL ? S::NV : (set == SET_MASS ? S::NM : S::NG);
    }
    static __device__ __forceinline__ const OvTab& tab(const Dev& d, int64_t k) {
        return d.ov[d.pcls ? d.pcls[k] : 0];
    }
    static __device__ __forceinline__ const Pix* tile(const Dev& d, const OvTab& o, int64_t k) {
        return (const Pix*)d.tiles + (d.tile_off ? d.tile_off[k] : (int64_t)k * o.P * o.P);
    }
    // mode S: a cell entirely wet (eta > -min z_b) gives V = eta + the sub-cell
    // mean depth and A = 1; entirely dry (eta <= -max z_b) gives V = A = 0;
    // otherwise the pixels are summed.  The per-cell bounds are optional (the
    // allocation-free residual has none): without them every sub-cell sums.
    static __device__ __forceinline__ bool shortcut(const Dev& d, int64_t k, double eta,
                                                    double zbar, double& V, double& A, bool& full) {
        if (d.zmin == nullptr) return false;
        if (eta > -d.zmin[k]) {
            V = eta + zbar;
            A = 1.0;
            full = true;
            return true;
        }
        if (!(eta > -d.zmax[k])) {
            V = 0.0;
            A = 0.0;
            full = false;
            return true;
        }
        return false;
    }
    // V, A of sub-cell (ia, ib) of point set `set` of cell k at elevation eta,
    // and whether every pixel of it is wet
    static __device__ __forceinline__ void VA(const Dev& d, const Tables& tb, int64_t k, int set,
                                              int ia, int ib, double eta, double& V, double& A,
                                              bool& full) {
        if (MODE == 0) {
            if (d.zmin != nullptr &&
                shortcut(d, k, eta, d.zpts[(size_t)k * S::NZP + offset(set) + ia + count(set) * ib],
                         V, A, full))
                return;
            const OvTab& o = tab(d, k);
            subgrid_S<Pix>(tile(d, o, k), o, set, ia, set, ib, eta, V, A, full);
        } else {
            subgrid_P(d.zpts[(size_t)k * S::NZP + offset(set) + ia + count(set) * ib], eta, V, A);
            full = A > 0.0;
        }
    }
    static __device__ __forceinline__ void VA(const Dev& d, const Tables& tb, int64_t k, int set,
                                              int ia, int ib, double eta, double& V, double& A) {
        bool full;
        VA(d, tb, k, set, ia, ib, eta, V, A, full);
    }
    // the strip of the coarse cell k on its face f under GLL point al of the
    // fine half face h (a 2:1 face): normal extent = its first/last mass
    // sub-interval, tangential extent = the fine point's sub-interval
    static __device__ __forceinline__ void VA_half(const Dev& d, int64_t k, int f, int h, int al,
                                                   double eta, double& V, double& A) {
        const double zh = d.zhang[(((size_t)k * 4 + f) * 2 + h) * S::NM + al];
        if (MODE == 0) {
            bool full;
            if (shortcut(d, k, eta, zh, V, A, full)) return;
            const OvTab& o = tab(d, k);
            const int m = (f == 0 || f == 2) ? 0 : S::NM - 1;
            if (f < 2)
                subgrid_S<Pix>(tile(d, o, k), o, SET_MASS, m, SET_HALF, h * S::NM + al, eta, V, A,
                               full);
            else
                subgrid_S<Pix>(tile(d, o, k), o, SET_HALF, h * S::NM + al, SET_MASS, m, eta, V, A,
                               full);
        } else {
            subgrid_P(zh, eta, V, A);
        }
    }
};

// mass-point index of the strip of face f at face point al
template <int NM>
__device__ __forceinline__ void face_site_index(int f, int al, int& ia, int& ib) {
    if (f == 0) { ia = 0; ib = al; }
    else if (f == 1) { ia = NM - 1; ib = al; }
    else if (f == 2) { ia = al; ib = 0; }
    else { ia = al; ib = NM - 1; }
}
// node index (a + ND1 b) of the j-th node along face f
template <int ND1>
__device__ __forceinline__ int face_node(int f, int j) {
    if (f == 0) return ND1 * j;
    if (f == 1) return (ND1 - 1) + ND1 * j;
    if (f == 2) return j;
    return j + ND1 * (ND1 - 1);
}

// the four fields of a cell at face point al of face f: sum_j B[al][j] u(node(f, j));
// fields are fstride apart; a field constant on the cell is that constant
template <int ND1>
__device__ __forceinline__ void face_trace(const double* u, size_t fstride, unsigned cm, int f,
                                           const double (*B)[MXN], int al, double t[4]) {
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
        const double* uf = u + fl * fstride;
        if (cm & (1u << fl)) {
            t[fl] = uf[0];
            continue;
        }
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < ND1; ++j) s += B[al][j] * uf[face_node<ND1>(f, j)];
        t[fl] = s;
    }
}

// Rusanov flux with hydrostatic reconstruction at one face point, seen from
// side A with outward normal (nx, ny) (Eqs. lxf_parameter, velocity,
// hydro_rec_vars, mass_rhs, discharge_rhs, r_concentration).  hA = V_A(zeta_A),
// hsA = min(V_A(zeta_A), V_B(zeta_A)).  out = {F, Gx_cons, Gy_cons, R}; the
// non-conservative pressure scalar g {{h*}} (h*A - h*B)/2 is returned apart.
__device__ __forceinline__ void rusanov(double qxA, double qyA, double cA, double hA, double hsA,
                                        double qxB, double qyB, double cB, double hB, double hsB,
                                        double nx, double ny, double g, double eps, double out[4],
                                        double& pres, double& lam) {
    double fA = vel_factor(hA, eps), fB = vel_factor(hB, eps);
    double uAx = fA * qxA, uAy = fA * qyA, uBx = fB * qxB, uBy = fB * qyB;
    double unA = uAx * nx + uAy * ny, unB = uBx * nx + uBy * ny;
    double l = fmax(fabs(unA) + sqrt(g * hA), fabs(unB) + sqrt(g * hB));
    double qsAx = hsA * uAx, qsAy = hsA * uAy, qsBx = hsB * uBx, qsBy = hsB * uBy;
    out[0] = 0.5 * ((qsAx + qsBx) * nx + (qsAy + qsBy) * ny) + 0.5 * l * (hsA - hsB);
    out[1] = 0.5 * (qsAx * unA + qsBx * unB) + 0.5 * l * (qsAx - qsBx);
    out[2] = 0.5 * (qsAy * unA + qsBy * unB) + 0.5 * l * (qsAy - qsBy);
    out[3] = 0.5 * ((qsAx * cA + qsBx * cB) * nx + (qsAy * cA + qsBy * cB) * ny) +
             0.5 * l * (hsA * cA - hsB * cB);
    pres = g * 0.5 * (hsA + hsB) * 0.5 * (hsA - hsB);
    lam = l;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// residual: volume terms on the volume Gauss-Legendre points, face terms on
// r+2 Gauss-Lobatto points per face (Eqs. mass_rhs, discharge_rhs,
// discharge_rhs_implicit, r_concentration)
// ---------------------------------------------------------------------------
template <int R>
constexpr int res_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 5 * S::ND1 * S::NV + 6 * S::NVP + 12 * S::NVP + 12 * S::NV * S::ND1 +
           32 * S::NM + 6 * S::ND;
}

template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(TPB)
    k_residual(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int buf,
               int stage, double c_stage, int want_dt) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NV = S::NV, NVP = S::NVP, NM = S::NM;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* su = smem + warp * res_smem<R>();
    double* tx = su + 4 * ND;        // [5][ND1][NV]
    double* pv = tx + 5 * ND1 * NV;  // unused slot kept for alignment of later arrays
    double* X = pv + 6 * NVP;        // [12][NVP]
    double* sy = X + 12 * NVP;       // [12][NV][ND1]
    double* fh = sy + 12 * NV * ND1; // [4 fields][4 faces][2 halves][NM]
    double* rs = fh + 32 * NM;       // [6][ND]
    const double g = d.g, eps = d.eps;
    const double t = (c_stage == 0.0) ? d.sc->t : d.sc->t + c_stage * get_dt(d);
    const int64_t n = d.n;

    for (int64_t k = (int64_t)blockIdx.x * WPB + warp; k < n; k += (int64_t)gridDim.x * WPB) {
        for (int i = lane; i < 4 * ND; i += 32)
            su[i] = ufield(d, buf, i / ND, ND)[k * ND + (i % ND)];
        const unsigned cm = d.cmask[(size_t)buf * n + k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double ihx = d.ihxhy ? d.ihxhy[2 * k] : 1.0 / hx;
        const double ihy = d.ihxhy ? d.ihxhy[2 * k + 1] : 1.0 / hy;
        const double man = d.manning[k];
        __syncwarp();
        // x-contraction of the four fields (values) and of zeta (d/dxi)
        for (int i = lane; i < 5 * ND1 * NV; i += 32) {
            int f = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
            const double* u = su + (f < 4 ? f : 0) * ND + ND1 * b;
            double s = 0.0;
            if (f < 4) {
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += tb.Bv[al][a] * u[a];
            } else {
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += tb.Dv[al][a] * u[a];
            }
            tx[i] = s;
        }
        __syncwarp();
        // y-contraction and pointwise physics, one volume point per lane
        for (int p = lane; p < NVP; p += 32) {
            const int al = p % NV, be = p / NV;
            double z = 0, zx = 0, zy = 0, qx = 0, qy = 0, c = 0;
#pragma unroll
            for (int b = 0; b < ND1; ++b) {
                const double B = tb.Bv[be][b], D = tb.Dv[be][b];
                z += B * tx[(0 * ND1 + b) * NV + al];
                qx += B * tx[(1 * ND1 + b) * NV + al];
                qy += B * tx[(2 * ND1 + b) * NV + al];
                c += B * tx[(3 * ND1 + b) * NV + al];
                zx += B * tx[(4 * ND1 + b) * NV + al];
                zy += D * tx[(0 * ND1 + b) * NV + al];
            }
            if (cm & 1u) { z = su[0]; zx = 0.0; zy = 0.0; }
            if (cm & 2u) qx = su[ND];
            if (cm & 4u) qy = su[2 * ND];
            if (cm & 8u) c = su[3 * ND];
            zx *= ihx;
            zy *= ihy;
            double h, A;
            ST::VA(d, tb, k, SET_VOL, al, be, z, h, A);
            const double fv = vel_factor(h, eps);
            const double ux = fv * qx, uy = fv * qy;
            const double gam = gamma_manning(man, h, qx, qy, g, eps);
            const double w = J * tb.wv[al] * tb.wv[be], wx = w * ihx, wy = w * ihy;
            X[0 * NVP + p] = wx * qx;
            X[1 * NVP + p] = wy * qy;
            X[2 * NVP + p] = wx * qx * ux;
            X[3 * NVP + p] = wy * qx * uy;
            X[4 * NVP + p] = -w * g * h * zx;
            X[5 * NVP + p] = wx * qy * ux;
            X[6 * NVP + p] = wy * qy * uy;
            X[7 * NVP + p] = -w * g * h * zy;
            X[8 * NVP + p] = wx * c * qx;
            X[9 * NVP + p] = wy * c * qy;
            X[10 * NVP + p] = -w * gam * qx;
            X[11 * NVP + p] = -w * gam * qy;
        }
        __syncwarp();
        // test integration, y-contraction: sy[c][0: grad-x part, 1: rest][al][b]
        // fields: F (0,1,-), Gx (2,3,4), Gy (5,6,7), R (8,9,-), Lx (-,-,10), Ly (-,-,11)
        for (int i = lane; i < 6 * NV * ND1; i += 32) {
            const int cf = i / (NV * ND1), r_ = i % (NV * ND1), al = r_ / ND1, b = r_ % ND1;
            const int ix = cf == 0 ? 0 : cf == 1 ? 2 : cf == 2 ? 5 : cf == 3 ? 8 : -1;
            const int iy = cf == 0 ? 1 : cf == 1 ? 3 : cf == 2 ? 6 : cf == 3 ? 9 : -1;
            const int iv = cf == 1 ? 4 : cf == 2 ? 7 : cf == 4 ? 10 : cf == 5 ? 11 : -1;
            double sx = 0.0, so = 0.0;
#pragma unroll
            for (int be = 0; be < NV; ++be) {
                const int p = al + NV * be;
                if (ix >= 0) sx += tb.Bv[be][b] * X[ix * NVP + p];
                if (iy >= 0) so += tb.Dv[be][b] * X[iy * NVP + p];
                if (iv >= 0) so += tb.Bv[be][b] * X[iv * NVP + p];
            }
            sy[((cf * 2 + 0) * NV + al) * ND1 + b] = sx;
            sy[((cf * 2 + 1) * NV + al) * ND1 + b] = so;
        }
        __syncwarp();
        for (int i = lane; i < 6 * ND; i += 32) {
            const int cf = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
            double s = 0.0;
#pragma unroll
            for (int al = 0; al < NV; ++al)
                s += tb.Dv[al][a] * sy[((cf * 2 + 0) * NV + al) * ND1 + b] +
                     tb.Bv[al][a] * sy[((cf * 2 + 1) * NV + al) * ND1 + b];
            rs[i] = s;
        }
        // faces: one (sub)face point per lane; a coarse cell integrates each
        // 2:1 face over the GLL points of both fine halves
        double dtl = 0.0;
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
            double tm[4];
            face_trace<ND1>(su, ND, cm, f, coarse ? tb.BmH[h] : tb.Bm, al, tm);
            int ia, ib;
            face_site_index<NM>(f, al, ia, ib);
            auto own_V = [&](double eta) {
                double V, A;
                if (coarse) ST::VA_half(d, k, f, h, al, eta, V, A);
                else ST::VA(d, tb, k, SET_MASS, ia, ib, eta, V, A);
                return V;
            };
            const int32_t s0 = d.nbr[k * 8 + f * 2];
            const double hm = own_V(tm[0]);
            double tp[4], hp, hsm, hsp, out[4], pres, lam;
            if (s0 >= 0) {
                const int64_t nb = coarse ? (int64_t)(h ? d.nbr[k * 8 + f * 2 + 1] : s0) : (int64_t)s0;
                const int fo = f ^ 1;
                face_trace<ND1>(ufield(d, buf, 0, ND) + nb * ND, (size_t)n * ND,
                                d.cmask[(size_t)buf * n + nb], fo, fine ? tb.BmH[half] : tb.Bm, al, tp);
                int ja, jb;
                face_site_index<NM>(fo, al, ja, jb);
                auto nb_V = [&](double eta) {
                    double V, A;
                    if (fine) ST::VA_half(d, nb, fo, half, al, eta, V, A);
                    else ST::VA(d, tb, nb, SET_MASS, ja, jb, eta, V, A);
                    return V;
                };
                hp = nb_V(tp[0]);
                hsm = fmin(hm, nb_V(tm[0]));  // min(V-(zeta-), V+(zeta-))
                hsp = fmin(hp, own_V(tp[0])); // min(V+(zeta+), V-(zeta+))
                // canonical side order: the lower cell index is side A, so both
                // cells of the face compute bit-identical fluxes
                const bool own_first = k < nb;
                if (own_first)
                    rusanov(tm[1], tm[2], tm[3], hm, hsm, tp[1], tp[2], tp[3], hp, hsp, nx, ny, g, eps,
                            out, pres, lam);
                else
                    rusanov(tp[1], tp[2], tp[3], hp, hsp, tm[1], tm[2], tm[3], hm, hsm, -nx, -ny, g,
                            eps, out, pres, lam);
                const double sg = own_first ? 1.0 : -1.0;
                // the pressure vector g {{h*}} (h*A - h*B)/2 n_A is the same for both sides
                const double pnx = own_first ? pres * nx : pres * (-nx);
                const double pny = own_first ? pres * ny : pres * (-ny);
                out[0] *= sg;
                out[1] = sg * out[1] - pnx;
                out[2] = sg * out[2] - pny;
                out[3] *= sg;
            } else {
                const int tag = -1 - s0;
                tp[0] = tm[0]; tp[1] = tm[1]; tp[2] = tm[2]; tp[3] = tm[3];
                if (d.bc_kind[tag] == 1) {
                    tp[0] = d.bc_amp[tag] * sin(2.0 * M_PI * t / d.bc_per[tag] + d.bc_ph[tag]);
                } else {
                    const double qn = tm[1] * nx + tm[2] * ny;
                    tp[1] = tm[1] - 2.0 * qn * nx;
                    tp[2] = tm[2] - 2.0 * qn * ny;
                }
                hp = own_V(tp[0]); // ghost: same sub-grid operator
                hsm = hm;
                hsp = hp;
                rusanov(tm[1], tm[2], tm[3], hm, hsm, tp[1], tp[2], tp[3], hp, hsp, nx, ny, g, eps, out,
                        pres, lam);
                out[1] -= pres * nx;
                out[2] -= pres * ny;
            }
            const double wl = L * tb.wm[al];
#pragma unroll
            for (int cf = 0; cf < 4; ++cf) fh[((cf * 4 + f) * 2 + h) * NM + al] = wl * out[cf];
            // lambda l / J for the positivity step (l = L, J = hx hy)
            dtl = fmax(dtl, fmax(lam, 1e-12) * ((f < 2) ? ihx : ihy) * (coarse ? 0.5 : 1.0));
        }
        if (want_dt) {
            const double m = warp_max(dtl);
            if (lane == 0) atomic_max_pos(&d.sc->rmax, m);
        }
        __syncwarp();
        // lift the face fluxes onto the nodes of each face
        for (int i = lane; i < 4 * ND; i += 32) {
            const int cf = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
            double s = 0.0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const bool on = (f == 0 && a == 0) || (f == 1 && a == ND1 - 1) || (f == 2 && b == 0) ||
                                (f == 3 && b == ND1 - 1);
                if (!on) continue;
                const int tn = f < 2 ? b : a; // tangential node index along the face
                const double* fp = fh + (cf * 4 + f) * 2 * NM;
                if ((fi[f] & 3) == FI_COARSE) {
                    for (int al = 0; al < NM; ++al)
                        s += tb.BmH[0][al][tn] * fp[al] + tb.BmH[1][al][tn] * fp[NM + al];
                } else {
                    for (int al = 0; al < NM; ++al) s += tb.Bm[al][tn] * fp[al];
                }
            }
            rs[cf * ND + j] -= s;
        }
        __syncwarp();
        for (int i = lane; i < 6 * ND; i += 32)
            rfield(d, stage, i / ND, ND)[k * ND + (i % ND)] = rs[i];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// warp-cooperative scalar Newton for Hbar(e) = target (r_K = 0 cells,
// Eqs. newton, initial_guess); returns iterations
// ---------------------------------------------------------------------------
template <int R, typename Pix, int MODE>
__device__ __forceinline__ void mass_scalar(const Dev& d, const Tables& tb, int64_t k, double J,
                                            double e, int lane, double& H, double& A) {
    using S = Sz<R>;
    double h = 0.0, a = 0.0;
    for (int p = lane; p < S::NMP; p += 32) {
        const int ia = p % S::NM, ib = p / S::NM;
        double V, Ap;
        Site<R, Pix, MODE>::VA(d, tb, k, SET_MASS, ia, ib, e, V, Ap);
        const double w = J * tb.wm[ia] * tb.wm[ib];
        h += w * V;
        a += w * Ap;
    }
    H = warp_sum(h);
    A = warp_sum(a);
}

template <int R, typename Pix, int MODE>
__device__ int scalar_newton(const Dev& d, const Tables& tb, int64_t k, double J, double target,
                             double& e, int lane) {
    constexpr int ND = Sz<R>::ND;
    double H, A;
    mass_scalar<R, Pix, MODE>(d, tb, k, J, e, lane, H, A);
    if (A == 0.0) e = -d.zmax[k] + d.eps0;
    int it = 0;
    for (int kk = 0; kk < d.newton_max; ++kk) {
        mass_scalar<R, Pix, MODE>(d, tb, k, J, e, lane, H, A);
        if (A == 0.0) break;
        const double dd = (H - target) / A;
        e -= dd;
        ++it;
        if (ND * fabs(dd) <= d.newton_tol * (ND * (1.0 + fabs(e) + d.zabs[k]))) break;
    }
    return it;
}

// ---------------------------------------------------------------------------
// step start: degree switch (Eq. criteria_p) with mass-exact remap, then
// H_i(zeta^n), C~_i^n (Eqs. depth_rhs, concentration_rhs) and their sums
// ---------------------------------------------------------------------------
template <int R>
constexpr int begin_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 4 * S::NMP + 2 * S::NM * S::NM + 3 * S::NGP + 2 * S::ND;
}

template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(TPB)
    k_step_begin(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int do_switch) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* su = smem + warp * begin_smem<R>();
    double* pe = su + 4 * ND;    // [NMP] zeta at mass points
    double* pc = pe + NMP;       // [NMP] c at mass points
    double* pV = pc + NMP;       // [NMP]
    double* px = pV + NMP;       // [NMP] scratch products
    double* tmp = px + NMP;      // [2 NM NM]
    double* pg = tmp + 2 * NM * NM; // [3][NGP]
    double* out = pg + 3 * NGP;  // [2][ND]
    const int64_t n = d.n;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.sc->rmax = 0ull;
        d.sc->maxits = 0;
    }
    for (int64_t k = (int64_t)blockIdx.x * WPB + warp; k < n; k += (int64_t)gridDim.x * WPB) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        unsigned cm = d.cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        __syncwarp();
        // zeta and c at the mass points
        tens_interp<ND1, NM>(tb.Bm, su, tmp, pe, lane);
        tens_interp<ND1, NM>(tb.Bm, su + 3 * ND, tmp, pc, lane);
        for (int p = lane; p < NMP; p += 32) {
            if (cm & 1u) pe[p] = su[0];
            if (cm & 8u) pc[p] = su[3 * ND];
            double V, A;
            ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pe[p], V, A);
            pV[p] = V;
        }
        __syncwarp();
        double mu = INFINITY;
        for (int p = lane; p < NMP; p += 32) mu = fmin(mu, pV[p]);
        mu = warp_min(mu);
        const int flag = (do_switch && !(mu > d.hlim)) ? 0 : R;
        if (flag == 0) {
            // remap to r_K = 0: mass-exact zeta, GL means of q, tracer-mass-exact c
            double m = 0.0, tr = 0.0;
            for (int p = lane; p < NMP; p += 32) {
                const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
                m += w * pV[p];
                tr += w * pV[p] * pc[p];
            }
            m = warp_sum(m);
            tr = warp_sum(tr);
            for (int f = 0; f < 3; ++f) {
                tens_interp<ND1, NG>(tb.Bg, su + (1 + f) * ND, tmp, pg + f * NGP, lane);
            }
            double mq[3] = {0.0, 0.0, 0.0};
            for (int p = lane; p < NGP; p += 32) {
                const double w = tb.wg[p % NG] * tb.wg[p / NG];
                for (int f = 0; f < 3; ++f) {
                    const double v = (cm & (2u << f)) ? su[(1 + f) * ND] : pg[f * NGP + p];
                    mq[f] += w * v;
                }
            }
            for (int f = 0; f < 3; ++f) mq[f] = warp_sum(mq[f]);
            const double cnew = (m > 1e-14 * J * d.hlim) ? tr / m : mq[2];
            double emax = -INFINITY;
            for (int p = lane; p < NMP; p += 32) emax = fmax(emax, pe[p]);
            emax = warp_max(emax);
            __syncwarp();
            if (!(cm & 8u))
                for (int i = lane; i < ND; i += 32) su[3 * ND + i] = cnew;
            if (!(cm & 2u))
                for (int i = lane; i < ND; i += 32) su[ND + i] = mq[0];
            if (!(cm & 4u))
                for (int i = lane; i < ND; i += 32) su[2 * ND + i] = mq[1];
            if (!(cm & 1u)) {
                double e;
                if (m <= 0.0) e = -d.zmax[k];
                else {
                    e = emax;
                    scalar_newton<R, Pix, MODE>(d, tb, k, J, m, e, lane);
                }
                for (int i = lane; i < ND; i += 32) su[i] = e;
            }
            __syncwarp();
            for (int i = lane; i < 4 * ND; i += 32) ufield(d, 0, i / ND, ND)[k * ND + (i % ND)] = su[i];
            cm = 15u;
            for (int p = lane; p < NMP; p += 32) {
                pe[p] = su[0];
                pc[p] = su[3 * ND];
                double V, A;
                ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pe[p], V, A);
                pV[p] = V;
            }
            __syncwarp();
        }
        // H_i(zeta^n), C~_i^n and their sums
        double hb = 0.0, cb = 0.0;
        for (int p = lane; p < NMP; p += 32) {
            const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
            hb += w * pV[p];
            cb += w * pV[p] * pc[p];
            px[p] = w * pV[p];
        }
        hb = warp_sum(hb);
        cb = warp_sum(cb);
        __syncwarp();
        tens_test<ND1, NM>(tb.Bm, px, tmp, out, lane);
        for (int p = lane; p < NMP; p += 32) px[p] *= pc[p];
        __syncwarp();
        tens_test<ND1, NM>(tb.Bm, px, tmp, out + ND, lane);
        for (int i = lane; i < ND; i += 32) {
            d.HN[k * ND + i] = out[i];
            d.CN[k * ND + i] = out[ND + i];
        }
        if (lane == 0) {
            d.HNbar[k] = hb;
            d.CNbar[k] = cb;
            d.flag[k] = (uint8_t)flag;
            d.cmask[k] = (uint8_t)cm;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// stage update for one cell: continuity Newton (Eq. newton, Eq. mass_matrix),
// momentum with the friction-modified mass matrix (Eq. mass_matrix_discharge)
// inverted as S^-1 D^-1 S^-T (Sec. 3.3), tracer with the depth-weighted mass
// matrix (Eq. mass_matrix_concentration) by Cholesky
// ---------------------------------------------------------------------------
struct StageArgs {
    int out_buf;   // state buffer written
    int prev_buf;  // state buffer of stage l-1 (friction coefficient)
    int nres;      // residual stages summed
    double wa[MXS], wat[MXS];
    double add;    // implicit diagonal a~_ll
    int use_llin;  // final: the last stage enters with its linearised friction term
    int make_llin; // this stage is the last one and implicit: store Llin
    int final_;    // final combination: update time and bookkeeping
};

template <int R>
constexpr int stage_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 5 * S::ND + 3 * S::NMP + 2 * S::NM * S::NM + S::ND1 * S::ND1 * S::NM +
           S::ND * S::ND + 6 * S::NGP + 4 * S::ND + S::ND +
           // mixed-precision solve: x, r (ND), q (NMP), float M, Y, inv, r
           2 * S::ND + S::NMP + (S::ND * S::ND + S::ND1 * S::ND1 * S::NM + 2 * S::ND + 1) / 2 + 1;
}

// Cholesky of the SPD matrix M (ND x ND, row-major, lower part used) on a
// warp, then M x = b in place by column-oriented forward and back
// substitution (one reciprocal per column, the updates spread over lanes);
// returns false on a non-positive pivot
template <int ND>
__device__ bool chol_solve(double* M, double* b, double* inv, int lane) {
    for (int j = 0; j < ND; ++j) {
        __syncwarp();
        const double djj = M[j * ND + j];
        if (!(djj > 0.0)) return false;
        const double ljj = sqrt(djj);
        const double r = 1.0 / ljj;
        __syncwarp();
        for (int i = j + 1 + lane; i < ND; i += 32) M[i * ND + j] *= r;
        if (lane == 0) {
            M[j * ND + j] = ljj;
            inv[j] = r;
        }
        __syncwarp();
        const int m = ND - j - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int i = j + 1 + idx / m, l = j + 1 + idx % m;
            if (l <= i) M[i * ND + l] -= M[i * ND + j] * M[l * ND + j];
        }
    }
    __syncwarp();
    for (int j = 0; j < ND; ++j) { // L y = b
        const double yj = b[j] * inv[j];
        __syncwarp();
        for (int i = j + 1 + lane; i < ND; i += 32) b[i] -= M[i * ND + j] * yj;
        if (lane == 0) b[j] = yj;
        __syncwarp();
    }
    for (int j = ND - 1; j >= 0; --j) { // L^T x = y
        const double xj = b[j] * inv[j];
        __syncwarp();
        for (int i = lane; i < j; i += 32) b[i] -= M[j * ND + i] * xj;
        if (lane == 0) b[j] = xj;
        __syncwarp();
    }
    return true;
}

// FP32 Cholesky factorisation (lower part of M, reciprocal pivots in inv);
// returns false on a non-positive pivot
template <int ND>
__device__ bool chol_factor_f(float* M, float* inv, int lane) {
    for (int j = 0; j < ND; ++j) {
        __syncwarp();
        const float djj = M[j * ND + j];
        if (!(djj > 0.0f)) return false;
        const float ljj = sqrtf(djj);
        const float r = 1.0f / ljj;
        __syncwarp();
        for (int i = j + 1 + lane; i < ND; i += 32) M[i * ND + j] *= r;
        if (lane == 0) {
            M[j * ND + j] = ljj;
            inv[j] = r;
        }
        __syncwarp();
        const int m = ND - j - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int i = j + 1 + idx / m, l = j + 1 + idx % m;
            if (l <= i) M[i * ND + l] -= M[i * ND + j] * M[l * ND + j];
        }
    }
    __syncwarp();
    return true;
}

// (L L^T)^-1 b in FP32 with the factor of chol_factor_f, in place
template <int ND>
__device__ void chol_subst_f(const float* M, const float* inv, float* b, int lane) {
    for (int j = 0; j < ND; ++j) {
        const float yj = b[j] * inv[j];
        __syncwarp();
        for (int i = j + 1 + lane; i < ND; i += 32) b[i] -= M[i * ND + j] * yj;
        if (lane == 0) b[j] = yj;
        __syncwarp();
    }
    for (int j = ND - 1; j >= 0; --j) {
        const float xj = b[j] * inv[j];
        __syncwarp();
        for (int i = lane; i < j; i += 32) b[i] -= M[j * ND + i] * xj;
        if (lane == 0) b[j] = xj;
        __syncwarp();
    }
}

// FP32 copy of M_(a,b),(c,d) = sum c_{al,be} Bm[al][a] Bm[al][c] Bm[be][b] Bm[be][d]
template <int ND1, int NM>
__device__ __forceinline__ void assemble_mass_f(const Tables& tb, const double* cw, float* Y,
                                                float* M, int lane) {
    constexpr int ND = ND1 * ND1;
    for (int i = lane; i < ND1 * ND1 * NM; i += 32) {
        const int a = i / (ND1 * NM), r_ = i % (ND1 * NM), c = r_ / NM, be = r_ % NM;
        float s = 0.0f;
#pragma unroll
        for (int al = 0; al < NM; ++al)
            s += (float)cw[al + NM * be] * (float)tb.Bm[al][a] * (float)tb.Bm[al][c];
        Y[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < ND * ND; i += 32) {
        const int r_ = i / ND, s_ = i % ND;
        const int a = r_ % ND1, b = r_ / ND1, c = s_ % ND1, dd = s_ / ND1;
        float s = 0.0f;
#pragma unroll
        for (int be = 0; be < NM; ++be)
            s += Y[(a * ND1 + c) * NM + be] * (float)tb.Bm[be][b] * (float)tb.Bm[be][dd];
        M[i] = s;
    }
    __syncwarp();
}

// M_(a,b),(c,d) = sum_{al,be} c_{al,be} Bm[al][a] Bm[al][c] Bm[be][b] Bm[be][d]
template <int ND1, int NM>
__device__ __forceinline__ void assemble_mass(const Tables& tb, const double* cw, double* Y,
                                              double* M, int lane) {
    constexpr int ND = ND1 * ND1;
    for (int i = lane; i < ND1 * ND1 * NM; i += 32) {
        const int a = i / (ND1 * NM), r_ = i % (ND1 * NM), c = r_ / NM, be = r_ % NM;
        double s = 0.0;
#pragma unroll
        for (int al = 0; al < NM; ++al) s += cw[al + NM * be] * tb.Bm[al][a] * tb.Bm[al][c];
        Y[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < ND * ND; i += 32) {
        const int r_ = i / ND, s_ = i % ND;
        const int a = r_ % ND1, b = r_ / ND1, c = s_ % ND1, dd = s_ / ND1;
        double s = 0.0;
#pragma unroll
        for (int be = 0; be < NM; ++be)
            s += Y[(a * ND1 + c) * NM + be] * tb.Bm[be][b] * tb.Bm[be][dd];
        M[i] = s;
    }
    __syncwarp();
}

// Solve H x = b for the depth-weighted mass matrix H = B^T diag(cw) B (the
// tracer matrix of Eq. mass_matrix_concentration, or the masked Jacobian of
// Eq. mass_matrix) by mixed-precision iterative refinement: H is assembled and
// factored in FP32, each correction is solved in FP32, and the residual
// b - H x is formed in FP64 matrix-free by sum factorisation.  If the
// corrections do not fall below 1e-15 of x within 6 sweeps (an ill-conditioned
// near-dry cell), the FP64 Cholesky decides.  x (FP64, in place of b on
// return).  Scratch: Mf, Yf (float), r, t (ND doubles), q (NMP doubles),
// tmp (2 NM NM doubles), M, Y (double, fallback).
template <int ND1, int NM>
__device__ bool solve_mass_mixed(const Tables& tb, const double* cw, double* b, float* Mf,
                                 float* Yf, float* invf, float* rf, double* x, double* r,
                                 double* q, double* tmp, double* M, double* Y, double* inv,
                                 int lane) {
    constexpr int ND = ND1 * ND1, NMP = NM * NM;
    assemble_mass_f<ND1, NM>(tb, cw, Yf, Mf, lane);
    bool ok = chol_factor_f<ND>(Mf, invf, lane);
    if (ok) {
        for (int i = lane; i < ND; i += 32) {
            x[i] = 0.0;
            r[i] = b[i];
        }
        __syncwarp();
        ok = false;
        for (int sweep = 0; sweep < 6; ++sweep) {
            for (int i = lane; i < ND; i += 32) rf[i] = (float)r[i];
            __syncwarp();
            chol_subst_f<ND>(Mf, invf, rf, lane);
            double dmax = 0.0, xmax = 0.0;
            for (int i = lane; i < ND; i += 32) {
                x[i] += (double)rf[i];
                dmax = fmax(dmax, fabs((double)rf[i]));
                xmax = fmax(xmax, fabs(x[i]));
            }
            dmax = warp_max(dmax);
            xmax = warp_max(xmax);
            if (!(dmax <= 1e-15 * xmax) && !(dmax == 0.0)) {
                // r = b - H x, H x = B^T (cw * (B x))
                __syncwarp();
                tens_interp<ND1, NM>(tb.Bm, x, tmp, q, lane);
                for (int p = lane; p < NMP; p += 32) q[p] *= cw[p];
                __syncwarp();
                tens_test<ND1, NM>(tb.Bm, q, tmp, r, lane);
                for (int i = lane; i < ND; i += 32) r[i] = b[i] - r[i];
                __syncwarp();
            } else {
                ok = true;
                break;
            }
        }
    }
    if (ok) {
        for (int i = lane; i < ND; i += 32) b[i] = x[i];
        __syncwarp();
        return true;
    }
    assemble_mass<ND1, NM>(tb, cw, Y, M, lane);
    return chol_solve<ND>(M, b, inv, lane);
}

template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(TPB)
    k_stage(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, const StageArgs sa) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* su = smem + warp * stage_smem<R>(); // [4][ND] state v^n
    double* T = su + 4 * ND;                    // [ND]
    double* rq = T + ND;                        // [2][ND]
    double* rc = rq + 2 * ND;                   // [ND]
    double* z = rc + ND;                        // [ND] Newton iterate
    double* pe = z + ND;                        // [NMP]
    double* pV = pe + NMP;                      // [NMP]
    double* pA = pV + NMP;                      // [NMP]
    double* tmp = pA + NMP;                     // [2 NM NM]
    double* Y = tmp + 2 * NM * NM;              // [ND1 ND1 NM]
    double* M = Y + ND1 * ND1 * NM;             // [ND ND]
    double* pg = M + ND * ND;                   // [6][NGP]
    double* o = pg + 6 * NGP;                   // [4][ND]
    double* pinv = o + 4 * ND;                  // [ND] reciprocal Cholesky pivots
    double* xs = pinv + ND;                     // [ND] refinement iterate
    double* rs = xs + ND;                       // [ND] refinement residual
    double* qs = rs + ND;                       // [NMP]
    float* Mf = (float*)(qs + NMP);             // [ND ND]
    float* Yf = Mf + ND * ND;                   // [ND1 ND1 NM]
    float* invf = Yf + ND1 * ND1 * NM;          // [ND]
    float* rf = invf + ND;                      // [ND]
    const int64_t n = d.n;
    const double dt = get_dt(d);
    const double g = d.g, eps = d.eps;
    int its_max = 0;
    int viol = 0, fb = 0, bad = 0;

    for (int64_t k = (int64_t)blockIdx.x * WPB + warp; k < n; k += (int64_t)gridDim.x * WPB) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        const unsigned cm0 = d.cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double man = d.manning[k];
        int flag = d.flag[k];
        // right-hand sides of Eqs. algebraic_elevation, algebraic_discharge, algebraic_concentration
        double tsum = 0.0;
        for (int i = lane; i < ND; i += 32) {
            double sf = 0.0, sgx = 0.0, sgy = 0.0, sr = 0.0;
            for (int m = 0; m < sa.nres; ++m) {
                const size_t idx = (size_t)k * ND + i;
                const bool lin = sa.use_llin && (m == sa.nres - 1);
                const double lx = lin ? d.llin[idx] : rfield(d, m, 4, ND)[idx];
                const double ly = lin ? d.llin[(size_t)n * ND + idx] : rfield(d, m, 5, ND)[idx];
                sf += sa.wa[m] * rfield(d, m, 0, ND)[idx];
                sgx += sa.wa[m] * rfield(d, m, 1, ND)[idx] + sa.wat[m] * lx;
                sgy += sa.wa[m] * rfield(d, m, 2, ND)[idx] + sa.wat[m] * ly;
                sr += sa.wa[m] * rfield(d, m, 3, ND)[idx];
            }
            T[i] = d.HN[k * ND + i] + dt * sf;
            tsum += dt * sf;
            rq[i] = dt * sgx;
            rq[ND + i] = dt * sgy;
            rc[i] = d.CN[k * ND + i] + dt * sr;
        }
        const double Tbar = d.HNbar[k] + warp_sum(tsum);
        if (Tbar < 0.0) viol++;
        bool scalar = (flag == 0);
        int its = 0;
        __syncwarp();
        if (!scalar) {
            for (int i = lane; i < ND; i += 32) z[i] = su[i];
            bool zc = (cm0 & 1u) != 0;
            bool prev_full = false;
            __syncwarp();
            // each pass evaluates V, A at the current iterate; the last pass is
            // the evaluation at the result (for the tracer matrix and the
            // completely-dry test)
            for (int kk = 0;; ++kk) {
                tens_interp<ND1, NM>(tb.Bm, z, tmp, pe, lane);
                int ndry = 0, npart = 0;
                for (int p = lane; p < NMP; p += 32) {
                    if (zc) pe[p] = z[0];
                    double V, A;
                    bool full;
                    ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pe[p], V, A, full);
                    pV[p] = J * tb.wm[p % NM] * tb.wm[p / NM] * V;
                    pA[p] = J * tb.wm[p % NM] * tb.wm[p / NM] * A;
                    if (A == 0.0) ndry++;
                    else if (!full) npart++;
                }
                ndry = __reduce_add_sync(0xffffffffu, ndry);
                npart = __reduce_add_sync(0xffffffffu, npart);
                if (ndry) { scalar = true; break; }
                // every pixel wet at the previous and at this iterate: H is affine
                // on the segment between them and M(previous) is its exact
                // Jacobian, so this iterate solves H = T (the fully wet case of
                // Sec. 3.4); no verification step is needed
                if (kk > 0 && prev_full && npart == 0) break;
                if (kk == d.newton_max) break;
                __syncwarp();
                tens_test<ND1, NM>(tb.Bm, pV, tmp, o, lane); // H_i(zeta_k)
                for (int i = lane; i < ND; i += 32) o[i] -= T[i];
                __syncwarp();
                if (npart == 0) {
                    // M is the constant mass matrix, inverted by its tensor factors
                    kron_apply<ND1, false, MXN>(tb.M1inv, o, tmp, o + ND, 1.0 / J, lane);
                } else {
                    for (int i = lane; i < ND; i += 32) o[ND + i] = o[i];
                    __syncwarp();
                    if (!solve_mass_mixed<ND1, NM>(tb, pA, o + ND, Mf, Yf, invf, rf, xs, rs, qs, tmp, M,
                                                   Y, pinv, lane)) {
                        scalar = true;
                        break;
                    }
                }
                double inc = 0.0, scale = 0.0;
                for (int i = lane; i < ND; i += 32) {
                    z[i] -= o[ND + i];
                    inc += fabs(o[ND + i]);
                    scale += 1.0 + fabs(z[i]) + d.zabs[k];
                }
                inc = warp_sum(inc);
                scale = warp_sum(scale);
                its++;
                prev_full = (npart == 0);
                __syncwarp();
                {
                    bool eq = true;
                    for (int i = lane; i < ND; i += 32) eq = eq && (z[i] == z[0]);
                    zc = __all_sync(0xffffffffu, eq);
                }
                if (inc <= d.newton_tol * scale) prev_full = false, kk = d.newton_max - 1;
            }
            if (scalar) {
                fb++;
                flag = 0;
                if (lane == 0) d.flag[k] = 0;
            }
            __syncwarp();
        }
        // friction coefficient of the previous stage on the momentum GL points
        double* gam = pg + 5 * NGP;
        const bool need_gam = (sa.add != 0.0 || sa.make_llin) && man != 0.0;
        if (need_gam) {
            const unsigned cmp = d.cmask[(size_t)sa.prev_buf * n + k];
            for (int f = 0; f < 3; ++f) {
                const double* up = ufield(d, sa.prev_buf, f, ND) + k * ND;
                for (int i = lane; i < ND; i += 32) o[i] = up[i];
                __syncwarp();
                tens_interp<ND1, NG>(tb.Bg, o, tmp, pg + f * NGP, lane);
                if (cmp & (1u << f))
                    for (int p = lane; p < NGP; p += 32) pg[f * NGP + p] = o[0];
                __syncwarp();
            }
            for (int p = lane; p < NGP; p += 32) {
                double V, A;
                ST::VA(d, tb, k, SET_MOM, p % NG, p / NG, pg[p], V, A);
                gam[p] = gamma_manning(man, V, pg[NGP + p], pg[2 * NGP + p], g, eps);
            }
        } else {
            for (int p = lane; p < NGP; p += 32) gam[p] = 0.0;
        }
        __syncwarp();
        if (scalar) {
            double e;
            if (cm0 & 1u) e = su[0];
            else {
                tens_interp<ND1, NM>(tb.Bm, su, tmp, pe, lane);
                double s = 0.0;
                for (int p = lane; p < NMP; p += 32) s += tb.wm[p % NM] * tb.wm[p / NM] * pe[p];
                e = warp_sum(s);
            }
            its = scalar_newton<R, Pix, MODE>(d, tb, k, J, Tbar, e, lane);
            // momentum: sums of the rows of the friction-modified mass matrix
            double den = 0.0, num[2] = {0.0, 0.0};
            for (int f = 0; f < 2; ++f) {
                tens_interp<ND1, NG>(tb.Bg, su + (1 + f) * ND, tmp, pg + (3 + f) * NGP, lane);
                if (cm0 & (2u << f))
                    for (int p = lane; p < NGP; p += 32) pg[(3 + f) * NGP + p] = su[(1 + f) * ND];
                __syncwarp();
            }
            for (int p = lane; p < NGP; p += 32) {
                const double w = J * tb.wg[p % NG] * tb.wg[p / NG];
                den += w * (1.0 + sa.add * dt * gam[p]);
                num[0] += w * pg[3 * NGP + p];
                num[1] += w * pg[4 * NGP + p];
            }
            double rs0 = 0.0, rs1 = 0.0, rcs = 0.0;
            for (int i = lane; i < ND; i += 32) {
                rs0 += rq[i];
                rs1 += rq[ND + i];
                rcs += rc[i] - d.CN[k * ND + i];
            }
            den = warp_sum(den);
            const double qxn = (warp_sum(num[0]) + warp_sum(rs0)) / den;
            const double qyn = (warp_sum(num[1]) + warp_sum(rs1)) / den;
            rcs = warp_sum(rcs);
            double Hs, As;
            mass_scalar<R, Pix, MODE>(d, tb, k, J, e, lane, Hs, As);
            const bool tr_ok = Hs > 1e-14 * J * d.hlim;
            const double cn = tr_ok ? (d.CNbar[k] + rcs) / Hs : 0.0;
            for (int i = lane; i < ND; i += 32) {
                o[i] = e;
                o[ND + i] = qxn;
                o[2 * ND + i] = qyn;
                o[3 * ND + i] = tr_ok ? cn : su[3 * ND + i];
            }
            __syncwarp();
            if (sa.make_llin) {
                for (int p = lane; p < NGP; p += 32) {
                    const double w = J * tb.wg[p % NG] * tb.wg[p / NG] * gam[p];
                    pg[3 * NGP + p] = -w * qxn;
                    pg[4 * NGP + p] = -w * qyn;
                }
                __syncwarp();
                tens_test<ND1, NG>(tb.Bg, pg + 3 * NGP, tmp, M, lane);
                tens_test<ND1, NG>(tb.Bg, pg + 4 * NGP, tmp, M + ND, lane);
                for (int i = lane; i < ND; i += 32) {
                    d.llin[(size_t)k * ND + i] = M[i];
                    d.llin[(size_t)n * ND + (size_t)k * ND + i] = M[ND + i];
                }
            }
        } else {
            // momentum: point values on the GL (r+1)^2 points, S Q = [D0 q^n + S^-T rq] / D
            for (int f = 0; f < 2; ++f) {
                tens_interp<ND1, NG>(tb.Bg, su + (1 + f) * ND, tmp, pg + (3 + f) * NGP, lane);
                if (cm0 & (2u << f))
                    for (int p = lane; p < NGP; p += 32) pg[(3 + f) * NGP + p] = su[(1 + f) * ND];
                __syncwarp();
                kron_apply<ND1, true, MXP>(tb.Bginv, rq + f * ND, tmp, pg + f * NGP, 1.0, lane);
            }
            for (int p = lane; p < NGP; p += 32) {
                const double w = J * tb.wg[p % NG] * tb.wg[p / NG];
                const double D = w * (1.0 + sa.add * dt * gam[p]);
                pg[0 * NGP + p] = (w * pg[3 * NGP + p] + pg[0 * NGP + p]) / D;
                pg[1 * NGP + p] = (w * pg[4 * NGP + p] + pg[1 * NGP + p]) / D;
            }
            __syncwarp();
            kron_apply<ND1, false, MXP>(tb.Bginv, pg, tmp, o + ND, 1.0, lane);
            kron_apply<ND1, false, MXP>(tb.Bginv, pg + NGP, tmp, o + 2 * ND, 1.0, lane);
            if (sa.make_llin) {
                for (int p = lane; p < NGP; p += 32) {
                    const double w = J * tb.wg[p % NG] * tb.wg[p / NG] * gam[p];
                    pg[3 * NGP + p] = -w * pg[p];
                    pg[4 * NGP + p] = -w * pg[NGP + p];
                }
                __syncwarp();
                tens_test<ND1, NG>(tb.Bg, pg + 3 * NGP, tmp, M, lane);
                tens_test<ND1, NG>(tb.Bg, pg + 4 * NGP, tmp, M + ND, lane);
                for (int i = lane; i < ND; i += 32) {
                    d.llin[(size_t)k * ND + i] = M[i];
                    d.llin[(size_t)n * ND + (size_t)k * ND + i] = M[ND + i];
                }
                __syncwarp();
            }
            // tracer: H(zeta^(l)) C = C~ + dt sum a R with the depth-weighted mass matrix
            for (int i = lane; i < ND; i += 32) {
                o[i] = z[i];
                o[3 * ND + i] = rc[i];
            }
            __syncwarp();
            solve_mass_mixed<ND1, NM>(tb, pV, o + 3 * ND, Mf, Yf, invf, rf, xs, rs, qs, tmp, M, Y,
                                      pinv, lane);
        }
        __syncwarp();
        // write v^(l) and its constant-field mask
        unsigned cmo = 0;
        for (int f = 0; f < 4; ++f) {
            bool eq = true;
            for (int i = lane; i < ND; i += 32) eq = eq && (o[f * ND + i] == o[f * ND]);
            if (__all_sync(0xffffffffu, eq)) cmo |= (1u << f);
        }
        bool fin = true;
        for (int i = lane; i < 4 * ND; i += 32) {
            const double v = o[i];
            fin = fin && isfinite(v);
            ufield(d, sa.out_buf, i / ND, ND)[k * ND + (i % ND)] = v;
        }
        if (!__all_sync(0xffffffffu, fin)) bad = 1;
        if (lane == 0) d.cmask[(size_t)sa.out_buf * n + k] = (uint8_t)cmo;
        its_max = max(its_max, its);
        __syncwarp();
    }
    if (lane == 0) {
        if (its_max) atomicMax(&d.sc->maxits, its_max);
        if (viol) atomicAdd(&d.sc->viol, viol);
        if (fb) atomicAdd(&d.sc->fallback, fb);
        if (bad) atomicOr(&d.sc->status, ST_NAN);
    }
    if (sa.final_ && blockIdx.x == 0 && threadIdx.x == 0) {
        d.sc->dt_last = dt;
        d.sc->t = d.sc->t + dt;
    }
}

// ---------------------------------------------------------------------------
// constant-field masks of a state buffer
// ---------------------------------------------------------------------------
template <int R>
__global__ void k_masks(const __grid_constant__ Dev d, int buf) {
    constexpr int ND = Sz<R>::ND;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t k = (int64_t)blockIdx.x * WPB + warp; k < d.n; k += (int64_t)gridDim.x * WPB) {
        unsigned cm = 0;
        for (int f = 0; f < 4; ++f) {
            const double* u = ufield(d, buf, f, ND) + k * ND;
            bool eq = true;
            for (int i = lane; i < ND; i += 32) eq = eq && (u[i] == u[0]);
            if (__all_sync(0xffffffffu, eq)) cm |= (1u << f);
        }
        if (lane == 0) d.cmask[(size_t)buf * d.n + k] = (uint8_t)cm;
    }
}

// ---------------------------------------------------------------------------
// diagnostics: per-cell wet mass (Eq. positivity-7), tracer mass, min depth
// ---------------------------------------------------------------------------
template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(TPB)
    k_cell_diag(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, double* part) {
    using S = Sz<R>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* su = smem + warp * (2 * ND + 2 * NMP + 2 * NM * NM);
    double* pe = su + 2 * ND;
    double* pc = pe + NMP;
    double* tmp = pc + NMP;
    for (int64_t k = (int64_t)blockIdx.x * WPB + warp; k < d.n; k += (int64_t)gridDim.x * WPB) {
        for (int i = lane; i < ND; i += 32) {
            su[i] = ufield(d, 0, 0, ND)[k * ND + i];
            su[ND + i] = ufield(d, 0, 3, ND)[k * ND + i];
        }
        const unsigned cm = d.cmask[k];
        const double J = d.hxhy[2 * k] * d.hxhy[2 * k + 1];
        __syncwarp();
        tens_interp<ND1, NM>(tb.Bm, su, tmp, pe, lane);
        tens_interp<ND1, NM>(tb.Bm, su + ND, tmp, pc, lane);
        double m = 0.0, tm = 0.0, hmin = INFINITY;
        for (int p = lane; p < NMP; p += 32) {
            const double e = (cm & 1u) ? su[0] : pe[p];
            const double c = (cm & 8u) ? su[ND] : pc[p];
            double V, A;
            Site<R, Pix, MODE>::VA(d, tb, k, SET_MASS, p % NM, p / NM, e, V, A);
            const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
            m += w * V;
            tm += w * V * c;
            hmin = fmin(hmin, V);
        }
        m = warp_sum(m);
        tm = warp_sum(tm);
        hmin = warp_min(hmin);
        if (lane == 0) {
            part[4 * k + 0] = m;
            part[4 * k + 1] = tm;
            part[4 * k + 2] = hmin;
            part[4 * k + 3] = d.flag[k] ? 1.0 : 0.0;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// zeta at gauge points (Lagrange product formula, Sec. 3.2)
// ---------------------------------------------------------------------------
template <int R>
__global__ void k_gauges(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int ng,
                         const double* xy, double* out) {
    constexpr int ND1 = R + 1, ND = ND1 * ND1;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    const double x = xy[2 * gi], y = xy[2 * gi + 1];
    double v = NAN;
    for (int64_t k = 0; k < d.n; ++k) {
        const double x0 = d.x0y0[2 * k], y0 = d.x0y0[2 * k + 1], hx = d.hxhy[2 * k],
                     hy = d.hxhy[2 * k + 1];
        if (x >= x0 && x <= x0 + hx && y >= y0 && y <= y0 + hy) {
            const double* u = ufield(d, 0, 0, ND) + k * ND;
            if (d.cmask[k] & 1u) { v = u[0]; break; }
            const double xi = (x - x0) / hx, eta = (y - y0) / hy;
            double lx[ND1], ly[ND1];
            for (int a = 0; a < ND1; ++a) {
                double px = 1.0, py = 1.0;
                for (int b = 0; b < ND1; ++b)
                    if (b != a) {
                        px *= (xi - tb.xs[b]) / (tb.xs[a] - tb.xs[b]);
                        py *= (eta - tb.xs[b]) / (tb.xs[a] - tb.xs[b]);
                    }
                lx[a] = px;
                ly[a] = py;
            }
            double s = 0.0;
            for (int b = 0; b < ND1; ++b)
                for (int a = 0; a < ND1; ++a) s += u[a + ND1 * b] * lx[a] * ly[b];
            v = s;
            break;
        }
    }
    out[gi] = v;
}

} // namespace swdg
