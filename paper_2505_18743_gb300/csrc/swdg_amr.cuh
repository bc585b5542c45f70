// swdg_amr.cuh -- kernels of dynamic h-adaptation (Sec. 3.4): the refinement
// indicators of Sec. 4.4 and Sec. 5 and the remap of a nodal state from one
// leaf set to the next.
#pragma once
#include "swdg_kernels.cuh"

namespace swdg {

// Lagrange polynomial a on the support nodes xs at x
__device__ __forceinline__ double lagrange_at(const double* xs, int n, int a, double x) {
    double v = 1.0;
    for (int b = 0; b < n; ++b)
        if (b != a) v *= (x - xs[b]) / (xs[a] - xs[b]);
    return v;
}

template <int R>
constexpr int indicator_smem() {
    using S = Sz<R>;
    return 4 * S::ND + 8 * S::ND1 * S::NV;
}

// eta_K = max over the volume Gauss points of |curl u| (kind 0, u = f(h) q,
// grad h = A grad zeta) or of |grad c| (kind 1)
template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(32 * MAXWPB)
    k_indicator(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int kind,
                double* eta) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NV = S::NV, NVP = S::NVP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* su = smem + warp * indicator_smem<R>();
    double* tx = su + 4 * ND; // [4 fields][2: Bv, Dv][ND1][NV]
    const int64_t n = d.n;
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        const unsigned cm = d.cmask[k];
        const double ihx = 1.0 / d.hxhy[2 * k], ihy = 1.0 / d.hxhy[2 * k + 1];
        __syncwarp();
        for (int i = lane; i < 8 * ND1 * NV; i += 32) {
            const int fd = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
            const int fl = fd >> 1, der = fd & 1;
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < ND1; ++a)
                s += (der ? tb.Dv[al][a] : tb.Bv[al][a]) * su[fl * ND + ND1 * b + a];
            tx[i] = s;
        }
        __syncwarp();
        double best = 0.0;
        for (int p = lane; p < NVP; p += 32) {
            const int al = p % NV, be = p / NV;
            double v[4], gx[4], gy[4];
#pragma unroll
            for (int fl = 0; fl < 4; ++fl) {
                double s = 0.0, sx = 0.0, sy = 0.0;
#pragma unroll
                for (int b = 0; b < ND1; ++b) {
                    s += tb.Bv[be][b] * tx[((2 * fl) * ND1 + b) * NV + al];
                    sx += tb.Bv[be][b] * tx[((2 * fl + 1) * ND1 + b) * NV + al];
                    sy += tb.Dv[be][b] * tx[((2 * fl) * ND1 + b) * NV + al];
                }
                const bool c0 = cm & (1u << fl);
                v[fl] = c0 ? su[fl * ND] : s;
                gx[fl] = c0 ? 0.0 : sx * ihx;
                gy[fl] = c0 ? 0.0 : sy * ihy;
            }
            double val;
            if (kind == 1) {
                val = hypot(gx[3], gy[3]);
            } else {
                double V, A;
                ST::VA(d, tb, k, SET_VOL, al, be, v[0], V, A);
                const double e = d.eps;
                double f = 0.0, df = 0.0;
                if (V >= e) {
                    f = 1.0 / V;
                    df = -1.0 / (V * V);
                } else if (V > 0.0) {
                    const double e4 = (e * e) * (e * e), h4 = (V * V) * (V * V);
                    f = sqrt(2.0) * V / sqrt(e4 + h4);
                    df = sqrt(2.0) * (e4 - h4) / ((e4 + h4) * sqrt(e4 + h4));
                }
                val = fabs(f * (gx[2] - gy[1]) + df * A * (v[2] * gx[0] - v[1] * gy[0]));
            }
            best = fmax(best, val);
        }
        best = warp_max(best);
        if (lane == 0) eta[k] = best;
        __syncwarp();
    }
}

// remap plan of one new cell: 0 copy old cell src[0]; 1 child of old cell
// src[0], its support points at (ox + xs s, oy + xs s) in the old cell's
// reference square; 2 parent of old cells src[0..3] (children (0,0), (1,0),
// (0,1), (1,1)): L2 projection
struct RemapArgs {
    const double* uold;  // [4][n_old][nd]
    int64_t n_old;
    const int8_t* type;  // [n_new]
    const int32_t* src;  // [n_new][4]
    const double* rel;   // [n_new][3]: s, ox, oy
    double* unew;        // [4][n_new][nd]
    int64_t n_new;
};

template <int R>
constexpr int remap_smem() {
    using S = Sz<R>;
    return 2 * S::NG * S::ND1 + 4 * S::NGP + 2 * S::ND + 2 * S::ND1 * S::NG;
}

template <int R>
__global__ void __launch_bounds__(32 * MAXWPB)
    k_remap(const __grid_constant__ Tables tb, const __grid_constant__ RemapArgs a) {
    using S = Sz<R>;
    constexpr int ND1 = S::ND1, ND = S::ND, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* Lm = smem + warp * remap_smem<R>(); // [2 offsets][NG points][ND1]
    double* pc = Lm + 2 * NG * ND1;             // [4 children][NGP]
    double* rhs = pc + 4 * NGP;                 // [ND]
    double* out = rhs + ND;                     // [ND]
    double* tmp = out + ND;                     // [2 ND1 NG]
    // parent basis at the Gauss points of each half
    for (int i = lane; i < 2 * NG * ND1; i += 32) {
        const int o = i / (NG * ND1), q = (i / ND1) % NG, b = i % ND1;
        Lm[i] = lagrange_at(tb.xs, ND1, b, 0.5 * (o + tb.xq[SET_MOM][q]));
    }
    __syncwarp();
    const size_t fo = (size_t)a.n_old * ND, fn = (size_t)a.n_new * ND;
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < a.n_new; k += (int64_t)gridDim.x * wpb) {
        const int t = a.type[k];
        if (t == 0) {
            const int64_t s0 = a.src[4 * k];
            for (int i = lane; i < 4 * ND; i += 32)
                a.unew[(i / ND) * fn + k * ND + (i % ND)] = a.uold[(i / ND) * fo + s0 * ND + (i % ND)];
        } else if (t == 1) {
            const int64_t s0 = a.src[4 * k];
            const double s = a.rel[3 * k], ox = a.rel[3 * k + 1], oy = a.rel[3 * k + 2];
            for (int i = lane; i < 4 * ND; i += 32) {
                const int f = i / ND, j = i % ND;
                const double xi = ox + tb.xs[j % ND1] * s, et = oy + tb.xs[j / ND1] * s;
                const double* u = a.uold + f * fo + s0 * ND;
                double v = 0.0;
                for (int bb = 0; bb < ND1; ++bb) {
                    const double lb = lagrange_at(tb.xs, ND1, bb, et);
                    for (int aa = 0; aa < ND1; ++aa)
                        v += lagrange_at(tb.xs, ND1, aa, xi) * lb * u[aa + ND1 * bb];
                }
                a.unew[f * fn + k * ND + j] = v;
            }
        } else {
            for (int f = 0; f < 4; ++f) {
                for (int c = 0; c < 4; ++c) {
                    tens_interp<ND1, NG>(tb.Bg, a.uold + f * fo + (int64_t)a.src[4 * k + c] * ND, tmp,
                                         pc + c * NGP, lane);
                }
                for (int i = lane; i < ND; i += 32) {
                    const int aa = i % ND1, bb = i / ND1;
                    double s = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        const int ocx = c & 1, ocy = c >> 1;
                        for (int qb = 0; qb < NG; ++qb)
                            for (int qa = 0; qa < NG; ++qa)
                                s += 0.25 * tb.wg[qa] * tb.wg[qb] * pc[c * NGP + qa + NG * qb] *
                                     Lm[(ocx * NG + qa) * ND1 + aa] * Lm[(ocy * NG + qb) * ND1 + bb];
                    }
                    rhs[i] = s;
                }
                __syncwarp();
                kron_apply<ND1, false, MXN>(tb.M1inv, rhs, tmp, out, 1.0, lane);
                for (int i = lane; i < ND; i += 32) a.unew[f * fn + k * ND + i] = out[i];
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// transpose of k_gauges: zb[k][a + (R+1) b] += gbar[g] lx_a(xi) ly_b(eta) for
// the cell k holding gauge g (cell[g], or the first containing cell when cell
// is null); a constant (r_K = 0) cell is differentiated as its polynomial.
// One thread per gauge; gauges sharing a cell add atomically.
template <int R>
__global__ void k_gauges_vjp(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int ng,
                             const double* xy, const double* gbar, double* zb, const int32_t* cell) {
    constexpr int ND1 = R + 1;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    const double x = xy[2 * gi], y = xy[2 * gi + 1];
    int64_t k0 = 0, k1 = d.n;
    if (cell) {
        k0 = cell[gi];
        k1 = k0 < 0 ? k0 : k0 + 1;
    }
    for (int64_t k = k0; k < k1; ++k) {
        const double x0 = d.x0y0[2 * k], y0 = d.x0y0[2 * k + 1], hx = d.hxhy[2 * k],
                     hy = d.hxhy[2 * k + 1];
        if (x >= x0 && x <= x0 + hx && y >= y0 && y <= y0 + hy) {
            const double xi = (x - x0) / hx, eta = (y - y0) / hy, g = gbar[gi];
            for (int b = 0; b < ND1; ++b) {
                const double ly = g * lagrange_at(tb.xs, ND1, b, eta);
                for (int a = 0; a < ND1; ++a)
                    atomicAdd(zb + k * ND1 * ND1 + a + ND1 * b, ly * lagrange_at(tb.xs, ND1, a, xi));
            }
            break;
        }
    }
}

} // namespace swdg
