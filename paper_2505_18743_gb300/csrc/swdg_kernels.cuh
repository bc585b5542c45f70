// swdg_kernels.cuh -- sm_103a kernels of the sub-grid DG shallow-water hot
// path (arXiv 2505.18743): residual (Sec. 3.2), degree switch (Eq.
// criteria_p), stage update (Sec. 3.1) and auxiliary reductions.
//
// Mapping: one warp per cell, a launch-time number of warps per block (1..8,
// chosen by the autotuner), grid-stride over cells; one launch covers every
// member of an ensemble.
// Each warp stages its cell in shared memory and evaluates the tensor-product
// operators by sum factorisation (1D contractions), one quadrature point,
// degree of freedom or face point per lane.
#pragma once
#include "swdg_common.cuh"

#include <utility>

namespace swdg {

constexpr int WPB = 4;    // default warps per block
constexpr int MAXWPB = 8; // largest block the kernels are compiled for

// ---------------------------------------------------------------------------
// small tensor contractions on a warp (all arrays in shared memory, x fastest)
// ---------------------------------------------------------------------------
// out[q1 NO + q0] = sum_b B[q1][b] sum_a B[q0][a] in[b NI + a]
template <int NI, int NO, typename T = double, int TL = 32>
__device__ __forceinline__ void tens_interp(const T (*B)[MXN], const T* in, T* tmp, T* out,
                                            int lane, unsigned tm = 0xffffffffu) {
    for (int i = lane; i < NI * NO; i += TL) {
        int b = i / NO, q0 = i % NO;
        T s = T(0);
#pragma unroll
        for (int a = 0; a < NI; ++a) s += B[q0][a] * in[b * NI + a];
        tmp[i] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < NO * NO; i += TL) {
        int q1 = i / NO, q0 = i % NO;
        T s = T(0);
#pragma unroll
        for (int b = 0; b < NI; ++b) s += B[q1][b] * tmp[b * NO + q0];
        out[i] = s;
    }
    __syncwarp(tm);
}

// out[b NI + a] = sum_q1 B[q1][b] sum_q0 B[q0][a] in[q1 NO + q0]   (transpose)
template <int NI, int NO, typename T = double, int TL = 32>
__device__ __forceinline__ void tens_test(const T (*B)[MXN], const T* in, T* tmp, T* out,
                                          int lane, unsigned tm = 0xffffffffu) {
    for (int i = lane; i < NO * NI; i += TL) {
        int q1 = i / NI, a = i % NI;
        T s = T(0);
#pragma unroll
        for (int q0 = 0; q0 < NO; ++q0) s += B[q0][a] * in[q1 * NO + q0];
        tmp[i] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < NI * NI; i += TL) {
        int b = i / NI, a = i % NI;
        T s = T(0);
#pragma unroll
        for (int q1 = 0; q1 < NO; ++q1) s += B[q1][b] * tmp[q1 * NI + a];
        out[i] = s;
    }
    __syncwarp(tm);
}

// out[b N + a] = scale * sum_d C(b,d) sum_c C(a,c) in[d N + c], C(i,j) = T ? M[j][i] : M[i][j]
template <int N, bool T, int LD, typename E = double, int TL = 32>
__device__ __forceinline__ void kron_apply(const E (*M)[LD], const E* in, E* tmp, E* out, E scale,
                                           int lane, unsigned tm = 0xffffffffu) {
    for (int i = lane; i < N * N; i += TL) {
        int d = i / N, a = i % N;
        E s = E(0);
#pragma unroll
        for (int c = 0; c < N; ++c) s += (T ? M[c][a] : M[a][c]) * in[d * N + c];
        tmp[i] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < N * N; i += TL) {
        int b = i / N, a = i % N;
        E s = E(0);
#pragma unroll
        for (int d = 0; d < N; ++d) s += (T ? M[d][b] : M[b][d]) * tmp[d * N + a];
        out[i] = scale * s;
    }
    __syncwarp(tm);
}

// the contractions above for two inputs at once (each output by the same sum,
// the two halves of the work side by side on the lanes)
template <int NI, int NO, typename T = double, int TL = 32>
__device__ __forceinline__ void tens_interp2(const T (*B)[MXN], const T* in0, const T* in1, T* tmp0,
                                             T* tmp1, T* out0, T* out1, int lane, unsigned tm = 0xffffffffu) {
    constexpr int M1 = NI * NO, M2 = NO * NO;
    for (int i = lane; i < 2 * M1; i += TL) {
        const int j = i < M1 ? i : i - M1;
        const T* in = i < M1 ? in0 : in1;
        const int b = j / NO, q0 = j % NO;
        T s = T(0);
#pragma unroll
        for (int a = 0; a < NI; ++a) s += B[q0][a] * in[b * NI + a];
        (i < M1 ? tmp0 : tmp1)[j] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < 2 * M2; i += TL) {
        const int j = i < M2 ? i : i - M2;
        const T* tmp = i < M2 ? tmp0 : tmp1;
        const int q1 = j / NO, q0 = j % NO;
        T s = T(0);
#pragma unroll
        for (int b = 0; b < NI; ++b) s += B[q1][b] * tmp[b * NO + q0];
        (i < M2 ? out0 : out1)[j] = s;
    }
    __syncwarp(tm);
}

template <int NI, int NO, typename T = double, int TL = 32>
__device__ __forceinline__ void tens_test2(const T (*B)[MXN], const T* in0, const T* in1, T* tmp0,
                                           T* tmp1, T* out0, T* out1, int lane, unsigned tm = 0xffffffffu) {
    constexpr int M1 = NO * NI, M2 = NI * NI;
    for (int i = lane; i < 2 * M1; i += TL) {
        const int j = i < M1 ? i : i - M1;
        const T* in = i < M1 ? in0 : in1;
        const int q1 = j / NI, a = j % NI;
        T s = T(0);
#pragma unroll
        for (int q0 = 0; q0 < NO; ++q0) s += B[q0][a] * in[q1 * NO + q0];
        (i < M1 ? tmp0 : tmp1)[j] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < 2 * M2; i += TL) {
        const int j = i < M2 ? i : i - M2;
        const T* tmp = i < M2 ? tmp0 : tmp1;
        const int b = j / NI, a = j % NI;
        T s = T(0);
#pragma unroll
        for (int q1 = 0; q1 < NO; ++q1) s += B[q1][b] * tmp[q1 * NI + a];
        (i < M2 ? out0 : out1)[j] = s;
    }
    __syncwarp(tm);
}

template <int N, bool T, int LD, typename E = double, int TL = 32>
__device__ __forceinline__ void kron_apply2(const E (*M)[LD], const E* in0, const E* in1, E* tmp0,
                                            E* tmp1, E* out0, E* out1, E scale, int lane, unsigned tm = 0xffffffffu) {
    constexpr int MM = N * N;
    for (int i = lane; i < 2 * MM; i += TL) {
        const int j = i < MM ? i : i - MM;
        const E* in = i < MM ? in0 : in1;
        const int d = j / N, a = j % N;
        E s = E(0);
#pragma unroll
        for (int c = 0; c < N; ++c) s += (T ? M[c][a] : M[a][c]) * in[d * N + c];
        (i < MM ? tmp0 : tmp1)[j] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < 2 * MM; i += TL) {
        const int j = i < MM ? i : i - MM;
        const E* tmp = i < MM ? tmp0 : tmp1;
        const int b = j / N, a = j % N;
        E s = E(0);
#pragma unroll
        for (int d = 0; d < N; ++d) s += (T ? M[d][b] : M[b][d]) * tmp[d * N + a];
        (i < MM ? out0 : out1)[j] = scale * s;
    }
    __syncwarp(tm);
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
    // The two tests run on order-preserving integer keys (integer pipe); they
    // decide exactly as eta > -zmin and !(eta > -zmax), a NaN eta reading as
    // dry as under IEEE comparisons.
    static __device__ __forceinline__ bool shortcut(const Dev& d, int64_t k, double eta,
                                                    double zbar, double& V, double& A, bool& full) {
        if (d.zmin == nullptr) return false;
        return shortcut_b(eta, d.zmin[k], d.zmax[k], zbar, V, A, full);
    }
    // the same tests against the bounds zlo <= z_k <= zhi of a set of pixels
    static __device__ __forceinline__ bool shortcut_b(double eta, double zlo, double zhi,
                                                      double zbar, double& V, double& A,
                                                      bool& full) {
        const bool nan = nan_bits(eta);
        const long long ek = okey(eta);
        if (!nan && ek > nkey_neg(zlo)) {
            V = eta + zbar;
            A = 1.0;
            full = true;
            return true;
        }
        if (nan || !(ek > nkey_neg(zhi))) {
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
            if (d.zmin != nullptr) {
                const size_t ip = (size_t)k * S::NZP + offset(set) + ia + count(set) * ib;
                const double zbar = d.zpts[ip];
                // the cell's depth bounds first (one value per cell, cached); where
                // the waterline crosses the cell, the sub-cell's own bounds, so that
                // only the sub-cells it crosses sum their pixels
                if (shortcut_b(eta, d.zmin[k], d.zmax[k], zbar, V, A, full)) return;
                if (d.zsb != nullptr) {
                    const float2 b = d.zsb[ip];
                    if (shortcut_b(eta, (double)b.x, (double)b.y, zbar, V, A, full)) return;
                }
            }
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

// The wave-speed bound's maximum (Eq. lxf_parameter).  For plain arithmetic
// types it is fmax; the adjoint's dual types overload it (found by
// argument-dependent lookup) with the symmetric subgradient at exact ties.
template <typename T>
__device__ __forceinline__ T wave_speed_max(T a, T b) {
    return fmax(a, b);
}

// Rusanov flux with hydrostatic reconstruction at one face point, seen from
// side A with outward normal (nx, ny) (Eqs. lxf_parameter, velocity,
// hydro_rec_vars, mass_rhs, discharge_rhs, r_concentration).  hA = V_A(zeta_A),
// hsA = min(V_A(zeta_A), V_B(zeta_A)).  out = {F, Gx_cons, Gy_cons, R}; the
// non-conservative pressure scalar g {{h*}} (h*A - h*B)/2 is returned apart.
// DC (the adjoint): dc = {dR/dcA, dR/dcB}, the tracer flux's partial
// derivatives in the two concentrations (it is linear in each).
template <typename T, bool DC = false>
__device__ __forceinline__ void rusanov(T qxA, T qyA, T cA, T hA, T hsA, T qxB, T qyB, T cB, T hB,
                                        T hsB, T dhAB, T nx, T ny, T g, T eps, T out[4], T& pres,
                                        T& lam, T* dc = nullptr) {
    // dhAB = h*A - h*B, formed in FP64 by the caller (the well-balanced part of
    // the reconstruction); the tracer jump h*A cA - h*B cB = dhAB cA + h*B (cA - cB)
    const T half = T(0.5);
    T fA = vel_factor<T>(hA, eps), fB = vel_factor<T>(hB, eps);
    T uAx = fA * qxA, uAy = fA * qyA, uBx = fB * qxB, uBy = fB * qyB;
    T unA = uAx * nx + uAy * ny, unB = uBx * nx + uBy * ny;
    T l = wave_speed_max(fabs(unA) + sqrt(g * hA), fabs(unB) + sqrt(g * hB));
    T qsAx = hsA * uAx, qsAy = hsA * uAy, qsBx = hsB * uBx, qsBy = hsB * uBy;
    out[0] = half * ((qsAx + qsBx) * nx + (qsAy + qsBy) * ny) + half * l * dhAB;
    out[1] = half * (qsAx * unA + qsBx * unB) + half * l * (qsAx - qsBx);
    out[2] = half * (qsAy * unA + qsBy * unB) + half * l * (qsAy - qsBy);
    out[3] = half * ((qsAx * cA + qsBx * cB) * nx + (qsAy * cA + qsBy * cB) * ny) +
             half * l * (dhAB * cA + hsB * (cA - cB));
    pres = g * half * (hsA + hsB) * half * dhAB;
    lam = l;
    if constexpr (DC) {
        // R = 1/2 (qs_A cA + qs_B cB).n + l/2 (h*A cA - h*B cB)
        dc[0] = half * (qsAx * nx + qsAy * ny) + half * l * hsA;
        dc[1] = half * (qsBx * nx + qsBy * ny) - half * l * hsB;
    }
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
template <int R, typename B>
constexpr int res_smem() {
    // in doubles: su [4 ND], tz [2 ND1 NV], Xd [4 NVP], sd [4 NV ND1], fh [32 NM], rs [6 ND],
    // tc [2 ND1 NV] (tracer diffusion), then B-typed: suB [4 ND], tB [3 ND1 NV] (B = double;
    // [5 ND1 NV] for B = float, with the elevation's two x-contractions), XB [8 NVP],
    // sB [8 NV ND1]
    using S = Sz<R>;
    constexpr int nd = 4 * S::ND + 2 * S::ND1 * S::NV + 4 * S::NVP + 4 * S::NV * S::ND1 +
                       32 * S::NM + 6 * S::ND + 2 * S::ND1 * S::NV;
    constexpr int ntb = sizeof(B) == sizeof(double) ? 3 : 5;
    constexpr int nb = 4 * S::ND + ntb * S::ND1 * S::NV + 8 * S::NVP + 8 * S::NV * S::ND1;
    return nd + (nb * (int)sizeof(B) + 7) / 8;
}

// traces of zeta (FP64) and of qx, qy, c (type B) at face point al of face f;
// u32 (B = float, nullable): the FP32 copy of u, same layout and stride
template <int ND1, typename B>
__device__ __forceinline__ void face_trace_mixed(const double* u, const float* u32, size_t fstride,
                                                 unsigned cm, int f, const double (*Bd)[MXN],
                                                 const B (*Bb)[MXN], int al, double& z, B t[3]) {
    if (cm & 1u) z = u[0];
    else {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < ND1; ++j) s += Bd[al][j] * u[face_node<ND1>(f, j)];
        z = s;
    }
#pragma unroll
    for (int fl = 1; fl < 4; ++fl) {
        const double* uf = u + fl * fstride;
        if constexpr (sizeof(B) == sizeof(float)) {
            if (u32 != nullptr) { // the same values as (float)uf[.], without conversions
                const float* vf = u32 + fl * fstride;
                if (cm & (1u << fl)) {
                    t[fl - 1] = vf[0];
                    continue;
                }
                B s = B(0);
#pragma unroll
                for (int j = 0; j < ND1; ++j) s += Bb[al][j] * vf[face_node<ND1>(f, j)];
                t[fl - 1] = s;
                continue;
            }
        }
        if (cm & (1u << fl)) {
            t[fl - 1] = (B)uf[0];
            continue;
        }
        B s = B(0);
#pragma unroll
        for (int j = 0; j < ND1; ++j) s += Bb[al][j] * (B)uf[face_node<ND1>(f, j)];
        t[fl - 1] = s;
    }
}

template <typename B>
__device__ __forceinline__ const B (*tab_or(const double (*d)[MXN], const float (*f)[MXN]))[MXN] {
    if constexpr (sizeof(B) == sizeof(double)) return (const B(*)[MXN])d;
    else return (const B(*)[MXN])f;
}

// B = double: the plain FP64 method.  B = float (FP32-bulk): elevation,
// sub-grid integrals, hydrostatic reconstruction and the continuity and
// tracer test integrals stay FP64 (so mass, tracer mass and c = 1 are kept to
// FP64 round-off and the lake at rest exactly); the momentum, friction and
// flux arithmetic is FP32.
// one face point (Sec. 3.2): the Rusanov flux with the hydrostatic
// reconstruction at GLL point al of half h of face f of cell k, whose state
// (4 fields, stride ustride) is uk with constant-field mask cm.  An interior
// point returns the flux of the canonical side order (the lower cell index is
// side A, so both cells of a face get bit-identical values) in raw, with the
// pressure term pres, own_first = (k is side A) and the neighbour nb; a
// boundary point returns k's final flux in raw (bnd = true, nb = -1).  lam is
// the wave speed bound of the point.
template <int R, typename Pix, int MODE, typename B>
__device__ __forceinline__ void face_point(const Dev& d, const Tables& tb, int64_t k, const double* uk,
                                           const float* ukF, size_t ustride, unsigned cm, int buf,
                                           int f, int h, int al,
                                           unsigned info, double hx, double hy, int mem, double t,
                                           B raw[4], B& pres, B& lam, bool& own_first, bool& bnd,
                                           int64_t& nb_out) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM;
    const int64_t n = d.n;
    const B gB = (B)d.g, epsB = (B)d.eps;
    const auto BmB = tab_or<B>(tb.Bm, tb.BmF);
    const bool coarse = (info & 3) == FI_COARSE, fine = (info & 3) == FI_FINE;
    const int half = (int)(info >> 2);
    const double nx = (f == 0) ? -1.0 : (f == 1) ? 1.0 : 0.0;
    const double ny = (f == 2) ? -1.0 : (f == 3) ? 1.0 : 0.0;
    double zm;
    B tm[3];
    face_trace_mixed<ND1, B>(uk, ukF, ustride, cm, f, coarse ? tb.BmH[h] : tb.Bm,
                             coarse ? tab_or<B>(tb.BmH[h], tb.BmHF[h]) : BmB, al, zm, tm);
    int ia, ib;
    face_site_index<NM>(f, al, ia, ib);
    auto own_V = [&](double eta) {
        double V, A;
        if (coarse) ST::VA_half(d, k, f, h, al, eta, V, A);
        else ST::VA(d, tb, k, SET_MASS, ia, ib, eta, V, A);
        return V;
    };
    const int32_t s0 = d.nbr[k * 8 + f * 2];
    const double hm = own_V(zm);
    double zp, hp, hsm, hsp;
    B tp[3];
    if (s0 >= 0) {
        const int64_t nb = coarse ? (int64_t)(h ? d.nbr[k * 8 + f * 2 + 1] : s0) : (int64_t)s0;
        const int fo = f ^ 1;
        face_trace_mixed<ND1, B>(ufield(d, buf, 0, ND) + nb * ND,
                                 d.uF ? ufieldF(d, buf, 0, ND) + nb * ND : nullptr, (size_t)n * ND,
                                 d.cmask[(size_t)buf * n + nb], fo, fine ? tb.BmH[half] : tb.Bm,
                                 fine ? tab_or<B>(tb.BmH[half], tb.BmHF[half]) : BmB, al, zp, tp);
        int ja, jb;
        face_site_index<NM>(fo, al, ja, jb);
        auto nb_V = [&](double eta) {
            double V, A;
            if (fine) ST::VA_half(d, nb, fo, half, al, eta, V, A);
            else ST::VA(d, tb, nb, SET_MASS, ja, jb, eta, V, A);
            return V;
        };
        hp = nb_V(zp);
        hsm = fmin(hm, nb_V(zm)); // min(V-(zeta-), V+(zeta-)), FP64
        hsp = fmin(hp, own_V(zp)); // min(V+(zeta+), V-(zeta+)), FP64
        own_first = k < nb;
        if (own_first)
            rusanov<B>(tm[0], tm[1], tm[2], (B)hm, (B)hsm, tp[0], tp[1], tp[2], (B)hp, (B)hsp,
                       (B)(hsm - hsp), (B)nx, (B)ny, gB, epsB, raw, pres, lam);
        else
            rusanov<B>(tp[0], tp[1], tp[2], (B)hp, (B)hsp, tm[0], tm[1], tm[2], (B)hm, (B)hsm,
                       (B)(hsp - hsm), (B)(-nx), (B)(-ny), gB, epsB, raw, pres, lam);
        bnd = false;
        nb_out = nb;
    } else {
        const int tag = -1 - s0;
        zp = zm;
        tp[0] = tm[0]; tp[1] = tm[1]; tp[2] = tm[2];
        const bool tide = d.mbc ? d.mbc[mem].kind[tag] == 1 : d.bc_kind[tag] == 1;
        if (tide) {
            const double amp = d.mbc ? d.mbc[mem].amp[tag] : d.bc_amp[tag];
            const double per = d.mbc ? d.mbc[mem].per[tag] : d.bc_per[tag];
            const double ph = d.mbc ? d.mbc[mem].ph[tag] : d.bc_ph[tag];
            zp = amp * sin(2.0 * M_PI * t / per + ph);
        } else {
            const B qn = tm[0] * (B)nx + tm[1] * (B)ny;
            tp[0] = tm[0] - B(2) * qn * (B)nx;
            tp[1] = tm[1] - B(2) * qn * (B)ny;
        }
        hp = own_V(zp); // ghost: same sub-grid operator
        hsm = hm;
        hsp = hp;
        rusanov<B>(tm[0], tm[1], tm[2], (B)hm, (B)hsm, tp[0], tp[1], tp[2], (B)hp, (B)hsp,
                   (B)(hsm - hsp), (B)nx, (B)ny, gB, epsB, raw, pres, lam);
        raw[1] -= pres * (B)nx;
        raw[2] -= pres * (B)ny;
        own_first = true;
        bnd = true;
        nb_out = -1;
    }
}

// the flux of an interior face point as seen from the cell whose face f it
// is: the canonical flux with the sign of that side, and the pressure vector
// g {{h*}} (h*A - h*B)/2 n_A, which is the same for both sides
template <typename B>
__device__ __forceinline__ void side_flux(const B raw[4], B pres, bool own_first, int f, B out[4]) {
    const double nx = (f == 0) ? -1.0 : (f == 1) ? 1.0 : 0.0;
    const double ny = (f == 2) ? -1.0 : (f == 3) ? 1.0 : 0.0;
    const B sg = own_first ? B(1) : B(-1);
    const B pnx = own_first ? pres * (B)nx : pres * (B)(-nx);
    const B pny = own_first ? pres * (B)ny : pres * (B)(-ny);
    out[0] = raw[0] * sg;
    out[1] = sg * raw[1] - pnx;
    out[2] = sg * raw[2] - pny;
    out[3] = raw[3] * sg;
}

// 96 registers for the FP64 form; 80 for B = float (six blocks of four
// warps per SM instead of five; measured 2 % faster despite a few spilled
// registers, while the FP32-bulk stage update is slower at 80 or 72)
template <int R, typename Pix, int MODE, typename B>
__global__ void __maxnreg__(sizeof(B) == 4 ? 80 : 96)
    k_residual(const __grid_constant__ Dev d, const __grid_constant__ Tables tb_g, int buf,
               int stage, double c_stage, int want_dt) {
    // the basis tables in shared memory: the contractions index them by lane
    // (a different row or column per lane), which the constant cache would
    // serialise (measured: -3 % per launch)
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
    double* su = smem + warp * res_smem<R, B>();
    double* tz = su + 4 * ND;           // [2][ND1][NV] x-contractions of zeta: value, d/dxi
    double* Xd = tz + 2 * ND1 * NV;     // [4][NVP]: F_x, F_y, R_x, R_y
    double* sd = Xd + 4 * NVP;          // [4][NV][ND1]
    double* fh = sd + 4 * NV * ND1;     // [4 fields][4 faces][2 halves][NM]
    double* rs = fh + 32 * NM;          // [6][ND]
    double* tc = rs + 6 * ND;           // [2][ND1][NV] x-contractions of c (value, d/dxi), FP64
    constexpr bool F64 = sizeof(B) == sizeof(double);
    B* suB = F64 ? (B*)su : (B*)(tc + 2 * ND1 * NV); // [4][ND] (the FP64 state itself when B = double)
    // [3][ND1][NV]: qx, qy, c; B = float: [5][ND1][NV], then zeta (value, d/dxi)
    B* tB = (B*)(tc + 2 * ND1 * NV) + 4 * ND;
    B* XB = tB + (F64 ? 3 : 5) * ND1 * NV; // [8][NVP]: Gx (x, y, v), Gy (x, y, v), Lx, Ly
    B* sB = XB + 8 * NVP;               // [8][NV][ND1]
    const auto BvB = tab_or<B>(tb.Bv, tb.BvF);
    const auto DvB = tab_or<B>(tb.Dv, tb.DvF);
    const auto BmB = tab_or<B>(tb.Bm, tb.BmF);
    const double g = d.g, eps = d.eps;
    const B gB = (B)g, epsB = (B)eps;
    const int64_t n = d.n;

    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        if constexpr (F64) {
            for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, buf, i / ND, ND)[k * ND + (i % ND)];
        } else {
            // B = float: all four fields in FP32 (the elevation enters FP32
            // arithmetic only through its gradient), from the FP32 copy of the
            // state where the context keeps one; in FP64 the elevation, and the
            // other fields only where something still reads them in FP64 (the
            // tracer diffusion, the inline face integration)
            const bool all64 = !d.uF || !d.fflux || (d.nu_c && d.nu_c[k] != 0.0);
            for (int i = lane; i < 4 * ND; i += 32) {
                const bool z64 = i < ND || all64;
                const double v = z64 ? ufield(d, buf, i / ND, ND)[k * ND + (i % ND)] : 0.0;
                su[i] = v;
                suB[i] = d.uF ? ufieldF(d, buf, i / ND, ND)[k * ND + (i % ND)] : (B)v;
            }
        }
        const unsigned cm = d.cmask[(size_t)buf * n + k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double ihx = d.ihxhy ? d.ihxhy[2 * k] : 1.0 / hx;
        const double ihy = d.ihxhy ? d.ihxhy[2 * k + 1] : 1.0 / hy;
        B manB, JB, ihxB, ihyB;
        if constexpr (F64) {
            manB = d.manning[k];
            JB = J;
            ihxB = ihx;
            ihyB = ihy;
        } else {
            // the four per-cell values converted once per warp (lanes 0..3),
            // since conversions occupy the FP64 pipe
            const int q = lane & 3;
            const float f = (float)(q == 0 ? d.manning[k] : q == 1 ? J : q == 2 ? ihx : ihy);
            manB = __shfl_sync(0xffffffffu, f, 0);
            JB = __shfl_sync(0xffffffffu, f, 1);
            ihxB = __shfl_sync(0xffffffffu, f, 2);
            ihyB = __shfl_sync(0xffffffffu, f, 3);
        }
        // the member's stage time t^n + c_l dt (boundary data)
        const int mem = member_of(d, k);
        const double t = (c_stage == 0.0) ? d.mb[mem].t : d.mb[mem].t + c_stage * get_dt(d, mem);
        __syncwarp();
        // x-contractions: zeta (value, d/dxi) in FP64, qx, qy, c in B
        if constexpr (F64) {
            // one job list over the five contractions, the table selected
            // per job (no branch inside a warp): jobs 0..1 zeta value and
            // d/dxi into tz, jobs 2..4 qx, qy, c into tB (B = double here)
            constexpr int NE = ND1 * NV;
            for (int i = lane; i < 5 * NE; i += 32) {
                const int f = i / NE, r_ = i % NE, b = r_ / NV, al = r_ % NV;
                const double(*Tb)[MXN] = f == 1 ? tb.Dv : tb.Bv;
                const double* u = su + (f < 2 ? 0 : f - 1) * ND + ND1 * b;
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += Tb[al][a] * u[a];
                if (f < 2) tz[i] = s;
                else tB[i - 2 * NE] = s;
            }
        } else {
            // the elevation's value in FP64 (the sub-grid depth); in B: qx, qy,
            // c, and the elevation's value and d/dxi for its gradient
            for (int i = lane; i < ND1 * NV; i += 32) {
                const int b = i / NV, al = i % NV;
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += tb.Bv[al][a] * su[ND1 * b + a];
                tz[i] = s;
            }
            for (int i = lane; i < 5 * ND1 * NV; i += 32) {
                const int f = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
                const B* u = suB + (f < 3 ? 1 + f : 0) * ND + ND1 * b;
                const B(*Tb)[MXN] = f == 4 ? DvB : BvB;
                B s = B(0);
#pragma unroll
                for (int a = 0; a < ND1; ++a) s += Tb[al][a] * u[a];
                tB[i] = s;
            }
        }
        // tracer numerical diffusion (Eq. numdiff): grad c in FP64
        const double nu = d.nu_c ? d.nu_c[k] : 0.0;
        if (nu != 0.0) {
            for (int i = lane; i < 2 * ND1 * NV; i += 32) {
                const int f = i / (ND1 * NV), r_ = i % (ND1 * NV), b = r_ / NV, al = r_ % NV;
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < ND1; ++a)
                    s += (f ? tb.Dv[al][a] : tb.Bv[al][a]) * su[3 * ND + ND1 * b + a];
                tc[i] = s;
            }
        }
        __syncwarp();
        // y-contraction and pointwise physics, one volume point per lane
        for (int p = lane; p < NVP; p += 32) {
            const int al = p % NV, be = p / NV;
            double z = 0.0;
            B qx = B(0), qy = B(0), c = B(0), zx, zy;
            if constexpr (F64) {
                double zxd = 0.0, zyd = 0.0;
#pragma unroll
                for (int b = 0; b < ND1; ++b) {
                    z += tb.Bv[be][b] * tz[b * NV + al];
                    zxd += tb.Bv[be][b] * tz[(ND1 + b) * NV + al];
                    zyd += tb.Dv[be][b] * tz[b * NV + al];
                }
                if (cm & 1u) { z = su[0]; zxd = 0.0; zyd = 0.0; }
                zx = zxd * ihx;
                zy = zyd * ihy;
            } else {
                // the gradient of the elevation in FP32 (it enters only the
                // FP32 pressure term g h grad zeta)
                B zxd = B(0), zyd = B(0);
#pragma unroll
                for (int b = 0; b < ND1; ++b) {
                    z += tb.Bv[be][b] * tz[b * NV + al];
                    zxd += BvB[be][b] * tB[(4 * ND1 + b) * NV + al];
                    zyd += DvB[be][b] * tB[(3 * ND1 + b) * NV + al];
                }
                if (cm & 1u) { z = su[0]; zxd = B(0); zyd = B(0); }
                zx = zxd * ihxB;
                zy = zyd * ihyB;
            }
#pragma unroll
            for (int b = 0; b < ND1; ++b) {
                const B Bb = BvB[be][b];
                qx += Bb * tB[(0 * ND1 + b) * NV + al];
                qy += Bb * tB[(1 * ND1 + b) * NV + al];
                c += Bb * tB[(2 * ND1 + b) * NV + al];
            }
            if (cm & 2u) qx = suB[ND];
            if (cm & 4u) qy = suB[2 * ND];
            if (cm & 8u) c = suB[3 * ND];
            double h, A;
            ST::VA(d, tb, k, SET_VOL, al, be, z, h, A);
            const B hB = (B)h;
            B fv, gam;
            vel_gamma<B>(manB, hB, qx, qy, gB, epsB, fv, gam);
            const B ux = fv * qx, uy = fv * qy;
            const double w = J * tb.wv[al] * tb.wv[be];
            B wB, wx, wy;
            if constexpr (F64) {
                wB = w;
                wx = w * ihx;
                wy = w * ihy;
            } else { // the weights of the FP32 terms in FP32 (no conversions per point)
                wB = JB * tb.wvF[al] * tb.wvF[be];
                wx = wB * ihxB;
                wy = wB * ihyB;
            }
            Xd[0 * NVP + p] = (double)(wx * qx);
            Xd[1 * NVP + p] = (double)(wy * qy);
            Xd[2 * NVP + p] = (double)(wx * c * qx);
            Xd[3 * NVP + p] = (double)(wy * c * qy);
            if (nu != 0.0 && !(cm & 8u)) {
                // -nu h grad c . grad psi: the reference derivatives of c at the point
                double cxd = 0.0, cyd = 0.0;
#pragma unroll
                for (int b = 0; b < ND1; ++b) {
                    cxd += tb.Bv[be][b] * tc[(ND1 + b) * NV + al];
                    cyd += tb.Dv[be][b] * tc[b * NV + al];
                }
                Xd[2 * NVP + p] -= w * nu * h * cxd * ihx * ihx;
                Xd[3 * NVP + p] -= w * nu * h * cyd * ihy * ihy;
            }
            XB[0 * NVP + p] = wx * qx * ux;
            XB[1 * NVP + p] = wy * qx * uy;
            XB[2 * NVP + p] = -wB * gB * hB * zx;
            XB[3 * NVP + p] = wx * qy * ux;
            XB[4 * NVP + p] = wy * qy * uy;
            XB[5 * NVP + p] = -wB * gB * hB * zy;
            XB[6 * NVP + p] = -wB * gam * qx;
            XB[7 * NVP + p] = -wB * gam * qy;
        }
        __syncwarp();
        // test integration, y-contraction.  FP64: F (x, y), R (x, y); B: Gx, Gy
        // (x; y + v), Lx, Ly (v)
        if constexpr (F64) {
            // every single 5-term sum is one job, so the lanes stay busy: jobs
            // 0,1 F/R x-part (Bv), 2,3 F/R y-part (Dv), 4,5 Gx/Gy x-part (Bv),
            // 6,7 Lx/Ly (Bv), NV ND1 entries each; then the Gx/Gy y + v parts
            constexpr int NE = NV * ND1;
            for (int i = lane; i < 8 * NE; i += 32) {
                const int job = i / NE, r_ = i % NE, al = r_ / ND1, b = r_ % ND1;
                const int c2 = job & 1, kind = job >> 1;
                const double(*Tb)[MXN] = kind == 1 ? tb.Dv : tb.Bv;
                const double* X = kind == 0   ? Xd + (2 * c2) * NVP
                                  : kind == 1 ? Xd + (2 * c2 + 1) * NVP
                                  : kind == 2 ? (const double*)XB + 3 * c2 * NVP
                                              : (const double*)XB + (6 + c2) * NVP;
                double* out = kind == 0   ? sd + ((c2 * 2 + 0) * NV + al) * ND1 + b
                              : kind == 1 ? sd + ((c2 * 2 + 1) * NV + al) * ND1 + b
                              : kind == 2 ? (double*)sB + ((c2 * 2 + 0) * NV + al) * ND1 + b
                                          : (double*)sB + (((2 + c2) * 2 + 1) * NV + al) * ND1 + b;
                double acc = 0.0;
#pragma unroll
                for (int be = 0; be < NV; ++be) acc += Tb[be][b] * X[al + NV * be];
                *out = acc;
            }
            for (int i = lane; i < 2 * NE; i += 32) {
                const int cg = i / NE, r_ = i % NE, al = r_ / ND1, b = r_ % ND1;
                const B* Xg = XB + 3 * cg * NVP;
                B so = B(0);
#pragma unroll
                for (int be = 0; be < NV; ++be) {
                    const int p = al + NV * be;
                    so += DvB[be][b] * Xg[NVP + p] + BvB[be][b] * Xg[2 * NVP + p];
                }
                sB[((cg * 2 + 1) * NV + al) * ND1 + b] = so;
            }
        } else {
            for (int i = lane; i < 2 * NV * ND1; i += 32) {
                const int cf = i / (NV * ND1), r_ = i % (NV * ND1), al = r_ / ND1, b = r_ % ND1;
                double sx = 0.0, so = 0.0;
#pragma unroll
                for (int be = 0; be < NV; ++be) {
                    const int p = al + NV * be;
                    sx += tb.Bv[be][b] * Xd[(2 * cf) * NVP + p];
                    so += tb.Dv[be][b] * Xd[(2 * cf + 1) * NVP + p];
                }
                sd[((cf * 2 + 0) * NV + al) * ND1 + b] = sx;
                sd[((cf * 2 + 1) * NV + al) * ND1 + b] = so;
            }
            // Gx, Gy: grad-x part, and grad-y + value parts
            for (int i = lane; i < 2 * NV * ND1; i += 32) {
                const int cg = i / (NV * ND1), r_ = i % (NV * ND1), al = r_ / ND1, b = r_ % ND1;
                const B* Xg = XB + 3 * cg * NVP;
                B sx = B(0), so = B(0);
#pragma unroll
                for (int be = 0; be < NV; ++be) {
                    const int p = al + NV * be;
                    sx += BvB[be][b] * Xg[p];
                    so += DvB[be][b] * Xg[NVP + p] + BvB[be][b] * Xg[2 * NVP + p];
                }
                sB[((cg * 2 + 0) * NV + al) * ND1 + b] = sx;
                sB[((cg * 2 + 1) * NV + al) * ND1 + b] = so;
            }
            // Lx, Ly: value parts only
            for (int i = lane; i < 2 * NV * ND1; i += 32) {
                const int cl = i / (NV * ND1), r_ = i % (NV * ND1), al = r_ / ND1, b = r_ % ND1;
                const B* Xl = XB + (6 + cl) * NVP;
                B so = B(0);
#pragma unroll
                for (int be = 0; be < NV; ++be) so += BvB[be][b] * Xl[al + NV * be];
                sB[(((2 + cl) * 2 + 1) * NV + al) * ND1 + b] = so;
            }
        }
        __syncwarp();
        // x-contraction into rs = [F, Gx, Gy, R, Lx, Ly]: F and R in FP64
        for (int i = lane; i < 2 * ND; i += 32) {
            const int cf = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
            double s = 0.0;
#pragma unroll
            for (int al = 0; al < NV; ++al)
                s += tb.Dv[al][a] * sd[((cf * 2 + 0) * NV + al) * ND1 + b] +
                     tb.Bv[al][a] * sd[((cf * 2 + 1) * NV + al) * ND1 + b];
            rs[(cf == 0 ? 0 : 3) * ND + j] = s;
        }
        for (int i = lane; i < 2 * ND; i += 32) { // Gx, Gy
            const int cg = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
            B s = B(0);
#pragma unroll
            for (int al = 0; al < NV; ++al)
                s += DvB[al][a] * sB[((cg * 2 + 0) * NV + al) * ND1 + b] +
                     BvB[al][a] * sB[((cg * 2 + 1) * NV + al) * ND1 + b];
            rs[(1 + cg) * ND + j] = (double)s;
        }
        for (int i = lane; i < 2 * ND; i += 32) { // Lx, Ly
            const int cl = i / ND, j = i % ND, a = j % ND1, b = j / ND1;
            B s = B(0);
#pragma unroll
            for (int al = 0; al < NV; ++al) s += BvB[al][a] * sB[(((2 + cl) * 2 + 1) * NV + al) * ND1 + b];
            rs[(4 + cl) * ND + j] = (double)s;
        }
        // faces: one (sub)face point per lane; a coarse cell integrates each
        // 2:1 face over the GLL points of both fine halves
        double dtl = 0.0;
        unsigned fi[4]; // indexed by constants only (registers)
#pragma unroll
        for (int f = 0; f < 4; ++f) fi[f] = d.finfo ? d.finfo[k * 4 + f] : 0;
        if (d.fflux) {
            // the face fluxes of this cell, computed once per face point by k_faces
            const double* F = d.fflux + k * (32 * NM);
            for (int i = lane; i < 32 * NM; i += 32) fh[i] = F[i];
        } else {
            // the face points of faces 0..3 start at 0, b1, b2, b3 (2 NM points
            // on a coarse 2:1 face, else NM)
            auto npts = [&](unsigned inf) { return (((inf & 3) == FI_COARSE) ? 2 : 1) * NM; };
            const int b1 = npts(fi[0]), b2 = b1 + npts(fi[1]), b3 = b2 + npts(fi[2]),
                      b4 = b3 + npts(fi[3]);
            for (int it = lane; it < b4; it += 32) {
                const int f = (it >= b1) + (it >= b2) + (it >= b3);
                const int r_ = it - (f == 0 ? 0 : f == 1 ? b1 : f == 2 ? b2 : b3), h = r_ / NM,
                          al = r_ % NM;
                const unsigned info = f == 0 ? fi[0] : f == 1 ? fi[1] : f == 2 ? fi[2] : fi[3];
                const bool coarse = (info & 3) == FI_COARSE;
                B raw[4], pres, lam, out[4];
                bool own_first, bnd;
                int64_t nb;
                face_point<R, Pix, MODE, B>(d, tb, k, su, nullptr, ND, cm, buf, f, h, al, info, hx, hy,
                                            mem, t, raw, pres, lam, own_first, bnd, nb);
                if (bnd) {
#pragma unroll
                    for (int cf = 0; cf < 4; ++cf) out[cf] = raw[cf];
                } else {
                    side_flux<B>(raw, pres, own_first, f, out);
                }
                const double L = ((f < 2) ? hy : hx) * (coarse ? 0.5 : 1.0);
                const double wl = L * tb.wm[al];
#pragma unroll
                for (int cf = 0; cf < 4; ++cf)
                    fh[((cf * 4 + f) * 2 + h) * NM + al] = wl * (double)out[cf];
                // lambda l / J for the positivity step (l = L, J = hx hy)
                dtl = fmax(dtl, fmax((double)lam, 1e-12) * ((f < 2) ? ihx : ihy) * (coarse ? 0.5 : 1.0));
            }
        }
        if (want_dt && !d.fflux) {
            const double m = warp_max(dtl);
            if (lane == 0) atomic_max_pos(&d.mb[mem].rmax, m);
        }
        __syncwarp();
        // lift the face fluxes onto the nodes of each face: one item per field,
        // face and node along it, the x faces (0, 1: node columns a = 0 and
        // ND1 - 1) in one pass and the y faces (2, 3: rows b = 0 and ND1 - 1) in
        // the next, so that the items of a pass touch distinct nodes and every
        // lane does the same work
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = lane; i < 4 * 2 * ND1; i += 32) {
                const int cf = i / (2 * ND1), r_ = i % (2 * ND1), f = 2 * pass + r_ / ND1;
                const int tn = r_ % ND1; // node index along the face
                const unsigned inf = f == 0 ? fi[0] : f == 1 ? fi[1] : f == 2 ? fi[2] : fi[3];
                const double* fp = fh + (cf * 4 + f) * 2 * NM;
                double s = 0.0;
                if ((inf & 3) == FI_COARSE) {
#pragma unroll
                    for (int al = 0; al < NM; ++al)
                        s += tb.BmH[0][al][tn] * fp[al] + tb.BmH[1][al][tn] * fp[NM + al];
                } else {
#pragma unroll
                    for (int al = 0; al < NM; ++al) s += tb.Bm[al][tn] * fp[al];
                }
                rs[cf * ND + face_node<ND1>(f, tn)] -= s;
            }
            __syncwarp();
        }
        for (int i = lane; i < 6 * ND; i += 32)
            rfield(d, stage, i / ND, ND)[k * ND + (i % ND)] = rs[i];
        __syncwarp();
    }
}

// every face point of the mesh once (the residual's face integrals, Sec. 3.2):
// job j of d.fjobs is cell k = job >> 8 with face f, half h and GLL point al
// packed as f | h << 2 | al << 3, k the lower cell index of the face (or the
// cell of a boundary face).  The flux as seen from each side, times that
// side's quadrature weight, goes to the side's slots of d.fflux
// ([cell][4 fields][4 faces][2 halves][NM], the residual's fh layout);
// with want_dt the wave speed bound of each side (lambda l / J) raises its
// member's rmax, as the residual does when it integrates the faces itself.
// One job per lane.
template <int R, typename Pix, int MODE, typename B>
__global__ void __maxnreg__(80)
    k_faces(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int buf, double c_stage,
            int want_dt) {
    using S = Sz<R>;
    constexpr int ND = S::ND, NM = S::NM, SL = 32 * NM;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = d.n;
    for (int64_t j0 = gw * 32; j0 < d.njobs; j0 += nw * 32) { // warp-uniform bounds
        const int64_t j = j0 + lane;
        double v = 0.0;
        int mem = -1;
        if (j < d.njobs) {
            const int64_t job = d.fjobs[j];
            const int64_t k = job >> 8;
            const int f = (int)(job & 3), h = (int)((job >> 2) & 1), al = (int)((job >> 3) & 31);
            const unsigned info = d.finfo ? d.finfo[k * 4 + f] : 0;
            const bool coarse = (info & 3) == FI_COARSE;
            const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1];
            const double ihx = d.ihxhy ? d.ihxhy[2 * k] : 1.0 / hx;
            const double ihy = d.ihxhy ? d.ihxhy[2 * k + 1] : 1.0 / hy;
            mem = member_of(d, k);
            const double t = (c_stage == 0.0) ? d.mb[mem].t : d.mb[mem].t + c_stage * get_dt(d, mem);
            B raw[4], pres, lam, out[4];
            bool own_first, bnd;
            int64_t nb;
            face_point<R, Pix, MODE, B>(d, tb, k, ufield(d, buf, 0, ND) + k * ND,
                                        d.uF ? ufieldF(d, buf, 0, ND) + k * ND : nullptr, (size_t)n * ND,
                                        d.cmask[(size_t)buf * n + k], buf, f, h, al, info, hx, hy,
                                        mem, t, raw, pres, lam, own_first, bnd, nb);
            if (bnd) {
#pragma unroll
                for (int cf = 0; cf < 4; ++cf) out[cf] = raw[cf];
            } else {
                side_flux<B>(raw, pres, own_first, f, out);
            }
            const double L = ((f < 2) ? hy : hx) * (coarse ? 0.5 : 1.0);
            const double wl = L * tb.wm[al];
            double* F = d.fflux + k * SL;
#pragma unroll
            for (int cf = 0; cf < 4; ++cf) F[((cf * 4 + f) * 2 + h) * NM + al] = wl * (double)out[cf];
            v = fmax((double)lam, 1e-12) * ((f < 2) ? ihx : ihy) * (coarse ? 0.5 : 1.0);
            if (!bnd && nb != k) {
                // the other side: its face fo, its half (the fine side of a 2:1
                // face has one) and its own weight
                const int fo = f ^ 1;
                const unsigned ninfo = d.finfo ? d.finfo[nb * 4 + fo] : 0;
                const bool ncoarse = (ninfo & 3) == FI_COARSE;
                const int hn = ((info & 3) == FI_FINE) ? (int)(info >> 2) : 0;
                const double nhx = d.hxhy[2 * nb], nhy = d.hxhy[2 * nb + 1];
                const double nihx = d.ihxhy ? d.ihxhy[2 * nb] : 1.0 / nhx;
                const double nihy = d.ihxhy ? d.ihxhy[2 * nb + 1] : 1.0 / nhy;
                side_flux<B>(raw, pres, !own_first, fo, out);
                const double Ln = ((fo < 2) ? nhy : nhx) * (ncoarse ? 0.5 : 1.0);
                const double wln = Ln * tb.wm[al];
                double* Fn = d.fflux + nb * SL;
#pragma unroll
                for (int cf = 0; cf < 4; ++cf)
                    Fn[((cf * 4 + fo) * 2 + hn) * NM + al] = wln * (double)out[cf];
                v = fmax(v, fmax((double)lam, 1e-12) * ((fo < 2) ? nihx : nihy) * (ncoarse ? 0.5 : 1.0));
            }
        }
        if (want_dt) {
            // one atomic per warp when its jobs share a member, else per job
            const int m0 = __shfl_sync(0xffffffffu, mem, 0);
            if (__all_sync(0xffffffffu, mem == m0 || mem < 0)) {
                const double m = team_max_nonneg(v, 0xffffffffu); // v >= 0, never NaN
                if (lane == 0 && m0 >= 0) atomic_max_pos(&d.mb[m0].rmax, m);
            } else if (mem >= 0) {
                atomic_max_pos(&d.mb[mem].rmax, v);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// warp-cooperative scalar Newton for Hbar(e) = target (r_K = 0 cells,
// Eqs. newton, initial_guess); returns iterations
// ---------------------------------------------------------------------------
template <int R, typename Pix, int MODE, int TL = 32>
__device__ __forceinline__ void mass_scalar(const Dev& d, const Tables& tb, int64_t k, double J,
                                            double e, int lane, double& H, double& A,
                                            unsigned tm = 0xffffffffu) {
    using S = Sz<R>;
    double h = 0.0, a = 0.0;
    for (int p = lane; p < S::NMP; p += TL) {
        const int ia = p % S::NM, ib = p / S::NM;
        double V, Ap;
        Site<R, Pix, MODE>::VA(d, tb, k, SET_MASS, ia, ib, e, V, Ap);
        const double w = J * tb.wm[ia] * tb.wm[ib];
        h += w * V;
        a += w * Ap;
    }
    team_sum2<TL>(h, a, tm);
    H = h;
    A = a;
}

// The same mean depth and wet area for a constant elevation e, in mode S as
// one sum over the cell's pixels: the mass sub-cells tile the cell, so the
// pixel k of a P x P tile carries 1/P^2 of the area whatever sub-cells it
// is split among, and Hbar(e) = J / P^2 sum_k max(e + z_k, 0), Abar = J / P^2
// #{e + z_k > 0} (equal to mass_scalar up to rounding, with P^2 terms
// instead of the sub-cells' split pixels).  Cells wholly wet or dry, and mode
// P, take mass_scalar (its shortcut makes it cheap there).
template <int R, typename Pix, int MODE, int TL = 32>
__device__ __forceinline__ void mass_scalar_pixels(const Dev& d, const Tables& tb, int64_t k,
                                                   double J, double e, int lane, double& H,
                                                   double& A, unsigned tm = 0xffffffffu) {
    using ST = Site<R, Pix, MODE>;
    const bool mixed = MODE == 0 && d.zmin != nullptr && !nan_bits(e) &&
                       !(okey(e) > nkey_neg(d.zmin[k])) && okey(e) > nkey_neg(d.zmax[k]);
    if (!mixed) {
        mass_scalar<R, Pix, MODE, TL>(d, tb, k, J, e, lane, H, A, tm);
        return;
    }
    const OvTab& o = ST::tab(d, k);
    const Pix* t = ST::tile(d, o, k);
    const int np = o.P * o.P;
    double h = 0.0;
    int a = 0;
    for (int i = lane; i < np; i += TL) {
        const double dd = e + (double)t[i];
        if (dd > 0.0) {
            h += dd;
            ++a;
        }
    }
    const double w = J / (double)np;
    H = w * team_sum<TL>(h, tm);
    A = w * (double)__reduce_add_sync(tm, a);
}

template <int R, typename Pix, int MODE, int TL = 32>
__device__ int scalar_newton(const Dev& d, const Tables& tb, int64_t k, double J, double target,
                             double& e, int lane, unsigned tm = 0xffffffffu) {
    constexpr int ND = Sz<R>::ND;
    double H, A;
    mass_scalar_pixels<R, Pix, MODE, TL>(d, tb, k, J, e, lane, H, A, tm);
    // the first iteration reuses this evaluation unless the start moves to the
    // dry start of Eq. initial_guess
    bool have = true;
    if (A == 0.0) {
        e = -d.zmax[k] + d.eps0;
        have = false;
    }
    int it = 0;
    for (int kk = 0; kk < d.newton_max; ++kk) {
        if (!have) mass_scalar_pixels<R, Pix, MODE, TL>(d, tb, k, J, e, lane, H, A, tm);
        have = false;
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
__global__ void __launch_bounds__(32 * MAXWPB)
    k_step_begin(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, int do_switch) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* su = smem + warp * begin_smem<R>();
    double* pe = su + 4 * ND;    // [NMP] zeta at mass points
    double* pc = pe + NMP;       // [NMP] c at mass points
    double* pV = pc + NMP;       // [NMP]
    double* px = pV + NMP;       // [NMP] scratch products
    double* tmp = px + NMP;      // [2 NM NM]
    double* pg = tmp + 2 * NM * NM; // [3][NGP]
    double* out = pg + 3 * NGP;  // [2][ND]
    const int64_t n = d.n;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < d.nmemb; i += blockDim.x) d.mb[i].rmax = 0ull;
        if (threadIdx.x == 0) d.sc->maxits = 0;
    }
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += 32) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        unsigned cm = d.cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        __syncwarp();
        // zeta and c at the mass points
        tens_interp<ND1, NM>(tb.Bm, su, tmp, pe, lane);
        tens_interp<ND1, NM>(tb.Bm, su + 3 * ND, tmp, pc, lane);
        bool allfull = true;
        for (int p = lane; p < NMP; p += 32) {
            if (cm & 1u) pe[p] = su[0];
            if (cm & 8u) pc[p] = su[3 * ND];
            double V, A;
            bool full;
            ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pe[p], V, A, full);
            pV[p] = V;
            allfull = allfull && full && !zero_bits(A);
        }
        allfull = __all_sync(0xffffffffu, allfull);
        __syncwarp();
        // r_K = 0 where the smallest wet depth of the mass points is at most
        // h_lim (a NaN depth never counts, as under fmin)
        bool low = false;
        for (int p = lane; p < NMP; p += 32) low = low || pV[p] <= d.hlim;
        const int flag = (do_switch && __any_sync(0xffffffffu, low)) ? 0 : R;
        if (flag == 0) {
            // remap to r_K = 0: mass-exact zeta, GL means of q, tracer-mass-exact c
            double m = 0.0, tr = 0.0;
            for (int p = lane; p < NMP; p += 32) {
                const double w = J * tb.wm[p % NM] * tb.wm[p / NM];
                m += w * pV[p];
                tr += w * pV[p] * pc[p];
            }
            team_sum2<32>(m, tr, 0xffffffffu);
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
            team_sum2<32>(mq[0], mq[1], 0xffffffffu);
            mq[2] = warp_sum(mq[2]);
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
            for (int i = lane; i < 4 * ND; i += 32) {
                ufield(d, 0, i / ND, ND)[k * ND + (i % ND)] = su[i];
                if (d.uF) ufieldF(d, 0, i / ND, ND)[k * ND + (i % ND)] = (float)su[i];
            }
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
            pc[p] = px[p] * pc[p]; // c is not needed beyond C~
        }
        team_sum2<32>(hb, cb, 0xffffffffu);
        __syncwarp();
        tens_test2<ND1, NM>(tb.Bm, px, pc, tmp, tmp + NM * NM, out, out + ND, lane);
        for (int i = lane; i < ND; i += 32) {
            d.HN[k * ND + i] = out[i];
            d.CN[k * ND + i] = out[ND + i];
        }
        // the discharges of v^n at the momentum points, the same for every
        // stage of the step (the stage update reads them rather than
        // interpolating v^n again; same sums, same constant fields)
        if (d.qpts) {
            tens_interp2<ND1, NG>(tb.Bg, su + ND, su + 2 * ND, tmp, tmp + NM * NM, pg, pg + NGP, lane);
            for (int p = lane; p < 2 * NGP; p += 32)
                d.qpts[k * 2 * NGP + p] = (cm & (2u << (p / NGP))) ? su[(1 + p / NGP) * ND] : pg[p];
        }
        if (lane == 0) {
            d.HNbar[k] = hb;
            d.CNbar[k] = cb;
            d.flag[k] = (uint8_t)flag;
            d.cmask[k] = (uint8_t)cm;
            if (d.wet0) d.wet0[k] = (uint8_t)(flag != 0 && allfull);
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
constexpr int stage_union() {
    // in doubles, one region for what is never live at the same time: the
    // friction points / the momentum block's point arrays [6 NGP] with its
    // nodal and tmp pairs (B-typed, sized in doubles); the FP32 solve's float
    // M, Y (8-byte padded); the FP64 fallback's M [ND ND]
    using S = Sz<R>;
    constexpr int mom = 6 * S::NGP + 2 * S::ND + 2 * S::ND1 * S::NG;
    constexpr int f32 = (S::ND * S::ND + S::ND1 * S::ND1 * S::NM + 1) / 2;
    constexpr int fb = S::ND * S::ND;
    constexpr int m = mom > f32 ? mom : f32;
    return m > fb ? m : fb;
}
template <int R>
constexpr int stage_smem() {
    using S = Sz<R>;
    // the FP64 fallback's Y [ND1 ND1 NM] overlays tmp, x, r (see k_stage)
    static_assert(S::ND1 * S::ND1 * S::NM <= 2 * S::NM * S::NM + 2 * S::ND, "fallback Y");
    return 4 * S::ND + 5 * S::ND + 3 * S::NMP + 2 * S::NM * S::NM + 2 * S::ND + 4 * S::ND +
           stage_union<R>();
}

// Cholesky of the SPD matrix M (ND x ND, row-major, lower part used) on a
// warp, then M x = b in place by column-oriented forward and back
// substitution (one reciprocal per column, the updates spread over lanes);
// returns false on a non-positive pivot
template <int ND, int TL = 32>
__device__ bool chol_solve(double* M, double* b, double* inv, int lane, unsigned tm = 0xffffffffu) {
    for (int j = 0; j < ND; ++j) {
        __syncwarp(tm);
        const double djj = M[j * ND + j];
        if (!(djj > 0.0)) return false;
        const double ljj = sqrt(djj);
        const double r = 1.0 / ljj;
        __syncwarp(tm);
        for (int i = j + 1 + lane; i < ND; i += TL) M[i * ND + j] *= r;
        if (lane == 0) {
            M[j * ND + j] = ljj;
            inv[j] = r;
        }
        __syncwarp(tm);
        const int m = ND - j - 1;
        for (int idx = lane; idx < m * m; idx += TL) {
            const int i = j + 1 + idx / m, l = j + 1 + idx % m;
            if (l <= i) M[i * ND + l] -= M[i * ND + j] * M[l * ND + j];
        }
    }
    __syncwarp(tm);
    for (int j = 0; j < ND; ++j) { // L y = b
        const double yj = b[j] * inv[j];
        __syncwarp(tm);
        for (int i = j + 1 + lane; i < ND; i += TL) b[i] -= M[i * ND + j] * yj;
        if (lane == 0) b[j] = yj;
        __syncwarp(tm);
    }
    for (int j = ND - 1; j >= 0; --j) { // L^T x = y
        const double xj = b[j] * inv[j];
        __syncwarp(tm);
        for (int i = lane; i < j; i += TL) b[i] -= M[j * ND + i] * xj;
        if (lane == 0) b[j] = xj;
        __syncwarp(tm);
    }
    return true;
}

// M_(a,b),(c,d) = sum_{al,be} c_{al,be} Bm[al][a] Bm[al][c] Bm[be][b] Bm[be][d]
template <int ND1, int NM, int TL = 32>
__device__ __forceinline__ void assemble_mass(const Tables& tb, const double* cw, double* Y,
                                              double* M, int lane, unsigned tm = 0xffffffffu) {
    constexpr int ND = ND1 * ND1;
    for (int i = lane; i < ND1 * ND1 * NM; i += TL) {
        const int a = i / (ND1 * NM), r_ = i % (ND1 * NM), c = r_ / NM, be = r_ % NM;
        double s = 0.0;
#pragma unroll
        for (int al = 0; al < NM; ++al) s += cw[al + NM * be] * tb.Bm[al][a] * tb.Bm[al][c];
        Y[i] = s;
    }
    __syncwarp(tm);
    for (int i = lane; i < ND * ND; i += TL) {
        const int r_ = i / ND, s_ = i % ND;
        const int a = r_ % ND1, b = r_ / ND1, c = s_ % ND1, dd = s_ / ND1;
        double s = 0.0;
#pragma unroll
        for (int be = 0; be < NM; ++be)
            s += Y[(a * ND1 + c) * NM + be] * tb.Bm[be][b] * tb.Bm[be][dd];
        M[i] = s;
    }
    __syncwarp(tm);
}

// Index of element (i, t) of an FP32 factor stored by rows.  For a
// power-of-two order the column is XOR-swizzled with i / 2, so that a team's
// lanes reading one element of each row, or of each column, hit distinct
// shared-memory banks; an odd order needs no swizzle.
template <int ND>
__device__ __forceinline__ int lrow_idx(int i, int t) {
    if constexpr ((ND & (ND - 1)) == 0) return i * ND + (t ^ ((i >> 1) & (ND - 1)));
    else return i * ND + t;
}

// The steps of a Cholesky factorisation with row i of the matrix in the
// lane's registers a (lower part used).  Step J takes the pivot from lane J,
// scales column J and updates the columns l > J with L_lJ from lane l.  The
// steps are expanded from index sequences, so that every index into a is a
// constant and the row stays in registers.  After a non-positive pivot the
// steps go on (no branch) and ok is false.
template <int ND, int TL, int J, int L>
__device__ __forceinline__ void chol_row_update(float (&a)[ND], int i, unsigned tm) {
    constexpr int l = J + 1 + L;
    const float llj = __shfl_sync(tm, a[J], l, TL); // L_lJ
    if (l <= i) a[l] -= a[J] * llj;
}
template <int ND, int TL, int J, int... L>
__device__ __forceinline__ void chol_row_step(float (&a)[ND], int i, float& rinv, bool& ok,
                                              unsigned tm, std::integer_sequence<int, L...>) {
    const float djj = __shfl_sync(tm, a[J], J, TL); // the same on every lane of the team
    ok = ok && djj > 0.0f;
    const float ljj = sqrtf(djj);
    const float r = 1.0f / ljj;
    if (i == J) {
        a[J] = ljj;
        rinv = r;
    } else if (i > J) {
        a[J] *= r;
    }
    (chol_row_update<ND, TL, J, L>(a, i, tm), ...);
}
template <int ND, int TL, int... J>
__device__ __forceinline__ void chol_rows(float (&a)[ND], int i, float& rinv, bool& ok, unsigned tm,
                                          std::integer_sequence<int, J...>) {
    (chol_row_step<ND, TL, J>(a, i, rinv, ok, tm, std::make_integer_sequence<int, ND - J - 1>{}),
     ...);
}

// FP32 copy of M_(a,b),(c,d) = sum c_{al,be} Bm[al][a] Bm[al][c] Bm[be][b] Bm[be][d],
// assembled and Cholesky-factored with one row per lane (ND <= TL).  The
// weights cw are converted once (conversions run on the FP64 pipe: converting
// inside the sums would cost one per term); lane i forms the lower part of
// row i of M from the FP32 basis table, the factor's column updates take the
// pivot column from the other lanes by shuffles, and L is stored by rows in
// Mf (lrow_idx).  The lane's reciprocal pivot 1/L_ii comes back in rinv.
// Returns false on a non-positive pivot.
template <int ND1, int NM, int TL>
__device__ bool mass_factor_rows_f(const Tables& tb, const double* cw, float* Y, float* Mf,
                                   float& rinv, int lane, unsigned tm) {
    constexpr int ND = ND1 * ND1;
    static_assert(ND <= TL, "one row per lane");
    static_assert(NM * NM <= ND * ND, "the weights are staged in Mf");
    float* cwf = Mf; // Mf is written only once the factor is done
    for (int p = lane; p < NM * NM; p += TL) cwf[p] = (float)cw[p];
    __syncwarp(tm);
    for (int i = lane; i < ND1 * ND1 * NM; i += TL) {
        const int a = i / (ND1 * NM), r_ = i % (ND1 * NM), c = r_ / NM, be = r_ % NM;
        float s = 0.0f;
#pragma unroll
        for (int al = 0; al < NM; ++al) s += cwf[al + NM * be] * tb.BmF[al][a] * tb.BmF[al][c];
        Y[i] = s;
    }
    __syncwarp(tm);
    // lanes past the last row repeat it and store nothing
    const int i = lane < ND ? lane : ND - 1;
    const int ar = i % ND1, br = i / ND1;
    float bb[NM];
#pragma unroll
    for (int be = 0; be < NM; ++be) bb[be] = tb.BmF[be][br];
    float a[ND];
#pragma unroll
    for (int t = 0; t < ND; ++t) {
        float s = 0.0f;
#pragma unroll
        for (int be = 0; be < NM; ++be)
            s += Y[(ar * ND1 + t % ND1) * NM + be] * bb[be] * tb.BmF[be][t / ND1];
        a[t] = s;
    }
    bool ok = true;
    rinv = 0.0f;
    chol_rows<ND, TL>(a, i, rinv, ok, tm, std::make_integer_sequence<int, ND>{});
    if (ok && lane < ND) {
#pragma unroll
        for (int t = 0; t < ND; ++t)
            if (t <= i) Mf[lrow_idx<ND>(i, t)] = a[t];
    }
    __syncwarp(tm);
    return ok;
}

// (L L^T)^-1 b in FP32 with the factor of mass_factor_rows_f: lane i brings
// b_i and gets x_i; the solved component of each step is passed by a
// shuffle (forward, then backward substitution, column by column).
template <int ND, int TL>
__device__ __forceinline__ float chol_subst_rows_f(const float* Mf, float rinv, float bv, int lane,
                                                   unsigned tm) {
    const int i = lane < ND ? lane : ND - 1;
    float lr[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) lr[j] = j < i ? Mf[lrow_idx<ND>(i, j)] : 0.0f; // row i of L
#pragma unroll
    for (int j = 0; j < ND; ++j) { // L y = b
        const float yj = __shfl_sync(tm, bv * rinv, j, TL);
        if (i == j) bv = yj;
        else if (i > j) bv -= lr[j] * yj;
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) lr[j] = j > i ? Mf[lrow_idx<ND>(j, i)] : 0.0f; // column i of L
#pragma unroll
    for (int j = ND - 1; j >= 0; --j) { // L^T x = y
        const float xj = __shfl_sync(tm, bv * rinv, j, TL);
        if (i == j) bv = xj;
        else if (i < j) bv -= lr[j] * xj;
    }
    return bv;
}

// Solve H x = b for the depth-weighted mass matrix H = B^T diag(cw) B (the
// tracer matrix of Eq. mass_matrix_concentration, or the masked Jacobian of
// Eq. mass_matrix) by mixed-precision iterative refinement: H is assembled and
// factored in FP32, each correction is solved in FP32, and the residual
// b - H x is formed in FP64 matrix-free by sum factorisation.  The sweeps stop
// when a correction, or the next one as predicted from the contraction of
// the last two, is below 1e-15 of x; if that does not happen within 6 sweeps
// (an ill-conditioned near-dry cell), the FP64 Cholesky decides.  x (FP64, in place of b on
// return).  Scratch: Mf [ND ND], Yf [ND1 ND1 NM] (float), x, r (ND doubles),
// q (NMP doubles), tmp (2 NM NM doubles), M, Y, inv (double, fallback).
template <int ND1, int NM, int TL = 32>
__device__ bool solve_mass_mixed(const Tables& tb, const double* cw, double* b, float* Mf,
                                 float* Yf, double* x, double* r, double* q, double* tmp,
                                 double* M, double* Y, double* inv, int lane,
                                 unsigned tm = 0xffffffffu) {
    constexpr int ND = ND1 * ND1, NMP = NM * NM;
    static_assert(ND <= TL, "one unknown per lane");
    float rinv; // the lane's reciprocal FP32 pivot
    bool ok = mass_factor_rows_f<ND1, NM, TL>(tb, cw, Yf, Mf, rinv, lane, tm);
    if (ok) {
        for (int i = lane; i < ND; i += TL) {
            x[i] = 0.0;
            r[i] = b[i];
        }
        __syncwarp(tm);
        ok = false;
        double dprev = 0.0; // max |correction| of the previous sweep
        for (int sweep = 0; sweep < 6; ++sweep) {
            // the lane's component of the correction
            const float v =
                chol_subst_rows_f<ND, TL>(Mf, rinv, lane < ND ? (float)r[lane] : 0.0f, lane, tm);
            // max |correction| and max |x| (a NaN counts as 0, as under fmax),
            // reduced on their bit patterns
            float da = 0.0f;
            double xa = 0.0;
            if (lane < ND) {
                x[lane] += (double)v;
                da = (v == v) ? fabsf(v) : 0.0f;
                const unsigned long long xb =
                    (unsigned long long)__double_as_longlong(x[lane]) & 0x7fffffffffffffffull;
                xa = __longlong_as_double((long long)(xb > 0x7ff0000000000000ull ? 0ull : xb));
            }
            const double dmax = (double)team_max_nonneg(da, tm);
            const double xmax = team_max_nonneg(xa, tm);
            // converged when this correction is below 1e-15 of x, or when the
            // next one is, as predicted from the contraction of the last two
            // (dmax / dprev, at most 1/2)
            const bool next_small =
                sweep > 0 && dmax <= 0.5 * dprev && dmax * dmax <= 1e-15 * xmax * dprev;
            if (!(dmax <= 1e-15 * xmax) && !(dmax == 0.0) && !next_small) {
                dprev = dmax;
                // r = b - H x, H x = B^T (cw * (B x))
                __syncwarp(tm);
                tens_interp<ND1, NM, double, TL>(tb.Bm, x, tmp, q, lane, tm);
                for (int p = lane; p < NMP; p += TL) q[p] *= cw[p];
                __syncwarp(tm);
                tens_test<ND1, NM, double, TL>(tb.Bm, q, tmp, r, lane, tm);
                for (int i = lane; i < ND; i += TL) r[i] = b[i] - r[i];
                __syncwarp(tm);
            } else {
                ok = true;
                break;
            }
        }
    }
    if (ok) {
        for (int i = lane; i < ND; i += TL) b[i] = x[i];
        __syncwarp(tm);
        return true;
    }
    assemble_mass<ND1, NM, TL>(tb, cw, Y, M, lane, tm);
    return chol_solve<ND, TL>(M, b, inv, lane, tm);
}

// Tracer stage solve of the FP32-bulk path (Eq. algebraic_concentration,
// H(zeta^(l)) C = b with the depth-weighted mass matrix H = B^T diag(cw) B):
// C = c0 + delta, where c0 = sum_i b_i / sum_i s_i is the cell's mean
// concentration (s = H 1, the row sums of H, i.e. H_i(zeta^(l)) of the
// continuity equation, in FP64), delta = H^-1 (b - c0 s) is solved once in
// FP32 (FP32 factor of mass_factor_rows_f), and a constant correction makes
// sum_i (H C)_i = sum_i s_i C_i equal sum_i b_i in FP64, so the tracer mass
// is kept to FP64 round-off and a constant tracer (b = c s) stays constant up
// to the rounding of b - c0 s.  A failed FP32 factor falls back to the FP64
// Cholesky.  b: right-hand side in, C out (FP64).  Scratch: Mf, Yf (float),
// s (ND doubles), tmp (2 NM NM doubles), M, Y, inv (fallback).  s_known: the
// continuity target T when the Newton solve ended on its certificate (H is
// affine between the last two iterates, so H(zeta^(l)) = T up to the
// rounding of the last update): it stands for s = H 1 = H(zeta^(l)); null:
// s is integrated from cw.
template <int ND1, int NM, int TL>
__device__ void solve_tracer_bulk(const Tables& tb, const double* cw, double* b, float* Mf,
                                  float* Yf, double* s, double* tmp, double* M, double* Y,
                                  double* inv, const double* s_known, int lane, unsigned tm) {
    constexpr int ND = ND1 * ND1;
    static_assert(ND <= TL, "one unknown per lane");
    float rinv;
    if (!mass_factor_rows_f<ND1, NM, TL>(tb, cw, Yf, Mf, rinv, lane, tm)) {
        assemble_mass<ND1, NM, TL>(tb, cw, Y, M, lane, tm);
        chol_solve<ND1 * ND1, TL>(M, b, inv, lane, tm);
        return;
    }
    if (s_known == nullptr) tens_test<ND1, NM, double, TL>(tb.Bm, cw, tmp, s, lane, tm); // s_i = (H 1)_i
    const double* sv = s_known ? s_known : s;
    const double bi = lane < ND ? b[lane] : 0.0, si = lane < ND ? sv[lane] : 0.0;
    double sb = bi, ss = si;
    team_sum2<TL>(sb, ss, tm);
    const double c0 = ss > 0.0 ? sb / ss : 0.0;
    const float v = chol_subst_rows_f<ND, TL>(Mf, rinv, (float)(bi - c0 * si), lane, tm);
    const double xi = lane < ND ? c0 + (double)v : 0.0;
    const double m = team_sum<TL>(si * xi, tm);
    const double alpha = ss > 0.0 ? (sb - m) / ss : 0.0;
    __syncwarp(tm);
    if (lane < ND) b[lane] = xi + alpha;
    __syncwarp(tm);
}

// Momentum stage solve of an r_K = r cell in arithmetic T (Eq. algebraic_discharge
// with the friction-modified mass matrix of Eq. mass_matrix_discharge on the
// (r+1)^2 Gauss-Legendre points, inverted as S^-1 D^-1 S^-T):
//   S Q = [D0 q^n + S^-T rq] / D,  D = D0 (1 + add dt gamma),  D0 = J w.
// gamma (of the previous stage) is formed here from prev (zeta in FP64 for the
// sub-grid depth, q in T).  Optionally the linearised friction term
// Llin = -S^T (J w gamma S Q).  Inputs su (v^n, FP64), rq [2][ND] (FP64);
// outputs Q [2][ND] (FP64) and llin [2][ND] (FP64).
template <int R, typename Pix, int MODE, typename T, int TL = 32>
__device__ void momentum_block(const Dev& d, const Tables& tb, int64_t k, double J, double man,
                               double dt, double add, bool need_gam, bool make_llin, int prev_buf,
                               const double* su, unsigned cm0, const double* rq, T* w0, T* w1,
                               T* pts, double* zp, double* tmpd, double* Q, double* llin, int lane,
                               unsigned tm = 0xffffffffu) {
    using S = Sz<R>;
    constexpr int ND1 = S::ND1, ND = S::ND, NG = S::NG, NGP = S::NGP;
    const auto Bg = tab_or<T>(tb.Bg, tb.BgF);
    const T(*Bginv)[MXP] = nullptr;
    if constexpr (sizeof(T) == sizeof(double)) Bginv = (const T(*)[MXP])tb.Bginv;
    else Bginv = (const T(*)[MXP])tb.BginvF;
    // w0: [2][ND] nodal pair; w1: [2][ND1 NG] tmp pair; pts: [6][NGP] point
    // arrays.  The two discharge components are contracted side by side.
    T* nod = w0;              // [2][ND]
    T* pg = pts;              // [6][NGP]: 0,1 S^-T rq / point values; 2 gamma; 3,4 q^n; 5 spare
    T* tmp = w1;
    T* tmp1 = w1 + ND1 * NG;
    T* gam = pg + 2 * NGP;
    const int64_t n = d.n;
    constexpr bool F64 = sizeof(T) == sizeof(double);
    // per-cell values in T: for T = float converted once per team (lanes
    // 0..4), since conversions occupy the FP64 pipe
    T JT, manT, gT, epsT, adtT;
    if constexpr (F64) {
        JT = J;
        manT = man;
        gT = d.g;
        epsT = d.eps;
        adtT = add * dt;
    } else {
        const int q = lane < 5 ? lane : 0;
        const float f = (float)(q == 0 ? J : q == 1 ? man : q == 2 ? d.g : q == 3 ? d.eps : add * dt);
        JT = __shfl_sync(tm, f, 0, TL);
        manT = __shfl_sync(tm, f, 1, TL);
        gT = __shfl_sync(tm, f, 2, TL);
        epsT = __shfl_sync(tm, f, 3, TL);
        adtT = __shfl_sync(tm, f, 4, TL);
    }
    // the quadrature weight of momentum point p (T = float: FP32 weights)
    auto wpt = [&](int p) -> T {
        if constexpr (F64) return J * tb.wg[p % NG] * tb.wg[p / NG];
        else return JT * tb.wgF[p % NG] * tb.wgF[p / NG];
    };
    if (need_gam) {
        const unsigned cmp = d.cmask[(size_t)prev_buf * n + k];
        const double* uz = ufield(d, prev_buf, 0, ND) + k * ND;
        tens_interp<ND1, NG, double, TL>(tb.Bg, uz, tmpd, zp, lane, tm); // zeta of v^(l-1), FP64
        if (cmp & 1u)
            for (int p = lane; p < NGP; p += TL) zp[p] = uz[0];
        const double* up0 = ufield(d, prev_buf, 1, ND) + k * ND;
        const double* up1 = ufield(d, prev_buf, 2, ND) + k * ND;
        for (int i = lane; i < 2 * ND; i += TL) nod[i] = (T)(i < ND ? up0[i] : up1[i - ND]);
        __syncwarp(tm);
        tens_interp2<ND1, NG, T, TL>(Bg, nod, nod + ND, tmp, tmp1, pg + 3 * NGP, pg + 4 * NGP, lane, tm);
        if (cmp & 2u)
            for (int p = lane; p < NGP; p += TL) pg[3 * NGP + p] = (T)up0[0];
        if (cmp & 4u)
            for (int p = lane; p < NGP; p += TL) pg[4 * NGP + p] = (T)up1[0];
        __syncwarp(tm);
        for (int p = lane; p < NGP; p += TL) {
            double V, A;
            Site<R, Pix, MODE>::VA(d, tb, k, SET_MOM, p % NG, p / NG, zp[p], V, A);
            gam[p] = gamma_manning<T>(manT, (T)V, pg[3 * NGP + p], pg[4 * NGP + p], gT, epsT);
        }
    } else {
        for (int p = lane; p < NGP; p += TL) gam[p] = T(0);
    }
    __syncwarp(tm);
    if (F64 && d.qpts != nullptr) { // q^n at the points, from the step start
        for (int p = lane; p < 2 * NGP; p += TL) pg[3 * NGP + p] = (T)d.qpts[k * 2 * NGP + p];
    } else {
        for (int i = lane; i < 2 * ND; i += TL) nod[i] = (T)su[ND + i];
        __syncwarp(tm);
        tens_interp2<ND1, NG, T, TL>(Bg, nod, nod + ND, tmp, tmp1, pg + 3 * NGP, pg + 4 * NGP, lane,
                                     tm);
        if (cm0 & 2u)
            for (int p = lane; p < NGP; p += TL) pg[3 * NGP + p] = (T)su[ND];
        if (cm0 & 4u)
            for (int p = lane; p < NGP; p += TL) pg[4 * NGP + p] = (T)su[2 * ND];
    }
    for (int i = lane; i < 2 * ND; i += TL) nod[i] = (T)rq[i];
    __syncwarp(tm);
    kron_apply2<ND1, true, MXP, T, TL>(Bginv, nod, nod + ND, tmp, tmp1, pg, pg + NGP, T(1), lane, tm);
    for (int p = lane; p < NGP; p += TL) {
        const T w = wpt(p);
        const T rD = T(1) / (w * (T(1) + adtT * gam[p]));
        pg[0 * NGP + p] = (w * pg[3 * NGP + p] + pg[0 * NGP + p]) * rD;
        pg[1 * NGP + p] = (w * pg[4 * NGP + p] + pg[1 * NGP + p]) * rD;
    }
    __syncwarp(tm);
    kron_apply2<ND1, false, MXP, T, TL>(Bginv, pg, pg + NGP, tmp, tmp1, nod, nod + ND, T(1), lane, tm);
    for (int i = lane; i < 2 * ND; i += TL) Q[i] = (double)nod[i];
    __syncwarp(tm);
    if (make_llin) {
        for (int p = lane; p < NGP; p += TL) {
            const T w = wpt(p) * gam[p];
            pg[3 * NGP + p] = -w * pg[p];
            pg[4 * NGP + p] = -w * pg[NGP + p];
        }
        __syncwarp(tm);
        tens_test2<ND1, NG, T, TL>(Bg, pg + 3 * NGP, pg + 4 * NGP, tmp, tmp1, nod, nod + ND, lane, tm);
        for (int i = lane; i < 2 * ND; i += TL) llin[i] = (double)nod[i];
        __syncwarp(tm);
    }
}

template <int R, typename Pix, int MODE, typename B>
__global__ void __maxnreg__(96)
    k_stage(const __grid_constant__ Dev d, const __grid_constant__ Tables tb,
            const __grid_constant__ StageArgs sa) {
    using S = Sz<R>;
    using ST = Site<R, Pix, MODE>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP, NG = S::NG, NGP = S::NGP;
    extern __shared__ double smem[];
    // two cells per warp, one per team of 16 lanes (a cell's loops run over 16
    // nodes and 16 momentum points): "warp" is the team within the block,
    // "lane" the lane within the team, wpb the teams per block
    constexpr int TL = 16;
    const int warp = threadIdx.x / TL, lane = threadIdx.x % TL, wpb = blockDim.x / TL;
    const unsigned tm = 0xFFFFu << (threadIdx.x & 16); // the team's lanes
    double* su = smem + warp * stage_smem<R>(); // [4][ND] state v^n
    double* T = su + 4 * ND;                    // [ND]
    double* rq = T + ND;                        // [2][ND]
    double* rc = rq + 2 * ND;                   // [ND]
    double* z = rc + ND;                        // [ND] Newton iterate
    double* pe = z + ND;                        // [NMP]
    double* pV = pe + NMP;                      // [NMP]
    double* pA = pV + NMP;                      // [NMP]
    double* tmp = pA + NMP;                     // [2 NM NM]
    double* xs = tmp + 2 * NM * NM;             // [ND] refinement iterate (also scratch [2 ND]
    double* rs = xs + ND;                       // [ND] refinement residual   with rs outside a solve)
    double* o = rs + ND;                        // [4][ND]
    // the refinement's q [NMP] is pe, idle inside a solve (pe holds the
    // interpolated iterate only while V and A are evaluated)
    double* qs = pe;
    // the last region: friction points pg (the scalar path's; the momentum
    // block's point arrays on the other path) with the momentum scratch, or
    // the FP32 solve's arrays, or the FP64 fallback's M.  The momentum block
    // runs between the two solves; the fallback runs only inside a solve, when
    // the FP32 arrays are given up, and its Y and pivots take tmp, x, r and q,
    // which are idle then.
    double* un = o + 4 * ND;
    double* pg = un;                            // [6][NGP]
    double* mw = pg + 6 * NGP;                  // momentum nodal pair [2 ND] (B)
    double* mt = mw + 2 * ND;                   // momentum tmp pair [2 ND1 NG] (B)
    float* Mf = (float*)un;                     // [ND ND]
    float* Yf = Mf + ND * ND;                   // [ND1 ND1 NM]
    double* M = un;                             // [ND ND] (fallback)
    double* Y = tmp;                            // [ND1 ND1 NM] (fallback)
    double* pinv = qs;                          // [ND] (fallback)
    const int64_t n = d.n;
    const double g = d.g, eps = d.eps;
    int its_max = 0;
    int viol = 0, fb = 0, bad = 0;

    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < n; k += (int64_t)gridDim.x * wpb) {
        for (int i = lane; i < 4 * ND; i += TL) su[i] = ufield(d, 0, i / ND, ND)[k * ND + (i % ND)];
        const unsigned cm0 = d.cmask[k];
        const double hx = d.hxhy[2 * k], hy = d.hxhy[2 * k + 1], J = hx * hy;
        const double man = d.manning[k];
        int flag = d.flag[k];
        const double dt = get_dt(d, member_of(d, k)); // the member's step
        // right-hand sides of Eqs. algebraic_elevation, algebraic_discharge, algebraic_concentration
        double tsum = 0.0;
        for (int i = lane; i < ND; i += TL) {
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
        const double Tbar = d.HNbar[k] + team_sum<TL>(tsum, tm);
        if (Tbar < 0.0) viol++;
        bool scalar = (flag == 0);
        int its = 0;
        __syncwarp(tm);
        bool cert = false; // the Newton solve ended on its one-step certificate
        if (!scalar) {
            for (int i = lane; i < ND; i += TL) z[i] = su[i];
            bool zc = (cm0 & 1u) != 0;
            bool prev_full = false;
            // every mass point fully wet at zeta^n (known from the step start,
            // which evaluated H(zeta^n) = HN from the same state by the same
            // arithmetic): the first Newton step needs no evaluation, since
            // H(zeta^n) - T = HN - T and M(zeta^n) is the constant mass matrix
            const bool full0 = d.wet0 != nullptr && d.wet0[k] != 0 && d.newton_max > 0;
            __syncwarp(tm);
            // each pass evaluates V, A at the current iterate; the last pass is
            // the evaluation at the result (for the tracer matrix and the
            // completely-dry test)
            for (int kk = 0;; ++kk) {
                int ndry = 0, npart = 0;
                if (kk == 0 && full0) {
                    for (int i = lane; i < ND; i += TL) o[i] = d.HN[k * ND + i] - T[i];
                } else {
                tens_interp<ND1, NM, double, TL>(tb.Bm, z, tmp, pe, lane, tm);
                for (int p = lane; p < NMP; p += TL) {
                    if (zc) pe[p] = z[0];
                    double V, A;
                    bool full;
                    ST::VA(d, tb, k, SET_MASS, p % NM, p / NM, pe[p], V, A, full);
                    pV[p] = J * tb.wm[p % NM] * tb.wm[p / NM] * V;
                    pA[p] = J * tb.wm[p % NM] * tb.wm[p / NM] * A;
                    if (zero_bits(A)) ndry++;
                    else if (!full) npart++;
                }
                ndry = __reduce_add_sync(tm, ndry);
                npart = __reduce_add_sync(tm, npart);
                if (ndry) { scalar = true; break; }
                // every pixel wet at the previous and at this iterate: H is affine
                // on the segment between them and M(previous) is its exact
                // Jacobian, so this iterate solves H = T (the fully wet case of
                // Sec. 3.4); no verification step is needed
                if (kk > 0 && prev_full && npart == 0) {
                    cert = true;
                    break;
                }
                if (kk == d.newton_max) break;
                __syncwarp(tm);
                tens_test<ND1, NM, double, TL>(tb.Bm, pV, tmp, o, lane, tm); // H_i(zeta_k)
                for (int i = lane; i < ND; i += TL) o[i] -= T[i];
                }
                __syncwarp(tm);
                if (npart == 0) {
                    // M is the constant mass matrix, inverted by its tensor factors
                    kron_apply<ND1, false, MXN, double, TL>(tb.M1inv, o, tmp, o + ND, 1.0 / J, lane, tm);
                } else {
                    for (int i = lane; i < ND; i += TL) o[ND + i] = o[i];
                    __syncwarp(tm);
                    if (!solve_mass_mixed<ND1, NM, TL>(tb, pA, o + ND, Mf, Yf, xs, rs, qs,
                                                       tmp, M, Y, pinv, lane, tm)) {
                        scalar = true;
                        break;
                    }
                }
                double inc = 0.0, scale = 0.0;
                for (int i = lane; i < ND; i += TL) {
                    z[i] -= o[ND + i];
                    inc += fabs(o[ND + i]);
                    scale += 1.0 + fabs(z[i]) + d.zabs[k];
                }
                team_sum2<TL>(inc, scale, tm);
                its++;
                prev_full = (npart == 0);
                __syncwarp(tm);
                {
                    bool eq = true;
                    for (int i = lane; i < ND; i += TL) eq = eq && same_bits(z[i], z[0]);
                    zc = __all_sync(tm, eq);
                }
                if (inc <= d.newton_tol * scale) prev_full = false, kk = d.newton_max - 1;
            }
            if (scalar) {
                fb++;
                flag = 0;
                if (lane == 0) d.flag[k] = 0;
            }
            __syncwarp(tm);
        }
        // friction coefficient of the previous stage on the momentum GL points
        // (scalar path; the r path forms it inside momentum_block)
        double* gam = pg + 5 * NGP;
        const bool need_gam = (sa.add != 0.0 || sa.make_llin) && man != 0.0;
        if (need_gam && scalar) {
            const unsigned cmp = d.cmask[(size_t)sa.prev_buf * n + k];
            for (int f = 0; f < 3; ++f) {
                const double* up = ufield(d, sa.prev_buf, f, ND) + k * ND;
                if (cmp & (1u << f)) { // a constant field: its value at every point
                    const double v0 = up[0];
                    for (int p = lane; p < NGP; p += TL) pg[f * NGP + p] = v0;
                } else {
                    for (int i = lane; i < ND; i += TL) o[i] = up[i];
                    __syncwarp(tm);
                    tens_interp<ND1, NG, double, TL>(tb.Bg, o, tmp, pg + f * NGP, lane, tm);
                }
                __syncwarp(tm);
            }
            for (int p = lane; p < NGP; p += TL) {
                double V, A;
                ST::VA(d, tb, k, SET_MOM, p % NG, p / NG, pg[p], V, A);
                gam[p] = gamma_manning<double>(man, V, pg[NGP + p], pg[2 * NGP + p], g, eps);
            }
        } else {
            for (int p = lane; p < NGP; p += TL) gam[p] = 0.0;
        }
        __syncwarp(tm);
        if (scalar) {
            double e;
            if (cm0 & 1u) e = su[0];
            else {
                tens_interp<ND1, NM, double, TL>(tb.Bm, su, tmp, pe, lane, tm);
                double s = 0.0;
                for (int p = lane; p < NMP; p += TL) s += tb.wm[p % NM] * tb.wm[p / NM] * pe[p];
                e = team_sum<TL>(s, tm);
            }
            its = scalar_newton<R, Pix, MODE, TL>(d, tb, k, J, Tbar, e, lane, tm);
            // momentum: sums of the rows of the friction-modified mass matrix
            double den = 0.0, num[2] = {0.0, 0.0};
            if (d.qpts) {
                for (int p = lane; p < 2 * NGP; p += TL) pg[3 * NGP + p] = d.qpts[k * 2 * NGP + p];
                __syncwarp(tm);
            } else {
                for (int f = 0; f < 2; ++f) {
                    if (cm0 & (2u << f))
                        for (int p = lane; p < NGP; p += TL) pg[(3 + f) * NGP + p] = su[(1 + f) * ND];
                    else
                        tens_interp<ND1, NG, double, TL>(tb.Bg, su + (1 + f) * ND, tmp,
                                                         pg + (3 + f) * NGP, lane, tm);
                    __syncwarp(tm);
                }
            }
            for (int p = lane; p < NGP; p += TL) {
                const double w = J * tb.wg[p % NG] * tb.wg[p / NG];
                den += w * (1.0 + sa.add * dt * gam[p]);
                num[0] += w * pg[3 * NGP + p];
                num[1] += w * pg[4 * NGP + p];
            }
            double rs0 = 0.0, rs1 = 0.0, rcs = 0.0;
            for (int i = lane; i < ND; i += TL) {
                rs0 += rq[i];
                rs1 += rq[ND + i];
                rcs += rc[i] - d.CN[k * ND + i];
            }
            team_sum2<TL>(den, rcs, tm);
            team_sum2<TL>(num[0], rs0, tm);
            team_sum2<TL>(num[1], rs1, tm);
            const double qxn = (num[0] + rs0) / den;
            const double qyn = (num[1] + rs1) / den;
            double Hs, As;
            mass_scalar_pixels<R, Pix, MODE, TL>(d, tb, k, J, e, lane, Hs, As, tm);
            const bool tr_ok = Hs > 1e-14 * J * d.hlim;
            const double cn = tr_ok ? (d.CNbar[k] + rcs) / Hs : 0.0;
            for (int i = lane; i < ND; i += TL) {
                o[i] = e;
                o[ND + i] = qxn;
                o[2 * ND + i] = qyn;
                o[3 * ND + i] = tr_ok ? cn : su[3 * ND + i];
            }
            __syncwarp(tm);
            if (sa.make_llin) {
                for (int p = lane; p < NGP; p += TL) {
                    const double w = J * tb.wg[p % NG] * tb.wg[p / NG] * gam[p];
                    pg[3 * NGP + p] = -w * qxn;
                    pg[4 * NGP + p] = -w * qyn;
                }
                __syncwarp(tm);
                tens_test<ND1, NG, double, TL>(tb.Bg, pg + 3 * NGP, tmp, xs, lane, tm);
                tens_test<ND1, NG, double, TL>(tb.Bg, pg + 4 * NGP, tmp, rs, lane, tm);
                for (int i = lane; i < ND; i += TL) {
                    d.llin[(size_t)k * ND + i] = xs[i];
                    d.llin[(size_t)n * ND + (size_t)k * ND + i] = xs[ND + i];
                }
            }
        } else {
            // momentum (FP64, or FP32 in the FP32-bulk path)
            momentum_block<R, Pix, MODE, B, TL>(d, tb, k, J, man, dt, sa.add, need_gam, sa.make_llin != 0,
                                            sa.prev_buf, su, cm0, rq, (B*)mw, (B*)mt, (B*)pg, pe, tmp,
                                            o + ND,
                                            xs, lane, tm);
            if (sa.make_llin) {
                for (int i = lane; i < ND; i += TL) {
                    d.llin[(size_t)k * ND + i] = xs[i];
                    d.llin[(size_t)n * ND + (size_t)k * ND + i] = xs[ND + i];
                }
                __syncwarp(tm);
            }
            // tracer: H(zeta^(l)) C = C~ + dt sum a R with the depth-weighted mass matrix
            for (int i = lane; i < ND; i += TL) {
                o[i] = z[i];
                o[3 * ND + i] = rc[i];
            }
            __syncwarp(tm);
            if constexpr (sizeof(B) == sizeof(float))
                solve_tracer_bulk<ND1, NM, TL>(tb, pV, o + 3 * ND, Mf, Yf, xs, tmp, M, Y, pinv,
                                               cert ? T : nullptr, lane, tm);
            else
                solve_mass_mixed<ND1, NM, TL>(tb, pV, o + 3 * ND, Mf, Yf, xs, rs, qs, tmp, M,
                                              Y, pinv, lane, tm);
        }
        __syncwarp(tm);
        // write v^(l) and its constant-field mask
        unsigned cmo = 0;
        for (int f = 0; f < 4; ++f) {
            bool eq = true;
            for (int i = lane; i < ND; i += TL) eq = eq && same_bits(o[f * ND + i], o[f * ND]);
            if (__all_sync(tm, eq)) cmo |= (1u << f);
        }
        bool fin = true;
        for (int i = lane; i < 4 * ND; i += TL) {
            const double v = o[i];
            fin = fin && finite_bits(v);
            ufield(d, sa.out_buf, i / ND, ND)[k * ND + (i % ND)] = v;
            if (d.uF) ufieldF(d, sa.out_buf, i / ND, ND)[k * ND + (i % ND)] = (float)v;
        }
        if (!__all_sync(tm, fin)) bad = 1;
        if (lane == 0) d.cmask[(size_t)sa.out_buf * n + k] = (uint8_t)cmo;
        its_max = max(its_max, its);
        __syncwarp(tm);
    }
    if (lane == 0) {
        if (its_max) atomicMax(&d.sc->maxits, its_max);
        if (viol) atomicAdd(&d.sc->viol, viol);
        if (fb) atomicAdd(&d.sc->fallback, fb);
        if (bad) atomicOr(&d.sc->status, ST_NAN);
    }
    if (sa.final_ && blockIdx.x == 0) {
        // every member advances by its own step (rmax is not written here)
        for (int i = threadIdx.x; i < d.nmemb; i += blockDim.x) {
            const double dti = get_dt(d, i);
            d.mb[i].dt_last = dti;
            d.mb[i].t = d.mb[i].t + dti;
        }
    }
}

// ---------------------------------------------------------------------------
// constant-field masks of a state buffer
// ---------------------------------------------------------------------------
template <int R>
__global__ void k_masks(const __grid_constant__ Dev d, int buf) {
    constexpr int ND = Sz<R>::ND;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < d.n; k += (int64_t)gridDim.x * wpb) {
        unsigned cm = 0;
        for (int f = 0; f < 4; ++f) {
            const double* u = ufield(d, buf, f, ND) + k * ND;
            bool eq = true;
            for (int i = lane; i < ND; i += 32) eq = eq && same_bits(u[i], u[0]);
            if (__all_sync(0xffffffffu, eq)) cm |= (1u << f);
            if (d.uF)
                for (int i = lane; i < ND; i += 32) ufieldF(d, buf, f, ND)[k * ND + i] = (float)u[i];
        }
        if (lane == 0) d.cmask[(size_t)buf * d.n + k] = (uint8_t)cm;
    }
}

// ---------------------------------------------------------------------------
// diagnostics: per-cell wet mass (Eq. positivity-7), tracer mass, min depth
// ---------------------------------------------------------------------------
template <int R, typename Pix, int MODE>
__global__ void __launch_bounds__(32 * MAXWPB)
    k_cell_diag(const __grid_constant__ Dev d, const __grid_constant__ Tables tb, double* part) {
    using S = Sz<R>;
    constexpr int ND1 = S::ND1, ND = S::ND, NM = S::NM, NMP = S::NMP;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double* su = smem + warp * (2 * ND + 2 * NMP + 2 * NM * NM);
    double* pe = su + 2 * ND;
    double* pc = pe + NMP;
    double* tmp = pc + NMP;
    for (int64_t k = (int64_t)blockIdx.x * wpb + warp; k < d.n; k += (int64_t)gridDim.x * wpb) {
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
                         const double* xy, double* out, int64_t k0, int64_t k1,
                         const int32_t* cell) {
    constexpr int ND1 = R + 1, ND = ND1 * ND1;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    const double x = xy[2 * gi], y = xy[2 * gi + 1];
    double v = NAN;
    // the cells searched: [k0, k1), or only the one located on the host (cell[gi], -1: none)
    if (cell) {
        k0 = cell[gi];
        k1 = k0 < 0 ? k0 : k0 + 1;
    }
    for (int64_t k = k0; k < k1; ++k) {
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
