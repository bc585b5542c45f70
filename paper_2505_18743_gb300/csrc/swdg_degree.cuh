// swdg_degree.cuh -- launchers of one polynomial degree (included once by each
// swdg_r{1,2,3}.cu with SWDG_DEGREE defined).
#pragma once
#include "swdg_adjoint.cuh"
#include "swdg_amr.cuh"
#include "swdg_kernels.cuh"
#include "swdg_launch.h"

namespace swdg {

template <int R, typename Pix, int MODE, typename B>
struct Launchers {
    using S = Sz<R>;
    static constexpr size_t res_b = sizeof(double) * res_smem<R, B>();   // per warp
    static constexpr size_t begin_b = sizeof(double) * begin_smem<R>();
    // k_stage runs two cells per warp (a team of 16 lanes each)
    static constexpr size_t stage_b = 2 * sizeof(double) * stage_smem<R>();
    static constexpr size_t diag_b = sizeof(double) * (2 * S::ND + 2 * S::NMP + 2 * S::NM * S::NM);
    static constexpr size_t vjp_b = sizeof(double) * vjp_smem<R>();
    static constexpr size_t svjp_b = 2 * sizeof(double) * stage_vjp_smem<R>(); // two cells per warp
    static constexpr size_t bvjp_b = sizeof(double) * begin_vjp_smem<R>();
    static constexpr size_t ind_b = sizeof(double) * indicator_smem<R>();
    static constexpr size_t remap_b = sizeof(double) * remap_smem<R>();

    static void residual(const Dev& d, const Tables& tb, int buf, int stage, double c_stage,
                         int want_dt, Shape s, cudaStream_t st) {
        k_residual<R, Pix, MODE, B><<<s.grid, 32 * s.wpb, res_b * s.wpb, st>>>(d, tb, buf, stage,
                                                                              c_stage, want_dt);
    }
    static void faces(const Dev& d, const Tables& tb, int buf, double c_stage, int want_dt,
                      cudaStream_t st) {
        if (d.njobs <= 0) return;
        const int64_t blocks = std::min<int64_t>((d.njobs + 255) / 256, 152 * 16);
        k_faces<R, Pix, MODE, B><<<(int)blocks, 256, 0, st>>>(d, tb, buf, c_stage, want_dt);
    }
    static void step_begin(const Dev& d, const Tables& tb, int do_switch, Shape s, cudaStream_t st) {
        k_step_begin<R, Pix, MODE><<<s.grid, 32 * s.wpb, begin_b * s.wpb, st>>>(d, tb, do_switch);
    }
    static void stage(const Dev& d, const Tables& tb, const StageArgs& sa, Shape s, cudaStream_t st) {
        // two cells per warp: no more blocks than 2 wpb cells each
        const int64_t need = (d.n + 2 * s.wpb - 1) / (2 * s.wpb);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(s.grid, need));
        k_stage<R, Pix, MODE, B><<<grid, 32 * s.wpb, stage_b * s.wpb, st>>>(d, tb, sa);
    }
    static void masks(const Dev& d, int buf, Shape s, cudaStream_t st) {
        k_masks<R><<<s.grid, 32 * s.wpb, 0, st>>>(d, buf);
    }
    static void cell_diag(const Dev& d, const Tables& tb, double* part, Shape s, cudaStream_t st) {
        k_cell_diag<R, Pix, MODE><<<s.grid, 32 * s.wpb, diag_b * s.wpb, st>>>(d, tb, part);
    }
    static void gauges(const Dev& d, const Tables& tb, int ng, const double* xy, double* out,
                       int64_t k0, int64_t k1, const int32_t* cell, cudaStream_t st) {
        k_gauges<R><<<(ng + 63) / 64, 64, 0, st>>>(d, tb, ng, xy, out, k0, k1, cell);
    }
    static void gauges_vjp(const Dev& d, const Tables& tb, int ng, const double* xy,
                           const double* gbar, double* zb, const int32_t* cell, cudaStream_t st) {
        k_gauges_vjp<R><<<(ng + 63) / 64, 64, 0, st>>>(d, tb, ng, xy, gbar, zb, cell);
    }
    static void residual_vjp(const Dev& d, const Tables& tb, const double* u, const uint8_t* cm,
                             const double* rbar, double* ubar, double* nbar, double* dbar,
                             int accumulate, Shape s, cudaStream_t st) {
        k_residual_vjp<R, Pix, MODE><<<s.grid, 32 * s.wpb, vjp_b * s.wpb, st>>>(
            d, tb, u, cm, rbar, ubar, nbar, dbar, accumulate);
    }
    static void stage_vjp(const Dev& d, const Tables& tb, const StageVjpArgs& a, Shape s,
                          cudaStream_t st) {
        const int64_t need = (d.n + 2 * s.wpb - 1) / (2 * s.wpb);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(s.grid, need));
        k_stage_vjp<R, Pix, MODE><<<grid, 32 * s.wpb, svjp_b * s.wpb, st>>>(d, tb, a);
    }
    static void begin_vjp(const Dev& d, const Tables& tb, const BeginVjpArgs& a, Shape s,
                          cudaStream_t st) {
        k_begin_vjp<R, Pix, MODE><<<s.grid, 32 * s.wpb, bvjp_b * s.wpb, st>>>(d, tb, a);
    }
    static void indicator(const Dev& d, const Tables& tb, int kind, double* eta, Shape s,
                          cudaStream_t st) {
        k_indicator<R, Pix, MODE><<<s.grid, 32 * s.wpb, ind_b * s.wpb, st>>>(d, tb, kind, eta);
    }
    static void remap(const Tables& tb, const RemapArgs& a, Shape s, cudaStream_t st) {
        k_remap<R><<<s.grid, 32 * s.wpb, remap_b * s.wpb, st>>>(tb, a);
    }
    template <typename K>
    static bool opt_in(K kern, size_t per_warp) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(per_warp * MAXWPB)) == cudaSuccess;
    }
    static bool prepare() {
        return opt_in(k_residual<R, Pix, MODE, B>, res_b) &&
               opt_in(k_step_begin<R, Pix, MODE>, begin_b) &&
               opt_in(k_stage<R, Pix, MODE, B>, stage_b) &&
               opt_in(k_cell_diag<R, Pix, MODE>, diag_b) &&
               opt_in(k_residual_vjp<R, Pix, MODE>, vjp_b) &&
               opt_in(k_stage_vjp<R, Pix, MODE>, svjp_b) &&
               opt_in(k_begin_vjp<R, Pix, MODE>, bvjp_b);
    }
    template <typename K>
    static int occ(K kern, int wpb, size_t per_warp) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * wpb, per_warp * wpb) !=
            cudaSuccess)
            return 0;
        return nb;
    }
    static int occupancy(int kind, int wpb) {
        if (wpb < 1 || wpb > MAXWPB) return 0;
        switch (kind) {
        case KK_BEGIN: return occ(k_step_begin<R, Pix, MODE>, wpb, begin_b);
        case KK_RESIDUAL: return occ(k_residual<R, Pix, MODE, B>, wpb, res_b);
        case KK_STAGE: return occ(k_stage<R, Pix, MODE, B>, wpb, stage_b);
        default: return occ(k_cell_diag<R, Pix, MODE>, wpb, diag_b);
        }
    }
    static void fill(Launch* L) {
        L->residual = &residual;
        L->faces = &faces;
        L->step_begin = &step_begin;
        L->stage = &stage;
        L->masks = &masks;
        L->cell_diag = &cell_diag;
        L->gauges = &gauges;
        L->gauges_vjp = &gauges_vjp;
        L->residual_vjp = &residual_vjp;
        L->stage_vjp = &stage_vjp;
        L->begin_vjp = &begin_vjp;
        L->indicator = &indicator;
        L->remap = &remap;
        L->prepare = &prepare;
        L->occupancy = &occupancy;
        L->nzp = Sz<R>::NZP;
    }
};

template <int R, typename B>
bool get_launch_prec(int mode, int pix, Launch* L) {
    if (mode == 1) Launchers<R, double, 1, B>::fill(L);
    else if (pix == 0) Launchers<R, float, 0, B>::fill(L);
    else if (pix == 1) Launchers<R, double, 0, B>::fill(L);
    else return false;
    return true;
}

// precision 0: FP64; 1: FP32-bulk residual arithmetic
template <int R>
bool get_launch_degree(int mode, int pix, int prec, Launch* L) {
    if (prec == 0) return get_launch_prec<R, double>(mode, pix, L);
    if (prec == 1) return get_launch_prec<R, float>(mode, pix, L);
    return false;
}

} // namespace swdg
