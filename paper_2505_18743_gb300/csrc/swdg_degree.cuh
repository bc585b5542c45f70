// swdg_degree.cuh -- launchers of one polynomial degree (included once by each
// swdg_r{1,2,3}.cu with SWDG_DEGREE defined).
#pragma once
#include "swdg_kernels.cuh"
#include "swdg_launch.h"

namespace swdg {

template <int R, typename Pix, int MODE, typename B>
struct Launchers {
    static void residual(const Dev& d, const Tables& tb, int buf, int stage, double c_stage,
                         int want_dt, int grid, cudaStream_t st) {
        size_t sm = sizeof(double) * res_smem<R, B>() * WPB;
        k_residual<R, Pix, MODE, B><<<grid, TPB, sm, st>>>(d, tb, buf, stage, c_stage, want_dt);
    }
    static void step_begin(const Dev& d, const Tables& tb, int do_switch, int grid, cudaStream_t st) {
        size_t sm = sizeof(double) * begin_smem<R>() * WPB;
        k_step_begin<R, Pix, MODE><<<grid, TPB, sm, st>>>(d, tb, do_switch);
    }
    static void stage(const Dev& d, const Tables& tb, const StageArgs& sa, int grid, cudaStream_t st) {
        size_t sm = sizeof(double) * stage_smem<R>() * WPB;
        k_stage<R, Pix, MODE, B><<<grid, TPB, sm, st>>>(d, tb, sa);
    }
    static void masks(const Dev& d, int buf, int grid, cudaStream_t st) {
        k_masks<R><<<grid, TPB, 0, st>>>(d, buf);
    }
    static void cell_diag(const Dev& d, const Tables& tb, double* part, int grid, cudaStream_t st) {
        using S = Sz<R>;
        size_t sm = sizeof(double) * (2 * S::ND + 2 * S::NMP + 2 * S::NM * S::NM) * WPB;
        k_cell_diag<R, Pix, MODE><<<grid, TPB, sm, st>>>(d, tb, part);
    }
    static void gauges(const Dev& d, const Tables& tb, int ng, const double* xy, double* out,
                       cudaStream_t st) {
        k_gauges<R><<<(ng + 63) / 64, 64, 0, st>>>(d, tb, ng, xy, out);
    }
    static void fill(Launch* L) {
        L->residual = &residual;
        L->step_begin = &step_begin;
        L->stage = &stage;
        L->masks = &masks;
        L->cell_diag = &cell_diag;
        L->gauges = &gauges;
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
