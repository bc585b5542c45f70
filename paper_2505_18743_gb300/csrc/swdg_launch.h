// swdg_launch.h -- per-degree launch table filled by the swdg_r{1,2,3}.cu
// translation units (compiled in parallel), used by swdg_api.cu.
#pragma once
#include "swdg_common.cuh"

namespace swdg {

struct StageArgs;
struct StageVjpArgs;
struct BeginVjpArgs;
struct RemapArgs;

// launch shape of one kernel: blocks and warps (cells in flight) per block
struct Shape {
    int grid, wpb;
};

// kernel kinds the autotuner shapes independently
enum { KK_BEGIN = 0, KK_RESIDUAL = 1, KK_STAGE = 2, KK_AUX = 3, KK_N = 4 };

struct Launch {
    void (*residual)(const Dev&, const Tables&, int buf, int stage, double c_stage, int want_dt,
                     Shape, cudaStream_t);
    // the face points of the residual, each once, into d.fflux (before residual)
    void (*faces)(const Dev&, const Tables&, int buf, double c_stage, int want_dt, cudaStream_t);
    void (*step_begin)(const Dev&, const Tables&, int do_switch, Shape, cudaStream_t);
    void (*stage)(const Dev&, const Tables&, const StageArgs&, Shape, cudaStream_t);
    void (*masks)(const Dev&, int buf, Shape, cudaStream_t);
    void (*cell_diag)(const Dev&, const Tables&, double* part, Shape, cudaStream_t);
    // zeta at gauge points (cell: the cell of each point, -1 none; null: search [k0, k1))
    void (*gauges)(const Dev&, const Tables&, int ng, const double* xy, double* out, int64_t k0,
                   int64_t k1, const int32_t* cell, cudaStream_t);
    // its transpose: zb [n][nd] += gbar [ng] times the interpolation weights
    void (*gauges_vjp)(const Dev&, const Tables&, int ng, const double* xy, const double* gbar,
                       double* zb, const int32_t* cell, cudaStream_t);
    // discrete adjoint of the residual (FP64): rbar [6][n][nd] -> ubar [4][n][nd],
    // nbar [n] (Manning), dbar [n] (bathymetry offset)
    void (*residual_vjp)(const Dev&, const Tables&, const double* u, const uint8_t* cmask,
                         const double* rbar, double* ubar, double* nbar, double* dbar,
                         int accumulate, Shape, cudaStream_t);
    // adjoints of a stage update / the final combination and of the step start (FP64)
    void (*stage_vjp)(const Dev&, const Tables&, const StageVjpArgs&, Shape, cudaStream_t);
    void (*begin_vjp)(const Dev&, const Tables&, const BeginVjpArgs&, Shape, cudaStream_t);
    // refinement indicator (kind 0 |curl u|, 1 |grad c|) and state remap (Sec. 3.4)
    void (*indicator)(const Dev&, const Tables&, int kind, double* eta, Shape, cudaStream_t);
    void (*remap)(const Tables&, const RemapArgs&, Shape, cudaStream_t);
    // opt every kernel in to the shared memory of MAXWPB warps; false on failure
    bool (*prepare)();
    // resident blocks per SM of kernel kind KK_* at wpb warps per block (0: cannot launch)
    int (*occupancy)(int kind, int wpb);
    int nzp; // mode P samples per cell
};

// mode: 0 S, 1 P; pix: 0 float32, 1 float64; prec: 0 FP64, 1 FP32-bulk
bool get_launch(int degree, int mode, int pix, int prec, Launch* out);
bool get_launch_r1(int mode, int pix, int prec, Launch* out);
bool get_launch_r2(int mode, int pix, int prec, Launch* out);
bool get_launch_r3(int mode, int pix, int prec, Launch* out);

} // namespace swdg
