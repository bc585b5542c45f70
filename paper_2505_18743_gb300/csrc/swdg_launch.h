// swdg_launch.h -- per-degree launch table filled by the swdg_r{1,2,3}.cu
// translation units (compiled in parallel), used by swdg_api.cu.
#pragma once
#include "swdg_common.cuh"

namespace swdg {

struct StageArgs;

struct Launch {
    void (*residual)(const Dev&, const Tables&, int buf, int stage, double c_stage, int want_dt,
                     int grid, cudaStream_t);
    void (*step_begin)(const Dev&, const Tables&, int do_switch, int grid, cudaStream_t);
    void (*stage)(const Dev&, const Tables&, const StageArgs&, int grid, cudaStream_t);
    void (*masks)(const Dev&, int buf, int grid, cudaStream_t);
    void (*cell_diag)(const Dev&, const Tables&, double* part, int grid, cudaStream_t);
    void (*gauges)(const Dev&, const Tables&, int ng, const double* xy, double* out, cudaStream_t);
    int nzp; // mode P samples per cell
};

// mode: 0 S, 1 P; pix: 0 float32, 1 float64; prec: 0 FP64, 1 FP32-bulk
bool get_launch(int degree, int mode, int pix, int prec, Launch* out);
bool get_launch_r1(int mode, int pix, int prec, Launch* out);
bool get_launch_r2(int mode, int pix, int prec, Launch* out);
bool get_launch_r3(int mode, int pix, int prec, Launch* out);

} // namespace swdg
