// swdg_r2.cu -- kernels of polynomial degree r = 2 (one translation unit per
// degree so that the three compile in parallel).
#include "swdg_degree.cuh"

namespace swdg {
bool get_launch_r2(int mode, int pix, int prec, Launch* out) {
    return get_launch_degree<2>(mode, pix, prec, out);
}
} // namespace swdg
