// swdg_r1.cu -- kernels of polynomial degree r = 1 (one translation unit per
// degree so that the three compile in parallel).
#include "swdg_degree.cuh"

namespace swdg {
bool get_launch_r1(int mode, int pix, int prec, Launch* out) {
    return get_launch_degree<1>(mode, pix, prec, out);
}
} // namespace swdg
