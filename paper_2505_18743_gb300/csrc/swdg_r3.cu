// swdg_r3.cu -- kernels of polynomial degree r = 3 (one translation unit per
// degree so that the three compile in parallel).
#include "swdg_degree.cuh"

namespace swdg {
bool get_launch_r3(int mode, int pix, int prec, Launch* out) {
    return get_launch_degree<3>(mode, pix, prec, out);
}
} // namespace swdg
