// FP32 kernels for processors that share an SM (lb_options.ctas_per_sm 2 or
// 4): the half-warp and twin kernels of exact nz 96 with 1/2 or 1/4 of their
// threads, so that the SM holds the same warps in total.  Used by the
// measurement study of costs under shared SMs (Sec. V).
#include "lb_step_kernel.cuh"

namespace lbk {

bool kernels_f32_shared_sm(int nz, bool twin, int ctas_per_sm, KernelInfo *out) {
    if (nz != 96) return false;
    if (twin) {
        if (ctas_per_sm == 2) { *out = kernel_entry<float, float, 96, true, 1, 256, false, 0, true, 2>(); return true; }
        if (ctas_per_sm == 4) { *out = kernel_entry<float, float, 96, true, 1, 128, false, 0, true, 4>(); return true; }
        return false;
    }
    if (ctas_per_sm == 2) { *out = kernel_entry<float, float, 96, true, 1, 384, true, 0, false, 2>(); return true; }
    if (ctas_per_sm == 4) { *out = kernel_entry<float, float, 96, true, 1, 192, true, 0, false, 4>(); return true; }
    return false;
}

}  // namespace lbk
