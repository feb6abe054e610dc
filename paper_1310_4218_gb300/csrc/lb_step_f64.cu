// FP64 storage, FP64 compute: the persistent step kernels.
#include "lb_step_kernel.cuh"

namespace lbk {

bool kernels_f64(int nz_max, int nz_min, bool same, KernelInfo *out) {
    (void)nz_min;
    if (same && nz_max == 32) { *out = kernel_entry<double, double, 32, true, 1, 256>(); return true; }
    if (nz_max <= 32) { *out = kernel_entry<double, double, 32, false, 1, 256>(); return true; }
    if (nz_max <= 64) { *out = kernel_entry<double, double, 64, false, 1, 256>(); return true; }
    return false;
}

}  // namespace lbk
