// FP32 storage, FP32 compute: the persistent step kernels specialised to
// one column length.
#include "lb_step_kernel.cuh"

namespace lbk {

bool kernels_f32(int nz_max, int nz_min, bool same, int threads_hint, KernelInfo *out) {
    if (same && nz_max == 32) { *out = kernel_entry<float, float, 32, true, 1, 512>(); return true; }
    if (same && nz_max == 64) { *out = kernel_entry<float, float, 64, true, 1, 512>(); return true; }
    if (same && nz_max == 96) {
        if (threads_hint == 512) *out = kernel_entry<float, float, 96, true, 1, 512>();
        else *out = kernel_entry<float, float, 96, true, 1, 384>();
        return true;
    }
    return kernels_f32_any(nz_max, nz_min, out);
}

}  // namespace lbk
