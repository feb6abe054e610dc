// FP32 storage, FP32 compute: the persistent step kernels specialised to
// one column length.
#include "lb_step_kernel.cuh"

namespace lbk {

// Default: split columns (two lanes per column); threads_hint 1 selects the
// one-lane-per-column kernels.
bool kernels_f32(int nz_max, int nz_min, bool same, int threads_hint, KernelInfo *out) {
    const bool one_lane = threads_hint == 1;
    if (same && nz_max == 32) {
        if (one_lane) *out = kernel_entry<float, float, 32, true, 1, 512>();
        else *out = kernel_entry<float, float, 32, true, 1, 1024, true>();
        return true;
    }
    if (same && nz_max == 64) {
        if (one_lane) *out = kernel_entry<float, float, 64, true, 1, 512>();
        else *out = kernel_entry<float, float, 64, true, 1, 768, true>();
        return true;
    }
    if (same && nz_max == 96) {
        if (one_lane) *out = kernel_entry<float, float, 96, true, 1, 384>();
        else *out = kernel_entry<float, float, 96, true, 1, 768, true>();
        return true;
    }
    return kernels_f32_any(nz_max, nz_min, one_lane, out);
}

}  // namespace lbk
