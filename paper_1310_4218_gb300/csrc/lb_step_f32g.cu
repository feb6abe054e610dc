// FP32 storage, FP32 compute: the persistent step kernels for any column
// length up to the variant (grids of different nz in one launch).
#include "lb_step_kernel.cuh"

namespace lbk {

bool kernels_f32_any(int nz_max, int nz_min, bool one_lane, KernelInfo *out) {
    // split columns with runtime nz (any nz >= 2 up to the bucket)
    if (!one_lane && nz_min >= 2) {
        if (nz_max <= 32) { *out = kernel_entry<float, float, 32, false, 1, 1024, true>(); return true; }
        if (nz_max <= 64) { *out = kernel_entry<float, float, 64, false, 1, 768, true>(); return true; }
        if (nz_max <= 96) { *out = kernel_entry<float, float, 96, false, 1, 768, true>(); return true; }
    }
    // one lane per column
    if (nz_max <= 32) { *out = kernel_entry<float, float, 32, false, 1, 512>(); return true; }
    if (nz_max <= 64) { *out = kernel_entry<float, float, 64, false, 1, 512>(); return true; }
    if (nz_max <= 96 && nz_min >= 32) { *out = kernel_entry<float, float, 96, false, 32, 384>(); return true; }
    if (nz_max <= 128) { *out = kernel_entry<float, float, 128, false, 1, 256>(); return true; }
    return false;
}

}  // namespace lbk
