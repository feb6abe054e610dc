// FP32 storage, FP32 compute: the persistent step kernels for any column
// length up to the variant (grids of different nz in one launch).
#include "lb_step_kernel.cuh"

namespace lbk {

// Default: twin halves (one lane per column) where the FP32 pivots
// converge; else split columns on half-warps.  threads_hint 1 one lane per column (plain Thomas), 2 half-warp
// split columns, 4 twin halves where the pivots allow.
bool kernels_f32_any(int nz_max, int nz_min, int threads_hint, bool wide, bool twin_ok,
                     KernelInfo *out) {
    const bool one_lane = threads_hint == 1;
    (void)wide;
    const bool twin = twin_ok && nz_min >= 2 && (threads_hint == 4 || threads_hint == 0);
    if (twin) {
        if (nz_max <= 32) { *out = kernel_entry<float, float, 32, false, 1, 1024, false, 0, true>(); return true; }
        if (nz_max <= 64) { *out = kernel_entry<float, float, 64, false, 1, 640, false, 0, true>(); return true; }
        if (nz_max <= 96) { *out = kernel_entry<float, float, 96, false, 1, 512, false, 0, true>(); return true; }
    }
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
