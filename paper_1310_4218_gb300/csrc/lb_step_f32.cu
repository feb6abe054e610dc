// FP32 storage, FP32 compute: the persistent step kernels specialised to
// one column length.
#include "lb_step_df.cuh"
#include "lb_step_tma.cuh"

namespace lbk {

// Exact nz 32 / 64 / 96.  Default: when the FP32 pivots converge (twin_ok),
// one lane per column with both twisted halves in packed pairs, items of 32
// columns; otherwise split columns on half-warps with 8 x 2 tiles.  threads_hint: 1 one lane per column (plain Thomas),
// 2 half-warps, 3 paired warps (16 x 2 tiles), 4 twin halves; `staged` the
// TMA-staged kernels (one box slot per warp, 147-221 KB of shared memory
// per SM).
bool kernels_f32(int nz_max, int nz_min, bool same, int threads_hint, bool staged, bool wide,
                 bool twin_ok, KernelInfo *out) {
    const bool one_lane = threads_hint == 1;
    const bool pair = threads_hint == 3;
    // twin halves wherever the pivots allow: with the scaled solves they
    // beat the half-warp split on narrow layouts as well
    (void)wide;
    const bool twin = twin_ok && nz_max / 2 > kTwinS0 && (threads_hint == 4 || threads_hint == 0);
    if (same && nz_max == 32) {
        if (one_lane) *out = kernel_entry<float, float, 32, true, 1, 512>();
        else if (staged) *out = kernel_entry_tma<32, 1024>();
        else if (twin) *out = kernel_entry_twin_df<32, 1024>();
        else if (pair) *out = kernel_entry<float, float, 32, true, 1, 960, true, 16>();
        else *out = kernel_entry<float, float, 32, true, 1, 1024, true>();
        return true;
    }
    if (same && nz_max == 64) {
        if (one_lane) *out = kernel_entry<float, float, 64, true, 1, 512>();
        else if (staged) *out = kernel_entry_tma<64, 768>();
        else if (twin) *out = kernel_entry_twin_df<64, 640>();
        else if (pair) *out = kernel_entry<float, float, 64, true, 1, 768, true, 16>();
        else *out = kernel_entry<float, float, 64, true, 1, 768, true>();
        return true;
    }
    if (same && nz_max == 96) {
        if (one_lane) *out = kernel_entry<float, float, 96, true, 1, 384>();
        else if (staged) *out = kernel_entry_tma<96, 512>();
        else if (twin) *out = kernel_entry_twin_df<96, 512>();
        else if (pair) *out = kernel_entry<float, float, 96, true, 1, 768, true, 16>();
        else *out = kernel_entry<float, float, 96, true, 1, 768, true>();
        return true;
    }
    return kernels_f32_any(nz_max, nz_min, threads_hint, wide, twin_ok, out);
}

}  // namespace lbk
