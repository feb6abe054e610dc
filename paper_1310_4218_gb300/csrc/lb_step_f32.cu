// FP32 storage, FP32 compute: the persistent step kernels specialised to
// one column length.
#include "lb_step_tma.cuh"

namespace lbk {

// Exact nz 32 / 64 / 96, split columns: on paired warps with 16 x 2 tiles
// when every VP width is a multiple of 16 (wide) or threads_hint is 3, else
// on half-warps with 8 x 2 tiles (narrower tiles idle fewer lanes at the
// edges of narrow VPs); threads_hint 2 forces half-warps, 1 selects the
// one-lane-per-column kernels; `staged` the TMA-staged kernels (one box
// slot per warp, 147-221 KB of shared memory per SM).
bool kernels_f32(int nz_max, int nz_min, bool same, int threads_hint, bool staged, bool wide,
                 KernelInfo *out) {
    const bool one_lane = threads_hint == 1;
    const bool pair = threads_hint == 3 || (threads_hint == 0 && wide);
    if (same && nz_max == 32) {
        if (one_lane) *out = kernel_entry<float, float, 32, true, 1, 512>();
        else if (staged) *out = kernel_entry_tma<32, 1024>();
        else if (pair) *out = kernel_entry<float, float, 32, true, 1, 960, true, 16>();
        else *out = kernel_entry<float, float, 32, true, 1, 1024, true>();
        return true;
    }
    if (same && nz_max == 64) {
        if (one_lane) *out = kernel_entry<float, float, 64, true, 1, 512>();
        else if (staged) *out = kernel_entry_tma<64, 768>();
        else if (pair) *out = kernel_entry<float, float, 64, true, 1, 768, true, 16>();
        else *out = kernel_entry<float, float, 64, true, 1, 768, true>();
        return true;
    }
    if (same && nz_max == 96) {
        if (one_lane) *out = kernel_entry<float, float, 96, true, 1, 384>();
        else if (staged) *out = kernel_entry_tma<96, 512>();
        else if (pair) *out = kernel_entry<float, float, 96, true, 1, 768, true, 16>();
        else *out = kernel_entry<float, float, 96, true, 1, 768, true>();
        return true;
    }
    return kernels_f32_any(nz_max, nz_min, one_lane, out);
}

}  // namespace lbk
