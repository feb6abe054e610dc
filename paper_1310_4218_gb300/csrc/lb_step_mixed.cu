// FP64 or BF16 storage with FP32 compute: the persistent step kernels.
#include "lb_step_kernel.cuh"

namespace lbk {

bool kernels_f64s(int nz_max, int nz_min, bool same, KernelInfo *out) {
    (void)nz_min;
    if (same && nz_max == 64) { *out = kernel_entry<double, float, 64, true, 1, 512>(); return true; }
    if (nz_max <= 64) { *out = kernel_entry<double, float, 64, false, 1, 512>(); return true; }
    if (nz_max <= 128) { *out = kernel_entry<double, float, 128, false, 1, 256>(); return true; }
    return false;
}

bool kernels_bf16(int nz_max, int nz_min, bool same, KernelInfo *out) {
    (void)nz_min;
    if (same && nz_max == 64) { *out = kernel_entry<__nv_bfloat16, float, 64, true, 1, 512>(); return true; }
    if (nz_max <= 64) { *out = kernel_entry<__nv_bfloat16, float, 64, false, 1, 512>(); return true; }
    if (nz_max <= 128) { *out = kernel_entry<__nv_bfloat16, float, 128, false, 1, 256>(); return true; }
    return false;
}

}  // namespace lbk
