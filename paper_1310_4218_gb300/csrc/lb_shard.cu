// Column copies between a grid's current field and a packed buffer: the
// halo exchange and VP migration of a sharded run (one rank per GPU, each
// owning a set of VPs; Sec. III / Sec. VI across processes).
#include <cuda_runtime.h>

#include <cstdint>

#include "lb_internal.h"

namespace lbk {

// Element (k, c) of the buffer is level k of column cells[c]; a thread per
// element, grid-stride, buffer-side coalesced.  T is the storage element
// moved as raw bits.  An index outside the plane is skipped and recorded.
template <class T, bool PACK>
__global__ void __launch_bounds__(256) k_columns(T *field, const int32_t *cells, int n, int nz,
                                                 int nx, int ny, int pitch, T *buf,
                                                 int32_t *status) {
    const int ncols = nx * ny;
    const size_t plane = (size_t)pitch * ny;
    const long long total = (long long)n * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), c = (int)(e - (long long)k * n);
        const int cell = cells[c];
        if (cell < 0 || cell >= ncols) {
            atomicCAS(status, 0, (int32_t)LB_EINVAL);
            continue;
        }
        const int j = cell / nx;
        const size_t f = (size_t)k * plane + (size_t)j * pitch + (cell - j * nx);
        if (PACK) buf[e] = field[f];
        else field[f] = buf[e];
    }
}

template <bool PACK>
static cudaError_t launch_columns(void *field, int esize, const int32_t *cells, int n, int nz,
                                  int nx, int ny, int pitch, void *buf, int32_t *status,
                                  cudaStream_t s) {
    const long long total = (long long)n * nz;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (esize == 8)
        k_columns<uint64_t, PACK><<<blocks, 256, 0, s>>>(static_cast<uint64_t *>(field), cells, n,
                                                          nz, nx, ny, pitch,
                                                          static_cast<uint64_t *>(buf),
                                                          status);
    else if (esize == 4)
        k_columns<uint32_t, PACK><<<blocks, 256, 0, s>>>(static_cast<uint32_t *>(field), cells, n,
                                                          nz, nx, ny, pitch,
                                                          static_cast<uint32_t *>(buf),
                                                          status);
    else
        k_columns<uint16_t, PACK><<<blocks, 256, 0, s>>>(static_cast<uint16_t *>(field), cells, n,
                                                          nz, nx, ny, pitch,
                                                          static_cast<uint16_t *>(buf),
                                                          status);
    return cudaGetLastError();
}

cudaError_t dev_columns(bool pack, void *field, int esize, const int32_t *cells, int n, int nz,
                        int nx, int ny, int pitch, void *buf, int32_t *status, cudaStream_t s) {
    return pack ? launch_columns<true>(field, esize, cells, n, nz, nx, ny, pitch, buf, status, s)
                : launch_columns<false>(field, esize, cells, n, nz, nx, ny, pitch, buf, status, s);
}

}  // namespace lbk
