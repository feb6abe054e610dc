// lb_step_noalloc: the persistent step for one grid without any memory
// allocation, for callers that cannot allocate device memory.
//
// Who needs it: a host program whose device memory is owned by another
// allocator (a framework's caching allocator that has already reserved the
// GPU, a fixed-budget pool in an embedded or real-time service) cannot let a
// library call cudaMalloc: the call may fail when the pool holds the memory,
// fragments the pool, and may synchronise the device at a moment the caller
// does not control.  lb_create allocates its tables with cudaMalloc; this
// entry point instead keeps every table and every scratch word of the step
// kernel in one file-scope device array of fixed size, compiled into the
// library.
//
// Properties the caller must know:
//   - The array (kScratchBytes below) is held by every GPU that loads the
//     library, until the process exits.
//   - The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it; make
//     that first call before any stream capture.  The cache lives as long
//     as the process: after a cudaDeviceReset of that device the address
//     may change, so the entry point must not be called again.
//   - All calls share the one array and it keeps the previous call's
//     contents: each call clears what must start at zero.  Calls whose work
//     overlaps on the GPU (two streams, or two host threads on one device)
//     race on the array and give wrong results; serialise them.
//   - Sizes beyond the fixed maxima are rejected with LB_EINVAL.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "lb.h"
#include "lb_internal.h"

using namespace lbk;

namespace {

constexpr int kMaxVps = LB_NOALLOC_MAX_VPS;
constexpr int kMaxItems = LB_NOALLOC_MAX_ITEMS;
constexpr int kMaxBins = 1024;
constexpr int kMaxDevices = 64;
constexpr int kMaxBitmapCols = 1 << 22;

// Byte offsets of every table inside the scratch array (256-byte aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffGrid = 0;
constexpr size_t kOffVps = al(kOffGrid + sizeof(GridDev));
constexpr size_t kOffItems = al(kOffVps + sizeof(VPDev) * kMaxVps);
constexpr size_t kOffBinStart = al(kOffItems + sizeof(int2) * kMaxItems);
constexpr size_t kOffZero = al(kOffBinStart + sizeof(int32_t) * (kMaxBins + 1));
// the region cleared by every call starts here
constexpr size_t kOffBar = kOffZero;
constexpr size_t kOffStatus = kOffBar + 2 * sizeof(unsigned);
constexpr size_t kOffQhead = kOffStatus + sizeof(int32_t) * 2;
constexpr size_t kOffMassSeq = al(kOffQhead + 2 * sizeof(unsigned));
constexpr size_t kOffVpCycles = al(kOffMassSeq + sizeof(unsigned long long));
constexpr size_t kOffBinBusy = al(kOffVpCycles + sizeof(unsigned long long) * kMaxVps);
constexpr size_t kZeroEnd = al(kOffBinBusy + sizeof(unsigned long long) * kMaxBins);
constexpr size_t kOffBinSmid = kZeroEnd;
constexpr size_t kOffBinCal = al(kOffBinSmid + sizeof(int32_t) * kMaxBins);
constexpr size_t kOffBinMass = al(kOffBinCal + sizeof(long long) * 4 * kMaxBins);
constexpr size_t kOffMassHist = al(kOffBinMass + sizeof(double) * 2 * kMaxBins);
constexpr size_t kOffMassT = al(kOffMassHist + sizeof(double) * 2 * kMassHist);
constexpr size_t kScratchBytes = al(kOffMassT + sizeof(long long) * kMassHist);
static_assert(kScratchBytes <= LB_NOALLOC_SCRATCH_BYTES, "scratch exceeds its stated maximum");

// The scratch array itself.  In host code this name is only a stand-in for
// the device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host staging for the tables (file scope: no heap use per call).
VPDev h_vps[kMaxVps];
int2 h_items[kMaxItems];
int32_t h_bin_start[kMaxBins + 1];
unsigned char h_cover[kMaxBitmapCols];
std::mutex g_mutex;
unsigned char *g_dev_scratch[kMaxDevices];

// errors are readable through lb_last_error(NULL), as for lb_create
lb_status fail(lb_status s, const char *msg) {
    set_ctxless_error(msg);
    return s;
}

// Pivots of the zero-flux operator for a column of nz rows (exact table)
// or the length-independent table plus the grid's last-row pivot.
void pivot_table(double r, int exact_nz, double *m) {
    for (int k = 0; k < kNzMax; ++k) {
        if (exact_nz > 0 && k >= exact_nz) { m[k] = 1.0; continue; }
        const bool last = exact_nz > 0 && k == exact_nz - 1;
        const int nb = (k > 0 ? 1 : 0) + (last ? 0 : 1);
        const double b = 1.0 + r * nb;
        m[k] = k == 0 ? 1.0 / b : 1.0 / (b - r * r * m[k - 1]);
    }
}

double last_row_pivot(double r, int nz) {
    if (nz == 1) return 1.0;
    double m = 1.0 / (1.0 + r);
    for (int k = 1; k < nz - 1; ++k) m = 1.0 / (1.0 + 2.0 * r - r * r * m);
    return 1.0 / (1.0 + r - r * r * m);
}

template <class TC>
cudaError_t launch_noalloc(const KernelInfo &ki, unsigned char *base, int nbins, int nvps,
                           int nitems, long long t0, int nsteps, double r, cudaStream_t st) {
    StepParams<TC> p;
    std::memset(&p, 0, sizeof(p));
    p.grids = reinterpret_cast<const GridDev *>(base + kOffGrid);
    p.vps = reinterpret_cast<const VPDev *>(base + kOffVps);
    p.items = reinterpret_cast<const int2 *>(base + kOffItems);
    p.bin_start = reinterpret_cast<const int32_t *>(base + kOffBinStart);
    p.ngrids = 1;
    p.nvps = nvps;
    p.nbins = nbins;
    p.nitems = nitems;
    p.queue_mode = 0;
    p.mass_every = 1;
    p.parity0 = 0;
    p.nsteps = nsteps;
    p.t0 = t0;
    p.timeout_ns = 2000000000LL;
    p.bar = reinterpret_cast<unsigned *>(base + kOffBar);
    p.status = reinterpret_cast<int32_t *>(base + kOffStatus);
    p.qhead = reinterpret_cast<unsigned *>(base + kOffQhead);
    p.vp_cycles = reinterpret_cast<unsigned long long *>(base + kOffVpCycles);
    p.bin_busy = reinterpret_cast<unsigned long long *>(base + kOffBinBusy);
    p.bin_smid = reinterpret_cast<int32_t *>(base + kOffBinSmid);
    p.bin_cal = reinterpret_cast<long long *>(base + kOffBinCal);
    p.bin_mass = reinterpret_cast<double *>(base + kOffBinMass);
    p.mass_hist = reinterpret_cast<double *>(base + kOffMassHist);
    p.mass_t = reinterpret_cast<long long *>(base + kOffMassT);
    p.mass_seq = reinterpret_cast<unsigned long long *>(base + kOffMassSeq);
    double m[kNzMax];
    pivot_table(r, (ki.exact && !ki.split) ? ki.nz_variant : 0, m);
    for (int k = 0; k < kNzMax; ++k) {
        p.coef.m[k] = (TC)m[k];
        p.coef.rm[k] = (TC)(r * m[k]);
    }
    const double a = ki.split ? r * m[ki.nz_variant / 2 - 1] : 0.0;
    p.coef.ifa = (TC)a;
    p.coef.ifc = (TC)(1.0 / (1.0 - a * a));
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nbins);
    cfg.blockDim = dim3(ki.threads);
    cfg.dynamicSmemBytes = sizeof(double) * (ki.threads / kWarp);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&p};
    return cudaLaunchKernelExC(&cfg, ki.fn, args);
}

}  // namespace

extern "C" lb_status lb_step_noalloc(const lb_grid_desc *grid, const lb_vp *vps, int32_t nvps,
                                     int64_t t0, int32_t nsteps, void *cuda_stream,
                                     double *mass_out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    // sizes and layout first: nothing touches the device before they pass
    if (!grid || !vps) return fail(LB_EINVAL, "grid and vps must be non-NULL");
    if (nvps < 1 || nvps > kMaxVps) return fail(LB_EINVAL, "nvps must be in 1..LB_NOALLOC_MAX_VPS");
    if (nsteps < 0) return fail(LB_EINVAL, "nsteps < 0");
    const lb_grid_desc &d = *grid;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nz > kNzMax)
        return fail(LB_EINVAL, "need nx, ny >= 1 and 1 <= nz <= 128");
    if ((long long)d.nx * d.ny * d.nz >= (1LL << 31)) return fail(LB_EINVAL, "nx*ny*nz must be below 2^31");
    if (d.dynamics != 0 && d.dynamics != 1) return fail(LB_EINVAL, "dynamics is 0 or 1");
    if (d.pad0 != 0) return fail(LB_EINVAL, "pad0 must be 0");
    if (d.dynamics == 0 &&
        (!std::isfinite(d.cx) || !std::isfinite(d.cy) || !std::isfinite(d.cz) ||
         std::fabs(d.cx) + std::fabs(d.cy) + std::fabs(d.cz) > 1.0 + 1e-12))
        return fail(LB_EINVAL, "need |cx|+|cy|+|cz| <= 1");
    if (d.dynamics == 1 && !(d.nu > 0.0 && d.nu <= 1.0 / 6.0 + 1e-15))
        return fail(LB_EINVAL, "Jacobi weight needs 0 < nu <= 1/6");
    if (!std::isfinite(d.r) || d.r < 0.0) return fail(LB_EINVAL, "need r >= 0");
    const bool ok_types = (d.storage == LB_F64 && (d.compute == LB_F64 || d.compute == LB_F32)) ||
                          (d.storage == LB_F32 && d.compute == LB_F32) ||
                          (d.storage == LB_BF16 && d.compute == LB_F32);
    if (!ok_types) return fail(LB_EINVAL, "unsupported storage/compute pair");
    if (d.compute == LB_F64 && d.nz > 64) return fail(LB_EINVAL, "FP64 compute supports nz <= 64");
    if (!d.q0 || !d.q1 || d.q0 == d.q1) return fail(LB_EINVAL, "q0 and q1 must be distinct device buffers");
    if (!d.kc_disk && !d.kc) return fail(LB_EINVAL, "kc array required");
    if (d.kc_disk && (d.k_in < 0 || d.k_out < 0 || d.disk_r < 0))
        return fail(LB_EINVAL, "disk needs k_in, k_out, R >= 0");
    KernelInfo ki;
    if (!find_step_kernel(d.storage, d.compute, d.nz, d.nz, true, &ki))
        return fail(LB_EINVAL, "no kernel variant for this grid");
    long long area = 0, nitems = 0;
    for (int v = 0; v < nvps; ++v) {
        const lb_vp &p = vps[v];
        if (p.grid != 0 || p.w < 1 || p.h < 1 || p.x0 < 0 || p.y0 < 0 || p.x0 + p.w > d.nx ||
            p.y0 + p.h > d.ny)
            return fail(LB_EINVAL, "a VP lies outside the grid (grid index must be 0)");
        area += (long long)p.w * p.h;
        nitems += items_of_vp(ki, p.w, p.h);
    }
    if (area != (long long)d.nx * d.ny) return fail(LB_EINVAL, "VPs do not tile the grid");
    if (nitems > kMaxItems) return fail(LB_EINVAL, "too many work items for LB_NOALLOC_MAX_ITEMS");
    if ((long long)d.nx * d.ny <= kMaxBitmapCols) {
        std::memset(h_cover, 0, (size_t)d.nx * d.ny);
        for (int v = 0; v < nvps; ++v)
            for (int j = vps[v].y0; j < vps[v].y0 + vps[v].h; ++j)
                for (int i = vps[v].x0; i < vps[v].x0 + vps[v].w; ++i) {
                    unsigned char &c = h_cover[(size_t)j * d.nx + i];
                    if (c) return fail(LB_EINVAL, "VPs overlap");
                    c = 1;
                }
    }
    if (nsteps == 0) return LB_OK;

    // per-device set-up: the scratch array's device address
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LB_ECUDA, "device index out of range");
    if (!g_dev_scratch[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
        g_dev_scratch[dev] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *base = g_dev_scratch[dev];

    int nsm = 0, occ = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki.fn, ki.threads,
                                                          sizeof(double) * (ki.threads / kWarp));
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
    if (occ < 1) return fail(LB_ENORESIDENT, "step kernel cannot be resident");
    const int nbins = nsm < kMaxBins ? nsm : kMaxBins;

    // tables: grid, VPs, work items of a static contiguous placement
    GridDev g;
    std::memset(&g, 0, sizeof(g));
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.kc_disk = d.kc_disk;
    g.plane = d.nx * d.ny;
    g.sx = d.cx >= 0 ? 1 : -1;
    g.sy = d.cy >= 0 ? 1 : -1;
    g.sz = d.cz >= 0 ? 1 : -1;
    g.q[0] = d.q0;
    g.q[1] = d.q1;
    g.kc = d.kc;
    g.disk_x0 = d.disk_x0;
    g.disk_y0 = d.disk_y0;
    g.disk_vx = d.disk_vx;
    g.disk_vy = d.disk_vy;
    g.disk_r = d.disk_r;
    g.k_in = d.k_in;
    g.k_out = d.k_out;
    const double w[4] = {1.0 - std::fabs(d.cx) - std::fabs(d.cy) - std::fabs(d.cz), std::fabs(d.cx),
                         std::fabs(d.cy), std::fabs(d.cz)};
    for (int n = 0; n < 4; ++n) {
        g.wd[n] = w[n];
        g.wf[n] = (float)w[n];
    }
    g.xy_only = (d.dynamics == 0 && w[0] == 0.0 && d.cz == 0.0) ? 1 : 0;
    g.jacobi = d.dynamics == 1 ? 1 : 0;
    g.nu_d = d.nu;
    g.w0j_d = 1.0 - 6.0 * d.nu;
    g.nu_f = (float)d.nu;
    g.w0j_f = (float)(1.0 - 6.0 * d.nu);
    g.sweeps_on = d.r > 0.0 ? 1 : 0;
    const double ml = last_row_pivot(d.r, d.nz);
    g.mlast_d = ml;
    g.rlast_d = d.r * ml;
    g.mlast_f = (float)ml;
    g.rlast_f = (float)(d.r * ml);
    if (d.nz >= 2) split_coupling(d.r, d.nz, &g.ifa_b_f, &g.ifa_t_f, &g.ifc_bt_f);
    int ni = 0;
    for (int b = 0, v = 0; b < nbins; ++b) {
        h_bin_start[b] = ni;
        const int vend = (int)(((long long)(b + 1) * nvps) / nbins);
        for (; v < vend; ++v) {
            const int n = items_of_vp(ki, vps[v].w, vps[v].h);
            for (int c = 0; c < n; ++c) h_items[ni++] = make_int2(v, c);
        }
    }
    h_bin_start[nbins] = ni;
    for (int v = 0; v < nvps; ++v)
        h_vps[v] = VPDev{0, vps[v].x0, vps[v].y0, vps[v].w, vps[v].h, vps[v].w * vps[v].h, 0, 0};

    cudaStream_t st = (cudaStream_t)cuda_stream;
    e = cudaMemcpyAsync(base + kOffGrid, &g, sizeof(g), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffVps, h_vps, sizeof(VPDev) * nvps, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffItems, h_items, sizeof(int2) * ni, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffBinStart, h_bin_start, sizeof(int32_t) * (nbins + 1),
                            cudaMemcpyHostToDevice, st);
    // barrier words, status, queue heads, global-sum counter, cost counters
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffZero, 0, kZeroEnd - kOffZero, st);
    if (e == cudaSuccess) {
        e = d.compute == LB_F64
                ? launch_noalloc<double>(ki, base, nbins, nvps, ni, t0, nsteps, d.r, st)
                : launch_noalloc<float>(ki, base, nbins, nvps, ni, t0, nsteps, d.r, st);
    }
    // the staging arrays are reused by the next call: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));

    int32_t status = 0;
    e = cudaMemcpy(&status, base + kOffStatus, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
    if (status == LB_ETIMEOUT) return fail(LB_ETIMEOUT, "grid barrier wait exceeded 2 s");
    if (status == LB_ENUMERIC) return fail(LB_ENUMERIC, "global sum is not finite");
    if (mass_out) {
        double ent[2];
        e = cudaMemcpy(ent, base + kOffMassHist + sizeof(double) * 2 * ((nsteps - 1) % kMassHist),
                       sizeof(ent), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
        *mass_out = ent[0] + ent[1];
    }
    return LB_OK;
}
