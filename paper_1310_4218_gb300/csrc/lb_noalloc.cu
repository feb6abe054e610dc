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
constexpr long long kMaxColumns = LB_NOALLOC_MAX_COLUMNS;

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
uint64_t h_cover[kMaxColumns / 64];   // one bit per column: covered by a VP
std::mutex g_mutex;
unsigned char *g_dev_scratch[kMaxDevices];

// errors are readable through lb_last_error(NULL), as for lb_create
lb_status fail(lb_status s, const char *msg) {
    set_ctxless_error(msg);
    return s;
}

// Marks columns [i0, i1) of row j covered; false if one of them already was.
bool cover_row(long long row0, int i0, int i1) {
    long long a = row0 + i0;
    const long long b = row0 + i1;
    while (a < b) {
        const long long w = a >> 6;
        const int lo = (int)(a & 63);
        const int hi = (b - (w << 6)) >= 64 ? 64 : (int)(b - (w << 6));
        const uint64_t mask = (hi == 64 ? ~0ull : ((1ull << hi) - 1)) & ~((1ull << lo) - 1);
        if (h_cover[w] & mask) return false;
        h_cover[w] |= mask;
        a = (w + 1) << 6;
    }
    return true;
}

template <class TC>
cudaError_t launch_noalloc(const KernelInfo &ki, unsigned char *base, int nbins, int nvps,
                           int nitems, long long t0, int nsteps, double r, long long timeout_ns,
                           cudaStream_t st) {
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
    p.timeout_ns = timeout_ns;
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
    fill_coef(r, ki, p.coef);
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nbins);
    cfg.blockDim = dim3(ki.threads);
    cfg.dynamicSmemBytes = step_dyn_smem(ki, 1);
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
                                     const lb_options *opt, int64_t t0, int32_t nsteps,
                                     void *cuda_stream, double *mass_out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    // sizes and layout first: nothing touches the device before they pass
    if (!grid || !vps) return fail(LB_EINVAL, "grid and vps must be non-NULL");
    if (nvps < 1 || nvps > kMaxVps) return fail(LB_EINVAL, "nvps must be in 1..LB_NOALLOC_MAX_VPS");
    if (nsteps < 0) return fail(LB_EINVAL, "nsteps < 0");
    const lb_grid_desc &d = *grid;
    if (const char *why = check_grid_desc(d)) return fail(LB_EINVAL, why);
    if ((long long)d.nx * d.ny > kMaxColumns)
        return fail(LB_EINVAL, "nx*ny above LB_NOALLOC_MAX_COLUMNS");
    lb_options o;
    if (opt) o = *opt;
    else lb_default_options(&o);
    const long long timeout_ns = o.barrier_timeout_ns > 0 ? o.barrier_timeout_ns : 2000000000LL;
    for (int v = 0; v < nvps; ++v) {
        const lb_vp &p = vps[v];
        if (p.grid != 0 || p.w < 1 || p.h < 1 || p.x0 < 0 || p.y0 < 0 || p.x0 > d.nx - p.w ||
            p.y0 > d.ny - p.h)
            return fail(LB_EINVAL, "a VP lies outside the grid (grid index must be 0)");
    }
    // the kernel lb_create would choose for this grid and layout
    KernelInfo ki;
    if (!choose_step_kernel(&d, 1, vps, nvps, o.threads_hint, false, &ki))
        return fail(LB_EINVAL, "no kernel variant for this grid");
    long long area = 0, nitems = 0;
    for (int v = 0; v < nvps; ++v) {
        area += (long long)vps[v].w * vps[v].h;
        nitems += items_of_vp(ki, vps[v].w, vps[v].h);
    }
    if (area != (long long)d.nx * d.ny) return fail(LB_EINVAL, "VPs do not tile the grid");
    // with the areas equal, no overlap means an exact tiling
    std::memset(h_cover, 0, sizeof(uint64_t) * (size_t)(((long long)d.nx * d.ny + 63) / 64));
    for (int v = 0; v < nvps; ++v)
        for (int j = vps[v].y0; j < vps[v].y0 + vps[v].h; ++j)
            if (!cover_row((long long)j * d.nx, vps[v].x0, vps[v].x0 + vps[v].w))
                return fail(LB_EINVAL, "VPs overlap");
    if (nitems > kMaxItems) return fail(LB_EINVAL, "too many work items for LB_NOALLOC_MAX_ITEMS");
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
    const size_t smem = step_dyn_smem(ki, 1);
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // kernels with staged buffers take more than the default 48 KB
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(ki.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki.fn, ki.threads, smem);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
    if (occ < 1) return fail(LB_ENORESIDENT, "step kernel cannot be resident");
    const int nbins = nsm < kMaxBins ? nsm : kMaxBins;

    // tables: grid, VPs, work items of a static contiguous placement
    GridDev g;
    fill_grid_dev(d, reinterpret_cast<int32_t *>(base + kOffStatus) + 1, g);
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
                ? launch_noalloc<double>(ki, base, nbins, nvps, ni, t0, nsteps, d.r, timeout_ns, st)
                : launch_noalloc<float>(ki, base, nbins, nvps, ni, t0, nsteps, d.r, timeout_ns, st);
    }
    // the staging arrays are reused by the next call: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));

    // status words: [0] sticky failure, [1] k_c range flag (cleared by the
    // next call's memset)
    int32_t status[2] = {0, 0};
    e = cudaMemcpy(status, base + kOffStatus, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
    if (status[0] == LB_ETIMEOUT) return fail(LB_ETIMEOUT, "grid barrier wait exceeded barrier_timeout_ns");
    if (status[0] == LB_ENUMERIC) return fail(LB_ENUMERIC, "global sum is not finite");
    if (status[0] != 0) return fail((lb_status)status[0], "device reported an error");
    if (mass_out) {
        double ent[2];
        e = cudaMemcpy(ent, base + kOffMassHist + sizeof(double) * 2 * ((nsteps - 1) % kMassHist),
                       sizeof(ent), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(LB_ECUDA, cudaGetErrorString(e));
        *mass_out = ent[0] + ent[1];
    }
    if (status[1] != 0)
        return fail(LB_EKCRANGE, "k_c array entries above LB_KC_MAX were clamped to it");
    return LB_OK;
}
