// Internal declarations shared by the library's translation units.
// Device-side tables of a ctx and the persistent step kernel's parameters.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lb.h"

namespace lbk {

constexpr int kNzMax = 128;        // longest register-resident column
constexpr int kMassHist = 1024;    // global sums kept per grid
constexpr int kMaxGrids = 512;
constexpr int kWarp = 32;
constexpr int kBoxW = 12, kBoxH = 3;   // TMA-staged kernel: box of an 8 x 2 tile
// Twin kernels: level from which the FP32 pivots m_s and r m_s of a zero-flux
// end must be one constant pair (checked by the host for every ctx that
// selects them).
constexpr int kTwinS0 = 8;

// One grid as the kernel sees it.
struct GridDev {
    int32_t nx, ny, nz, kc_disk;
    int32_t plane;                 // pitch*ny: elements between levels
    int32_t pitch;                 // elements between rows (nx when dense)
    int32_t sx, sy, sz;            // upwind direction per axis (+1: neighbour at -1)
    void *q[2];                    // ping-pong fields
    const int32_t *kc;             // k_c array (kc_disk == 0)
    int32_t *kc_range;             // set to 1 when an array entry above LB_KC_MAX was clamped
    int32_t disk_x0, disk_y0, disk_vx, disk_vy, disk_r, k_in, k_out;
    int32_t xy_only;               // w0 == 0 and wz == 0: two-neighbour stencil
    int32_t sweeps_on;             // r > 0
    int32_t jacobi;                // 1: weighted Jacobi sweep instead of advection
    float nu_f, w0j_f;             // Jacobi weights nu, 1 - 6 nu (FP32 compute)
    double nu_d, w0j_d;            // same for FP64 compute
    float wf[4];                   // w0, |cx|, |cy|, |cz| for FP32 compute
    double wd[4];                  // same for FP64 compute
    float mlast_f, rlast_f;        // last-row coefficients (runtime-nz kernels)
    double mlast_d, rlast_d;
    // runtime-nz split kernels: lower half ceil(nz/2) levels, upper half
    // floor(nz/2); middle coupling a_b = r m[Hb-1], a_t = r m[Ht-1],
    // c = 1 / (1 - a_b a_t)
    float ifa_b_f, ifa_t_f, ifc_bt_f, pad1;
};

// One VP (rectangle of columns of one grid).
struct VPDev {
    int32_t grid, x0, y0, w, h, ncols, pad0, pad1;
};

// Thomas coefficients of the zero-flux operator for the kernel's compute
// type: m[k] = 1/pivot_k, rm[k] = r*m[k] (FP64 values rounded once).
//
// Split-family kernels (half-warp, paired-warp, twin, TMA-staged) solve in
// units of the converged pivot m_inf = lim m_k: a solve maps y to
// M^-1 y / m_inf, whose forward elimination is q_k = e_k y_k + r m_k q_{k-1}
// with e_k = m_k / m_inf -- exactly 1 in FP32 once the pivots have
// converged, so the multiply drops out there -- and whose back substitution
// (x_k = q_k + r m_k x_{k+1}) and middle 2x2 system are unchanged.  After k
// solves the column is M^-k y / m_inf^k; the store multiplies it by
// f[k] = m_inf^k (in the same FMA that adds back the shift).  To stay in
// range, every resc_every solves the column is multiplied by resc =
// m_inf^resc_every, and f[k] divides those factors out again (FP64, one
// rounding).
template <class TC>
struct Coef {
    TC m[kNzMax];
    TC rm[kNzMax];
    TC ifa, ifc;   // split kernels: interface coupling a = r m_{H-1}, 1/(1-a^2)
    TC e[kNzMax];              // forward multipliers m_k / m_inf
    TC f[LB_KC_MAX + 1];       // f[k] = m_inf^k / resc^floor(k / resc_every)
    TC resc;                   // m_inf^resc_every
    int32_t resc_every;
    // twin kernels' head levels as packed pairs (c, c) of the FP32 values
    float2 e2[kTwinS0], rm2[kTwinS0];
};

// Dataflow launches (lb_options.dataflow): the per-launch state, zeroed by
// the host before each launch.  Items of every step come from one queue
// (index step * nitems + item); steps are reduced in order through
// kDfSlots slots of per-step counts and sums.
constexpr int kDfSlots = 4;
constexpr int kDfDeps = 16;        // dependencies per item held inline (else the CSR)
struct DfState {
    unsigned long long qhead;      // next queue index
    unsigned reduced;              // steps of this launch reduced, in order
    unsigned started;              // CTAs that have read the step clock
    unsigned cnt[kDfSlots];        // finished items of the step in each slot
};

template <class TC>
struct StepParams {
    const GridDev *grids;
    const VPDev *vps;
    const int2 *items;             // work items {vp, chunk}: table or queue order
    const int32_t *bin_start;      // [nbins+1] item ranges per processor
    int32_t ngrids, nvps, nbins, nitems;
    int32_t queue_mode, mass_every, parity0, nsteps;
    int64_t t0;
    int64_t timeout_ns;
    unsigned *bar;                 // [0] arrivals, [1] generation
    int32_t *status;               // sticky lb_status of device failures
    unsigned *qhead;               // [2] queue counters (step parity)
    unsigned long long *vp_cycles; // [nvps] summed work-item cycles
    unsigned long long *bin_busy;  // [nbins] summed busy cycles per step
    int32_t *bin_smid;             // [nbins]
    long long *bin_cal;            // [nbins][4]: globaltimer0, clock0, globaltimer1, clock1
    double *bin_mass;              // [2][nbins][ngrids]
    double *mass_hist;             // [kMassHist][ngrids][2] (sum, comp)
    long long *mass_t;             // [kMassHist] step index of each entry
    unsigned long long *mass_seq;  // number of entries written so far
    unsigned long long *sweeps;    // cell-sweep updates performed (may be null)
    unsigned *bin_ctr;             // [2][nbins] per-processor item counters (stealing)
    int32_t steal;                 // 1: processors that run out take others' items
    int32_t serial_warps;          // > 0: only this many warps per processor run items
    long long *dclock;             // [0] step index, [1] buffer parity: read at start
                                   // instead of t0/parity0, advanced at the end (may be null)
    const void *tmaps;             // TMA-staged kernels: [ngrids][2] tensor maps of the
                                   // fields (128 bytes each), else null
    DfState *df;                   // dataflow launches: per-launch state (else null)
    double *df_mass;               // [kDfSlots][ngrids] global-sum partials per step slot
    int32_t *df_done;              // [nitems] steps each queue item has finished
    const int32_t *df_dep_start;   // [nitems + 1] CSR of each queue item's dependencies:
    const int32_t *df_deps;        // the items owning its closed 4-neighbourhood
    const int32_t *df_inl;         // [nitems][kDfDeps] the same lists padded with -1
                                   // (null when an item has more than kDfDeps)
    Coef<TC> coef;
};

// Kernel lookup: returns the persistent kernel for a (storage, compute,
// nz-variant) triple, or nullptr.  exact=1: specialised to nz == variant.
struct KernelInfo {
    const void *fn;
    const void *df_fn;  // the dataflow variant of fn (exact-nz twin kernels), else null
    int threads;
    int nz_variant;
    int exact;
    int split;          // 1: two lanes per column (twisted factorisation)
    int cols_per_item;  // columns of one work item: 32, or 16 when split
    int tile_w, tile_h; // split kernels: an item is a tile_w x tile_h tile of
                        // the VP (row-major over tiles); 0: runs of
                        // cols_per_item columns in the VP's row-major order
    int twin_s0;        // twin kernels: level from which the FP32 pivots must be one
                        // constant pair, else 0
    int tma_slots;      // TMA-staged kernel: shared-memory box slots (one per warp), else 0
    int tma_slot_bytes; // bytes of one box
};

// Dynamic shared memory of a step launch: the per-warp global-sum partials
// [warps][ngrids] (doubles); TMA-staged kernels add their slots at launch
// set-up.
inline size_t step_dyn_smem(const KernelInfo &k, int ngrids) {
    return sizeof(double) * (size_t)(k.threads / kWarp) * (size_t)ngrids;
}

// Split kernels' work items: 8 x 2 column tiles.  A compact tile spans less
// of a smooth k_c field than a 16 x 1 run, so its lanes' sweep counts differ
// less (the warp runs the largest); each row of 8 FP32 columns is one
// 32-byte sector when the VP's x extent is a multiple of 8.
constexpr int kTileW = 8, kTileH = 2;

// Work items of a w x h VP.
inline int items_of_vp(const KernelInfo &k, int w, int h) {
    if (k.tile_w > 0) return ((w + k.tile_w - 1) / k.tile_w) * ((h + k.tile_h - 1) / k.tile_h);
    return (w * h + k.cols_per_item - 1) / k.cols_per_item;
}
// staged: allow the TMA-staged kernel (the caller then provides tensor maps);
// wide: at least 3/4 of the columns lie in VPs whose width is a multiple of
// 16 (the twin kernels are the default there); twin_ok: the FP32 pivots are
// one constant pair from level kTwinS0 on (twin kernels may run).
// ctas_per_sm > 1: a variant with 1/ctas_per_sm of the threads where one
// exists (exact nz 96, half-warp and twin kernels), so that that many
// processors share an SM with the same warps per SM.
bool find_step_kernel(int storage, int compute, int nz_max, int nz_min, bool all_same_nz,
                      KernelInfo *out, int threads_hint = 0, bool staged = false,
                      bool wide = false, bool twin_ok = false, int ctas_per_sm = 1);

// Per-type kernel tables (one translation unit each, compiled in parallel).
bool kernels_f32(int nz_max, int nz_min, bool same, int threads_hint, bool staged, bool wide,
                 bool twin_ok, KernelInfo *out);
bool kernels_f64(int nz_max, int nz_min, bool same, KernelInfo *out);
bool kernels_f64s(int nz_max, int nz_min, bool same, KernelInfo *out);
bool kernels_bf16(int nz_max, int nz_min, bool same, KernelInfo *out);
bool kernels_f32_any(int nz_max, int nz_min, int threads_hint, bool wide, bool twin_ok,
                     KernelInfo *out);
bool kernels_f32_shared_sm(int nz, bool twin, int ctas_per_sm, KernelInfo *out);

// Middle coupling of the runtime-nz split kernels for a column of nz >= 2
// rows: lower half hb = ceil(nz/2) rows, upper ht = floor(nz/2), each
// eliminated from its zero-flux end with the nz-independent pivots m_k
// (m_0 = 1/(1+r), m_k = 1/(1+2r-r^2 m_{k-1})); a_b = r m_{hb-1},
// a_t = r m_{ht-1}, c = 1/(1 - a_b a_t); FP64, rounded once.
inline void split_coupling(double r, int nz, float *ab, float *at, float *c) {
    const int hb = (nz + 1) / 2, ht = nz / 2;
    double m = 0.0, mb = 0.0, mt = 0.0;
    for (int k = 0; k < hb; ++k) {
        m = k == 0 ? 1.0 / (1.0 + r) : 1.0 / (1.0 + 2.0 * r - r * r * m);
        if (k == hb - 1) mb = m;
        if (k == ht - 1) mt = m;
    }
    const double a_b = ht >= 1 ? r * mb : 0.0, a_t = ht >= 1 ? r * mt : 0.0;
    *ab = (float)a_b;
    *at = (float)a_t;
    *c = (float)(1.0 / (1.0 - a_b * a_t));
}

// Device balancer (lb_device_balance.cu): limits, state words, history.
constexpr int kDevBalMaxVps = 8192;
constexpr int kDevBalMaxBins = 1024;
constexpr int kDevBalMaxSms = 1024;
constexpr int kBalHist = 1024;        // rows kept
constexpr int kBalHistCols = 8;       // step, strategy, migrations, predicted
                                      // max/mean, measured SM max/mean,
                                      // granularity floor, refine iterations,
                                      // 1 if the table was kept (threshold)
enum {
    kStHave = 0,       // 1 once costs exist (measured or set)
    kStRebal = 1,      // table rebalances so far (decides LB_AUTO*)
    kStMeasStep = 2,   // step index of the last measurement
    kStStrategy = 3,   // strategy of the current table
    kStHist = 4,       // history rows written
    kStForce = 5,      // 1: costs were rescaled, the next threshold test must rebalance
    kStKept = 6,       // 1: the last call kept the table (the table kernel skips)
    kStWords = 8
};

struct DevBal {
    int32_t nvps, nbins, nsm, nitems;
    double ema_alpha, refine_tol, fallback_ns_per_cycle;
    unsigned long long *vp_cycles;  // step kernel accumulators (reset here)
    unsigned long long *bin_busy;
    const int32_t *bin_smid;
    const long long *bin_cal;
    const long long *dclock;        // [0] step index
    int32_t *status;                // sticky device status
    unsigned *ticket;               // k_measure completion counter (0 between calls)
    double *cost;                   // [nvps] cost average, ns per step
    double *last;                   // [nvps] last measured cost, ns per step
    int32_t *assign;                // [nvps] VP -> processor
    int32_t *order;                 // [nvps] scratch: VPs by (cost desc, id asc)
    long long *q;                   // [nvps] scratch: costs on the fixed-point grid
    const int32_t *spatial;         // [nvps] VPs in spatial order
    const int32_t *nchunks;         // [nvps] work items per VP
    long long *state;               // [kStWords]
    double *pend;                   // [2] measured SM max/mean of the last measurement,
                                    // kappa of the last cost rescale
    double *hist;                   // [kBalHist][kBalHistCols]
    int2 *items;                    // processor tables (written)
    int32_t *bin_start;             // [nbins + 1] (written)
    // predictive cost model (lb_set_kc with predict_kc)
    const VPDev *vps;
    const GridDev *grids;
    int32_t cols_per_item;
    int32_t tile_w, tile_h;         // item shape (KernelInfo)
    double kc_overhead;             // fallback per-item overhead, in k_c sweeps
    double *feat1;                  // [nvps] items * nz
    double *feat2;                  // [nvps] sum over items of max k_c * nz (current array)
    double *feat_new;               // [nvps] the same for a new array
    double *fit;                    // [kFitBlocks][5] partial sums of the cost fit
};
constexpr int kFitThreads = 256;
constexpr int kFitBlocks = (kDevBalMaxVps + kFitThreads - 1) / kFitThreads;
size_t dev_balance_smem(int nvps, int nbins);
cudaError_t dev_balance_init();
cudaError_t dev_measure(const DevBal &p, cudaStream_t s);
cudaError_t dev_rebalance(const DevBal &p, int strategy, double threshold, cudaStream_t s);
// Point a grid's k_c source at a new array, in stream order.
cudaError_t dev_set_kc(GridDev *g, const int32_t *kc, cudaStream_t s);
// Predictive cost model: item features of `grid`'s VPs under array kc
// (into feat2 when initial, else feat_new and then rescale the averages).
cudaError_t dev_kc_features(const DevBal &p, int grid, const int32_t *kc, bool initial,
                            cudaStream_t s);

// Column copies of a sharded run (lb_shard.cu): pack (field -> buf) or
// unpack (buf -> field) n columns of nz levels; esize = storage bytes.
cudaError_t dev_columns(bool pack, void *field, int esize, const int32_t *cells, int n, int nz,
                        int nx, int ny, int pitch, void *buf, int32_t *status, cudaStream_t s);

// Text returned by lb_last_error(NULL) (calls without a ctx).
void set_ctxless_error(const char *msg);

// Host set-up shared by lb_create and lb_step_noalloc (lb_setup.cpp).
// Per-grid argument checks: nullptr when the descriptor is valid, else the
// reason (a static string).
const char *check_grid_desc(const lb_grid_desc &d);
// Pivots m[kNzMax] of the zero-flux operator: exact_nz > 0, the table of a
// column of that length; 0, the length-independent table (rows 0..nz-2 of
// any column), the last row coming from zero_flux_last_pivot.
void zero_flux_pivots(double r, int exact_nz, double *m);
double zero_flux_last_pivot(double r, int nz);
// From level kTwinS0 on, the FP32 forward multipliers m_s / m_inf are 1 and
// r m_s is one constant (the twin kernels' packed elimination).
bool twin_pivots_converge(double r);
// The converged pivot m_inf of the zero-flux elimination (1 when r = 0).
double converged_pivot(double r);
// At least 3/4 of the columns lie in VPs whose width is a multiple of 16,
// or a grid runs the Jacobi sweep: the twin kernels are the default.
bool layout_is_wide(const lb_vp *vps, int nvps, bool any_jacobi);
// The step kernel for these grids and VPs (the choice lb_create makes).
bool choose_step_kernel(const lb_grid_desc *grids, int ngrids, const lb_vp *vps, int nvps,
                        int threads_hint, bool staged, KernelInfo *out, int ctas_per_sm = 1);
// The pivot table and coefficients the chosen kernel reads.
void pivots_for_kernel(double r, const KernelInfo &k, double *m);
void fill_coef(double r, const KernelInfo &k, Coef<float> &c);
void fill_coef(double r, const KernelInfo &k, Coef<double> &c);
// The device record of one grid; kc_range is the device word the kernel
// sets when it clamps a k_c array entry.
void fill_grid_dev(const lb_grid_desc &d, int32_t *kc_range, GridDev &h);

}  // namespace lbk
