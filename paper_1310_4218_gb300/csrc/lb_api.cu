// C ABI of liblb.so: ctx life cycle, validation, work tables, launches,
// load measurement and rebalancing.  Declarations and contracts: lb.h.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_balance.h"
#include "lb_internal.h"

using namespace lbk;

struct lb_ctx {
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0;
    std::vector<lb_grid_desc> grids;
    std::vector<lb_vp> vps;
    lb_options opt;
    KernelInfo kinfo{};
    int nbins = 0, threads = 0, max_ctas_per_sm = 0, regs = 0;
    int storage = LB_F32, compute = LB_F32;
    size_t dyn_smem = 0;
    int nitems = 0;

    GridDev *d_grids = nullptr;
    VPDev *d_vps = nullptr;
    int2 *d_items = nullptr;     // processor-table order
    int2 *d_qitems = nullptr;    // queue order
    int32_t *d_bin_start = nullptr;
    unsigned *d_bar = nullptr;
    int32_t *d_status = nullptr;
    unsigned *d_qhead = nullptr;
    unsigned long long *d_vp_cycles = nullptr;
    unsigned long long *d_bin_busy = nullptr;
    int32_t *d_bin_smid = nullptr;
    long long *d_bin_cal = nullptr;
    double *d_bin_mass = nullptr;
    double *d_mass_hist = nullptr;
    long long *d_mass_t = nullptr;
    unsigned long long *d_mass_seq = nullptr;
    unsigned long long *d_sweeps = nullptr;
    long long *d_clock = nullptr;      // [step, parity] mirrored on the device
    unsigned *d_bin_ctr = nullptr;     // [2][nbins] per-processor counters (stealing)
    // device balancer: mirrors of cost / assign and its own state
    double *d_cost = nullptr;
    double *d_last = nullptr;
    int32_t *d_assign = nullptr;
    int32_t *d_order = nullptr;
    long long *d_q = nullptr;          // fixed-point costs (device balancer scratch)
    int32_t *d_spatial = nullptr;
    int32_t *d_nchunks = nullptr;
    long long *d_bstate = nullptr;
    double *d_pend = nullptr;
    double *d_bhist = nullptr;
    unsigned *d_ticket = nullptr;
    double *d_feat1 = nullptr, *d_feat2 = nullptr, *d_featn = nullptr;   // predictive cost model
    double *d_fit = nullptr;
    CUtensorMap *d_tmaps = nullptr;    // TMA-staged kernel: [ngrids][2] field maps
    // dataflow launches (lb_options.dataflow): one block holding the DfState,
    // the [kDfSlots][ngrids] step sums and the [nitems] done flags, zeroed
    // before each launch; the queue items' dependency lists (CSR)
    unsigned char *d_df = nullptr;
    size_t df_mass_off = 0, df_done_off = 0;
    int32_t *d_df_dep_start = nullptr;
    int32_t *d_df_deps = nullptr;
    size_t df_deps_cap = 0;
    int32_t *d_df_inl = nullptr;       // [nitems][kDfDeps] lists padded with -1
    bool df_inline = false;            // every item has at most kDfDeps
    bool predict = false;              // predict_kc active
    bool dev_newer = false;            // device balancer state newer than the host copy
    std::string devbal_off;            // why the device balancer is unavailable ("" = available)
    double fallback_npc = 1.0;
    long long cells = 0;               // cells of all grids
    long long cell_steps = 0;

    std::vector<GridDev> h_grids;
    std::vector<int> assign;           // VP -> processor (static-type strategies)
    std::vector<int> vp_nchunks;
    int strategy = LB_STATIC;
    bool queue_mode = false;
    int rebalances = 0;
    std::vector<double> cost;          // per-VP cost average, ns per step
    std::vector<double> last;          // per-VP cost of the last measurement
    bool have_costs = false;
    long long step = 0;
    int parity = 0;
    long long steps_since_measure = 0;
    Coef<float> coef_f;
    Coef<double> coef_d;
    struct GraphRec {
        int steps;      // time steps per replay
        bool balances;  // replays run the device balancer
    };
    std::map<cudaGraphExec_t, GraphRec> graph_steps;   // graphs made for this ctx
    std::string err;
};

static thread_local std::string g_create_err;

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return fail(ctx, LB_ECUDA, std::string(#call ": ") + \
                                                              cudaGetErrorString(e_)); \
    } while (0)

void lbk::set_ctxless_error(const char *msg) { g_create_err = msg; }

static lb_status fail(lb_ctx *ctx, lb_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return s;
}

static size_t dtype_size(int t) { return t == LB_F64 ? 8 : (t == LB_F32 ? 4 : 2); }

extern "C" void lb_default_options(lb_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->ctas_per_sm = 1;
    opt->queue_order = 0;
    opt->mass_every = 1;
    opt->device_balancer = 0;
    opt->ema_alpha = 0.5;
    opt->refine_tol = 0.05;
    opt->barrier_timeout_ns = 2000000000LL;
}

// ------------------------------------------------------------------ helpers
static DevBal make_devbal(lb_ctx *ctx);

// The device status words: [0] the sticky failure (lb_status), [1] the k_c
// range flag.  A failure is reported (and cleared) first, a clamp on the
// next call.
static lb_status check_status(lb_ctx *ctx) {
    int32_t w[2] = {0, 0};
    CK(cudaMemcpyAsync(w, ctx->d_status, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int32_t st = w[0];
    if (st == 0 && w[1] != 0) {
        int32_t zero = 0;
        CK(cudaMemcpyAsync(ctx->d_status + 1, &zero, sizeof(zero), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return fail(ctx, LB_EKCRANGE,
                    "k_c array entries above LB_KC_MAX were clamped to it in the steps since the "
                    "last report");
    }
    if (st != 0) {
        int32_t zero = 0;
        CK(cudaMemcpyAsync(ctx->d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (st == LB_ETIMEOUT)
            return fail(ctx, LB_ETIMEOUT, "grid barrier wait exceeded barrier_timeout_ns");
        if (st == LB_ENUMERIC) return fail(ctx, LB_ENUMERIC, "global sum is not finite");
        if (st == LB_ESTATE)
            return fail(ctx, LB_ESTATE,
                        "device balancer: no step since the last measurement, or no costs yet");
        if (st == LB_EINVAL)
            return fail(ctx, LB_EINVAL,
                        "a column index given to lb_pack_columns or lb_unpack_columns was outside "
                        "the grid (that column was skipped)");
        return fail(ctx, (lb_status)st, "device reported an error");
    }
    return LB_OK;
}

// Host copies of what the device balancer owns: costs, assignment and its
// state words.  The device copy is newer after lb_device_* calls and graph
// replays that balance (pull before the host reads), the host copy after
// every host-side change (push).
static lb_status pull_state(lb_ctx *ctx) {
    if (!ctx->dev_newer) return LB_OK;
    const size_t nv = ctx->vps.size();
    long long stw[kStWords];
    std::vector<int32_t> a(nv);
    CK(cudaMemcpyAsync(ctx->cost.data(), ctx->d_cost, sizeof(double) * nv, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->last.data(), ctx->d_last, sizeof(double) * nv, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(a.data(), ctx->d_assign, sizeof(int32_t) * nv, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(stw, ctx->d_bstate, sizeof(stw), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->assign.assign(a.begin(), a.end());
    ctx->have_costs = stw[kStHave] != 0;
    ctx->rebalances = (int)stw[kStRebal];
    ctx->steps_since_measure = ctx->step - stw[kStMeasStep];
    ctx->strategy = (int)stw[kStStrategy];
    ctx->dev_newer = false;
    return LB_OK;
}

static lb_status push_state(lb_ctx *ctx) {
    const size_t nv = ctx->vps.size();
    std::vector<int32_t> a(ctx->assign.begin(), ctx->assign.end());
    long long stw[4] = {ctx->have_costs ? 1 : 0, ctx->rebalances,
                        ctx->step - ctx->steps_since_measure, ctx->strategy};
    CK(cudaMemcpyAsync(ctx->d_cost, ctx->cost.data(), sizeof(double) * nv, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_last, ctx->last.data(), sizeof(double) * nv, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_assign, a.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_bstate, stw, sizeof(stw), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LB_OK;
}

// VP ids in spatial order: grid, then row, then column (then id).
static std::vector<int> spatial_order(const lb_ctx *ctx) {
    std::vector<int> order(ctx->vps.size());
    for (size_t v = 0; v < order.size(); ++v) order[v] = (int)v;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const lb_vp &A = ctx->vps[a], &B = ctx->vps[b];
        if (A.grid != B.grid) return A.grid < B.grid;
        if (A.y0 != B.y0) return A.y0 < B.y0;
        if (A.x0 != B.x0) return A.x0 < B.x0;
        return a < b;
    });
    return order;
}

// Work items {vp, chunk} for the processor tables and the queue.
// Dataflow launches: for each queue item, the queue items owning a column
// of its closed 4-neighbourhood (periodic, itself included), as CSR.  The
// columns of an item are those the kernel gives its lanes: cols_per_item
// consecutive columns of the VP in row-major order.
static void df_dependencies(const lb_ctx *ctx, const std::vector<int2> &qitems,
                            std::vector<int32_t> &start, std::vector<int32_t> &deps) {
    const int cpi = ctx->kinfo.cols_per_item;
    std::vector<std::vector<int32_t>> owner(ctx->grids.size());
    for (size_t g = 0; g < ctx->grids.size(); ++g)
        owner[g].assign((size_t)ctx->grids[g].nx * ctx->grids[g].ny, -1);
    auto each_col = [&](int q, auto &&fn) {
        const int2 it = qitems[q];
        const lb_vp &vp = ctx->vps[it.x];
        const int ncols = vp.w * vp.h;
        for (int l = 0; l < cpi; ++l) {
            const int k = it.y * cpi + l;
            if (k >= ncols) break;
            const int ly = k / vp.w;
            fn(vp.grid, vp.x0 + (k - ly * vp.w), vp.y0 + ly);
        }
    };
    for (int q = 0; q < (int)qitems.size(); ++q)
        each_col(q, [&](int g, int i, int j) { owner[g][(size_t)j * ctx->grids[g].nx + i] = q; });
    start.assign(qitems.size() + 1, 0);
    deps.clear();
    std::vector<int32_t> nb;
    const int di[5] = {0, 1, -1, 0, 0}, dj[5] = {0, 0, 0, 1, -1};
    for (int q = 0; q < (int)qitems.size(); ++q) {
        nb.clear();
        each_col(q, [&](int g, int i, int j) {
            const int nx = ctx->grids[g].nx, ny = ctx->grids[g].ny;
            for (int d = 0; d < 5; ++d) {
                const int ii = (i + di[d] + nx) % nx, jj = (j + dj[d] + ny) % ny;
                const int o = owner[g][(size_t)jj * nx + ii];
                if (o >= 0) nb.push_back(o);
            }
        });
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        deps.insert(deps.end(), nb.begin(), nb.end());
        start[q + 1] = (int32_t)deps.size();
    }
}

static lb_status upload_items(lb_ctx *ctx) {
    const int nv = (int)ctx->vps.size();
    std::vector<int2> items;
    items.reserve(ctx->nitems);
    std::vector<int32_t> start(ctx->nbins + 1, 0);
    std::vector<std::vector<int>> per(ctx->nbins);
    for (int v = 0; v < nv; ++v) per[ctx->assign[v]].push_back(v);
    // each processor visits its VPs in spatial order (grid, row, column): all
    // processors then sweep the grids in the same direction at about the
    // same pace, so the halo and boundary sectors a VP shares with its
    // neighbours are still in L2 when the neighbour needs them
    for (auto &lst : per)
        std::sort(lst.begin(), lst.end(), [&](int a, int b) {
            const lb_vp &A = ctx->vps[a], &B = ctx->vps[b];
            if (A.grid != B.grid) return A.grid < B.grid;
            if (A.y0 != B.y0) return A.y0 < B.y0;
            if (A.x0 != B.x0) return A.x0 < B.x0;
            return a < b;
        });
    for (int b = 0; b < ctx->nbins; ++b) {
        start[b] = (int32_t)items.size();
        for (int v : per[b])
            for (int c = 0; c < ctx->vp_nchunks[v]; ++c) items.push_back(make_int2(v, c));
    }
    start[ctx->nbins] = (int32_t)items.size();
    std::vector<int> order(nv);
    for (int v = 0; v < nv; ++v) order[v] = v;
    if (ctx->opt.queue_order == 1 && ctx->have_costs)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return ctx->cost[a] > ctx->cost[b]; });
    std::vector<int2> qitems;
    qitems.reserve(ctx->nitems);
    for (int v : order)
        for (int c = 0; c < ctx->vp_nchunks[v]; ++c) qitems.push_back(make_int2(v, c));
    // pageable sources are staged before these calls return; the copies are
    // ordered on the ctx stream after any step already enqueued
    CK(cudaMemcpyAsync(ctx->d_items, items.data(), sizeof(int2) * items.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_qitems, qitems.data(), sizeof(int2) * qitems.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_bin_start, start.data(), sizeof(int32_t) * start.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int32_t> dstart, deps, inl;
    if (ctx->d_df) {
        df_dependencies(ctx, qitems, dstart, deps);
        if (deps.size() > ctx->df_deps_cap) {
            // the old list may still be read by a launch in flight: cudaFree
            // waits for the device
            if (ctx->d_df_deps) cudaFree(ctx->d_df_deps);
            ctx->d_df_deps = nullptr;
            ctx->df_deps_cap = 0;
            CK(cudaMalloc((void **)&ctx->d_df_deps, sizeof(int32_t) * std::max<size_t>(deps.size(), 1)));
            ctx->df_deps_cap = deps.size();
        }
        CK(cudaMemcpyAsync(ctx->d_df_dep_start, dstart.data(), sizeof(int32_t) * dstart.size(),
                           cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_df_deps, deps.data(), sizeof(int32_t) * deps.size(),
                           cudaMemcpyHostToDevice, ctx->stream));
        ctx->df_inline = true;
        for (size_t q = 0; q + 1 < dstart.size(); ++q)
            ctx->df_inline = ctx->df_inline && dstart[q + 1] - dstart[q] <= kDfDeps;
        if (ctx->df_inline) {
            inl.assign((dstart.size() - 1) * kDfDeps, -1);
            for (size_t q = 0; q + 1 < dstart.size(); ++q)
                for (int32_t k = dstart[q]; k < dstart[q + 1]; ++k)
                    inl[q * kDfDeps + (k - dstart[q])] = deps[k];
            CK(cudaMemcpyAsync(ctx->d_df_inl, inl.data(), sizeof(int32_t) * inl.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return push_state(ctx);
}

static void free_ctx(lb_ctx *ctx) {
    void *ptrs[] = {ctx->d_grids,     ctx->d_vps,      ctx->d_items,     ctx->d_qitems,
                    ctx->d_bin_start, ctx->d_bar,      ctx->d_status,    ctx->d_qhead,
                    ctx->d_vp_cycles, ctx->d_bin_busy, ctx->d_bin_smid,  ctx->d_bin_cal,
                    ctx->d_bin_mass,  ctx->d_mass_hist, ctx->d_mass_t,   ctx->d_mass_seq,
                    ctx->d_sweeps,    ctx->d_clock,    ctx->d_bin_ctr,   ctx->d_cost,
                    ctx->d_last,      ctx->d_assign,   ctx->d_order,     ctx->d_spatial,
                    ctx->d_nchunks,   ctx->d_bstate,   ctx->d_pend,      ctx->d_bhist,
                    ctx->d_ticket,    ctx->d_q,        ctx->d_feat1,     ctx->d_feat2,
                    ctx->d_featn,     ctx->d_fit,      ctx->d_tmaps,     ctx->d_df,
                    ctx->d_df_dep_start, ctx->d_df_deps, ctx->d_df_inl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete ctx;
}

template <class T>
static cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(n, 1));
}

// ------------------------------------------------------------------ TMA maps
// Tensor maps of every grid's two field buffers for the TMA-staged kernel:
// FP32, dims (nx, ny, nz) x-fastest, box kBoxW x kBoxH x nz (the 12 x 3
// column neighbourhood of an 8 x 2 tile, all levels), zero fill outside.
// The kernel applies when every buffer is 16-byte aligned and rows are a
// multiple of 16 bytes (nx % 4 == 0), TMA's addressing rules.
static bool staged_eligible(const std::vector<lb_grid_desc> &grids) {
    for (const auto &d : grids) {
        // the box holds the upwind neighbours only: advection grids
        if (d.dynamics != 0) return false;
        if (d.storage != LB_F32 || d.compute != LB_F32 || d.nx % 4 != 0) return false;
        if ((d.pitch ? d.pitch : d.nx) % 4 != 0) return false;
        if ((reinterpret_cast<uintptr_t>(d.q0) | reinterpret_cast<uintptr_t>(d.q1)) & 15u) return false;
    }
    return true;
}

static bool encode_tmaps(const std::vector<lb_grid_desc> &grids, int nz_box,
                         std::vector<CUtensorMap> &maps, std::string &why) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    maps.assign(2 * grids.size(), CUtensorMap{});
    for (size_t g = 0; g < grids.size(); ++g) {
        const lb_grid_desc &d = grids[g];
        const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
        const cuuint64_t pitch = (cuuint64_t)(d.pitch ? d.pitch : d.nx);
        const cuuint64_t strides[2] = {pitch * 4, pitch * d.ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)kBoxH, (cuuint32_t)nz_box};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2; ++b) {
            CUresult r = encode(&maps[2 * g + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                b ? d.q1 : d.q0, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
                return false;
            }
        }
    }
    return true;
}

// ------------------------------------------------------------------ create
static lb_status validate(const lb_grid_desc *grids, int32_t ngrids, const lb_vp *vps,
                          int32_t nvps) {
    if (!grids || ngrids < 1 || ngrids > kMaxGrids)
        return fail(nullptr, LB_EINVAL, "ngrids must be in 1..512 and grids non-NULL");
    if (!vps || nvps < 1) return fail(nullptr, LB_EINVAL, "need at least one VP");
    for (int g = 0; g < ngrids; ++g) {
        const lb_grid_desc &d = grids[g];
        const std::string pre = "grid " + std::to_string(g) + ": ";
        if (const char *why = check_grid_desc(d)) return fail(nullptr, LB_EINVAL, pre + why);
        if (d.storage != grids[0].storage || d.compute != grids[0].compute)
            return fail(nullptr, LB_EINVAL, pre + "all grids must share storage and compute");
        if (d.r != grids[0].r) return fail(nullptr, LB_EINVAL, pre + "all grids must share r");
    }
    // the VPs must tile every grid exactly
    std::vector<std::vector<unsigned char>> cover(ngrids);
    for (int g = 0; g < ngrids; ++g) cover[g].assign((size_t)grids[g].nx * grids[g].ny, 0);
    for (int v = 0; v < nvps; ++v) {
        const lb_vp &p = vps[v];
        if (p.grid < 0 || p.grid >= ngrids)
            return fail(nullptr, LB_EINVAL, "VP " + std::to_string(v) + ": grid out of range");
        const lb_grid_desc &d = grids[p.grid];
        if (p.w < 1 || p.h < 1 || p.x0 < 0 || p.y0 < 0 || p.x0 + p.w > d.nx || p.y0 + p.h > d.ny)
            return fail(nullptr, LB_EINVAL, "VP " + std::to_string(v) + ": outside its grid");
        for (int j = p.y0; j < p.y0 + p.h; ++j)
            for (int i = p.x0; i < p.x0 + p.w; ++i) {
                unsigned char &c = cover[p.grid][(size_t)j * d.nx + i];
                if (c) return fail(nullptr, LB_EINVAL, "VP " + std::to_string(v) + ": overlaps another VP");
                c = 1;
            }
    }
    for (int g = 0; g < ngrids; ++g)
        for (unsigned char c : cover[g])
            if (!c) return fail(nullptr, LB_EINVAL, "grid " + std::to_string(g) + ": VPs leave a gap");
    return LB_OK;
}

extern "C" lb_status lb_create(const lb_grid_desc *grids, int32_t ngrids, const lb_vp *vps,
                               int32_t nvps, const lb_options *opt, void *cuda_stream,
                               lb_ctx **out) {
    if (!out) return fail(nullptr, LB_EINVAL, "out is NULL");
    *out = nullptr;
    lb_status st = validate(grids, ngrids, vps, nvps);
    if (st != LB_OK) return st;
    lb_ctx *ctx = new lb_ctx();
    if (opt) ctx->opt = *opt;
    else lb_default_options(&ctx->opt);
    if (ctx->opt.ctas_per_sm < 1) ctx->opt.ctas_per_sm = 1;
    if (ctx->opt.mass_every < 0) ctx->opt.mass_every = 0;
    ctx->opt.dataflow = ctx->opt.dataflow ? 1 : 0;
    if (!(ctx->opt.ema_alpha > 0.0 && ctx->opt.ema_alpha <= 1.0)) ctx->opt.ema_alpha = 0.5;
    if (!(ctx->opt.refine_tol >= 0.0)) ctx->opt.refine_tol = 0.05;
    if (ctx->opt.barrier_timeout_ns <= 0) ctx->opt.barrier_timeout_ns = 2000000000LL;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->grids.assign(grids, grids + ngrids);
    ctx->vps.assign(vps, vps + nvps);
    ctx->storage = grids[0].storage;
    ctx->compute = grids[0].compute;

    auto bail = [&](lb_status s) {
        g_create_err = ctx->err;
        free_ctx(ctx);
        return s;
    };
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (e != cudaSuccess) {
        ctx->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return bail(LB_ECUDA);
    }
    if (!coop) {
        ctx->err = "device does not support cooperative launch";
        return bail(LB_ENORESIDENT);
    }

    // kernel variant: twin halves for FP32 grids where the FP32 pivots
    // converge, else split columns on half-warps (threads_hint overrides)
    const bool staged = ctx->opt.staged_loads && staged_eligible(ctx->grids);
    if (!choose_step_kernel(grids, ngrids, vps, nvps, ctx->opt.threads_hint, staged, &ctx->kinfo,
                            ctx->opt.ctas_per_sm)) {
        ctx->err = "no kernel variant for these grids";
        return bail(LB_EINVAL);
    }
    std::vector<CUtensorMap> maps;
    if (ctx->kinfo.tma_slots > 0) {
        // the ring and the per-warp sums must fit the shared memory of a CTA
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        const size_t need = 128 + (size_t)ctx->kinfo.tma_slots * ctx->kinfo.tma_slot_bytes +
                            sizeof(double) * (size_t)(ctx->kinfo.threads / kWarp) * ngrids + 4096;
        std::string why;
        if (need > (size_t)optin || !encode_tmaps(ctx->grids, ctx->kinfo.nz_variant, maps, why)) {
            // register-load kernel instead
            maps.clear();
            choose_step_kernel(grids, ngrids, vps, nvps, ctx->opt.threads_hint, false, &ctx->kinfo,
                               ctx->opt.ctas_per_sm);
        }
    }
    ctx->threads = ctx->kinfo.threads;
    ctx->dyn_smem = step_dyn_smem(ctx->kinfo, ngrids);
    if (ctx->kinfo.tma_slots > 0)
        ctx->dyn_smem += 128 + (size_t)ctx->kinfo.tma_slots * ctx->kinfo.tma_slot_bytes;
    if (ctx->dyn_smem > 48 * 1024) {
        // the limit is per kernel, not per ctx: raise it to the device
        // maximum so that no ctx lowers it under another one's needs
        int optin = 0;
        cudaFuncAttributes fa0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa0, ctx->kinfo.fn);
        if (e == cudaSuccess && ctx->dyn_smem + fa0.sharedSizeBytes > (size_t)optin) {
            ctx->err = "work tables need more shared memory than the device has";
            return bail(LB_EINVAL);
        }
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ctx->kinfo.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa0.sharedSizeBytes);
        if (e != cudaSuccess) {
            ctx->err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return bail(LB_ECUDA);
        }
    }
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, ctx->kinfo.fn);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->max_ctas_per_sm, ctx->kinfo.fn,
                                                          ctx->threads, ctx->dyn_smem);
    if (e != cudaSuccess) {
        ctx->err = std::string("occupancy query: ") + cudaGetErrorString(e);
        return bail(LB_ECUDA);
    }
    ctx->regs = fa.numRegs;
    if (ctx->max_ctas_per_sm < ctx->opt.ctas_per_sm) {
        ctx->err = "requested processors per SM cannot be co-resident (max " +
                   std::to_string(ctx->max_ctas_per_sm) + ")";
        return bail(LB_ENORESIDENT);
    }
    ctx->nbins = ctx->opt.ctas_per_sm * ctx->nsm;

    // coefficients and grid table (the k_c range flag pointer is set once
    // the status words exist)
    fill_coef(grids[0].r, ctx->kinfo, ctx->coef_d);
    fill_coef(grids[0].r, ctx->kinfo, ctx->coef_f);
    ctx->h_grids.resize(ngrids);
    for (int g = 0; g < ngrids; ++g) ctx->cells += (long long)grids[g].nx * grids[g].ny * grids[g].nz;
    for (int g = 0; g < ngrids; ++g) fill_grid_dev(grids[g], nullptr, ctx->h_grids[g]);

    // VP table and work items
    std::vector<VPDev> hv(nvps);
    ctx->vp_nchunks.resize(nvps);
    ctx->nitems = 0;
    for (int v = 0; v < nvps; ++v) {
        const lb_vp &p = vps[v];
        hv[v] = VPDev{p.grid, p.x0, p.y0, p.w, p.h, p.w * p.h, 0, 0};
        ctx->vp_nchunks[v] = items_of_vp(ctx->kinfo, p.w, p.h);
        ctx->nitems += ctx->vp_nchunks[v];
    }
    static_blocks(nvps, ctx->nbins, ctx->assign);
    ctx->cost.assign(nvps, 0.0);
    ctx->last.assign(nvps, 0.0);

    const int nb = ctx->nbins;
    e = dalloc(&ctx->d_grids, ngrids);
    if (e == cudaSuccess) e = dalloc(&ctx->d_vps, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_items, ctx->nitems);
    if (e == cudaSuccess) e = dalloc(&ctx->d_qitems, ctx->nitems);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_start, nb + 1);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bar, 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_status, 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_qhead, 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_vp_cycles, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_busy, nb);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_smid, nb);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_cal, 4 * (size_t)nb);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_mass, 2 * (size_t)nb * ngrids);
    if (e == cudaSuccess) e = dalloc(&ctx->d_mass_hist, (size_t)kMassHist * ngrids * 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_mass_t, kMassHist);
    if (e == cudaSuccess) e = dalloc(&ctx->d_mass_seq, 1);
    if (e == cudaSuccess) e = dalloc(&ctx->d_sweeps, 1);
    if (e == cudaSuccess) e = dalloc(&ctx->d_clock, 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bin_ctr, 2 * (size_t)nb);
    if (e == cudaSuccess) e = dalloc(&ctx->d_cost, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_last, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_assign, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_order, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_q, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_feat1, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_feat2, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_featn, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_fit, (size_t)kFitBlocks * 5);
    if (e == cudaSuccess) e = dalloc(&ctx->d_spatial, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_nchunks, nvps);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bstate, kStWords);
    if (e == cudaSuccess) e = dalloc(&ctx->d_pend, 2);
    if (e == cudaSuccess) e = dalloc(&ctx->d_bhist, (size_t)kBalHist * kBalHistCols);
    if (e == cudaSuccess) e = dalloc(&ctx->d_ticket, 1);
    if (e == cudaSuccess && !maps.empty()) e = dalloc(&ctx->d_tmaps, maps.size());
    if (e == cudaSuccess && ctx->opt.dataflow && ctx->kinfo.df_fn) {
        ctx->df_mass_off = (sizeof(DfState) + 255) / 256 * 256;
        ctx->df_done_off =
            ctx->df_mass_off + (sizeof(double) * kDfSlots * (size_t)ngrids + 255) / 256 * 256;
        e = dalloc(&ctx->d_df, ctx->df_done_off + sizeof(int32_t) * (size_t)ctx->nitems);
        if (e == cudaSuccess) e = dalloc(&ctx->d_df_dep_start, (size_t)ctx->nitems + 1);
        if (e == cudaSuccess) e = dalloc(&ctx->d_df_inl, (size_t)ctx->nitems * kDfDeps);
    }
    if (e == cudaSuccess && !maps.empty())
        e = cudaMemcpyAsync(ctx->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                            cudaMemcpyHostToDevice, ctx->stream);
    const std::vector<int> sp = spatial_order(ctx);
    std::vector<int32_t> sp32(sp.begin(), sp.end()), nch(ctx->vp_nchunks.begin(), ctx->vp_nchunks.end());
    cudaStream_t sm = ctx->stream;
    for (auto &h : ctx->h_grids) h.kc_range = ctx->d_status + 1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_grids, ctx->h_grids.data(), sizeof(GridDev) * ngrids,
                            cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_vps, hv.data(), sizeof(VPDev) * nvps, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, 2 * sizeof(int32_t), sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_vp_cycles, 0, sizeof(unsigned long long) * nvps, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bin_busy, 0, sizeof(unsigned long long) * nb, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_mass_seq, 0, sizeof(unsigned long long), sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_sweeps, 0, sizeof(unsigned long long), sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_clock, 0, 2 * sizeof(long long), sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bin_cal, 0, sizeof(long long) * 4 * nb, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bin_smid, 0xff, sizeof(int32_t) * nb, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_spatial, sp32.data(), sizeof(int32_t) * nvps, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_nchunks, nch.data(), sizeof(int32_t) * nvps, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bstate, 0, sizeof(long long) * kStWords, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_pend, 0, sizeof(double) * 2, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_ticket, 0, sizeof(unsigned), sm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) {
        ctx->err = std::string("device tables: ") + cudaGetErrorString(e);
        return bail(LB_ECUDA);
    }
    {
        int khz = 0;
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
        ctx->fallback_npc = khz > 0 ? 1e6 / khz : 1.0;
    }
    if (nvps > kDevBalMaxVps) ctx->devbal_off = "more than " + std::to_string(kDevBalMaxVps) + " VPs";
    else if (nb > kDevBalMaxBins) ctx->devbal_off = "more than " + std::to_string(kDevBalMaxBins) + " processors";
    else if (ctx->nsm > kDevBalMaxSms) ctx->devbal_off = "more SMs than the device balancer handles";
    else if (dev_balance_init() != cudaSuccess) {
        cudaGetLastError();
        ctx->devbal_off = "device balancer kernel needs more shared memory than the device offers";
    }
    st = upload_items(ctx);
    if (st != LB_OK) return bail(st);
    if (ctx->opt.predict_kc && ctx->devbal_off.empty()) {
        // item features: f1 = items * nz per VP, f2 under each array's k_c
        std::vector<double> f1(nvps), zero(nvps, 0.0);
        for (int v = 0; v < nvps; ++v) f1[v] = (double)ctx->vp_nchunks[v] * grids[vps[v].grid].nz;
        e = cudaMemcpyAsync(ctx->d_feat1, f1.data(), sizeof(double) * nvps, cudaMemcpyHostToDevice, sm);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->d_feat2, zero.data(), sizeof(double) * nvps, cudaMemcpyHostToDevice, sm);
        for (int g = 0; g < ngrids && e == cudaSuccess; ++g)
            if (!grids[g].kc_disk) e = dev_kc_features(make_devbal(ctx), g, grids[g].kc, true, sm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
        if (e != cudaSuccess) {
            ctx->err = std::string("cost model features: ") + cudaGetErrorString(e);
            return bail(LB_ECUDA);
        }
        ctx->predict = true;
    }
    *out = ctx;
    return LB_OK;
}

// ------------------------------------------------------------------ step
// lb_step runs the dataflow kernel: asked for, the kernel has one, queue mode
static bool df_active(const lb_ctx *ctx) {
    return ctx->d_df && ctx->kinfo.df_fn && ctx->queue_mode;
}

template <class TC>
static lb_status launch(lb_ctx *ctx, int nsteps, const Coef<TC> &coef, int serial_warps = 0) {
    StepParams<TC> p;
    std::memset(&p, 0, sizeof(p));
    p.serial_warps = serial_warps;
    p.grids = ctx->d_grids;
    p.vps = ctx->d_vps;
    p.items = ctx->queue_mode ? ctx->d_qitems : ctx->d_items;
    p.bin_start = ctx->d_bin_start;
    p.ngrids = (int)ctx->grids.size();
    p.nvps = (int)ctx->vps.size();
    p.nbins = ctx->nbins;
    p.nitems = ctx->nitems;
    p.queue_mode = ctx->queue_mode ? 1 : 0;
    p.mass_every = ctx->opt.mass_every;
    p.parity0 = ctx->parity;
    p.nsteps = nsteps;
    p.t0 = ctx->step;
    p.timeout_ns = ctx->opt.barrier_timeout_ns;
    p.bar = ctx->d_bar;
    p.status = ctx->d_status;
    p.qhead = ctx->d_qhead;
    p.vp_cycles = ctx->d_vp_cycles;
    p.bin_busy = ctx->d_bin_busy;
    p.bin_smid = ctx->d_bin_smid;
    p.bin_cal = ctx->d_bin_cal;
    p.bin_mass = ctx->d_bin_mass;
    p.mass_hist = ctx->d_mass_hist;
    p.mass_t = ctx->d_mass_t;
    p.mass_seq = ctx->d_mass_seq;
    p.sweeps = ctx->d_sweeps;
    p.dclock = ctx->d_clock;
    p.bin_ctr = ctx->d_bin_ctr;
    p.steal = ctx->opt.steal ? 1 : 0;
    p.tmaps = ctx->d_tmaps;
    p.coef = coef;

    CK(cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_qhead, 0, 2 * sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_bin_ctr, 0, 2 * sizeof(unsigned) * ctx->nbins, ctx->stream));
    const bool df = df_active(ctx) && serial_warps == 0;
    if (df) {
        p.df = reinterpret_cast<DfState *>(ctx->d_df);
        p.df_mass = reinterpret_cast<double *>(ctx->d_df + ctx->df_mass_off);
        p.df_done = reinterpret_cast<int32_t *>(ctx->d_df + ctx->df_done_off);
        p.df_dep_start = ctx->d_df_dep_start;
        p.df_deps = ctx->d_df_deps;
        p.df_inl = ctx->df_inline ? ctx->d_df_inl : nullptr;
        CK(cudaMemsetAsync(ctx->d_df, 0, ctx->df_done_off + sizeof(int32_t) * ctx->nitems,
                           ctx->stream));
    }
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(ctx->nbins);
    cfg.blockDim = dim3(ctx->threads);
    cfg.dynamicSmemBytes = df ? 0 : ctx->dyn_smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&p};
    CK(cudaLaunchKernelExC(&cfg, df ? ctx->kinfo.df_fn : ctx->kinfo.fn, args));
    return LB_OK;
}

static lb_status step_launch(lb_ctx *ctx, int32_t nsteps, int serial_warps) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, LB_EINVAL, "nsteps < 0");
    if (nsteps == 0) return LB_OK;
    lb_status st = ctx->compute == LB_F64 ? launch<double>(ctx, nsteps, ctx->coef_d, serial_warps)
                                          : launch<float>(ctx, nsteps, ctx->coef_f, serial_warps);
    if (st != LB_OK) return st;
    ctx->step += nsteps;
    ctx->cell_steps += ctx->cells * nsteps;
    ctx->parity ^= (nsteps & 1);
    ctx->steps_since_measure += nsteps;
    return LB_OK;
}

extern "C" lb_status lb_step(lb_ctx *ctx, int32_t nsteps) { return step_launch(ctx, nsteps, 0); }

extern "C" lb_status lb_step_serial(lb_ctx *ctx, int32_t nsteps) {
    if (ctx && (ctx->kinfo.tma_slots > 0 || (ctx->kinfo.tile_w == 16 && ctx->kinfo.split)))
        return fail(ctx, LB_ESTATE,
                    "lb_step_serial: the TMA-staged and paired-warp kernels run every warp");
    return step_launch(ctx, nsteps, 1);
}

// ------------------------------------------------------------------ graphs
extern "C" lb_status lb_graph_create(lb_ctx *ctx, int32_t nsteps, void **graph_exec) {
    if (!ctx || !graph_exec || nsteps < 1) return fail(ctx, LB_EINVAL, "lb_graph_create: bad arguments");
    *graph_exec = nullptr;
    CK(cudaStreamSynchronize(ctx->stream));
    // capture on a private stream: the ctx stream may be the legacy default
    // stream, which cannot be captured; the graph does not depend on it
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t own = ctx->stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    lb_status st = LB_OK;
    if (e == cudaSuccess) {
        ctx->stream = cap;
        st = ctx->compute == LB_F64 ? launch<double>(ctx, nsteps, ctx->coef_d)
                                    : launch<float>(ctx, nsteps, ctx->coef_f);
        ctx->stream = own;
        e = cudaStreamEndCapture(cap, &graph);
    }
    cudaStreamDestroy(cap);
    if (st != LB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(ctx, LB_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, LB_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    ctx->graph_steps[exec] = lb_ctx::GraphRec{nsteps, false};
    *graph_exec = exec;
    return LB_OK;
}

extern "C" lb_status lb_graph_launch(lb_ctx *ctx, void *graph_exec) {
    if (!ctx || !graph_exec) return fail(ctx, LB_EINVAL, "lb_graph_launch: bad arguments");
    auto it = ctx->graph_steps.find((cudaGraphExec_t)graph_exec);
    if (it == ctx->graph_steps.end()) return fail(ctx, LB_EINVAL, "graph was not made for this ctx");
    CK(cudaGraphLaunch((cudaGraphExec_t)graph_exec, ctx->stream));
    const int n = it->second.steps;
    ctx->step += n;
    ctx->cell_steps += ctx->cells * n;
    ctx->parity ^= (n & 1);
    ctx->steps_since_measure += n;
    if (it->second.balances) ctx->dev_newer = true;
    return LB_OK;
}

extern "C" lb_status lb_graph_destroy(lb_ctx *ctx, void *graph_exec) {
    if (!ctx || !graph_exec) return fail(ctx, LB_EINVAL, "lb_graph_destroy: bad arguments");
    ctx->graph_steps.erase((cudaGraphExec_t)graph_exec);
    CK(cudaGraphExecDestroy((cudaGraphExec_t)graph_exec));
    return LB_OK;
}

// ------------------------------------------------------------------ device balancer
static DevBal make_devbal(lb_ctx *ctx) {
    DevBal p;
    std::memset(&p, 0, sizeof(p));
    p.nvps = (int)ctx->vps.size();
    p.nbins = ctx->nbins;
    p.nsm = ctx->nsm;
    p.nitems = ctx->nitems;
    p.ema_alpha = ctx->opt.ema_alpha;
    p.refine_tol = ctx->opt.refine_tol;
    p.fallback_ns_per_cycle = ctx->fallback_npc;
    p.vp_cycles = ctx->d_vp_cycles;
    p.bin_busy = ctx->d_bin_busy;
    p.bin_smid = ctx->d_bin_smid;
    p.bin_cal = ctx->d_bin_cal;
    p.dclock = ctx->d_clock;
    p.status = ctx->d_status;
    p.ticket = ctx->d_ticket;
    p.cost = ctx->d_cost;
    p.last = ctx->d_last;
    p.assign = ctx->d_assign;
    p.order = ctx->d_order;
    p.q = ctx->d_q;
    p.spatial = ctx->d_spatial;
    p.nchunks = ctx->d_nchunks;
    p.state = ctx->d_bstate;
    p.pend = ctx->d_pend;
    p.hist = ctx->d_bhist;
    p.items = ctx->d_items;
    p.bin_start = ctx->d_bin_start;
    p.vps = ctx->d_vps;
    p.grids = ctx->d_grids;
    p.cols_per_item = ctx->kinfo.cols_per_item;
    p.tile_w = ctx->kinfo.tile_w;
    p.tile_h = ctx->kinfo.tile_h;
    p.kc_overhead = 6.0;
    p.feat1 = ctx->d_feat1;
    p.feat2 = ctx->d_feat2;
    p.feat_new = ctx->d_featn;
    p.fit = ctx->d_fit;
    return p;
}

static bool table_strategy(int s) {
    return s == LB_STATIC || s == LB_GREEDY || s == LB_REFINE_SWAP || s == LB_AUTO ||
           s == LB_GREEDY_SPATIAL || s == LB_AUTO_SPATIAL || s == LB_GREEDY_BLOCKED;
}

static lb_status devbal_check(lb_ctx *ctx, int strategy, bool need_strategy) {
    if (!ctx->devbal_off.empty())
        return fail(ctx, LB_EINVAL, "device balancer unavailable: " + ctx->devbal_off);
    if (need_strategy && strategy == LB_ATOMIC_QUEUE) {
        if (!ctx->queue_mode)
            return fail(ctx, LB_ESTATE, "device balancer: LB_ATOMIC_QUEUE records queue-mode periods; "
                                        "enter queue mode with lb_rebalance");
        return LB_OK;
    }
    if (need_strategy && !table_strategy(strategy))
        return fail(ctx, LB_EINVAL, "device balancer: unknown strategy");
    if (need_strategy && ctx->queue_mode)
        return fail(ctx, LB_ESTATE, "device balancer: ctx is in atomic-queue mode (leave it with lb_rebalance)");
    return LB_OK;
}

extern "C" lb_status lb_device_measure(lb_ctx *ctx) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = devbal_check(ctx, 0, false);
    if (st != LB_OK) return st;
    CK(dev_measure(make_devbal(ctx), ctx->stream));
    ctx->dev_newer = true;
    return LB_OK;
}

extern "C" lb_status lb_device_rebalance_if(lb_ctx *ctx, int32_t strategy, double threshold) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (!(threshold == threshold)) return fail(ctx, LB_EINVAL, "threshold is NaN");
    lb_status st = devbal_check(ctx, strategy, true);
    if (st != LB_OK) return st;
    CK(dev_rebalance(make_devbal(ctx), strategy, threshold, ctx->stream));
    ctx->dev_newer = true;
    return LB_OK;
}

extern "C" lb_status lb_device_rebalance(lb_ctx *ctx, int32_t strategy) {
    return lb_device_rebalance_if(ctx, strategy, 0.0);
}

extern "C" lb_status lb_get_costs(lb_ctx *ctx, double *avg_ns, double *last_ns) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    st = pull_state(ctx);
    if (st != LB_OK) return st;
    for (size_t v = 0; v < ctx->vps.size(); ++v) {
        if (avg_ns) avg_ns[v] = ctx->cost[v];
        if (last_ns) last_ns[v] = ctx->last[v];
    }
    return LB_OK;
}

extern "C" lb_status lb_balance_history(lb_ctx *ctx, double *rows, int32_t max, int32_t *n) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    long long stw[kStWords];
    CK(cudaMemcpyAsync(stw, ctx->d_bstate, sizeof(stw), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const long long written = stw[kStHist];
    const long long cnt = std::min<long long>(std::min<long long>(written, kBalHist), std::max(max, 0));
    if (n) *n = (int32_t)cnt;
    if (cnt == 0 || !rows) return LB_OK;
    std::vector<double> h((size_t)kBalHist * kBalHistCols);
    CK(cudaMemcpyAsync(h.data(), ctx->d_bhist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (long long i = 0; i < cnt; ++i) {
        const long long r = (written - cnt + i) % kBalHist;
        for (int c = 0; c < kBalHistCols; ++c) rows[i * kBalHistCols + c] = h[(size_t)r * kBalHistCols + c];
    }
    return LB_OK;
}

extern "C" lb_status lb_graph_create_periods(lb_ctx *ctx, int32_t nsteps, int32_t strategy,
                                             int32_t nperiods, double threshold,
                                             void **graph_exec) {
    if (!ctx || !graph_exec || nsteps < 1 || nperiods < 1 || !(threshold == threshold))
        return fail(ctx, LB_EINVAL, "lb_graph_create_periods: bad arguments");
    *graph_exec = nullptr;
    lb_status st = devbal_check(ctx, strategy, true);
    if (st != LB_OK) return st;
    if ((long long)nsteps * nperiods > 0x7fffffffLL)
        return fail(ctx, LB_EINVAL, "lb_graph_create_periods: too many steps");
    CK(cudaStreamSynchronize(ctx->stream));
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t own = ctx->stream;
    cudaGraph_t graph = nullptr;
    const DevBal db = make_devbal(ctx);
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        ctx->stream = cap;
        for (int k = 0; k < nperiods && st == LB_OK && e == cudaSuccess; ++k) {
            st = ctx->compute == LB_F64 ? launch<double>(ctx, nsteps, ctx->coef_d)
                                        : launch<float>(ctx, nsteps, ctx->coef_f);
            if (st == LB_OK) e = dev_measure(db, cap);
            if (st == LB_OK && e == cudaSuccess) e = dev_rebalance(db, strategy, threshold, cap);
        }
        ctx->stream = own;
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cap);
    if (st != LB_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st != LB_OK) return st;
        return fail(ctx, LB_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, LB_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    ctx->graph_steps[exec] = lb_ctx::GraphRec{nsteps * nperiods, true};
    *graph_exec = exec;
    return LB_OK;
}

extern "C" lb_status lb_sync(lb_ctx *ctx) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    return check_status(ctx);
}

// ------------------------------------------------------------------ loads
extern "C" lb_status lb_measure_loads(lb_ctx *ctx, double *vp_cost_ns, double *sm_busy_ns,
                                      int32_t *nsm) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    if (nsm) *nsm = ctx->nsm;
    st = pull_state(ctx);
    if (st != LB_OK) return st;
    if (ctx->steps_since_measure <= 0) return fail(ctx, LB_ESTATE, "no step since the last measurement");
    const int nv = (int)ctx->vps.size(), nb = ctx->nbins;
    std::vector<unsigned long long> cyc(nv), busy(nb);
    std::vector<int32_t> sm(nb);
    std::vector<long long> cal(4 * (size_t)nb);
    cudaStream_t s0 = ctx->stream;
    CK(cudaMemcpyAsync(cyc.data(), ctx->d_vp_cycles, sizeof(unsigned long long) * nv,
                       cudaMemcpyDeviceToHost, s0));
    CK(cudaMemcpyAsync(busy.data(), ctx->d_bin_busy, sizeof(unsigned long long) * nb,
                       cudaMemcpyDeviceToHost, s0));
    CK(cudaMemcpyAsync(sm.data(), ctx->d_bin_smid, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s0));
    CK(cudaMemcpyAsync(cal.data(), ctx->d_bin_cal, sizeof(long long) * 4 * nb,
                       cudaMemcpyDeviceToHost, s0));
    CK(cudaMemsetAsync(ctx->d_vp_cycles, 0, sizeof(unsigned long long) * nv, s0));
    CK(cudaMemsetAsync(ctx->d_bin_busy, 0, sizeof(unsigned long long) * nb, s0));
    CK(cudaStreamSynchronize(s0));
    // ns per SM cycle from each processor's globaltimer / clock64 pair:
    // integer sums (exact in any order), one FP64 division
    long long ns = 0, cy = 0;
    for (int b = 0; b < nb; ++b) {
        const long long dn = cal[4 * b + 2] - cal[4 * b + 0];
        const long long dc = cal[4 * b + 3] - cal[4 * b + 1];
        if (dn > 0 && dc > 0) {
            ns += dn;
            cy += dc;
        }
    }
    double ns_per_cycle = (cy > 0) ? (double)ns / (double)cy : 0.0;
    if (!(ns_per_cycle > 0)) ns_per_cycle = ctx->fallback_npc;
    const double steps = (double)ctx->steps_since_measure;
    const double a = ctx->opt.ema_alpha;
    for (int v = 0; v < nv; ++v) {
        double c = (double)cyc[v] * ns_per_cycle / steps;
        ctx->cost[v] = ctx->have_costs ? a * c + (1.0 - a) * ctx->cost[v] : c;
        ctx->last[v] = c;
        if (vp_cost_ns) vp_cost_ns[v] = c;
    }
    ctx->have_costs = true;
    if (sm_busy_ns) {
        for (int s = 0; s < ctx->nsm; ++s) sm_busy_ns[s] = 0.0;
        for (int b = 0; b < nb; ++b)
            if (sm[b] >= 0 && sm[b] < ctx->nsm) sm_busy_ns[sm[b]] += (double)busy[b] * ns_per_cycle / steps;
    }
    ctx->steps_since_measure = 0;
    return push_state(ctx);
}

// ------------------------------------------------------------------ balance
extern "C" lb_status lb_plan(int32_t strategy, const double *costs, int32_t nvps, int32_t nprocs,
                             const int32_t *current, double refine_tol, int32_t *out,
                             int32_t *mig, double *pred) {
    if (!costs || !out || nvps < 1 || nprocs < 1)
        return fail(nullptr, LB_EINVAL, "lb_plan: bad arguments");
    std::vector<double> c(costs, costs + nvps);
    for (double x : c)
        if (!std::isfinite(x) || x < 0) return fail(nullptr, LB_EINVAL, "lb_plan: costs must be finite and >= 0");
    std::vector<int> cur, res;
    if (current) {
        cur.assign(current, current + nvps);
        for (int b : cur)
            if (b < 0 || b >= nprocs) return fail(nullptr, LB_EINVAL, "lb_plan: current out of range");
    } else {
        static_blocks(nvps, nprocs, cur);
    }
    if (strategy == LB_STATIC) static_blocks(nvps, nprocs, res);
    else if (strategy == LB_GREEDY) greedy(c, nprocs, res);
    else if (strategy == LB_REFINE_SWAP) refine_swap(c, cur, nprocs, refine_tol, res);
    else if (strategy == LB_GREEDY_SPATIAL || strategy == LB_GREEDY_BLOCKED) {
        std::vector<int> order(nvps);
        for (int v = 0; v < nvps; ++v) order[v] = v;
        if (strategy == LB_GREEDY_SPATIAL) greedy_ordered(c, nprocs, order, res);
        else greedy_blocked(c, nprocs, order, res);
    } else
        return fail(nullptr, LB_EINVAL,
                    "lb_plan: strategy must be STATIC, GREEDY, REFINE_SWAP, GREEDY_SPATIAL or "
                    "GREEDY_BLOCKED");
    for (int v = 0; v < nvps; ++v) out[v] = res[v];
    if (mig) *mig = migrations(cur, res);
    if (pred) *pred = max_over_mean(c, res, nprocs);
    return LB_OK;
}

extern "C" lb_status lb_set_costs(lb_ctx *ctx, const double *costs) {
    if (!ctx || !costs) return fail(ctx, LB_EINVAL, "lb_set_costs: bad arguments");
    for (size_t v = 0; v < ctx->vps.size(); ++v)
        if (!std::isfinite(costs[v]) || costs[v] < 0) return fail(ctx, LB_EINVAL, "costs must be finite and >= 0");
    lb_status st = pull_state(ctx);
    if (st != LB_OK) return st;
    ctx->cost.assign(costs, costs + ctx->vps.size());
    ctx->have_costs = true;
    return push_state(ctx);
}

extern "C" lb_status lb_rebalance(lb_ctx *ctx, int32_t strategy, int32_t *mig, double *pred) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (strategy < LB_STATIC || strategy > LB_GREEDY_BLOCKED) return fail(ctx, LB_EINVAL, "unknown strategy");
    {
        lb_status ps = pull_state(ctx);
        if (ps != LB_OK) return ps;
    }
    if (strategy == LB_AUTO) strategy = ctx->rebalances == 0 ? LB_GREEDY : LB_REFINE_SWAP;
    if (strategy == LB_AUTO_SPATIAL)
        strategy = ctx->rebalances == 0 ? LB_GREEDY_SPATIAL : LB_REFINE_SWAP;
    const int nv = (int)ctx->vps.size();
    if ((strategy == LB_GREEDY || strategy == LB_REFINE_SWAP || strategy == LB_GREEDY_SPATIAL ||
         strategy == LB_GREEDY_BLOCKED) &&
        !ctx->have_costs)
        return fail(ctx, LB_ESTATE, "no measured costs yet");
    std::vector<int> res;
    int m = 0;
    double pr = 1.0;
    if (strategy == LB_ATOMIC_QUEUE) {
        ctx->queue_mode = true;
        // no table: report the granularity floor max(max c, mean) / mean
        double tot = 0.0, mx = 0.0;
        for (double c : ctx->cost) {
            tot += c;
            mx = std::max(mx, c);
        }
        double mean = tot / ctx->nbins;
        pr = (ctx->have_costs && mean > 0) ? std::max(mx, mean) / mean : 1.0;
    } else {
        if (strategy == LB_STATIC) static_blocks(nv, ctx->nbins, res);
        else if (strategy == LB_GREEDY) greedy(ctx->cost, ctx->nbins, res);
        else if (strategy == LB_GREEDY_SPATIAL) greedy_ordered(ctx->cost, ctx->nbins, spatial_order(ctx), res);
        else if (strategy == LB_GREEDY_BLOCKED) greedy_blocked(ctx->cost, ctx->nbins, spatial_order(ctx), res);
        else refine_swap(ctx->cost, ctx->assign, ctx->nbins, ctx->opt.refine_tol, res);
        m = migrations(ctx->assign, res);
        pr = ctx->have_costs ? max_over_mean(ctx->cost, res, ctx->nbins) : 1.0;
        ctx->assign = res;
        ctx->queue_mode = false;
        if (strategy != LB_STATIC) ctx->rebalances++;
    }
    ctx->strategy = strategy;
    lb_status st = upload_items(ctx);
    if (st != LB_OK) return st;
    if (mig) *mig = m;
    if (pred) *pred = pr;
    return LB_OK;
}

extern "C" lb_status lb_get_assignment(lb_ctx *ctx, int32_t *vp_to_proc, int32_t *nprocs) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = pull_state(ctx);
    if (st != LB_OK) return st;
    if (vp_to_proc)
        for (size_t v = 0; v < ctx->assign.size(); ++v) vp_to_proc[v] = ctx->assign[v];
    if (nprocs) *nprocs = ctx->nbins;
    return LB_OK;
}

extern "C" lb_status lb_set_assignment(lb_ctx *ctx, const int32_t *vp_to_proc) {
    if (!ctx || !vp_to_proc) return fail(ctx, LB_EINVAL, "bad arguments");
    for (size_t v = 0; v < ctx->vps.size(); ++v)
        if (vp_to_proc[v] < 0 || vp_to_proc[v] >= ctx->nbins)
            return fail(ctx, LB_EINVAL, "processor index out of range");
    lb_status st = pull_state(ctx);
    if (st != LB_OK) return st;
    ctx->assign.assign(vp_to_proc, vp_to_proc + ctx->vps.size());
    ctx->queue_mode = false;
    ctx->strategy = LB_STATIC;
    return upload_items(ctx);
}

// ------------------------------------------------------------------ sharding
extern "C" lb_status lb_set_owned(lb_ctx *ctx, const uint8_t *owned) {
    if (!ctx || !owned) return fail(ctx, LB_EINVAL, "lb_set_owned: bad arguments");
    const int nv = (int)ctx->vps.size();
    int any = 0;
    for (int v = 0; v < nv; ++v) {
        if (owned[v] > 1) return fail(ctx, LB_EINVAL, "lb_set_owned: entries must be 0 or 1");
        any |= owned[v];
    }
    if (!any) return fail(ctx, LB_EINVAL, "lb_set_owned: no VP owned");
    lb_status st = pull_state(ctx);
    if (st != LB_OK) return st;
    ctx->nitems = 0;
    std::vector<double> f1(nv, 0.0);
    for (int v = 0; v < nv; ++v) {
        const lb_vp &p = ctx->vps[v];
        ctx->vp_nchunks[v] = owned[v] ? items_of_vp(ctx->kinfo, p.w, p.h) : 0;
        ctx->nitems += ctx->vp_nchunks[v];
        f1[v] = (double)ctx->vp_nchunks[v] * ctx->grids[p.grid].nz;
    }
    std::vector<int32_t> nch(ctx->vp_nchunks.begin(), ctx->vp_nchunks.end());
    CK(cudaMemcpyAsync(ctx->d_nchunks, nch.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice,
                       ctx->stream));
    if (ctx->predict) {
        CK(cudaMemcpyAsync(ctx->d_feat1, f1.data(), sizeof(double) * nv, cudaMemcpyHostToDevice,
                           ctx->stream));
        for (int g = 0; g < (int)ctx->grids.size(); ++g)
            if (!ctx->grids[g].kc_disk)
                CK(dev_kc_features(make_devbal(ctx), g, ctx->grids[g].kc, true, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return upload_items(ctx);
}

static lb_status columns(lb_ctx *ctx, bool pack, int32_t grid, const int32_t *cells, int32_t n,
                         void *buf) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)ctx->grids.size() || n < 0 || (n > 0 && (!cells || !buf)))
        return fail(ctx, LB_EINVAL, "lb_pack_columns / lb_unpack_columns: bad arguments");
    if (n == 0) return LB_OK;
    const lb_grid_desc &d = ctx->grids[grid];
    void *field = ctx->parity ? d.q1 : d.q0;
    CK(dev_columns(pack, field, (int)dtype_size(d.storage), cells, n, d.nz, d.nx, d.ny,
                   d.pitch ? d.pitch : d.nx, buf, ctx->d_status, ctx->stream));
    return LB_OK;
}

extern "C" lb_status lb_pack_columns(lb_ctx *ctx, int32_t grid, const int32_t *cells, int32_t n,
                                     void *buf) {
    return columns(ctx, true, grid, cells, n, buf);
}

extern "C" lb_status lb_unpack_columns(lb_ctx *ctx, int32_t grid, const int32_t *cells, int32_t n,
                                       const void *buf) {
    return columns(ctx, false, grid, cells, n, const_cast<void *>(buf));
}

// ------------------------------------------------------------------ fields
extern "C" lb_status lb_set_kc(lb_ctx *ctx, int32_t grid, const int32_t *dev_kc) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)ctx->grids.size() || !dev_kc)
        return fail(ctx, LB_EINVAL, "lb_set_kc: bad grid or NULL array");
    if (ctx->grids[grid].kc_disk) return fail(ctx, LB_ESTATE, "grid uses the disk rule");
    ctx->grids[grid].kc = dev_kc;
    ctx->h_grids[grid].kc = dev_kc;
    // a one-thread kernel, so the switch is stream-ordered and needs no sync
    CK(dev_set_kc(&ctx->d_grids[grid], dev_kc, ctx->stream));
    if (ctx->predict) {
        CK(dev_kc_features(make_devbal(ctx), grid, dev_kc, false, ctx->stream));
        ctx->dev_newer = true;
    }
    return LB_OK;
}

extern "C" lb_status lb_work_done(lb_ctx *ctx, int64_t *cell_sweeps, int64_t *cell_steps) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, ctx->d_sweeps, sizeof(n), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (cell_sweeps) *cell_sweeps = (int64_t)n;
    if (cell_steps) *cell_steps = ctx->cell_steps;
    return LB_OK;
}

extern "C" lb_status lb_current_field(lb_ctx *ctx, int32_t grid, void **dev_ptr) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)ctx->grids.size() || !dev_ptr)
        return fail(ctx, LB_EINVAL, "bad grid or NULL output");
    *dev_ptr = ctx->parity ? ctx->grids[grid].q1 : ctx->grids[grid].q0;
    return LB_OK;
}

extern "C" lb_status lb_mass_history(lb_ctx *ctx, int32_t grid, double *sums, int32_t max,
                                     int32_t *n) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)ctx->grids.size()) return fail(ctx, LB_EINVAL, "bad grid");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    unsigned long long seq = 0;
    CK(cudaMemcpyAsync(&seq, ctx->d_mass_seq, sizeof(seq), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int ng = (int)ctx->grids.size();
    long long avail = (long long)std::min<unsigned long long>(seq, kMassHist);
    long long cnt = std::min<long long>(avail, std::max(max, 0));
    if (n) *n = (int32_t)cnt;
    if (cnt == 0 || !sums) return LB_OK;
    std::vector<double> hist((size_t)kMassHist * ng * 2);
    CK(cudaMemcpyAsync(hist.data(), ctx->d_mass_hist, sizeof(double) * hist.size(),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (long long i = 0; i < cnt; ++i) {
        unsigned long long s = seq - cnt + i;
        const double *e = &hist[((size_t)(s % kMassHist) * ng + grid) * 2];
        sums[i] = e[0] + e[1];
    }
    return LB_OK;
}

extern "C" lb_status lb_mass(lb_ctx *ctx, int32_t grid, double *sum, double *comp) {
    if (!ctx) return fail(nullptr, LB_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)ctx->grids.size()) return fail(ctx, LB_EINVAL, "bad grid");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    unsigned long long seq = 0;
    CK(cudaMemcpyAsync(&seq, ctx->d_mass_seq, sizeof(seq), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (seq == 0) return fail(ctx, LB_ESTATE, "no global sum computed yet");
    const int ng = (int)ctx->grids.size();
    double e[2];
    CK(cudaMemcpyAsync(e, ctx->d_mass_hist + ((size_t)((seq - 1) % kMassHist) * ng + grid) * 2,
                       sizeof(e), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (sum) *sum = e[0] + e[1];
    if (comp) *comp = e[1];
    return LB_OK;
}

// ------------------------------------------------------------------ checkpoint
static const char kMagic[8] = {'L', 'B', 'C', 'K', 'P', 'T', '0', '1'};

extern "C" lb_status lb_checkpoint(lb_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, LB_EINVAL, "bad arguments");
    lb_status st = check_status(ctx);
    if (st != LB_OK) return st;
    st = pull_state(ctx);
    if (st != LB_OK) return st;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, LB_EIO, std::string("cannot open ") + path);
    bool ok = true;
    auto W = [&](const void *p, size_t n) { ok = ok && std::fwrite(p, 1, n, f) == n; };
    int32_t hdr[6] = {(int32_t)ctx->grids.size(), (int32_t)ctx->vps.size(), ctx->nbins,
                      ctx->parity, ctx->strategy, ctx->queue_mode ? 1 : 0};
    int32_t hdr2[2] = {ctx->rebalances, ctx->have_costs ? 1 : 0};
    W(kMagic, 8);
    W(hdr, sizeof(hdr));
    W(hdr2, sizeof(hdr2));
    W(&ctx->step, sizeof(ctx->step));
    for (auto &g : ctx->grids) {
        int32_t dims[4] = {g.nx, g.ny, g.nz, g.storage};
        W(dims, sizeof(dims));
    }
    W(ctx->assign.data(), sizeof(int) * ctx->assign.size());
    W(ctx->cost.data(), sizeof(double) * ctx->cost.size());
    std::vector<char> buf;
    for (auto &g : ctx->grids) {
        size_t bytes = (size_t)(g.pitch ? g.pitch : g.nx) * g.ny * g.nz * dtype_size(g.storage);
        buf.resize(bytes);
        cudaError_t e = cudaMemcpyAsync(buf.data(), ctx->parity ? g.q1 : g.q0, bytes,
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, LB_ECUDA, cudaGetErrorString(e));
        }
        W(buf.data(), bytes);
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, LB_EIO, std::string("write failed: ") + path);
    return LB_OK;
}

extern "C" lb_status lb_restore(lb_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, LB_EINVAL, "bad arguments");
    CK(cudaStreamSynchronize(ctx->stream));
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, LB_EIO, std::string("cannot open ") + path);
    bool ok = true;
    auto R = [&](void *p, size_t n) { ok = ok && std::fread(p, 1, n, f) == n; };
    char magic[8];
    int32_t hdr[6], hdr2[2];
    long long step = 0;
    R(magic, 8);
    R(hdr, sizeof(hdr));
    R(hdr2, sizeof(hdr2));
    R(&step, sizeof(step));
    if (!ok || std::memcmp(magic, kMagic, 8) != 0 || hdr[0] != (int32_t)ctx->grids.size() ||
        hdr[1] != (int32_t)ctx->vps.size()) {
        std::fclose(f);
        return fail(ctx, LB_EINVAL, "checkpoint does not match this ctx");
    }
    for (auto &g : ctx->grids) {
        int32_t dims[4];
        R(dims, sizeof(dims));
        if (!ok || dims[0] != g.nx || dims[1] != g.ny || dims[2] != g.nz || dims[3] != g.storage) {
            std::fclose(f);
            return fail(ctx, LB_EINVAL, "checkpoint grid dimensions differ");
        }
    }
    std::vector<int> assign(ctx->vps.size());
    std::vector<double> cost(ctx->vps.size());
    R(assign.data(), sizeof(int) * assign.size());
    R(cost.data(), sizeof(double) * cost.size());
    const int parity = hdr[3] & 1;
    std::vector<char> buf;
    for (auto &g : ctx->grids) {
        size_t bytes = (size_t)(g.pitch ? g.pitch : g.nx) * g.ny * g.nz * dtype_size(g.storage);
        buf.resize(bytes);
        R(buf.data(), bytes);
        if (!ok) break;
        cudaError_t e = cudaMemcpyAsync(parity ? g.q1 : g.q0, buf.data(), bytes,
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, LB_ECUDA, cudaGetErrorString(e));
        }
    }
    std::fclose(f);
    if (!ok) return fail(ctx, LB_EIO, "checkpoint truncated");
    if (hdr[2] != ctx->nbins) {
        // different processor count: keep the static placement
        static_blocks((int)ctx->vps.size(), ctx->nbins, assign);
    }
    for (int b : assign)
        if (b < 0 || b >= ctx->nbins) return fail(ctx, LB_EINVAL, "checkpoint assignment out of range");
    ctx->assign = assign;
    ctx->cost = cost;
    ctx->have_costs = hdr2[1] != 0;
    ctx->rebalances = hdr2[0];
    ctx->strategy = hdr[4];
    ctx->queue_mode = hdr[5] != 0;
    ctx->step = step;
    ctx->parity = parity;
    ctx->steps_since_measure = 0;
    ctx->dev_newer = false;
    long long clk[2] = {step, parity};
    CK(cudaMemcpyAsync(ctx->d_clock, clk, sizeof(clk), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemsetAsync(ctx->d_vp_cycles, 0, sizeof(unsigned long long) * ctx->vps.size(), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_bin_busy, 0, sizeof(unsigned long long) * ctx->nbins, ctx->stream));
    return upload_items(ctx);
}

// ------------------------------------------------------------------ misc
extern "C" lb_status lb_get_info(lb_ctx *ctx, lb_info *info) {
    if (!ctx || !info) return fail(ctx, LB_EINVAL, "bad arguments");
    lb_status st = pull_state(ctx);
    if (st != LB_OK) return st;
    info->nprocs = ctx->nbins;
    info->nsm = ctx->nsm;
    info->threads_per_cta = ctx->threads;
    info->max_ctas_per_sm = ctx->max_ctas_per_sm;
    info->nz_variant = ctx->kinfo.nz_variant;
    info->exact_nz = ctx->kinfo.exact;
    info->step = ctx->step;
    info->work_items = ctx->nitems;
    info->strategy = ctx->queue_mode ? LB_ATOMIC_QUEUE : ctx->strategy;
    info->regs_per_thread = ctx->regs;
    info->item_w = ctx->kinfo.tile_w ? ctx->kinfo.tile_w : ctx->kinfo.cols_per_item;
    info->item_h = ctx->kinfo.tile_w ? ctx->kinfo.tile_h : 0;
    info->staged_slots = ctx->kinfo.tma_slots;
    info->dataflow = df_active(ctx) ? 1 : 0;
    return LB_OK;
}

extern "C" const char *lb_last_error(const lb_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

extern "C" void lb_destroy(lb_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->graph_steps) cudaGraphExecDestroy(kv.first);
    free_ctx(ctx);
}

namespace lbk {
bool find_step_kernel(int storage, int compute, int nz_max, int nz_min, bool same, KernelInfo *out,
                      int threads_hint, bool staged, bool wide, bool twin_ok, int ctas_per_sm) {
    if (storage == LB_F32 && compute == LB_F32) {
        if (!kernels_f32(nz_max, nz_min, same, threads_hint, staged, wide, twin_ok, out)) return false;
        // processors sharing an SM: the same kernel with fewer threads
        const bool twin = out->twin_s0 > 0;
        const bool half = out->split && !twin && out->tile_w == kTileW && out->tma_slots == 0;
        if (ctas_per_sm > 1 && same && (twin || half)) {
            KernelInfo k;
            if (kernels_f32_shared_sm(nz_max, twin, ctas_per_sm, &k)) *out = k;
        }
        return true;
    }
    if (storage == LB_F64 && compute == LB_F64) return kernels_f64(nz_max, nz_min, same, out);
    if (storage == LB_F64 && compute == LB_F32) return kernels_f64s(nz_max, nz_min, same, out);
    if (storage == LB_BF16 && compute == LB_F32) return kernels_bf16(nz_max, nz_min, same, out);
    return false;
}
}  // namespace lbk
