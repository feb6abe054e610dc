/*
 * lb.h -- C ABI of the GB300 column-physics load-balancing library (liblb.so).
 *
 * The library runs the hot path of "Dynamic Load Balancing in GPU-Based
 * Systems - Early Experiments" (Fazenda, Mendes, Kale, Panetta, Rodrigues)
 * on one GPU.  The paper over-decomposes a grid into virtual processors
 * (VPs, Sec. III), measures each VP's load on the device (Sec. V) and
 * migrates VPs between processors with GreedyLB and RefineSwapLB (Sec. VI).
 * Here a VP is a rectangle of grid columns, a "processor" is a CTA of one
 * persistent kernel (one CTA per SM by default), and a migration rewrites a
 * device-resident assignment table: field data never moves.
 *
 * One time step of a grid (the application loop of Fig. 2):
 *   1. dynamics: first-order upwind advection, convex donor-cell form
 *        q* = (1-|cx|-|cy|-|cz|) q + |cx| q[i-sx] + |cy| q[j-sy] + |cz| q[k-sz]
 *      (s = sign of the velocity), periodic in x and y, zero flux through
 *      the bottom and top faces; or, with lb_grid_desc.dynamics = 1, one
 *      weighted Jacobi sweep of the 7-point stencil (the paper's "3D Jacobi
 *      solver" phase, Sec. IV);
 *   2. physics: per column, k_c(i,j,t) passes of the implicit vertical
 *      diffusion solve M x = d, M = tridiag(-r, 1+2r, -r) with zero-flux
 *      ends (first and last diagonal 1+r) -- the serial-in-k recurrence of
 *      Fig. 1 whose trip count the load array C(i,j) multiplies (Fig. 4,
 *      Sec. VI-B);
 *   3. the load array moves through the domain (Sec. VI-B): either a disk
 *      of radius R centred at (x0,y0) + t (vx,vy) (periodic, minimum-image
 *      distance, integer cells) with k_in inside and k_out outside, or a
 *      caller-supplied array;
 *   4. optional diagnostic: compensated FP64 global sum of the new field.
 *
 * Layout of every field: x fastest, element (i,j,k) at (k*ny + j)*nx + i,
 * or (k*ny + j)*pitch + i with a row pitch (lb_grid_desc.pitch).
 *
 * Conventions for every entry point:
 *   - Returns an lb_status and never aborts or exits the process.
 *   - Device-side failures (grid-barrier timeout, non-finite sum) and
 *     clamped k_c entries are recorded in device status words and reported
 *     by the next call that synchronises (lb_measure_loads, lb_mass,
 *     lb_mass_history, lb_checkpoint, lb_sync, lb_get_costs,
 *     lb_balance_history); a failure is reported before a clamp, and each
 *     once.
 *   - lb_last_error(ctx) returns a text for the last failure of that ctx.
 *   - A ctx is not thread-safe; one host thread drives it at a time.
 *   - Work is issued on the stream given to lb_create (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).
 */
#ifndef LB_H
#define LB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,       /* invalid argument; nothing changed */
    LB_ECUDA = 2,        /* a CUDA runtime call failed */
    LB_ETIMEOUT = 3,     /* a grid-barrier wait ran past barrier_timeout_ns */
    LB_ENUMERIC = 4,     /* the global sum of a field became NaN or Inf */
    LB_ESTATE = 5,       /* call not valid in the ctx's current state */
    LB_ENORESIDENT = 6,  /* the requested CTAs cannot all be co-resident */
    LB_EIO = 7,          /* checkpoint file could not be written or read */
    LB_EKCRANGE = 8      /* a k_c array held entries above LB_KC_MAX; the
                            steps ran with those entries clamped to it */
} lb_status;

/*
 * Largest number of k_c solves a column runs in one step.  The kernels read
 * a k_c array entry e as min(max(e, 0), LB_KC_MAX): an array of garbage
 * (for instance one read before its copy has landed) then bounds the
 * launch instead of running it for hours.  A clamped entry sets a device
 * flag that the next call that synchronises reports once as LB_EKCRANGE.
 * The disk rule's k_in and k_out must not exceed it (LB_EINVAL).  The paper
 * puts no limit on its load array (Sec. VI-B); this one is a safety bound
 * of the library, far above the workloads' 64.
 */
#define LB_KC_MAX 1024

typedef enum { LB_F64 = 0, LB_F32 = 1, LB_BF16 = 2 } lb_dtype;

/*
 * Assignment strategies (Sec. VI):
 *   LB_STATIC       contiguous runs of VPs per processor (Table V, first row)
 *   LB_GREEDY       GreedyLB: VPs by measured cost descending (ties: lower
 *                   VP id) each to the least-loaded processor (ties: lower id)
 *   LB_REFINE_SWAP  RefineSwapLB: move/swap VPs off the most loaded
 *                   processor until max load <= (1+refine_tol) * mean
 *   LB_ATOMIC_QUEUE no table: warps pop work items from one global counter
 *                   every step (the dynamic task-queue scheme of Sec. II)
 *   LB_AUTO         GreedyLB on the first rebalance of a ctx, RefineSwapLB
 *                   afterwards -- the schedule the paper recommends (Sec. VII)
 *   LB_GREEDY_SPATIAL GreedyLB's rule (each VP to the least-loaded
 *                   processor) with the VPs taken in spatial order (grid,
 *                   y0, x0) instead of heaviest first.  Every processor
 *                   visits its VPs in that order, so the whole GPU sweeps
 *                   the grids together and neighbouring VPs' halo data is
 *                   still in L2 when it is needed.
 *   LB_AUTO_SPATIAL LB_GREEDY_SPATIAL on the first rebalance, RefineSwapLB
 *                   afterwards
 *   LB_GREEDY_BLOCKED GreedyLB applied block by block to the VPs in spatial
 *                   order: within each run of nprocs consecutive VPs, the
 *                   heaviest goes to the least-loaded processor, the next
 *                   heaviest to the next, one VP per processor.  Every
 *                   processor takes one VP of each block, so all sweep the
 *                   grids in lockstep; the spread of processor loads stays
 *                   below the largest VP cost.  (With nvps <= nprocs and
 *                   positive costs it is LB_GREEDY.)
 */
typedef enum {
    LB_STATIC = 0,
    LB_GREEDY = 1,
    LB_REFINE_SWAP = 2,
    LB_ATOMIC_QUEUE = 3,
    LB_AUTO = 4,
    LB_GREEDY_SPATIAL = 5,
    LB_AUTO_SPATIAL = 6,
    LB_GREEDY_BLOCKED = 7
} lb_strategy;

/*
 * One grid.  q0/q1 are caller-owned device buffers of nx*ny*nz elements of
 * the storage type, borrowed for the ctx's lifetime; q0 holds the initial
 * field.  Steps ping-pong between them; lb_current_field says which holds
 * the latest field.  |cx|+|cy|+|cz| <= 1, r >= 0, 1 <= nz <= 128 (<= 64
 * with LB_F64 compute), nx, ny >= 1, nx*ny*nz < 2^31.  storage/compute is
 * F64/F64, F64/F32, F32/F32 or BF16/F32, the same for every grid of a ctx,
 * as is r.
 */
typedef struct {
    int32_t nx, ny, nz;
    double cx, cy, cz;        /* Courant numbers (cells per step) */
    double r;                 /* diffusion number kappa*dt/dz^2 */
    int32_t storage;          /* lb_dtype of q0/q1 */
    int32_t compute;          /* lb_dtype of the arithmetic: LB_F32 or LB_F64 */
    void *q0;
    void *q1;
    const int32_t *kc;        /* device int32 [ny*nx] (row j, column i); read
                                 every step when kc_disk == 0, caller-owned.
                                 Each entry is that column's solve count:
                                 entries <= 0 mean none, entries above
                                 LB_KC_MAX run LB_KC_MAX solves and are
                                 reported as LB_EKCRANGE */
    int32_t kc_disk;          /* 1: moving-disk rule below; 0: kc array */
    int32_t disk_x0, disk_y0, disk_vx, disk_vy, disk_r;
    int32_t k_in, k_out;      /* k_c inside / outside the disk, 0..LB_KC_MAX */
    int32_t dynamics;         /* the step's first phase (Sec. IV dynamics):
                                 0 upwind advection with cx, cy, cz; 1 one
                                 weighted Jacobi sweep of the 7-point stencil,
                                 q* = (1 - 6 nu) q + nu * (sum of the six face
                                 neighbours), periodic in x/y, mirror ghosts
                                 (zero flux) in z; cx, cy, cz are then unused */
    int32_t pitch;            /* elements from one row (j) of q0/q1 to the
                                 next: 0 = nx (dense), else >= nx, so that
                                 rows can start on 32-byte sectors; the
                                 buffers then hold pitch*ny*nz elements,
                                 level k at k*pitch*ny, and the padding
                                 columns nx..pitch-1 are never read or
                                 written.  k_c arrays stay dense [ny*nx] */
    double nu;                /* Jacobi weight, 0 < nu <= 1/6 (dynamics 1) */
} lb_grid_desc;

/* One VP: columns x0 <= i < x0+w, y0 <= j < y0+h of grid `grid`.  The VPs
   of a ctx must tile every grid exactly (no gap, no overlap). */
typedef struct {
    int32_t grid, x0, y0, w, h;
} lb_vp;

typedef struct {
    int32_t ctas_per_sm;          /* processors per SM (default 1); with 2 or
                                     4, FP32 grids of nz 96 on the half-warp
                                     or twin kernels run a variant with 1/2
                                     or 1/4 of the threads, so the SM holds
                                     the same warps as with 1 */
    int32_t queue_order;          /* ATOMIC_QUEUE order: 0 VP id order,
                                     1 last measured cost, heaviest first;
                                     other values act as 0 */
    int32_t mass_every;           /* global sum every n-th step; 0 = never
                                     (default 1) */
    int32_t device_balancer;      /* reserved, must be 0 */
    double ema_alpha;             /* weight of the newest measurement in the
                                     per-VP cost average (default 0.5) */
    double refine_tol;            /* RefineSwapLB tolerance (default 0.05) */
    int64_t barrier_timeout_ns;   /* grid-barrier wait limit (default 2 s) */
    int32_t threads_hint;         /* kernel variant for FP32 grids: 0 default
                                     (one lane per column with packed
                                     twisted halves when r lets the FP32
                                     pivots converge; else split columns on
                                     half-warps), 1 one lane per column, 2
                                     split columns on half-warps, 3 split
                                     columns on paired warps (nz 32, 64,
                                     96), 4 packed twisted halves where the
                                     pivots allow */
    int32_t steal;                /* 1: with processor tables, a processor
                                     that finishes its VPs takes the next
                                     work items of the processor with the
                                     most left (default 0) */
    int32_t predict_kc;           /* 1: lb_set_kc also rescales each VP's cost
                                     average for the new k_c array (see
                                     lb_set_kc); default 0 */
    int32_t staged_loads;         /* 1: the TMA-staged kernel where it applies
                                     (FP32 split columns of nz 32, 64 or 96,
                                     nx % 4 == 0, 16-byte aligned fields);
                                     default 0 */
    int32_t dataflow;             /* 1: with the ATOMIC_QUEUE strategy, the
                                     exact-nz twin kernels (FP32 grids of nz
                                     32, 64 or 96) run a launch's steps
                                     without a grid barrier: a work item of
                                     step s starts once the items owning its
                                     columns' 4-neighbours have finished step
                                     s - 1 (same fields bit for bit; global
                                     sums added in another order); other
                                     configurations run the barrier kernel
                                     (lb_info.dataflow says which); default 0 */
    int32_t reserved[3];          /* must be 0 */
} lb_options;

/* Fill *opt with the defaults listed above. */
void lb_default_options(lb_options *opt);

/*
 * Create a ctx: validates the grids and the VP layout (Sec. III
 * over-decomposition), builds the VP and work tables, places VPs with
 * LB_STATIC, and checks that all processors can be co-resident
 * (LB_ENORESIDENT otherwise).  grids[ngrids], vps[nvps] are host arrays,
 * copied.  opt may be NULL (defaults).  On success *out owns device tables
 * of O(nvps + columns/32) entries; the field buffers stay caller-owned.
 */
lb_status lb_create(const lb_grid_desc *grids, int32_t ngrids, const lb_vp *vps,
                    int32_t nvps, const lb_options *opt, void *cuda_stream,
                    lb_ctx **out);

/*
 * Enqueue nsteps time steps (Fig. 2's inner loop) as one persistent
 * cooperative launch on the ctx stream; returns without waiting.  Every VP
 * is processed once per step under the current assignment or the atomic
 * queue; per-VP device cost (clock64 cycles per work item, Sec. V) and
 * per-processor busy time are accumulated for lb_measure_loads.  nsteps=0
 * is a no-op.
 */
lb_status lb_step(lb_ctx *ctx, int32_t nsteps);

/*
 * Like lb_step, but every processor runs its work items on one warp at a
 * time while its other warps idle: the serialized measurement of Sec. V
 * (Table I's synchronous mode), in which each VP's measured cost carries
 * no interference from other work on its SM.  The results are those of
 * lb_step; the steps are slower.  Costs read by the next
 * lb_measure_loads include these steps.  LB_ESTATE with the TMA-staged or
 * paired-warp kernels.
 */
lb_status lb_step_serial(lb_ctx *ctx, int32_t nsteps);

/*
 * Synchronise the stream, read the loads accumulated since the previous
 * call (Sec. V), fold them into the per-VP cost average (FP64 EMA) and reset
 * the accumulators.  Outputs (host, may be NULL):
 *   vp_cost_ns[nvps]  mean measured cost per step of each VP, ns
 *   sm_busy_ns[*nsm]  mean busy time per step of each SM, ns (SMs that ran
 *                     no processor report 0); *nsm = number of SMs
 * Returns LB_ESTATE if no step ran since the previous call.
 */
lb_status lb_measure_loads(lb_ctx *ctx, double *vp_cost_ns, double *sm_busy_ns,
                           int32_t *nsm);

/*
 * Re-map VPs to processors from the averaged costs (Sec. VI): strategy is
 * an lb_strategy.  The new table takes effect for the next lb_step.
 * migrations: VPs whose processor changed (host, may be NULL).
 * pred_max_over_mean: predicted max/mean processor load under the new
 * assignment (host, may be NULL).  LB_ESTATE if costs were never measured
 * and the strategy needs them.
 */
lb_status lb_rebalance(lb_ctx *ctx, int32_t strategy, int32_t *migrations,
                       double *pred_max_over_mean);

/*
 * Host-only planning with the library's balancers (Sec. VI; no ctx, no
 * GPU): the assignment `strategy` (LB_STATIC, LB_GREEDY, LB_REFINE_SWAP,
 * LB_GREEDY_SPATIAL or LB_GREEDY_BLOCKED, the last two taking the VPs in id
 * order here) produces for
 * FP64 costs[nvps] on nprocs processors.  current[nvps] is the present
 * assignment (needed by LB_REFINE_SWAP and for counting migrations; may be
 * NULL, meaning the static placement).  out[nvps] receives the assignment;
 * migrations and pred_max_over_mean may be NULL.
 */
lb_status lb_plan(int32_t strategy, const double *costs, int32_t nvps, int32_t nprocs,
                  const int32_t *current, double refine_tol, int32_t *out,
                  int32_t *migrations, double *pred_max_over_mean);

/* Replace the ctx's per-VP cost average by costs[nvps] (host, FP64, >= 0,
   finite): lets a caller balance on a cost model instead of the loads
   measured on the device (Sec. V). */
lb_status lb_set_costs(lb_ctx *ctx, const double *costs);

/* Read the current VP -> processor table (host int32[nvps]), the mapping the
   balancers of Sec. VI rewrite (Table V prints such tables); *nprocs =
   number of processors.  Under LB_ATOMIC_QUEUE the table of the last
   static-type strategy is returned. */
lb_status lb_get_assignment(lb_ctx *ctx, int32_t *vp_to_proc, int32_t *nprocs);

/* Install a caller-made VP -> processor table (host int32[nvps], each in
   [0, nprocs)); leaves queue mode.  Effective from the next lb_step. */
lb_status lb_set_assignment(lb_ctx *ctx, const int32_t *vp_to_proc);

/* Point grid `grid`'s k_c source at a new device array int32[ny*nx] (the
   load array C(i,j) of Fig. 4 and Sec. VI-B, re-drawn between segments).  The switch is enqueued on the
   ctx stream (no synchronisation): steps enqueued after this call read the
   new array, which stays caller-owned and must stay valid while they run.

   With lb_options.predict_kc (and the device balancer available), the call
   also predicts the costs the new array will cause, so that a rebalance
   made before any step has run on it is already right -- the predictive
   cost model of measured load balancing with a known load change.  Each
   VP's work is modelled as kappa * f1 + f2 with f1 = items * nz and f2 =
   sum over its work items of (largest k_c among the item's columns) * nz;
   kappa (per-item overhead in sweeps) is fitted by least squares to the
   last measured per-VP costs against (f1, f2) of the old array, or 6 when
   that fit is ill-posed.  Every cost average of the grid's VPs is then
   multiplied by (kappa f1 + f2_new) / (kappa f1 + f2_old).  Enqueued on
   the ctx stream; host calls that read costs see the result. */
lb_status lb_set_kc(lb_ctx *ctx, int32_t grid, const int32_t *dev_kc);

/* Compensated FP64 global sum of grid `grid` after the latest step that
   computed one (synchronises).  A diagnostic of this library: the paper
   prints no such quantity; conservation of the sum checks the step.  sum: the sum; comp: its compensation term
   (may be NULL). */
lb_status lb_mass(lb_ctx *ctx, int32_t grid, double *sum, double *comp);

/* Global sums of grid `grid` for the last *n steps that computed one
   (oldest first, up to max entries, at most 1024 kept); synchronises. */
lb_status lb_mass_history(lb_ctx *ctx, int32_t grid, double *sums, int32_t max,
                          int32_t *n);

/* Work done since lb_create, counted on the device (synchronises); the
   numerator of the cell-sweep throughput this library reports (the
   paper reports execution times, Sec. VI, Tables III-V):
   cell_sweeps = sum over steps and columns of nz * k_c (the implicit-solve
   row updates actually performed); cell_steps = sum over steps of the cells
   advanced.  Either pointer may be NULL. */
lb_status lb_work_done(lb_ctx *ctx, int64_t *cell_sweeps, int64_t *cell_steps);

/* Device pointer of the ping-pong buffer that holds grid `grid`'s field
   after every step enqueued so far (no synchronisation: the value is
   there once those steps have finished, e.g. after lb_sync). */
lb_status lb_current_field(lb_ctx *ctx, int32_t grid, void **dev_ptr);

/*
 * CUDA graphs of the step (the Fig. 2 inner loop replayed without host
 * launch work).  lb_graph_create captures one persistent launch of nsteps
 * steps into an executable graph (a cudaGraphExec_t, returned as void*).
 * The kernel reads the step index and the ping-pong parity from a device
 * word that every launch advances, so each replay continues where the ctx
 * stands.  lb_graph_launch replays it on the ctx stream and advances the
 * ctx's host-side counters; only graphs made for the same ctx are accepted.
 * A graph keeps the assignment mode it was captured with (processor tables
 * or atomic queue): rebalancing between table strategies is picked up (the
 * tables live in device memory), switching to or from LB_ATOMIC_QUEUE needs
 * a new graph.  lb_destroy frees a ctx's remaining graphs.
 */
lb_status lb_graph_create(lb_ctx *ctx, int32_t nsteps, void **graph_exec);
lb_status lb_graph_launch(lb_ctx *ctx, void *graph_exec);
lb_status lb_graph_destroy(lb_ctx *ctx, void *graph_exec);

/*
 * Device-side measurement and rebalancing: the same cost average and the
 * same balancers as lb_measure_loads / lb_rebalance, run as kernels on the
 * ctx stream.  Both calls only enqueue work (no synchronisation, no host
 * copies), so a rebalance period -- lb_step, lb_device_measure,
 * lb_device_rebalance -- runs back to back on the GPU and can be captured
 * in one CUDA graph (lb_graph_create_periods).
 *
 * lb_device_measure folds the loads accumulated since the previous
 * measurement into the per-VP cost average (Sec. V) with exactly
 * lb_measure_loads's FP64 arithmetic, and records the period's SM busy
 * max/mean.  With no step since the previous measurement it changes
 * nothing and the next synchronising call returns LB_ESTATE.
 *
 * lb_device_rebalance remaps VPs from the device cost average (Sec. VI)
 * and rewrites the processor tables in device memory; the next step uses
 * them.  strategy: LB_STATIC, LB_GREEDY, LB_REFINE_SWAP, LB_AUTO,
 * LB_GREEDY_SPATIAL, LB_AUTO_SPATIAL or LB_GREEDY_BLOCKED (LB_AUTO* decide
 * on the device, from
 * the number of table rebalances so far).  For equal costs and current
 * assignment the new assignment equals lb_rebalance's bit for bit.  Its
 * migrations and predicted max/mean are recorded in the balance history.
 * Without costs (never measured or set) the next synchronising call
 * returns LB_ESTATE.  In LB_ATOMIC_QUEUE mode only strategy LB_ATOMIC_QUEUE
 * is accepted (LB_ESTATE otherwise): it changes nothing and records the
 * period in the balance history, with the granularity floor as its
 * predicted max/mean.  Not available for more than 8192 VPs or 1024
 * processors (LB_EINVAL).
 *
 * Host calls that read or change costs or the assignment (lb_measure_loads,
 * lb_rebalance, lb_set_costs, lb_get_assignment, lb_set_assignment,
 * lb_checkpoint, lb_get_info) first wait for pending device-side
 * rebalancing work and see its result.
 */
lb_status lb_device_measure(lb_ctx *ctx);
lb_status lb_device_rebalance(lb_ctx *ctx, int32_t strategy);

/*
 * Threshold-triggered rebalancing (the paper's future-work item, Sec. VII)
 * on the device: like lb_device_rebalance, but the current table is kept
 * when its predicted max/mean processor load under the current cost
 * averages is at most threshold -- unless lb_set_kc rescaled the costs
 * since the last rebalance, which forces one.  A kept table is recorded in
 * the balance history (migrations 0, last column 1).  threshold <= 0:
 * always rebalance.  (Measured SM busy times are no criterion with work
 * stealing, which evens them out whatever the table.)
 */
lb_status lb_device_rebalance_if(lb_ctx *ctx, int32_t strategy, double threshold);

/* Per-VP costs, ns per step (host double[nvps] each, may be NULL): the
   cost average balancers use and the last measurement (the per-object
   loads of Sec. V).  Synchronises. */
lb_status lb_get_costs(lb_ctx *ctx, double *avg_ns, double *last_ns);

/*
 * The last *n (at most max, at most 1024 kept) device rebalances (Sec. VI
 * balancer calls), oldest first, 8 doubles each: step index, strategy applied (LB_AUTO* resolved),
 * migrations, predicted max/mean processor load, measured SM busy max/mean
 * of the preceding measurement, granularity floor max(max cost, mean)/mean,
 * RefineSwapLB iterations, 1 if the table was kept by
 * lb_device_rebalance_if (else 0).  rows: host double[max*8].  Synchronises.
 */
lb_status lb_balance_history(lb_ctx *ctx, double *rows, int32_t max, int32_t *n);

/*
 * One executable graph of nperiods rebalance periods (Fig. 2's loop): each
 * period is one persistent launch of nsteps steps, lb_device_measure and
 * lb_device_rebalance_if(strategy, threshold) (threshold <= 0: always
 * rebalance).  Replay with lb_graph_launch (the ctx's step counters advance
 * by nsteps*nperiods); destroy with lb_graph_destroy.  lb_set_kc between
 * replays switches the k_c array (and rescales costs with predict_kc).
 * Same availability rules as lb_device_rebalance.
 */
lb_status lb_graph_create_periods(lb_ctx *ctx, int32_t nsteps, int32_t strategy,
                                  int32_t nperiods, double threshold, void **graph_exec);

/* Wait for all work enqueued on the ctx stream, then report a device-side
   error recorded since the last report: LB_ETIMEOUT (a grid-barrier wait
   ran out of barrier_timeout_ns), LB_ENUMERIC (a global sum was not
   finite) or LB_ESTATE (a device balancer call came with no step since the
   last measurement, or before any costs).
   Reporting clears the status word, so each error is reported once.  The
   ctx stays usable: the steps of a launch that timed out leave undefined
   field values, and later steps run normally on them. */
lb_status lb_sync(lb_ctx *ctx);

/*
 * Write / read the whole run state to / from a file: step index, current
 * fields, assignment, cost averages (the paper's full device-to-host copy
 * around a migration, Fig. 2, becomes a checkpoint here).  lb_restore needs
 * a ctx created with the same grids and VPs; a resumed run is bitwise equal
 * to an uninterrupted one.
 */
lb_status lb_checkpoint(lb_ctx *ctx, const char *path);
lb_status lb_restore(lb_ctx *ctx, const char *path);

typedef struct {
    int32_t nprocs;           /* processors (CTAs of the persistent kernel) */
    int32_t nsm;              /* SMs of the device */
    int32_t threads_per_cta;
    int32_t max_ctas_per_sm;  /* co-residency limit of the chosen kernel */
    int32_t nz_variant;       /* register-resident column length of the kernel */
    int32_t exact_nz;         /* 1: kernel specialised to the grids' nz */
    int64_t step;             /* global index of the next step */
    int64_t work_items;       /* items of 32 columns per step */
    int32_t strategy;         /* strategy of the current table */
    int32_t regs_per_thread;
    int32_t item_w, item_h;   /* work item shape: an item_w x item_h tile of a
                                 VP (tiles row-major), or item_h == 0: runs of
                                 item_w columns of the VP in row-major order */
    int32_t staged_slots;     /* TMA-staged kernel: shared-memory box slots
                                 per processor (one per warp, each holding
                                 the next work item's input); 0: each warp
                                 loads its own items */
    int32_t dataflow;         /* 1: lb_step currently runs the dataflow
                                 kernel (lb_options.dataflow) */
} lb_info;

/* Fill *info (fields above).  Synchronises only when a device balancer call
   or graph replay has changed the assignment since the host last read it. */
lb_status lb_get_info(lb_ctx *ctx, lb_info *info);

/* Text of the last error of ctx (or of the last lb_create failure when ctx
   is NULL).  Owned by the library, valid until the next call on ctx. */
const char *lb_last_error(const lb_ctx *ctx);

/* Free the ctx's device tables; the caller's buffers are untouched.
   Synchronises the stream first.  NULL is a no-op. */
void lb_destroy(lb_ctx *ctx);

/*
 * Sharding across ranks (processes, one GPU each): every rank's ctx covers
 * the whole grid, holds full-size field buffers and runs only the VPs it
 * owns -- the paper's processors of a distributed run (Sec. III, Fig. 2),
 * with migration of VPs between them (Sec. VI).  Between steps the ranks
 * exchange the upwind halo columns of their VPs and move migrated VPs'
 * columns with lb_pack_columns / lb_unpack_columns.
 *
 * lb_set_owned: owned[nvps] (host), 1 = this ctx runs the VP, 0 = it does
 * not.  VPs that are not owned get no work items: their columns are not
 * written, their costs are not measured, and the global sum (lb_mass)
 * covers the owned columns only.  Takes effect for the next lb_step and
 * balancer call; CUDA graphs made earlier keep the old tables, so make
 * them again.  LB_EINVAL when no VP is owned or an entry is not 0 or 1.
 */
lb_status lb_set_owned(lb_ctx *ctx, const uint8_t *owned);

/*
 * Copy n columns (all nz levels) of the grid's current field into buf
 * (pack) or from buf into the current field (unpack), on the ctx stream.
 * cells (device int32 [n]): column indices j*nx + i.  buf (device, n*nz
 * elements of the grid's storage type): level-major, element (k, c) at
 * k*n + c.  Both stay caller-owned and must stay valid until the stream
 * has passed the copy.  An index outside [0, nx*ny) is skipped on the
 * device and reported as LB_EINVAL by the next call that synchronises;
 * n < 0, or a NULL pointer with n > 0, returns LB_EINVAL at once.  n = 0
 * is a no-op.
 */
lb_status lb_pack_columns(lb_ctx *ctx, int32_t grid, const int32_t *cells, int32_t n, void *buf);
lb_status lb_unpack_columns(lb_ctx *ctx, int32_t grid, const int32_t *cells, int32_t n,
                            const void *buf);

/*
 * lb_step_noalloc -- nsteps time steps of one grid without allocating any
 * memory.  (This entry point has no counterpart in the paper.)
 *
 * For callers that cannot call cudaMalloc: programs whose device memory is
 * owned by another allocator (a framework's caching allocator that has
 * already reserved the GPU, a fixed-budget pool in an embedded or real-time
 * service), where a library allocation could fail, fragment the pool, or
 * synchronise the device at a moment the caller does not control.  lb_create
 * allocates tables; this call keeps all of the step kernel's tables and
 * scratch in one fixed device array compiled into the library
 * (LB_NOALLOC_SCRATCH_BYTES, under 2 MiB), which every GPU that loads the
 * library holds until the process exits.
 *
 * Arguments: grid (host struct; q0 holds the input field, q1 is the other
 * ping-pong buffer; after the call the result is in q0 when nsteps is even,
 * in q1 when odd), vps[nvps] (host, grid index 0, must tile the grid),
 * opt (host, may be NULL for the defaults; barrier_timeout_ns and
 * threads_hint are used, as lb_create uses them), t0 (global index of the
 * first step: moves the k_c disk), nsteps, the stream, and mass_out (host,
 * may be NULL): the compensated global sum after the last step, left
 * unchanged when nsteps is 0.  VPs are placed statically, contiguous runs
 * per SM; the kernel is the one lb_create chooses for the same grid, VPs
 * and options, so the field after each call equals lb_step's bit for bit
 * (the global sum adds the same values in another order).
 *
 * Limits: nvps <= LB_NOALLOC_MAX_VPS, work items (per VP, the item count
 * of the chosen kernel: ceil(w*h/32) or 8x2 tiles) <= LB_NOALLOC_MAX_ITEMS,
 * nx*ny <= LB_NOALLOC_MAX_COLUMNS (the host bitmap that checks the tiling);
 * larger inputs return LB_EINVAL, with the reason in lb_last_error(NULL).
 * A k_c array entry above LB_KC_MAX returns LB_EKCRANGE after the steps
 * have run with it clamped (mass_out is written).  The call synchronises
 * the stream before returning.  The first call on a device looks up the
 * array's device address with that device current; make it before any
 * stream capture.  The address is cached for the life of the process:
 * after a cudaDeviceReset of that device, do not call this entry point
 * again.  Every call reuses the same array and clears the parts that must
 * start at zero; calls whose GPU work overlaps (two streams, two host
 * threads on one device) race on the array -- serialise them.
 */
#define LB_NOALLOC_MAX_VPS 8192
#define LB_NOALLOC_MAX_ITEMS 65536
#define LB_NOALLOC_MAX_COLUMNS (1 << 27)
#define LB_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u)
lb_status lb_step_noalloc(const lb_grid_desc *grid, const lb_vp *vps, int32_t nvps,
                          const lb_options *opt, int64_t t0, int32_t nsteps, void *cuda_stream,
                          double *mass_out);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
