// Device-side load measurement and rebalancing: the per-VP cost average
// (Sec. V) and GreedyLB / list scheduling / RefineSwapLB (Sec. VI) run as
// kernels on the ctx stream, so a whole rebalance period -- steps,
// measurement, balancer, new work tables -- can be enqueued, or captured in
// one CUDA graph, without a host round trip.
//
// Every FP64 result equals the host balancers' (lb_balance.cpp) bit for bit
// for equal inputs: the same operations in the same order, written as
// explicitly rounded intrinsics (__dadd_rn and friends are never contracted
// into FMAs).  Orders of FP64 values are taken on order-preserving 64-bit
// integer keys: FP64 compares run on GB300's narrow FP64 pipe, integer
// compares on the full-rate ALUs.
//
// Kernels (all on the ctx stream):
//   k_measure  one thread per VP: cycles -> ns per step -> EMA; the last
//              block to finish (threadfence ticket) records SM busy times
//              and the measurement step
//   k_rank     one thread per VP: rank by (cost desc, id asc) -- GreedyLB's
//              order; exits at once unless the resolved strategy is GreedyLB
//   k_balance  one CTA of 1024 threads: static / GreedyLB / list
//              scheduling in spatial order / RefineSwapLB on a shared-memory
//              copy of the assignment; migrations and predicted max/mean
//   k_items    one CTA per processor: its work-item range and its items in
//              spatial order (the tables the step kernel reads)
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace lbk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBalThreads = 1024;
constexpr int kBalWarps = kBalThreads / kWarp;
constexpr int kRankThreads = 256;
constexpr int kItemThreads = 256;
constexpr unsigned kNone = 0x7fffffffu;

// a < b (IEEE, -0 == +0, no NaN) iff okey(a) < okey(b)
__device__ __forceinline__ unsigned long long okey(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if (b == 0x8000000000000000ull) b = 0ull;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ int resolve(int s, long long rebalances) {
    if (s == LB_AUTO) return rebalances == 0 ? LB_GREEDY : LB_REFINE_SWAP;
    if (s == LB_AUTO_SPATIAL) return rebalances == 0 ? LB_GREEDY_SPATIAL : LB_REFINE_SWAP;
    return s;
}

// Lexicographic minimum of (key, id) over a full warp; every lane gets the id.
__device__ __forceinline__ unsigned warp_min_key_id(unsigned long long k, unsigned id) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mh = __reduce_min_sync(kFull, hi);
    const unsigned ml = __reduce_min_sync(kFull, hi == mh ? lo : ~0u);
    return __reduce_min_sync(kFull, (hi == mh && lo == ml) ? id : ~0u);
}

// Bin with the lowest (load, id), skipping `skip` and every bin at or before
// (after_key, after_id) in that order when after_id >= 0.  One full warp.
__device__ unsigned warp_next_bin(const double *s_load, int nb, int skip,
                                  unsigned long long after_key, int after_id) {
    const int lane = threadIdx.x % kWarp;
    unsigned long long bk = ~0ull;
    unsigned bi = kNone;
    for (int b = lane; b < nb; b += kWarp) {
        if (b == skip) continue;
        const unsigned long long k = okey(s_load[b]);
        if (after_id >= 0 && (k < after_key || (k == after_key && b <= after_id))) continue;
        if (k < bk) {
            bk = k;
            bi = (unsigned)b;
        }
    }
    return warp_min_key_id(bk, bi);
}

// Lexicographic minimum of (key, id) over a full warp, both parts returned.
__device__ __forceinline__ void warp_min_pair(unsigned long long &k, unsigned &id) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mh = __reduce_min_sync(kFull, hi);
    const unsigned ml = __reduce_min_sync(kFull, hi == mh ? lo : ~0u);
    id = __reduce_min_sync(kFull, (hi == mh && lo == ml) ? id : ~0u);
    k = ((unsigned long long)mh << 32) | ml;
}

// Block-wide lexicographic minimum of (key, idx) (1024 threads); every
// thread gets it.  (~0, ~0) means none.
__device__ void block_min_key_idx(unsigned long long &k, unsigned &idx, unsigned long long *s_wk,
                                  unsigned *s_wi) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    warp_min_pair(k, idx);
    if (lane == 0) {
        s_wk[warp] = k;
        s_wi[warp] = idx;
    }
    __syncthreads();
    if (warp == 0) {
        unsigned long long k2 = s_wk[lane];
        unsigned i2 = s_wi[lane];
        warp_min_pair(k2, i2);
        if (lane == 0) {
            s_wk[kBalWarps] = k2;
            s_wi[kBalWarps] = i2;
        }
    }
    __syncthreads();
    k = s_wk[kBalWarps];
    idx = s_wi[kBalWarps];
    __syncthreads();
}

__device__ __forceinline__ double from_okey(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

__device__ int block_sum_int(int v, int *s_w) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    const int nw = blockDim.x / kWarp;
    v = __reduce_add_sync(kFull, v);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += s_w[w];
    __syncthreads();
    return t;
}

// Per-bin loads, each the FP64 sum of its VPs' costs in increasing VP id
// (bin_loads); warp w sums bins w, w + 32, ...
__device__ void bin_loads_dev(const int *s_assign, const double *cost, int nv, int nb,
                              double *s_load) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    for (int b = warp; b < nb; b += kBalWarps) {
        double acc = 0.0;
        for (int base = 0; base < nv; base += kWarp) {
            const int v = base + lane;
            unsigned m = __ballot_sync(kFull, v < nv && s_assign[v] == b);
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                acc = __dadd_rn(acc, cost[base + j]);
            }
        }
        if (lane == 0) s_load[b] = acc;
    }
    __syncthreads();
}

// GreedyLB's rule over VPs in a given order (ov[i], with costs oc[i]): each
// to the bin with the lowest (load, id); loads summed in assignment order.
// One warp; lane l keeps the loads of bins l, l + 32, ... in registers.
template <int NBL>
__device__ void greedy_warp(const int *ov, const double *oc, int nv, int nb, int *s_assign) {
    const int lane = threadIdx.x % kWarp;
    double ld[NBL];
#pragma unroll
    for (int j = 0; j < NBL; ++j) ld[j] = 0.0;
    unsigned long long mk = lane < nb ? okey(0.0) : ~0ull;
    unsigned mi = lane < nb ? (unsigned)lane : kNone;
    for (int i = 0; i < nv; ++i) {
        const int v = ov[i];
        const double c = oc[i];
        const unsigned w = warp_min_key_id(mk, mi);
        if (lane == 0) s_assign[v] = (int)w;
        if ((int)(w % kWarp) == lane) {
            const int slot = (int)(w / kWarp);
            unsigned long long bk = ~0ull;
            unsigned bi = kNone;
#pragma unroll
            for (int j = 0; j < NBL; ++j) {
                if (j == slot) ld[j] = __dadd_rn(ld[j], c);
                const int b = lane + kWarp * j;
                if (b < nb) {
                    const unsigned long long k = okey(ld[j]);
                    if (k < bk) {
                        bk = k;
                        bi = (unsigned)b;
                    }
                }
            }
            mk = bk;
            mi = bi;
        }
        __syncwarp();
    }
}

// Same rule with the loads in shared memory (any bin count).
__device__ void greedy_warp_smem(const int *ov, const double *oc, int nv, int nb, int *s_assign,
                                 double *s_load) {
    const int lane = threadIdx.x % kWarp;
    for (int b = lane; b < nb; b += kWarp) s_load[b] = 0.0;
    __syncwarp();
    unsigned long long mk = lane < nb ? okey(0.0) : ~0ull;
    unsigned mi = lane < nb ? (unsigned)lane : kNone;
    for (int i = 0; i < nv; ++i) {
        const int v = ov[i];
        const double c = oc[i];
        const unsigned w = warp_min_key_id(mk, mi);
        if (lane == 0) s_assign[v] = (int)w;
        if ((int)(w % kWarp) == lane) {
            s_load[w] = __dadd_rn(s_load[w], c);
            unsigned long long bk = ~0ull;
            unsigned bi = kNone;
            for (int b = lane; b < nb; b += kWarp) {
                const unsigned long long k = okey(s_load[b]);
                if (k < bk) {
                    bk = k;
                    bi = (unsigned)b;
                }
            }
            mk = bk;
            mi = bi;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- kernels
__global__ void __launch_bounds__(256) k_measure(const DevBal p) {
    __shared__ double s_npc, s_steps;
    __shared__ int s_last;
    __shared__ unsigned long long s_busy[kDevBalMaxSms];
    if (threadIdx.x == 0) {
        // ns per SM cycle from every processor's globaltimer / clock64 pair
        double ns = 0.0, cy = 0.0;
        for (int b = 0; b < p.nbins; ++b) {
            const double dn = __ll2double_rn(p.bin_cal[4 * b + 2] - p.bin_cal[4 * b + 0]);
            const double dc = __ll2double_rn(p.bin_cal[4 * b + 3] - p.bin_cal[4 * b + 1]);
            if (dn > 0.0 && dc > 0.0) {
                ns = __dadd_rn(ns, dn);
                cy = __dadd_rn(cy, dc);
            }
        }
        double npc = cy > 0.0 ? __ddiv_rn(ns, cy) : 0.0;
        if (!(npc > 0.0)) npc = p.fallback_ns_per_cycle;
        s_npc = npc;
        s_steps = __ll2double_rn(p.dclock[0] - p.state[kStMeasStep]);
    }
    __syncthreads();
    const double steps = s_steps;
    if (!(steps > 0.0)) {   // no step since the last measurement
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(p.status, 0, (int)LB_ESTATE);
        return;
    }
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < p.nvps) {
        const double c = __ddiv_rn(__dmul_rn(__ull2double_rn(p.vp_cycles[v]), s_npc), steps);
        const double a = p.ema_alpha;
        p.cost[v] = p.state[kStHave]
                        ? __dadd_rn(__dmul_rn(a, c), __dmul_rn(__dsub_rn(1.0, a), p.cost[v]))
                        : c;
        p.last[v] = c;
        p.vp_cycles[v] = 0ull;
    }
    // the last block records per-SM busy time and the measurement step
    // (every block has read the state words before taking its ticket)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int s = threadIdx.x; s < p.nsm; s += blockDim.x) s_busy[s] = 0ull;
    __syncthreads();
    for (int b = threadIdx.x; b < p.nbins; b += blockDim.x) {
        const int sm = p.bin_smid[b];
        if (sm >= 0 && sm < p.nsm) atomicAdd(&s_busy[sm], p.bin_busy[b]);
        p.bin_busy[b] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0, tot = 0.0;
        int n = 0;
        for (int s = 0; s < p.nsm; ++s)
            if (s_busy[s] > 0ull) {
                const double x = (double)s_busy[s];
                mx = x > mx ? x : mx;
                tot += x;
                ++n;
            }
        p.pend[0] = (n > 0 && tot > 0.0) ? mx / (tot / n) : 0.0;
        p.state[kStHave] = 1;
        p.state[kStMeasStep] = p.dclock[0];
        *p.ticket = 0u;
    }
}

__global__ void __launch_bounds__(kRankThreads) k_rank(const DevBal p, int strategy) {
    __shared__ unsigned long long s_key[kRankThreads];
    if (resolve(strategy, p.state[kStRebal]) != LB_GREEDY) return;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long kv = v < p.nvps ? okey(p.cost[v]) : 0ull;
    int rank = 0;
    for (int base = 0; base < p.nvps; base += kRankThreads) {
        const int u = base + threadIdx.x;
        s_key[threadIdx.x] = u < p.nvps ? okey(p.cost[u]) : 0ull;
        __syncthreads();
        const int n = min(kRankThreads, p.nvps - base);
        for (int j = 0; j < n; ++j) {
            const unsigned long long ku = s_key[j];
            rank += (ku > kv) || (ku == kv && base + j < v);
        }
        __syncthreads();
    }
    if (v < p.nvps) p.order[rank] = v;
}

__global__ void __launch_bounds__(kBalThreads, 1) k_balance(const DevBal p, int strategy) {
    extern __shared__ double s_dyn[];
    const int nv = p.nvps, nb = p.nbins;
    double *s_load = s_dyn;                          // [nb]
    int *s_assign = (int *)(s_load + nb);            // [nv]
    int *s_pl = s_assign + nv;                       // [nv] members of P (unordered)
    int *s_ps = s_pl + nv;                           // [nv] members of P, (cost desc, id asc)
    int *s_ql = s_ps + nv;                           // [nv] members of Q (unordered)
    int *s_qs = s_ql + nv;                           // [nv] members of Q, (cost asc, id asc)
    double *s_oc = (double *)s_ps;                   // [nv] greedy: costs in visiting order
                                                     // (over s_ps and s_ql; 8-byte aligned)
    __shared__ int s_strat, s_skip, s_P, s_Q, s_np, s_nq, s_iters;
    __shared__ unsigned s_found;
    __shared__ double s_thr;
    __shared__ unsigned long long s_wk[kBalWarps + 1];
    __shared__ unsigned s_wi[kBalWarps + 1];
    __shared__ int s_wsum[kBalWarps];
    const int tid = threadIdx.x, lane = tid % kWarp, warp = tid / kWarp;

    if (tid == 0) {
        const int st = resolve(strategy, p.state[kStRebal]);
        s_strat = st;
        s_skip = st != LB_STATIC && !p.state[kStHave];
        if (s_skip) atomicCAS(p.status, 0, (int)LB_ESTATE);
        s_iters = 0;
    }
    __syncthreads();
    if (s_skip) return;
    const int st = s_strat;
    for (int v = tid; v < nv; v += kBalThreads) s_assign[v] = p.assign[v];
    __syncthreads();

    if (st == LB_STATIC) {
        for (int v = tid; v < nv; v += kBalThreads) s_assign[v] = (int)(((long long)v * nb) / nv);
    } else if (st == LB_GREEDY || st == LB_GREEDY_SPATIAL) {
        const int *ord = st == LB_GREEDY ? p.order : p.spatial;
        for (int i = tid; i < nv; i += kBalThreads) {
            const int v = ord[i];
            s_pl[i] = v;
            s_oc[i] = p.cost[v];
        }
        __syncthreads();
        if (warp == 0) {
            if (nb <= 8 * kWarp) greedy_warp<8>(s_pl, s_oc, nv, nb, s_assign);
            else greedy_warp_smem(s_pl, s_oc, nv, nb, s_assign, s_load);
        }
    } else {
        // RefineSwapLB (lb_balance.cpp: refine_swap)
        bin_loads_dev(s_assign, p.cost, nv, nb, s_load);
        if (tid == 0) {
            double t = 0.0;
            for (int b = 0; b < nb; ++b) t = __dadd_rn(t, s_load[b]);
            s_thr = __dmul_rn(__dadd_rn(1.0, p.refine_tol), __ddiv_rn(t, (double)nb));
        }
        __syncthreads();
        const double thr = s_thr;
        for (long long it = 0; it < 4LL * nv; ++it) {
            if (warp == 0) {
                // P: largest load, lowest id
                unsigned long long bk = ~0ull;
                unsigned bi = kNone;
                for (int b = lane; b < nb; b += kWarp) {
                    const unsigned long long k = ~okey(s_load[b]);
                    if (k < bk) {
                        bk = k;
                        bi = (unsigned)b;
                    }
                }
                const unsigned P = warp_min_key_id(bk, bi);
                const unsigned Q0 = warp_next_bin(s_load, nb, (int)P, 0ull, -1);
                if (lane == 0) {
                    s_P = (int)P;
                    s_Q = (int)Q0;
                    s_np = 0;
                    s_found = kNone;
                }
            }
            __syncthreads();
            const int P = s_P;
            if (!(s_load[P] > thr)) break;
            if (tid == 0) ++s_iters;
            for (int v = tid; v < nv; v += kBalThreads)
                if (s_assign[v] == P) s_pl[atomicAdd(&s_np, 1)] = v;
            __syncthreads();
            const int np = s_np;
            for (int i = tid; i < np; i += kBalThreads) {
                const int vi = s_pl[i];
                const unsigned long long ki = okey(p.cost[vi]);
                int r = 0;
                for (int j = 0; j < np; ++j) {
                    const int vj = s_pl[j];
                    const unsigned long long kj = okey(p.cost[vj]);
                    r += (kj > ki) || (kj == ki && vj < vi);
                }
                s_ps[r] = vi;
            }
            __syncthreads();
            // move: the first member of P (in that order) with a positive
            // cost that fits under the threshold on the least loaded other
            // bin Q0.  If none fits on Q0 none fits anywhere (every other
            // bin is at least as loaded), so later bins only try swaps.
            const int Q0 = s_Q;
            if (Q0 < nb) {
                const double lq = s_load[Q0];
                for (int i = tid; i < np; i += kBalThreads) {
                    const double c = p.cost[s_ps[i]];
                    if (c > 0.0 && __dadd_rn(lq, c) <= thr) atomicMin(&s_found, (unsigned)i);
                }
            }
            __syncthreads();
            if (s_found != kNone) {
                if (tid == 0) {
                    const int o = s_ps[s_found];
                    const double c = p.cost[o];
                    s_load[P] = __dsub_rn(s_load[P], c);
                    s_load[Q0] = __dadd_rn(s_load[Q0], c);
                    s_assign[o] = Q0;
                }
                __syncthreads();
                continue;
            }
            // swaps, bins Q in (load asc, id asc) order
            bool done = false;
            int Q = Q0;
            while (Q < nb) {
                if (tid == 0) s_nq = 0;
                __syncthreads();
                for (int v = tid; v < nv; v += kBalThreads)
                    if (s_assign[v] == Q) s_ql[atomicAdd(&s_nq, 1)] = v;
                __syncthreads();
                const int nq = s_nq;
                for (int i = tid; i < nq; i += kBalThreads) {
                    const int vi = s_ql[i];
                    const unsigned long long ki = okey(p.cost[vi]);
                    int r = 0;
                    for (int j = 0; j < nq; ++j) {
                        const int vj = s_ql[j];
                        const unsigned long long kj = okey(p.cost[vj]);
                        r += (kj < ki) || (kj == ki && vj < vi);
                    }
                    s_qs[r] = vi;
                }
                __syncthreads();
                // the first pair (o-order, then o'-order) of least
                // max(load P - d, load Q + d) below load P
                const double LP = s_load[P], LQ = s_load[Q];
                unsigned long long bk = ~0ull;
                unsigned bi = ~0u;
                const long long npairs = (long long)np * nq;
                for (long long e = tid; e < npairs; e += kBalThreads) {
                    const int i = (int)(e / nq), j = (int)(e % nq);
                    const double co = p.cost[s_ps[i]], c2 = p.cost[s_qs[j]];
                    if (!(co > c2)) continue;
                    const double d = __dsub_rn(co, c2);
                    const double a = __dsub_rn(LP, d), b = __dadd_rn(LQ, d);
                    const double m = (a < b) ? b : a;
                    if (!(m < LP)) continue;
                    const unsigned long long k = okey(m);
                    if (k < bk || (k == bk && (unsigned)e < bi)) {
                        bk = k;
                        bi = (unsigned)e;
                    }
                }
                block_min_key_idx(bk, bi, s_wk, s_wi);
                if (bi != ~0u) {
                    if (tid == 0) {
                        const int o = s_ps[bi / nq], o2 = s_qs[bi % nq];
                        const double d = __dsub_rn(p.cost[o], p.cost[o2]);
                        s_load[P] = __dsub_rn(s_load[P], d);
                        s_load[Q] = __dadd_rn(s_load[Q], d);
                        s_assign[o] = Q;
                        s_assign[o2] = P;
                    }
                    __syncthreads();
                    done = true;
                    break;
                }
                if (warp == 0) {
                    const unsigned nQ = warp_next_bin(s_load, nb, P, okey(s_load[Q]), Q);
                    if (lane == 0) s_Q = (int)nQ;
                }
                __syncthreads();
                Q = s_Q;
            }
            if (!done) break;
        }
    }
    __syncthreads();

    // migrations, new table, predicted max/mean, record
    int mig = 0;
    unsigned long long cmax = okey(0.0);
    for (int v = tid; v < nv; v += kBalThreads) {
        mig += s_assign[v] != p.assign[v];
        const unsigned long long k = okey(p.cost[v]);
        cmax = k > cmax ? k : cmax;
    }
    mig = block_sum_int(mig, s_wsum);
    {
        unsigned long long nk = ~cmax;
        unsigned ni = 0u;
        block_min_key_idx(nk, ni, s_wk, s_wi);
        cmax = ~nk;
    }
    for (int v = tid; v < nv; v += kBalThreads) p.assign[v] = s_assign[v];
    bin_loads_dev(s_assign, p.cost, nv, nb, s_load);
    if (tid == 0) {
        double total = 0.0;
        unsigned long long mk = 0ull;
        int mb = 0;
        for (int b = 0; b < nb; ++b) {
            total = __dadd_rn(total, s_load[b]);
            const unsigned long long k = okey(s_load[b]);
            if (k > mk) {
                mk = k;
                mb = b;
            }
        }
        const double mean = __ddiv_rn(total, (double)nb);
        const double pred = mean > 0.0 ? __ddiv_rn(s_load[mb], mean) : 1.0;
        const double cm = from_okey(cmax);
        const double floor = mean > 0.0 ? (cm > mean ? cm : mean) / mean : 1.0;
        const long long n = p.state[kStHist];
        double *row = p.hist + (size_t)(n % kBalHist) * kBalHistCols;
        row[0] = (double)p.dclock[0];
        row[1] = (double)st;
        row[2] = (double)mig;
        row[3] = pred;
        row[4] = p.pend[0];
        row[5] = floor;
        row[6] = (double)s_iters;
        row[7] = 0.0;
        p.state[kStHist] = n + 1;
        if (st != LB_STATIC) p.state[kStRebal] += 1;
        p.state[kStStrategy] = st;
    }
}

__global__ void __launch_bounds__(kItemThreads) k_items(const DevBal p) {
    __shared__ int s_w[kItemThreads / kWarp];
    __shared__ int s_wscan[kItemThreads / kWarp];
    const int b = blockIdx.x;
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    int acc = 0;
    for (int v = threadIdx.x; v < p.nvps; v += kItemThreads)
        if (p.assign[v] < b) acc += p.nchunks[v];
    const int start = block_sum_int(acc, s_w);
    if (threadIdx.x == 0) {
        p.bin_start[b] = start;
        if (b == p.nbins - 1) p.bin_start[p.nbins] = p.nitems;
    }
    // this processor's VPs in spatial order, each expanded into its items
    int carry = 0;
    for (int base = 0; base < p.nvps; base += kItemThreads) {
        const int s = base + threadIdx.x;
        const int v = s < p.nvps ? p.spatial[s] : -1;
        const int w = (v >= 0 && p.assign[v] == b) ? p.nchunks[v] : 0;
        int incl = w;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == kWarp - 1) s_wscan[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < kItemThreads / kWarp; ++q) {
            before += q < warp ? s_wscan[q] : 0;
            total += s_wscan[q];
        }
        const int pos = start + carry + before + incl - w;
        for (int c = 0; c < w; ++c) p.items[pos + c] = make_int2(v, c);
        carry += total;
        __syncthreads();
    }
}

}  // namespace

size_t dev_balance_smem(int nvps, int nbins) {
    return sizeof(double) * (size_t)nbins + sizeof(int) * 5 * (size_t)nvps;
}

// The attribute is per function: set the largest size any ctx can need, so
// that one ctx never lowers the limit under another.
cudaError_t dev_balance_init() {
    return cudaFuncSetAttribute(k_balance, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dev_balance_smem(kDevBalMaxVps, kDevBalMaxBins));
}

cudaError_t dev_measure(const DevBal &p, cudaStream_t s) {
    k_measure<<<(p.nvps + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t dev_rebalance(const DevBal &p, int strategy, cudaStream_t s) {
    k_rank<<<(p.nvps + kRankThreads - 1) / kRankThreads, kRankThreads, 0, s>>>(p, strategy);
    k_balance<<<1, kBalThreads, dev_balance_smem(p.nvps, p.nbins), s>>>(p, strategy);
    k_items<<<p.nbins, kItemThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace lbk
