// Device-side load measurement and rebalancing: the per-VP cost average
// (Sec. V) and GreedyLB / list scheduling / RefineSwapLB (Sec. VI) run as
// kernels on the ctx stream, so a whole rebalance period -- steps,
// measurement, balancer, new work tables -- can be enqueued, or captured in
// one CUDA graph, without a host round trip.
//
// The balancers work on the fixed-point cost grid of lb_balance.cpp: each
// cost rounded once to an integer, every load and total an integer below
// 2^53.  Loads are int64 sums (exact in any order), so the device reproduces
// the host balancers' assignments bit for bit while adding in parallel, and
// no FP64 work is needed (a dependent FP64 add costs ~64 cycles on GB300
// and the FP64 pipe is narrow; integer ops cost a few).  The cost average
// itself stays FP64, with the host's operations in the host's order
// (explicitly rounded intrinsics, never contracted into FMAs).
//
// Kernels (all on the ctx stream):
//   k_measure  one thread per VP: cycles -> ns per step -> cost average;
//              the last block to finish (threadfence ticket) records SM
//              busy times and the measurement step
//   k_prep     one thread per VP: costs on the fixed-point grid; for
//              GreedyLB each VP's rank by (cost desc, id asc), for the
//              blocked variant its rank inside its block
//   k_balance  one CTA of 1024 threads: static / GreedyLB / list scheduling
//              in spatial order (one warp) / RefineSwapLB (whole CTA) on
//              shared-memory copies of the assignment and the costs;
//              migrations and predicted max/mean
//   k_items    one CTA per processor: its work-item range and its items in
//              spatial order (the tables the step kernel reads)
//   k_features, k_fit, k_rescale  cost rescale for a new k_c array
//              (lb_set_kc with predict_kc): item features, least-squares
//              fit of the per-item overhead, rescaled cost averages
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace lbk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBalThreads = 1024;
constexpr int kBalWarps = kBalThreads / kWarp;
constexpr int kPrepThreads = 256;
constexpr int kItemThreads = 1024;
constexpr int kMeasThreads = 256;
constexpr unsigned kNone = 0x7fffffffu;
constexpr int kIdBits = 10;                   // bins < 1024 = 2^kIdBits
constexpr unsigned long long kIdMask = (1ull << kIdBits) - 1;

__device__ __forceinline__ int resolve(int s, long long rebalances) {
    if (s == LB_AUTO) return rebalances == 0 ? LB_GREEDY : LB_REFINE_SWAP;
    if (s == LB_AUTO_SPATIAL) return rebalances == 0 ? LB_GREEDY_SPATIAL : LB_REFINE_SWAP;
    return s;
}

__device__ __forceinline__ int bit_length(long long n) { return n > 0 ? 64 - __clzll(n) : 0; }

// x with 2^(x-1) <= c < 2^x, for c > 0 (frexp's exponent), from the bits.
__device__ __forceinline__ int exponent_of(double c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffull;
    const int E = (int)(b >> 52);
    return E ? E - 1022 : bit_length((long long)(b & ((1ull << 52) - 1))) - 1074;
}

// round-half-even(c * 2^e) for c >= 0 with c * 2^e < 2^53, in integer
// arithmetic: c = M * 2^(E - 1075), so the result is M shifted by
// E - 1075 + e with the bits shifted out rounded.  Equal to
// llrint(ldexp(c, e)); FP64 work would run on GB300's narrow FP64 pipe.
__device__ __forceinline__ long long fixed_q(double c, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffull;
    if (b == 0ull) return 0;
    int E = (int)(b >> 52);
    unsigned long long M = b & ((1ull << 52) - 1);
    if (E == 0) E = 1;
    else M |= 1ull << 52;
    const int s = E - 1075 + e;
    if (s >= 0) return (long long)(M << s);
    const int sh = -s;
    if (sh >= 64) return 0;
    const unsigned long long qf = M >> sh;
    const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    return (long long)(qf + (unsigned long long)(rem > half || (rem == half && (qf & 1ull))));
}

// Warp minimum / maximum of a 64-bit key; every lane gets it.
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long k) {
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mh = __reduce_min_sync(kFull, hi);
    const unsigned ml = __reduce_min_sync(kFull, hi == mh ? lo : ~0u);
    return ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ unsigned long long warp_max64(unsigned long long k) {
    return ~warp_min64(~k);
}

// Block minimum of a 64-bit key (blockDim a multiple of 32); every thread
// gets it.  s_w holds one word per warp plus one.
__device__ unsigned long long block_min64(unsigned long long k, unsigned long long *s_w) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    const int nw = blockDim.x / kWarp;
    k = warp_min64(k);
    if (lane == 0) s_w[warp] = k;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < nw ? s_w[lane] : ~0ull;
        x = warp_min64(x);
        if (lane == 0) s_w[nw] = x;
    }
    __syncthreads();
    k = s_w[nw];
    __syncthreads();
    return k;
}

__device__ unsigned long long block_sum64(unsigned long long v, unsigned long long *s_w) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    const int nw = blockDim.x / kWarp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < nw; ++w) t += s_w[w];
    __syncthreads();
    return t;
}

// Graham's list scheduling -- each VP of ord[0..nv) in turn to the bin with
// the lowest (load, id), loads summed in assignment order (GreedyLB's rule)
// -- reproduced exactly in rounds by one warp.  Keys load * 2^10 + bin are
// unique and ordered like (load, bin); cur holds the bins' keys in ascending
// order.  With the bins in that order as s_0, s_1, ..., the sequential rule
// gives VPs i, i+1, ... to s_0, s_1, ... for as long as each next s_j is
// still below every key already updated in this round (its key plus the
// VP's cost); the first VP for which that fails starts the next round.  The
// new order merges the updated keys into the untouched ones.
template <int R>   // candidates per lane: nb <= 32 * R
__device__ __noinline__ void list_schedule(const int32_t *ord, const long long *s_q, int nv, int nb,
                              int *s_assign, unsigned long long *sk0, unsigned long long *sk1,
                              unsigned long long *s_t) {
    const int lane = threadIdx.x % kWarp;
    for (int b = lane; b < nb; b += kWarp) sk0[b] = (unsigned long long)b;
    __syncwarp();
    unsigned long long *cur = sk0, *nxt = sk1;
    for (int i = 0; i < nv;) {
        const int n = min(nb, nv - i);
        unsigned long long k[R], u[R];
        int vv[R];
        unsigned long long run = ~0ull;   // min of u over this lane's candidates
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = lane * R + r;
            k[r] = ~0ull;
            u[r] = ~0ull;
            vv[r] = -1;
            if (j < n) {
                k[r] = cur[j];
                vv[r] = ord[i + j];
                u[r] = k[r] + ((unsigned long long)s_q[vv[r]] << kIdBits);
            }
            run = u[r] < run ? u[r] : run;
        }
        unsigned long long incl = run;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o && y < incl) incl = y;
        }
        unsigned long long pre = __shfl_up_sync(kFull, incl, 1);   // earlier lanes
        if (lane == 0) pre = ~0ull;
        unsigned first = ~0u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = lane * R + r;
            if (first == ~0u && j >= 1 && j < n && !(k[r] < pre)) first = (unsigned)j;
            pre = u[r] < pre ? u[r] : pre;
        }
        const unsigned f = __reduce_min_sync(kFull, first);
        const int K = f == ~0u ? n : (int)f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = lane * R + r;
            if (j < K) {
                s_assign[vv[r]] = (int)(k[r] & kIdMask);
                s_t[j] = u[r];
            }
        }
        __syncwarp();
        for (int j = lane; j < nb; j += kWarp) {
            unsigned long long key;
            int pos;
            if (j < K) {
                key = s_t[j];
                int lo = K, hi = nb;   // untouched keys below key
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cur[mid] < key) lo = mid + 1;
                    else hi = mid;
                }
                pos = lo - K;
            } else {
                key = cur[j];
                pos = j - K;
            }
            for (int t = 0; t < K; ++t) pos += s_t[t] < key;
            nxt[pos] = key;
        }
        __syncwarp();
        unsigned long long *tmp = cur;
        cur = nxt;
        nxt = tmp;
        i += K;
    }
}

// ---------------------------------------------------------------- kernels
__global__ void __launch_bounds__(kMeasThreads) k_measure(const DevBal p) {
    __shared__ double s_npc, s_steps;
    __shared__ int s_last;
    __shared__ unsigned long long s_w[kMeasThreads / kWarp + 1];
    __shared__ unsigned long long s_busy[kDevBalMaxSms];
    // ns per SM cycle from every processor's globaltimer / clock64 pair:
    // integer sums (exact in any order), one FP64 division
    unsigned long long ns = 0, cy = 0;
    for (int b = threadIdx.x; b < p.nbins; b += blockDim.x) {
        const long long dn = p.bin_cal[4 * b + 2] - p.bin_cal[4 * b + 0];
        const long long dc = p.bin_cal[4 * b + 3] - p.bin_cal[4 * b + 1];
        if (dn > 0 && dc > 0) {
            ns += (unsigned long long)dn;
            cy += (unsigned long long)dc;
        }
    }
    ns = block_sum64(ns, s_w);
    cy = block_sum64(cy, s_w);
    if (threadIdx.x == 0) {
        double npc = cy > 0 ? __ddiv_rn(__ll2double_rn((long long)ns), __ll2double_rn((long long)cy))
                            : 0.0;
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
    unsigned long long mx = 0, tot = 0, used = 0;
    for (int s = threadIdx.x; s < p.nsm; s += blockDim.x) {
        const unsigned long long x = s_busy[s];
        mx = x > mx ? x : mx;
        tot += x;
        used += x > 0;
    }
    mx = ~block_min64(~mx, s_w);
    tot = block_sum64(tot, s_w);
    used = block_sum64(used, s_w);
    if (threadIdx.x == 0) {
        p.pend[0] = (used > 0 && tot > 0) ? (double)mx / ((double)tot / (double)used) : 0.0;
        p.state[kStHave] = 1;
        p.state[kStMeasStep] = p.dclock[0];
        *p.ticket = 0u;
    }
}

// Costs on the fixed-point grid (lb_balance.cpp: fixed_point) into p.q,
// and the orders that do not depend on loads: GreedyLB's (cost desc, id
// asc) over all VPs, or for the blocked variant the same order inside each
// block of nbins VPs in spatial order.  Every block rounds all costs into
// shared memory and handles its own range.
__global__ void __launch_bounds__(kPrepThreads) k_prep(const DevBal p, int strategy) {
    extern __shared__ long long s_qall[];          // [nvps]
    __shared__ unsigned long long s_w[kPrepThreads / kWarp + 1];
    const int nv = p.nvps, nb = p.nbins;
    unsigned long long kmax = 0ull;                // costs >= 0: bit patterns order them
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const unsigned long long k =
            (unsigned long long)__double_as_longlong(p.cost[v]) & 0x7fffffffffffffffull;
        kmax = k > kmax ? k : kmax;
    }
    kmax = ~block_min64(~kmax, s_w);
    const double cmax = __longlong_as_double((long long)kmax);
    const int e = kmax ? 53 - bit_length(nv) - exponent_of(cmax) : 0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) s_qall[v] = kmax ? fixed_q(p.cost[v], e) : 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nv) return;
    p.q[t] = s_qall[t];
    const int st = resolve(strategy, p.state[kStRebal]);
    if (st == LB_GREEDY) {
        const long long qv = s_qall[t];
        int rank = 0;
        for (int u = 0; u < nv; ++u) {
            const long long qu = s_qall[u];
            rank += (int)((qu > qv) | ((qu == qv) & (u < t)));
        }
        p.order[rank] = t;
    } else if (st == LB_GREEDY_BLOCKED) {
        const int base = (t / nb) * nb, m = min(nb, nv - base);
        const int v = p.spatial[t];
        const long long qv = s_qall[v];
        int rank = 0;
        for (int c = 0; c < m; ++c) {
            const int u = p.spatial[base + c];
            const long long qu = s_qall[u];
            rank += (int)((qu > qv) | ((qu == qv) & (u < v)));
        }
        p.order[base + rank] = v;
    }
}

__global__ void __launch_bounds__(kBalThreads, 1) k_balance(const DevBal p, int strategy,
                                                            double threshold) {
    extern __shared__ long long s_dyn[];
    const int nv = p.nvps, nb = p.nbins;
    long long *s_q = s_dyn;                                          // [nv] fixed-point costs
    unsigned long long *s_load = (unsigned long long *)(s_q + nv);   // [nb]
    unsigned long long *s_k0 = s_load + nb;                          // [nb] list-scheduling keys
    unsigned long long *s_k1 = s_k0 + nb;                            // [nb]
    unsigned long long *s_t = s_k1 + nb;                             // [nb]
    int *s_assign = (int *)(s_t + nb);                               // [nv]
    int *s_ul = s_assign + nv;       // [nv] members of P or Q (unordered)
    int *s_ps = s_ul + nv;           // [nv] members of P, (cost desc, id asc)
    int *s_qs = s_ps + nv;           // [nv] members of Q, (cost asc, id asc)
    __shared__ int s_strat, s_skip, s_P, s_Q, s_np, s_nq, s_iters;
    __shared__ unsigned s_found;
    __shared__ double s_thr;
    __shared__ unsigned long long s_w[kBalWarps + 1];
    const int tid = threadIdx.x, lane = tid % kWarp, warp = tid / kWarp;

    if (tid == 0) {
        const int st = resolve(strategy, p.state[kStRebal]);
        s_strat = st;
        s_skip = st != LB_STATIC && st != LB_ATOMIC_QUEUE && !p.state[kStHave];
        if (s_skip) atomicCAS(p.status, 0, (int)LB_ESTATE);
        s_iters = 0;
    }
    __syncthreads();
    if (s_skip) return;
    const int st = s_strat;
    for (int v = tid; v < nv; v += kBalThreads) {
        s_assign[v] = p.assign[v];
        s_q[v] = p.q[v];
    }
    __syncthreads();

    // threshold-triggered rebalancing: keep the table while its predicted
    // max/mean under the current costs stays at or below the threshold
    // (unless the costs were just rescaled for a new k_c array)
    if (threshold > 0.0 && st != LB_STATIC && st != LB_ATOMIC_QUEUE && !p.state[kStForce]) {
        for (int b = tid; b < nb; b += kBalThreads) s_load[b] = 0ull;
        __syncthreads();
        unsigned long long tot = 0, qmax = 0;
        for (int v = tid; v < nv; v += kBalThreads) {
            const unsigned long long q = (unsigned long long)s_q[v];
            atomicAdd(&s_load[s_assign[v]], q);
            tot += q;
            qmax = q > qmax ? q : qmax;
        }
        tot = block_sum64(tot, s_w);
        qmax = ~block_min64(~qmax, s_w);
        unsigned long long lmax = 0;
        for (int b = tid; b < nb; b += kBalThreads) lmax = s_load[b] > lmax ? s_load[b] : lmax;
        lmax = ~block_min64(~lmax, s_w);
        const double mean = __ddiv_rn(__ull2double_rn(tot), (double)nb);
        const double pred = mean > 0.0 ? __ddiv_rn(__ull2double_rn(lmax), mean) : 1.0;
        if (pred <= threshold) {
            if (tid == 0) {
                const double cm = __ull2double_rn(qmax);
                const long long n = p.state[kStHist];
                double *row = p.hist + (size_t)(n % kBalHist) * kBalHistCols;
                row[0] = (double)p.dclock[0];
                row[1] = (double)st;
                row[2] = 0.0;
                row[3] = pred;
                row[4] = p.pend[0];
                row[5] = mean > 0.0 ? (cm > mean ? cm : mean) / mean : 1.0;
                row[6] = 0.0;
                row[7] = 1.0;
                p.state[kStHist] = n + 1;
                p.state[kStKept] = 1;
            }
            return;
        }
    }

    if (st == LB_ATOMIC_QUEUE) {
        // no table: the period is only recorded
    } else if (st == LB_STATIC) {
        for (int v = tid; v < nv; v += kBalThreads) s_assign[v] = (int)(((long long)v * nb) / nv);
    } else if (st == LB_GREEDY || st == LB_GREEDY_SPATIAL) {
        if (warp == 0) {
            const int32_t *ord = st == LB_GREEDY ? p.order : p.spatial;
            if (nb <= 5 * kWarp) list_schedule<5>(ord, s_q, nv, nb, s_assign, s_k0, s_k1, s_t);
            else if (nb <= 8 * kWarp) list_schedule<8>(ord, s_q, nv, nb, s_assign, s_k0, s_k1, s_t);
            else list_schedule<kDevBalMaxBins / kWarp>(ord, s_q, nv, nb, s_assign, s_k0, s_k1, s_t);
        }
    } else if (st == LB_GREEDY_BLOCKED) {
        // GreedyLB block by block over the VPs in spatial order
        // (lb_balance.cpp: greedy_blocked).  The order of the VPs inside
        // each block (cost desc, id asc) does not depend on the loads:
        // k_prep ranked all blocks at once.  Block by block, the bins are
        // ranked by (load asc, id asc) and the VP of rank r goes to the bin
        // of rank r.
        const int32_t *s_byr = p.order;   // VPs of each block by rank (k_prep)
        int *s_bin = s_qs;                // [nb] bins by rank (first m used)
        for (int b = tid; b < nb; b += kBalThreads) s_load[b] = 0ull;
        // bin ranks: G threads per bin (a power of two dividing 32)
        const int G = nb * 8 <= kBalThreads ? 8 : (nb * 4 <= kBalThreads ? 4
                    : (nb * 2 <= kBalThreads ? 2 : 1));
        for (int base = 0; base < nv; base += nb) {
            const int m = min(nb, nv - base);
            for (int b = tid; b < nb; b += kBalThreads)
                s_k0[b] = (s_load[b] << kIdBits) | (unsigned long long)b;
            __syncthreads();
            for (int g0 = 0; g0 < nb * G; g0 += kBalThreads) {
                const int gi = g0 + tid;
                const int b = gi / G, sub = gi % G;
                int r = 0;
                if (b < nb) {
                    const unsigned long long kb = s_k0[b];
                    const int c0 = (nb * sub) / G, c1 = (nb * (sub + 1)) / G;
#pragma unroll 8
                    for (int c = c0; c < c1; ++c) r += (int)(s_k0[c] < kb);
                }
                for (int o = 1; o < G; o <<= 1) r += __shfl_xor_sync(kFull, r, o);
                if (b < nb && sub == 0 && r < m) s_bin[r] = b;
            }
            __syncthreads();
            for (int r = tid; r < m; r += kBalThreads) {
                const int v = s_byr[base + r], b = s_bin[r];
                s_assign[v] = b;
                s_load[b] += (unsigned long long)s_q[v];
            }
            __syncthreads();
        }
    } else {
        // RefineSwapLB (lb_balance.cpp: refine_swap); loads are exact
        // integers, so they may be summed in any order
        for (int b = tid; b < nb; b += kBalThreads) s_load[b] = 0ull;
        __syncthreads();
        unsigned long long tot = 0;
        for (int v = tid; v < nv; v += kBalThreads) {
            atomicAdd(&s_load[s_assign[v]], (unsigned long long)s_q[v]);
            tot += (unsigned long long)s_q[v];
        }
        tot = block_sum64(tot, s_w);
        if (tid == 0)
            s_thr = __dmul_rn(__dadd_rn(1.0, p.refine_tol),
                              __ddiv_rn(__ull2double_rn(tot), (double)nb));
        __syncthreads();
        const double thr = s_thr;
        for (long long it = 0; it < 4LL * nv; ++it) {
            if (warp == 0) {
                // P: largest load, lowest id; Q0: smallest (load, id) other than P
                unsigned long long kp = 0ull;
                for (int b = lane; b < nb; b += kWarp) {
                    const unsigned long long k = (s_load[b] << kIdBits) | (kIdMask - b);
                    kp = k > kp ? k : kp;
                }
                kp = warp_max64(kp);
                const int P = (int)(kIdMask - (kp & kIdMask));
                unsigned long long kq = ~0ull;
                for (int b = lane; b < nb; b += kWarp) {
                    const unsigned long long k = (s_load[b] << kIdBits) | (unsigned long long)b;
                    if (b != P && k < kq) kq = k;
                }
                kq = warp_min64(kq);
                if (lane == 0) {
                    s_P = P;
                    s_Q = kq == ~0ull ? (int)kNone : (int)(kq & kIdMask);
                    s_np = 0;
                    s_found = kNone;
                }
            }
            __syncthreads();
            const int P = s_P;
            if (__ull2double_rn(s_load[P]) <= thr) break;
            if (tid == 0) ++s_iters;
            for (int v = tid; v < nv; v += kBalThreads)
                if (s_assign[v] == P) s_ul[atomicAdd(&s_np, 1)] = v;
            __syncthreads();
            const int np = s_np;
            for (int i = tid; i < np; i += kBalThreads) {
                const int vi = s_ul[i];
                const long long qi = s_q[vi];
                int r = 0;
                for (int j = 0; j < np; ++j) {
                    const int vj = s_ul[j];
                    const long long qj = s_q[vj];
                    r += (qj > qi) || (qj == qi && vj < vi);
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
                const unsigned long long lq = s_load[Q0];
                for (int i = tid; i < np; i += kBalThreads) {
                    const long long c = s_q[s_ps[i]];
                    if (c > 0 && __ull2double_rn(lq + (unsigned long long)c) <= thr)
                        atomicMin(&s_found, (unsigned)i);
                }
            }
            __syncthreads();
            if (s_found != kNone) {
                if (tid == 0) {
                    const int o = s_ps[s_found];
                    const unsigned long long c = (unsigned long long)s_q[o];
                    s_load[P] -= c;
                    s_load[Q0] += c;
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
                    if (s_assign[v] == Q) s_ul[atomicAdd(&s_nq, 1)] = v;
                __syncthreads();
                const int nq = s_nq;
                for (int i = tid; i < nq; i += kBalThreads) {
                    const int vi = s_ul[i];
                    const long long qi = s_q[vi];
                    int r = 0;
                    for (int j = 0; j < nq; ++j) {
                        const int vj = s_ul[j];
                        const long long qj = s_q[vj];
                        r += (qj < qi) || (qj == qi && vj < vi);
                    }
                    s_qs[r] = vi;
                }
                __syncthreads();
                // the first pair (o-order, then o'-order) of least
                // m = max(load P - d, load Q + d) below load P: the least m,
                // then the least pair index among the holders of it
                const long long LP = (long long)s_load[P], LQ = (long long)s_load[Q];
                unsigned long long bm = ~0ull, be = ~0ull;
                const long long npairs = (long long)np * nq;
                for (long long e = tid; e < npairs; e += kBalThreads) {
                    const int i = (int)(e / nq), j = (int)(e % nq);
                    const long long qo = s_q[s_ps[i]], q2 = s_q[s_qs[j]];
                    if (!(qo > q2)) continue;
                    const long long d = qo - q2;
                    const long long a = LP - d, b = LQ + d;
                    const long long m = a < b ? b : a;
                    if (!(m < LP)) continue;
                    if ((unsigned long long)m < bm ||
                        ((unsigned long long)m == bm && (unsigned long long)e < be)) {
                        bm = (unsigned long long)m;
                        be = (unsigned long long)e;
                    }
                }
                const unsigned long long gm = block_min64(bm, s_w);
                const unsigned long long ge = block_min64(bm == gm ? be : ~0ull, s_w);
                if (gm != ~0ull) {
                    if (tid == 0) {
                        const int o = s_ps[ge / nq], o2 = s_qs[ge % nq];
                        const unsigned long long d = (unsigned long long)(s_q[o] - s_q[o2]);
                        s_load[P] -= d;
                        s_load[Q] += d;
                        s_assign[o] = Q;
                        s_assign[o2] = P;
                    }
                    __syncthreads();
                    done = true;
                    break;
                }
                if (warp == 0) {
                    const unsigned long long after = (s_load[Q] << kIdBits) | (unsigned long long)Q;
                    unsigned long long kq = ~0ull;
                    for (int b = lane; b < nb; b += kWarp) {
                        const unsigned long long k = (s_load[b] << kIdBits) | (unsigned long long)b;
                        if (b != P && k > after && k < kq) kq = k;
                    }
                    kq = warp_min64(kq);
                    if (lane == 0) s_Q = kq == ~0ull ? (int)kNone : (int)(kq & kIdMask);
                }
                __syncthreads();
                Q = s_Q;
            }
            if (!done) break;
        }
    }
    __syncthreads();

    // migrations, new table, predicted max/mean, record
    for (int b = tid; b < nb; b += kBalThreads) s_load[b] = 0ull;
    __syncthreads();
    unsigned long long mig = 0, qmax = 0, tot = 0;
    for (int v = tid; v < nv; v += kBalThreads) {
        mig += s_assign[v] != p.assign[v];
        const unsigned long long q = (unsigned long long)s_q[v];
        qmax = q > qmax ? q : qmax;
        tot += q;
        atomicAdd(&s_load[s_assign[v]], q);
    }
    mig = block_sum64(mig, s_w);
    tot = block_sum64(tot, s_w);
    qmax = ~block_min64(~qmax, s_w);
    unsigned long long lmax = 0;
    for (int b = tid; b < nb; b += kBalThreads) lmax = s_load[b] > lmax ? s_load[b] : lmax;
    lmax = ~block_min64(~lmax, s_w);
    for (int v = tid; v < nv; v += kBalThreads) p.assign[v] = s_assign[v];
    if (tid == 0) {
        const double mean = __ddiv_rn(__ull2double_rn(tot), (double)nb);
        const double cm = __ull2double_rn(qmax);
        const double floor = mean > 0.0 ? (cm > mean ? cm : mean) / mean : 1.0;
        // the queue's prediction is its granularity floor
        const double pred = st == LB_ATOMIC_QUEUE
                                ? floor
                                : (mean > 0.0 ? __ddiv_rn(__ull2double_rn(lmax), mean) : 1.0);
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
        p.state[kStKept] = 0;
        p.state[kStForce] = 0;
        if (st != LB_STATIC && st != LB_ATOMIC_QUEUE) {
            p.state[kStRebal] += 1;
            p.state[kStStrategy] = st;
        }
    }
}

__global__ void __launch_bounds__(kItemThreads) k_items(const DevBal p) {
    __shared__ unsigned long long s_w[kItemThreads / kWarp + 1];
    __shared__ int s_wscan[kItemThreads / kWarp];
    const int b = blockIdx.x;
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    if (p.state[kStKept]) return;     // table unchanged
    unsigned long long acc = 0;
    for (int v = threadIdx.x; v < p.nvps; v += kItemThreads)
        if (p.assign[v] < b) acc += (unsigned long long)p.nchunks[v];
    const int start = (int)block_sum64(acc, s_w);
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

__global__ void k_set_kc(GridDev *g, const int32_t *kc) { g->kc = kc; }

// Item features of grid `grid`'s VPs under k_c array kc, one warp per VP:
// out[v] = nz * sum over the VP's work items of the largest k_c among the
// item's columns (the sweeps a warp runs for it).  Items are the kernel's:
// tile_w x tile_h tiles (row-major over tiles), or runs of cols_per_item
// columns in row-major order; either way a warp pass over 32 item slots
// covers whole items (32 is a multiple of the item size).
__global__ void __launch_bounds__(256) k_features(const DevBal p, int grid, const int32_t *kc,
                                                  double *out) {
    const int v = (int)((blockIdx.x * blockDim.x + threadIdx.x) / kWarp);
    const int lane = threadIdx.x % kWarp;
    if (v >= p.nvps) return;                 // whole warps
    const VPDev vp = p.vps[v];
    if (vp.grid != grid) return;
    if (p.nchunks[v] == 0) {                 // a VP this ctx does not run (lb_set_owned)
        if (lane == 0) out[v] = 0.0;
        return;
    }
    const GridDev &g = p.grids[grid];
    const bool tiles = p.tile_w > 0;
    const int isz = tiles ? p.tile_w * p.tile_h : p.cols_per_item;
    const int tiles_x = tiles ? (vp.w + p.tile_w - 1) / p.tile_w : 1;
    const int nitems = tiles ? tiles_x * ((vp.h + p.tile_h - 1) / p.tile_h)
                             : (vp.ncols + isz - 1) / isz;
    long long sum = 0;
    for (int base = 0; base < nitems * isz; base += kWarp) {
        const int slot = base + lane;
        const int it = slot / isz, c = slot - it * isz;
        int xi, yi;
        bool ok;
        if (tiles) {
            const int ty = it / tiles_x, tx = it - ty * tiles_x;
            xi = tx * p.tile_w + c % p.tile_w;
            yi = ty * p.tile_h + c / p.tile_w;
            ok = it < nitems && xi < vp.w && yi < vp.h;
        } else {
            const int q = it * isz + c;
            yi = q / vp.w;
            xi = q - yi * vp.w;
            ok = q < vp.ncols;
        }
        int k = 0;
        if (ok) {
            const int kv = kc[(size_t)(vp.y0 + yi) * g.nx + vp.x0 + xi];
            k = kv > 0 ? (kv < LB_KC_MAX ? kv : LB_KC_MAX) : 0;   // as the step kernel reads it
        }
        for (int o = isz / 2; o > 0; o >>= 1) {
            const int k2 = __shfl_xor_sync(kFull, k, o);
            k = k2 > k ? k2 : k;
        }
        if (lane % isz == 0) sum += k;
    }
    sum = (long long)__reduce_add_sync(kFull, (unsigned)sum);
    if (lane == 0) out[v] = (double)sum * (double)g.nz;
}

__device__ double block_sum_f64(double x, double *s_d) {
    const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
    const int nw = blockDim.x / kWarp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0) s_d[warp] = x;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += s_d[w];
    __syncthreads();
    return t;
}

// Cost rescale for a new k_c array of grid `grid`, part 1: per block of
// kFitThreads VPs the sums of the least-squares fit of the last measured
// costs y to a f1 + b f2 (old array): sum x1^2, x1 x2, x2^2, x1 y, x2 y.
__global__ void __launch_bounds__(kFitThreads) k_fit(const DevBal p, int grid) {
    __shared__ double s_d[kFitThreads / kWarp];
    const int v = blockIdx.x * kFitThreads + threadIdx.x;
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (v < p.nvps && p.vps[v].grid == grid) {
        const double x1 = p.feat1[v], x2 = p.feat2[v], y = p.last[v];
        t[0] = x1 * x1;
        t[1] = x1 * x2;
        t[2] = x2 * x2;
        t[3] = x1 * y;
        t[4] = x2 * y;
    }
    for (int k = 0; k < 5; ++k) {
        const double sum = block_sum_f64(t[k], s_d);
        if (threadIdx.x == 0) p.fit[blockIdx.x * 5 + k] = sum;
    }
}

// Part 2: every block adds the partial sums in block order (the same kappa
// everywhere) -- kappa = a / b, p.kc_overhead when the fit is ill-posed --
// and rescales its VPs: cost *= (kappa f1 + f2_new) / (kappa f1 + f2_old);
// the new features become the current ones.
__global__ void __launch_bounds__(kFitThreads) k_rescale(const DevBal p, int grid, int nblocks) {
    __shared__ double s_kappa;
    if (threadIdx.x == 0) {
        double a11 = 0.0, a12 = 0.0, a22 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int k = 0; k < nblocks; ++k) {
            a11 += p.fit[k * 5 + 0];
            a12 += p.fit[k * 5 + 1];
            a22 += p.fit[k * 5 + 2];
            b1 += p.fit[k * 5 + 3];
            b2 += p.fit[k * 5 + 4];
        }
        double kappa = p.kc_overhead;
        const double det = a11 * a22 - a12 * a12;
        if (det > 1e-9 * a11 * a22 && a22 > 0.0) {
            const double a = (b1 * a22 - b2 * a12) / det, b = (a11 * b2 - a12 * b1) / det;
            if (b > 0.0 && a >= 0.0) kappa = a / b;
        }
        s_kappa = kappa;
        if (blockIdx.x == 0) p.pend[1] = kappa;
    }
    __syncthreads();
    const bool have = p.state[kStHave] != 0;
    const double kappa = s_kappa;
    const int v = blockIdx.x * kFitThreads + threadIdx.x;
    if (v < p.nvps && p.vps[v].grid == grid) {
        const double f1 = p.feat1[v], fo = p.feat2[v], fn = p.feat_new[v];
        const double den = kappa * f1 + fo;
        if (have && den > 0.0) p.cost[v] = p.cost[v] * ((kappa * f1 + fn) / den);
        p.feat2[v] = fn;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && have) p.state[kStForce] = 1;
}

}  // namespace

cudaError_t dev_set_kc(GridDev *g, const int32_t *kc, cudaStream_t s) {
    k_set_kc<<<1, 1, 0, s>>>(g, kc);
    return cudaGetLastError();
}

cudaError_t dev_kc_features(const DevBal &p, int grid, const int32_t *kc, bool initial,
                            cudaStream_t s) {
    const int blocks = (p.nvps * kWarp + 255) / 256;
    k_features<<<blocks, 256, 0, s>>>(p, grid, kc, initial ? p.feat2 : p.feat_new);
    if (!initial) {
        const int nb = (p.nvps + kFitThreads - 1) / kFitThreads;
        k_fit<<<nb, kFitThreads, 0, s>>>(p, grid);
        k_rescale<<<nb, kFitThreads, 0, s>>>(p, grid, nb);
    }
    return cudaGetLastError();
}

size_t dev_balance_smem(int nvps, int nbins) {
    return sizeof(long long) * (size_t)nvps + sizeof(unsigned long long) * 4 * (size_t)nbins +
           sizeof(int) * 4 * (size_t)nvps;
}

static size_t prep_smem(int nvps) { return sizeof(long long) * (size_t)nvps; }

// The attributes are per function: set the largest sizes any ctx can need,
// so that one ctx never lowers the limit under another.
cudaError_t dev_balance_init() {
    cudaError_t e = cudaFuncSetAttribute(k_balance, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dev_balance_smem(kDevBalMaxVps, kDevBalMaxBins));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)prep_smem(kDevBalMaxVps));
    return e;
}

cudaError_t dev_measure(const DevBal &p, cudaStream_t s) {
    k_measure<<<(p.nvps + kMeasThreads - 1) / kMeasThreads, kMeasThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t dev_rebalance(const DevBal &p, int strategy, double threshold, cudaStream_t s) {
    k_prep<<<(p.nvps + kPrepThreads - 1) / kPrepThreads, kPrepThreads, prep_smem(p.nvps), s>>>(
        p, strategy);
    k_balance<<<1, kBalThreads, dev_balance_smem(p.nvps, p.nbins), s>>>(p, strategy, threshold);
    if (strategy != LB_ATOMIC_QUEUE) k_items<<<p.nbins, kItemThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace lbk
