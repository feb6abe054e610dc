// Host balancers (Sec. VI): static placement, GreedyLB, RefineSwapLB, and
// GreedyLB's rule over a given VP order (list scheduling) or block by block
// (blocked GreedyLB).
//
// Costs arrive as FP64 and are rounded once to a fixed-point grid
// (fixed_point): integers whose every sum stays below 2^53.  Loads are then
// exact int64 sums in any order and exactly representable in FP64, so the
// device balancer reproduces these assignments bit for bit.
#include "lb_balance.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>
#include <utility>

namespace lbk {

void static_blocks(int nvps, int nbins, std::vector<int> &out) {
    out.resize(nvps);
    for (int v = 0; v < nvps; ++v) out[v] = (int)(((long long)v * nbins) / nvps);
}

int bit_length(long long n) {
    int L = 0;
    while (n > 0) {
        ++L;
        n >>= 1;
    }
    return L;
}

// q_v = c_v * 2^e rounded to nearest (ties to even), e = 53 - L - x with L
// the bit length of the VP count and 2^(x-1) <= max c < 2^x.
void fixed_point(const std::vector<double> &costs, std::vector<long long> &q) {
    const size_t n = costs.size();
    q.assign(n, 0);
    double cmax = 0.0;
    for (double c : costs) cmax = c > cmax ? c : cmax;
    if (!(cmax > 0.0)) return;
    int x = 0;
    std::frexp(cmax, &x);
    const int e = 53 - bit_length((long long)n) - x;
    for (size_t v = 0; v < n; ++v) q[v] = std::llrint(std::ldexp(costs[v], e));
}

void bin_loads(const std::vector<long long> &q, const std::vector<int> &assign, int nbins,
               std::vector<long long> &loads) {
    loads.assign(nbins, 0);
    for (size_t v = 0; v < assign.size(); ++v) loads[assign[v]] += q[v];
}

double max_over_mean(const std::vector<double> &costs, const std::vector<int> &assign, int nbins) {
    std::vector<long long> q, loads;
    fixed_point(costs, q);
    bin_loads(q, assign, nbins, loads);
    long long total = 0;
    for (long long x : q) total += x;
    const double mean = (double)total / (double)nbins;
    const long long mx = *std::max_element(loads.begin(), loads.end());
    return mean > 0.0 ? (double)mx / mean : 1.0;
}

int migrations(const std::vector<int> &a, const std::vector<int> &b) {
    int m = 0;
    for (size_t v = 0; v < a.size(); ++v) m += a[v] != b[v];
    return m;
}

// Graham's list scheduling: VPs in `order`, each to the bin with the least
// load so far (ties: lowest id).
static void list_schedule(const std::vector<long long> &q, int nbins, const std::vector<int> &order,
                          std::vector<int> &out) {
    typedef std::pair<long long, int> Item;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int b = 0; b < nbins; ++b) heap.push(Item(0, b));
    out.assign(q.size(), 0);
    for (int v : order) {
        Item top = heap.top();
        heap.pop();
        out[v] = top.second;
        heap.push(Item(top.first + q[v], top.second));
    }
}

// GreedyLB: "always assigns the heaviest object to the least loaded
// processor" (Sec. VI-A).  Objects by (cost desc, id asc).
void greedy(const std::vector<double> &costs, int nbins, std::vector<int> &out) {
    std::vector<long long> q;
    fixed_point(costs, q);
    std::vector<int> order(q.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (q[a] != q[b]) return q[a] > q[b];
        return a < b;
    });
    list_schedule(q, nbins, order, out);
}

// GreedyLB's rule with the objects in a caller-given order.  With the VPs in
// spatial order and every processor visiting its VPs in that order, all
// processors sweep the grid in step: the order the GPU's L2 needs.
void greedy_ordered(const std::vector<double> &costs, int nbins, const std::vector<int> &order,
                    std::vector<int> &out) {
    std::vector<long long> q;
    fixed_point(costs, q);
    list_schedule(q, nbins, order, out);
}

// GreedyLB over consecutive blocks of nbins objects of `order`: within a
// block, objects by (cost desc, id asc) to bins by (load asc, id asc), one
// each.  Every processor takes one object of each full block, so with the
// VPs in spatial order all processors sweep the grid in lockstep; the load
// spread stays below the largest cost.
void greedy_blocked(const std::vector<double> &costs, int nbins, const std::vector<int> &order,
                    std::vector<int> &out) {
    std::vector<long long> q, loads(nbins, 0);
    fixed_point(costs, q);
    out.assign(q.size(), 0);
    std::vector<int> block, bins(nbins);
    for (size_t base = 0; base < order.size(); base += (size_t)nbins) {
        const size_t end = std::min(order.size(), base + (size_t)nbins);
        block.assign(order.begin() + base, order.begin() + end);
        std::sort(block.begin(), block.end(), [&](int a, int b) {
            if (q[a] != q[b]) return q[a] > q[b];
            return a < b;
        });
        std::iota(bins.begin(), bins.end(), 0);
        std::sort(bins.begin(), bins.end(), [&](int a, int b) {
            if (loads[a] != loads[b]) return loads[a] < loads[b];
            return a < b;
        });
        for (size_t k = 0; k < block.size(); ++k) {
            out[block[k]] = bins[k];
            loads[bins[k]] += q[block[k]];
        }
    }
}

// RefineSwapLB (Sec. VI-B): move objects off the most loaded processor
// toward the mean; swap when no single move fits.  The paper gives no
// constants; the reading implemented (q: fixed-point costs):
//   T = (1 + tol) * ((double)sum(q) / nbins).
//   Repeat at most 4*nvps times:
//     stop if max load <= T; P = most loaded (ties: lowest id);
//     for Q in (load asc, id asc), Q != P:
//       move: first o of P in (cost desc, id asc) with q_o > 0 and
//             load(Q) + q_o <= T  -> move, restart;
//       swap: over o in that order and o' of Q in (cost asc, id asc) with
//             q_o > q_o', the first pair minimising
//             max(load(P) - d, load(Q) + d), d = q_o - q_o'; if below
//             load(P) -> swap, restart;
//     no Q worked -> stop.
void refine_swap(const std::vector<double> &costs, const std::vector<int> &assign_in, int nbins,
                 double tol, std::vector<int> &assign) {
    std::vector<long long> q, loads;
    fixed_point(costs, q);
    const int nv = (int)q.size();
    assign = assign_in;
    bin_loads(q, assign, nbins, loads);
    long long total = 0;
    for (long long x : q) total += x;
    const double thr = (1.0 + tol) * ((double)total / (double)nbins);
    std::vector<std::vector<int>> members(nbins);
    for (int v = 0; v < nv; ++v) members[assign[v]].push_back(v);
    auto erase = [](std::vector<int> &vec, int x) {
        vec.erase(std::find(vec.begin(), vec.end(), x));
    };
    std::vector<int> qorder(nbins), porder, q2;
    for (long long it = 0; it < 4LL * nv; ++it) {
        int P = 0;
        for (int b = 1; b < nbins; ++b)
            if (loads[b] > loads[P]) P = b;
        if ((double)loads[P] <= thr) break;
        porder = members[P];
        std::sort(porder.begin(), porder.end(), [&](int a, int b) {
            if (q[a] != q[b]) return q[a] > q[b];
            return a < b;
        });
        std::iota(qorder.begin(), qorder.end(), 0);
        std::sort(qorder.begin(), qorder.end(), [&](int a, int b) {
            if (loads[a] != loads[b]) return loads[a] < loads[b];
            return a < b;
        });
        bool done = false;
        for (int Q : qorder) {
            if (Q == P) continue;
            for (int o : porder) {
                if (q[o] > 0 && (double)(loads[Q] + q[o]) <= thr) {
                    loads[P] -= q[o];
                    loads[Q] += q[o];
                    erase(members[P], o);
                    members[Q].push_back(o);
                    assign[o] = Q;
                    done = true;
                    break;
                }
            }
            if (done) break;
            q2 = members[Q];
            std::sort(q2.begin(), q2.end(), [&](int a, int b) {
                if (q[a] != q[b]) return q[a] < q[b];
                return a < b;
            });
            long long best = loads[P];
            int bo = -1, bo2 = -1;
            for (int o : porder)
                for (int o2 : q2) {
                    if (!(q[o] > q[o2])) continue;
                    const long long d = q[o] - q[o2];
                    const long long m = std::max(loads[P] - d, loads[Q] + d);
                    if (m < best) {
                        best = m;
                        bo = o;
                        bo2 = o2;
                    }
                }
            if (bo >= 0) {
                const long long d = q[bo] - q[bo2];
                loads[P] -= d;
                loads[Q] += d;
                erase(members[P], bo);
                members[Q].push_back(bo);
                erase(members[Q], bo2);
                members[P].push_back(bo2);
                assign[bo] = Q;
                assign[bo2] = P;
                done = true;
                break;
            }
        }
        if (!done) break;
    }
}

}  // namespace lbk
