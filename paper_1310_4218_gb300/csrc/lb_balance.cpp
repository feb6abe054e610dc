// Host balancers (Sec. VI): static placement, GreedyLB, RefineSwapLB.
//
// Costs are FP64; every load is accumulated with the same FP64 additions in
// the same order as stated below, so results are reproducible bit for bit.
// Built with -ffp-contract=off.
#include "lb_balance.h"

#include <algorithm>
#include <numeric>
#include <queue>
#include <utility>

namespace lbk {

void static_blocks(int nvps, int nbins, std::vector<int> &out) {
    out.resize(nvps);
    for (int v = 0; v < nvps; ++v) out[v] = (int)(((long long)v * nbins) / nvps);
}

void bin_loads(const std::vector<double> &costs, const std::vector<int> &assign, int nbins,
               std::vector<double> &loads) {
    loads.assign(nbins, 0.0);
    for (size_t v = 0; v < assign.size(); ++v) loads[assign[v]] += costs[v];
}

// Sum of the processor loads, processors in id order.
double total_load(const std::vector<double> &loads) {
    double total = 0.0;
    for (double x : loads) total += x;
    return total;
}

double max_over_mean(const std::vector<double> &costs, const std::vector<int> &assign, int nbins) {
    std::vector<double> loads;
    bin_loads(costs, assign, nbins, loads);
    double mean = total_load(loads) / nbins;
    double mx = *std::max_element(loads.begin(), loads.end());
    return mean > 0.0 ? mx / mean : 1.0;
}

int migrations(const std::vector<int> &a, const std::vector<int> &b) {
    int m = 0;
    for (size_t v = 0; v < a.size(); ++v) m += a[v] != b[v];
    return m;
}

// GreedyLB: "always assigns the heaviest object to the least loaded
// processor" (Sec. VI-A).  Objects by (cost desc, id asc); processor with
// the least load so far (ties: lowest id); loads summed in assignment order.
void greedy(const std::vector<double> &costs, int nbins, std::vector<int> &out) {
    const int nv = (int)costs.size();
    std::vector<int> order(nv);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (costs[a] != costs[b]) return costs[a] > costs[b];
        return a < b;
    });
    typedef std::pair<double, int> Item;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int b = 0; b < nbins; ++b) heap.push(Item(0.0, b));
    out.assign(nv, 0);
    for (int v : order) {
        Item top = heap.top();
        heap.pop();
        out[v] = top.second;
        heap.push(Item(top.first + costs[v], top.second));
    }
}

// GreedyLB's rule with the objects in a caller-given order (Graham's list
// scheduling).  With the VPs in spatial order and every processor visiting
// its VPs in that order, all processors sweep the grid in step: the order
// the GPU's L2 needs.
void greedy_ordered(const std::vector<double> &costs, int nbins, const std::vector<int> &order,
                    std::vector<int> &out) {
    typedef std::pair<double, int> Item;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int b = 0; b < nbins; ++b) heap.push(Item(0.0, b));
    out.assign(costs.size(), 0);
    for (int v : order) {
        Item top = heap.top();
        heap.pop();
        out[v] = top.second;
        heap.push(Item(top.first + costs[v], top.second));
    }
}

// RefineSwapLB (Sec. VI-B): move objects off the most loaded processor
// toward the mean; swap when no single move fits.  The paper gives no
// constants; the reading implemented:
//   T = (1 + tol) * mean, mean = total_load(loads) / nbins.
//   Repeat at most 4*nvps times:
//     stop if max load <= T; P = most loaded (ties: lowest id);
//     for Q in (load asc, id asc), Q != P:
//       move: first o of P in (cost desc, id asc) with cost > 0 and
//             load(Q) + cost <= T  -> move, restart;
//       swap: over o in that order and o' of Q in (cost asc, id asc) with
//             c_o > c_o', the first pair minimising
//             max(load(P) - d, load(Q) + d), d = c_o - c_o'; if below
//             load(P) -> swap, restart;
//     no Q worked -> stop.
//   Loads: source -= c (or d), then target += c (or d).
void refine_swap(const std::vector<double> &costs, const std::vector<int> &assign_in, int nbins,
                 double tol, std::vector<int> &assign) {
    const int nv = (int)costs.size();
    assign = assign_in;
    std::vector<double> loads;
    bin_loads(costs, assign, nbins, loads);
    const double thr = (1.0 + tol) * (total_load(loads) / nbins);
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
        if (loads[P] <= thr) break;
        porder = members[P];
        std::sort(porder.begin(), porder.end(), [&](int a, int b) {
            if (costs[a] != costs[b]) return costs[a] > costs[b];
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
                if (costs[o] > 0.0 && loads[Q] + costs[o] <= thr) {
                    loads[P] -= costs[o];
                    loads[Q] += costs[o];
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
                if (costs[a] != costs[b]) return costs[a] < costs[b];
                return a < b;
            });
            double best = loads[P];
            int bo = -1, bo2 = -1;
            for (int o : porder)
                for (int o2 : q2) {
                    if (!(costs[o] > costs[o2])) continue;
                    double d = costs[o] - costs[o2];
                    double m = std::max(loads[P] - d, loads[Q] + d);
                    if (m < best) {
                        best = m;
                        bo = o;
                        bo2 = o2;
                    }
                }
            if (bo >= 0) {
                double d = costs[bo] - costs[bo2];
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
