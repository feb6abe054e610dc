// Host balancers (Sec. VI): static placement, GreedyLB, RefineSwapLB, list
// scheduling and blocked GreedyLB, on the fixed-point cost grid.
#pragma once

#include <vector>

namespace lbk {

int bit_length(long long n);
void fixed_point(const std::vector<double> &costs, std::vector<long long> &q);
void static_blocks(int nvps, int nbins, std::vector<int> &out);
void bin_loads(const std::vector<long long> &q, const std::vector<int> &assign, int nbins,
               std::vector<long long> &loads);
double max_over_mean(const std::vector<double> &costs, const std::vector<int> &assign, int nbins);
int migrations(const std::vector<int> &a, const std::vector<int> &b);
void greedy(const std::vector<double> &costs, int nbins, std::vector<int> &out);
void greedy_ordered(const std::vector<double> &costs, int nbins, const std::vector<int> &order,
                    std::vector<int> &out);
void greedy_blocked(const std::vector<double> &costs, int nbins, const std::vector<int> &order,
                    std::vector<int> &out);
void refine_swap(const std::vector<double> &costs, const std::vector<int> &assign_in, int nbins,
                 double tol, std::vector<int> &assign);

}  // namespace lbk
