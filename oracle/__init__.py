"""FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
may import this package.  It shares no code with the CUDA library and the
library never calls it.

  step.py     -- the column-physics step (advection or the Jacobi sweep, k_c
                 Thomas sweeps, k_c rule, compensated mass), thin ctypes
                 wrapper over lb_oracle.c
  balance.py  -- the balancers: GreedyLB, RefineSwapLB, static placement
"""
from .step import (OracleGrid, kc_field, thomas, advect, jacobi, step, run, run_window,
                   compensated_sum, build_oracle)
from .balance import (static_blocks, greedy, greedy_ordered, refine_swap, migrations, bin_loads,
                      max_over_mean, fixed_point, greedy_blocked)

__all__ = ["OracleGrid", "kc_field", "thomas", "advect", "jacobi", "step", "run",
           "run_window", "compensated_sum", "build_oracle", "static_blocks",
           "greedy", "greedy_ordered", "refine_swap", "migrations", "bin_loads", "max_over_mean",
           "fixed_point", "greedy_blocked"]
