"""Seeded synthetic inputs for the column-physics load-balancing workloads.

This package holds no arithmetic of the method itself (no advection, no
diffusion solve, no load rule, no balancer).  It only draws the inputs that
both the CUDA library and the CPU oracle consume: initial fields, k_c arrays,
VP layouts and the workload definitions.
"""
from .rng import splitmix64, uniform01, std_normal, subseed
from .fields import gaussian_blob
from .layouts import regular_blocks, guillotine, layout_stats
from .kcfield import lognormal_kc
from .configs import CONFIGS, GridSpec, Workload, get_config

__all__ = [
    "splitmix64", "uniform01", "std_normal", "subseed", "gaussian_blob",
    "regular_blocks", "guillotine", "layout_stats", "lognormal_kc",
    "CONFIGS", "GridSpec", "Workload", "get_config",
]
