"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This package holds data containers, workload sizes and seeded random draws
only -- none of the butterfly method's arithmetic.  Both sides of every parity
check (the FP64 oracle and the CUDA library) receive their inputs from here.
"""
from .factors import ButterflyFactors, tree_sizes
from .workloads import (CONFIGS, BatchMember, Config, batched_workload, complex_normal, sample_rows,
                        sketch_blocks, synthetic_factors)

__all__ = [
    "ButterflyFactors", "tree_sizes", "CONFIGS", "Config", "complex_normal",
    "synthetic_factors", "sample_rows", "BatchMember", "batched_workload", "sketch_blocks",
]
