"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds no arithmetic of the solver: it only draws grids, sparsity
patterns and matrix values.  The right-hand side ``b = A @ x_true`` is formed
with SciPy's sparse product, a library primitive.
"""
from .acopf import (CONFIGS, KKTSequence, make_grid, kkt_sequence, config_sequence,
                    random_sparse_pattern, random_dd_values)

__all__ = ["CONFIGS", "KKTSequence", "make_grid", "kkt_sequence", "config_sequence",
           "random_sparse_pattern", "random_dd_values"]
