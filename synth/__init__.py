"""Seeded synthetic inputs shared by the oracle side and the GPU side."""
from .circuits import (CircuitSpec, CircuitMatrix, WORKLOADS, make, nd_order, rhs,
                       random_pattern_matrix)

__all__ = ["CircuitSpec", "CircuitMatrix", "WORKLOADS", "make", "nd_order", "rhs",
           "random_pattern_matrix"]
