"""Seeded synthetic inputs shared by the oracle checks, the GPU tests and the bench.

This module only draws data. It holds none of the arithmetic of the method
(no embedding, no nearest-neighbour search, no weights, no correlation), so
both sides of a parity check can take their inputs from it.
"""

from .coupled_maps import (
    WorkloadSpec,
    WORKLOADS,
    BatchedSpec,
    coupled_logistic,
    workload,
    batched_specs,
    batched_dataset,
    sample_pairs,
    sine_series,
    logistic_series,
    white_noise,
    library_subsets,
)

__all__ = [
    "WorkloadSpec",
    "WORKLOADS",
    "BatchedSpec",
    "coupled_logistic",
    "workload",
    "batched_specs",
    "batched_dataset",
    "sample_pairs",
    "sine_series",
    "logistic_series",
    "white_noise",
    "library_subsets",
]
