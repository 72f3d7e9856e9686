"""Seeded synthetic inputs for DET-LSH (data, queries, random draws).

This package holds input generators only: no step of the method's arithmetic
lives here. Both the CUDA path's tests/bench and the CPU oracle's tests draw
their inputs from it, so the two sides see identical inputs.
"""

from .synthetic import (  # noqa: F401
    WORKLOADS,
    Workload,
    gaussian_projection,
    make_workload,
    paa_projection,
    sample_ids,
)
