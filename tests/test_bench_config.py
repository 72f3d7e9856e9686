"""Host-side configuration of bench.py: the projection each method builds on."""

import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import gaussian_projection, paa_projection  # noqa: E402


def test_det_lsh_uses_the_gaussian_hash_vectors():
    w = dict(bench.WORKLOAD)
    A = bench.projection_for(w)
    assert A.shape == (w["L"] * w["K"], w["d"])
    assert torch.equal(A, gaussian_projection(w["L"], w["K"], w["d"]))


def test_det_only_uses_one_tree_over_paa():
    w = dict(bench.WORKLOAD, method="det-only", L=1)
    A = bench.projection_for(w)
    assert A.shape == (w["K"], w["d"])
    assert torch.equal(A, paa_projection(w["K"], w["d"]))
    seg = w["d"] // w["K"]
    assert torch.allclose(A.sum(1), torch.ones(w["K"]))
    assert (A[0, :seg] == 1.0 / seg).all() and (A[0, seg:] == 0).all()
