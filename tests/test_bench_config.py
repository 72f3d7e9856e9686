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


def test_gather_kernel_names_follow_the_library_dispatch():
    # FP32 rows of at most 128 coordinates (a multiple of 4) take the
    # eight-lanes-per-row gather, other widths the general one, a shortlist
    # the BF16 coarse gather
    assert bench.gather_kernel(128, 0) == "k_dist_g8"
    assert bench.gather_kernel(96, 0) == "k_dist_g8"
    assert bench.gather_kernel(4, 0) == "k_dist_g8"
    assert bench.gather_kernel(132, 0) == "k_dist"
    assert bench.gather_kernel(960, 0) == "k_dist"
    assert bench.gather_kernel(126, 0) == "k_dist"
    assert bench.gather_kernel(128, 64) == "k_dist_bf16"


def test_ncu_traffic_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    import hashlib
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "k_x_mid.md"
    prof.write_text(f"# k_x\n\ntraffic_bytes_per_unit: 66.0 candidate kernel.cu {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._ncu_traffic_per_unit("k_x") == 66.0
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench._ncu_traffic_per_unit("k_x") is None
    assert bench._ncu_traffic_per_unit("k_missing") is None
