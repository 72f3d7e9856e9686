"""The checked build (compiled with DETLSH_CHECKED): the query kernels check
their data-dependent indices on the device — leaf numbers and id-array entries
in the walk, dedup bitmap words, candidate ids and list positions in the
distance gathers, id ranges and pair places in the grouping, block and list
places in the round expansion, list lengths in the final top-k, point ids in
the leaf-major producer — and record any failure instead of making the
access. The GPU parity suites run here under that build in a child process;
an autouse fixture fails every test after which a check had failed."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_mirror.py", "tests/test_gpu_bf16.py",
          "tests/test_gpu_id_ranges.py", "tests/test_gpu_plan.py"]


def test_checked_build_reports_itself():
    env = dict(os.environ, DETLSH_CHECKED="1")
    code = ("import paper_2406_10938_gb300 as pkg; import torch; torch.zeros(1, device='cuda:0'); "
            "st = pkg.detlsh_check_status(); assert st == (0, 0, 0), st; print('checked')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked" in r.stdout, r.stdout + r.stderr


def test_parity_suites_pass_with_device_index_checks():
    env = dict(os.environ, DETLSH_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
