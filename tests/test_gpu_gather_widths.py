"""FP32 candidate distances at every row width the gathers handle: d = 4, 36,
60, 100, 128 (one to four 4-coordinate slices per lane of the eight-lanes-per-
row gather, with idle lanes where d is not a multiple of 32) and d = 132, 200
(the general gather). The returned distances must be the FP64 distances of
the returned ids within 1e-5, and the gather grouped by point-id range must
give the walk-order gather's results bit for bit."""

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from parity_helpers import DEV
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("d", [4, 36, 60, 100, 128, 132, 200])
def test_gather_widths(d):
    n, nq, k, beta = 20_000, 40, 20, 0.5
    X, Q = make_workload("precision", n=n, nq=nq, d=d)
    idx = pkg.detlsh_build(X.to(DEV), gaussian_projection(4, 16, d).to(DEV), sample_ids(n, n // 10).to(DEV), 16, 4,
                           256, 128)
    Qd = Q.to(DEV)
    runs = {}
    for name, t in (("walk", {"id_bucket_log2": -1}), ("auto", {}), ("ranges", {"id_bucket_log2": 10})):
        runs[name] = pkg.detlsh_query(idx, Qd, k, 1.5, 0.0, k_max=k, beta=beta, tuning=t)
    for name in ("auto", "ranges"):
        for a, b in zip(runs["walk"][:3], runs[name][:3]):
            assert torch.equal(a, b), (d, name)
    ids, dist, st = (x.cpu().numpy() for x in runs["walk"][:3])
    assert (st[:, 3] == 0).all() and (ids >= 0).all()
    X64, Q64 = X.numpy().astype(np.float64), Q.numpy().astype(np.float64)
    for qi in range(nq):
        true = np.sqrt(((X64[ids[qi]] - Q64[qi]) ** 2).sum(axis=1))
        assert np.allclose(dist[qi], true, rtol=1e-5, atol=1e-6), (d, qi)
        assert (np.diff(dist[qi]) >= 0).all()
    idx.free()
