"""The per-candidate distance gather takes a batch's candidates grouped by
point-id range (all queries' candidates among ids [0, 2^x) first, then the
next range, ...), so that the rows read at the same time stay in L2. Each
distance is the same computation and goes to its list position, so the
results equal the walk-order gather's bit for bit, for the FP32, uint8 and
BF16-shortlist gathers, one range or many, in one batch or several."""

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


CASES = [
    # name, n, d, nq, k, beta, max_leaf, proj_mode, shortlist
    ("mid", 40_000, 128, 40, 50, 0.1, 256, 0, 0),       # FP32 gather
    ("batching", 60_000, 96, 30, 100, 0.05, 1_024, 0, 0),
    ("serving", 60_000, 128, 30, 10, 0.05, 1_024, 0, 0),  # uint8 (integer dot products)
    ("mid", 40_000, 128, 24, 20, 0.1, 256, 1, 256),      # BF16 coarse gather of the shortlist mode
]


@pytest.mark.parametrize("name,n,d,nq,k,beta,max_leaf,proj_mode,shortlist", CASES)
def test_gather_by_id_range_equals_walk_order(name, n, d, nq, k, beta, max_leaf, proj_mode, shortlist):
    X, Q = make_workload(name, n=n, nq=nq, d=d)
    idx = pkg.detlsh_build(X.to(DEV), gaussian_projection(4, 16, d).to(DEV), sample_ids(n, n // 10).to(DEV), 16, 4,
                           256, max_leaf, proj_mode=proj_mode)
    g = torch.Generator().manual_seed(nq + d)
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32).to(DEV)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)].to(DEV)
    rm = torch.zeros(nq, device=DEV)
    Qd = Q.to(DEV)

    def run(**tuning):
        tuning.setdefault("coarse_gather", 1)
        return pkg.detlsh_query(idx, Qd, ks, cs, rm, k_max=k, beta=beta, shortlist=shortlist, tuning=tuning)

    walk = run(id_bucket_log2=-1)
    for t in ({}, {"id_bucket_log2": 10}, {"id_bucket_log2": 12, "batch": 7}, {"id_bucket_log2": 31}):
        got = run(**t)
        for a, b in zip(walk[:3], got[:3]):
            assert torch.equal(a, b), t
    assert (walk[2][:, 3] == 0).all()
    idx.free()


def test_bad_range_size_is_refused():
    X, Q = make_workload("tiny", n=2_000, nq=2, d=32)
    idx = pkg.detlsh_build(X.to(DEV), gaussian_projection(4, 16, 32).to(DEV), sample_ids(2_000, 200).to(DEV), 16, 4,
                           16, 256)
    for bad in (5, -2, 32):
        with pytest.raises(pkg.DetlshError):
            pkg.detlsh_query(idx, Q.to(DEV), 5, 1.5, 0.0, k_max=5, tuning={"id_bucket_log2": bad})
    idx.free()
