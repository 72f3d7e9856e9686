"""GPU parity of query plans (preallocated batches, CUDA-graph replay), of the
launch-shape tuning and of the autotuner.

The launch shapes and the route (direct launches or one graph launch per
batch) must not change any result: on exact-arithmetic inputs every plan
result equals the oracle's bit for bit, for batch sizes that span several
chunks and a ragged last chunk, and every tuning gives the default's results.
"""

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O
from parity_helpers import DEV, gpu_build, oracle_queries
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu
EINVAL = -1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _case(name="tiny", n=10_000, d=32, K=16, L=4, Nr=16, n_s=1_000, max_leaf=64, nq=150, k=10, seed=7,
          proj_mode=0):
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    g = torch.Generator().manual_seed(seed)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    ks[0] = k
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=proj_mode)
    return X, Q, A, ids, ks, cs, idx


def _same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x.cpu(), y.cpu())


@pytest.mark.parametrize("graph", [True, False])
def test_plan_matches_oracle_bit_exact(graph):
    K, L, Nr, max_leaf, beta = 16, 4, 16, 64, 0.05
    X, Q, A, ids, ks, cs, idx = _case(nq=150, max_leaf=max_leaf)
    eps = O.eps_from_lemma3(K, L)
    plan = pkg.Plan(idx, nq_max=64, k_max=10, eps=eps, beta=beta, graph=graph)
    info = plan.info()
    assert info["batch"] == 64
    got = pkg.detlsh_plan_query(plan, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0)
    assert pkg.detlsh_plan_status(plan) == 0
    info = plan.info()
    assert info["batches"] == 3                       # 64 + 64 + 22 queries
    assert info["graph_launches"] == (3 if graph else 0)
    if graph:
        assert info["graph_kernels"] >= 8
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    res = oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), np.zeros(150), eps, beta, keep=False)
    out_ids, out_dist, stats = (t.cpu().numpy() for t in got)
    for qi, r in enumerate(res):
        kq = int(ks[qi])
        assert (stats[qi, 0], stats[qi, 1], stats[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        assert np.array_equal(out_ids[qi, :kq], r.ids[:kq]), qi
        assert (out_ids[qi, kq:] == -1).all()
        assert np.array_equal(out_dist[qi, :kq], np.float32(r.dist[:kq])), qi
    # the direct query gives the same bits
    _same(got, pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=10, eps=eps, beta=beta)[:3])
    plan.destroy()
    idx.free()


def test_graph_replay_any_batch_size():
    """One captured graph serves batches of 1, 37 and 64 queries, host and device memory."""
    beta = 0.1
    X, Q, A, ids, ks, cs, idx = _case(nq=64, seed=11)
    plan = pkg.Plan(idx, nq_max=64, k_max=10, beta=beta, graph=True)
    for m in (1, 37, 64, 5):
        want = pkg.detlsh_query(idx, Q[:m].to(DEV), ks[:m].to(DEV), cs[:m].to(DEV), 0.0, k_max=10, beta=beta)[:3]
        got = pkg.detlsh_plan_query(plan, Q[:m].to(DEV), ks[:m].to(DEV), cs[:m].to(DEV), 0.0)
        assert pkg.detlsh_plan_status(plan) == 0
        _same(got, want)
        got_h = pkg.detlsh_plan_query(plan, Q[:m], ks[:m], cs[:m], 0.0)
        _same(got_h, want)
    assert plan.info()["graph_launches"] == 8
    plan.destroy()
    idx.free()


def test_plan_flags_bad_device_argument_and_recovers():
    X, Q, A, ids, ks, cs, idx = _case(nq=20, seed=3)
    plan = pkg.Plan(idx, nq_max=32, k_max=10, graph=True)
    bad = ks.clone()
    bad[7] = 11                                       # k > k_max
    pkg.detlsh_plan_query(plan, Q.to(DEV), bad.to(DEV), cs.to(DEV), 0.0)
    assert pkg.detlsh_plan_status(plan) == EINVAL
    assert pkg.detlsh_plan_status(plan) == 0           # the flag is cleared by reading it
    got = pkg.detlsh_plan_query(plan, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0)
    assert pkg.detlsh_plan_status(plan) == 0
    _same(got, pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=10)[:3])
    with pytest.raises(pkg.DetlshError):               # host arguments are checked on the host
        pkg.detlsh_plan_query(plan, Q, bad, cs, 0.0)
    plan.destroy()
    idx.free()


@pytest.mark.parametrize("tuning", [
    {"walk_ctas_per_sm": 1},
    {"dist_rows": 64, "dist_ctas_per_sm": 1},
    {"dist_rows": 1024, "dist_ctas_per_sm": 2},
    {"batch": 7, "walk_ctas_per_sm": 2, "dist_rows": 128},
    {"batch": 9, "streams": 2},
    {"batch": 9, "streams": 1, "dist_ctas_per_sm": 3},
    {"dist_ctas_per_sm": 4, "id_bucket_log2": 12},
])
def test_tuning_does_not_change_results(tuning):
    X, Q, A, ids, ks, cs, idx = _case("mid", n=20_000, d=128, Nr=256, n_s=2_000, max_leaf=64, nq=40, k=50)
    base = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, cand_cap=20_000)
    got = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, cand_cap=20_000,
                           tuning=tuning)
    _same(got[:3], base[:3])
    for qi in range(40):
        m = int(base[2][qi, 0])
        assert torch.equal(torch.sort(got[3][qi, :m].cpu())[0], torch.sort(base[3][qi, :m].cpu())[0])
    idx.free()


def test_tuning_rejects_bad_shapes():
    X, Q, A, ids, ks, cs, idx = _case(nq=4)
    for bad in ({"dist_rows": 100}, {"dist_ctas_per_sm": 5}, {"walk_ctas_per_sm": 9}, {"batch": -1},
                {"streams": 3}):
        with pytest.raises(pkg.DetlshError):
            pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=10, tuning=bad)
    idx.free()


def test_autotune_fp32_index():
    X, Q, A, ids, ks, cs, idx = _case("mid", n=20_000, d=128, Nr=256, n_s=2_000, max_leaf=64, nq=300, k=50)
    t = pkg.detlsh_autotune(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, min_agreement=0.99)
    assert t["walk_ctas_per_sm"] in (0, 1, 2, 3, 4)
    assert t["dist_rows"] % 64 == 0 and 64 <= t["dist_rows"] <= 8192
    assert t["dist_ctas_per_sm"] in (0, 1, 2, 3, 4)
    assert t["streams"] in (0, 1, 2)
    assert t["batch"] in (0, 1024, 2048, 4096, 8192, 16384)
    assert t["shortlist"] == 0                         # no BF16 copy to re-rank from
    base = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1)
    _same(pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, tuning=t)[:3], base[:3])
    idx.free()


def test_autotune_bf16_shortlist_and_plan():
    """The picked shortlist agrees with the exact top-k on the sample, and a
    BF16 plan with it gives detlsh_query's results."""
    X, Q = make_workload("mid", n=20_000, nq=200, d=128)
    A = gaussian_projection(4, 16, 128)
    ids = sample_ids(20_000, 2_000)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), 16, 4, 256, 64, proj_mode=1)
    ks = torch.full((200,), 50, dtype=torch.int32)
    cs = torch.full((200,), 1.5)
    t = pkg.detlsh_autotune(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, min_agreement=0.99)
    assert t["shortlist"] in (0, 64, 128, 256, 512, 1024, 2048, 4096)
    sl = t["shortlist"] or 256
    exact = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1)[0].cpu()
    got = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=50, beta=0.1, shortlist=sl,
                           tuning=t)
    agree = np.mean([len(set(exact[i].tolist()) & set(got[0][i].cpu().tolist())) / 50 for i in range(200)])
    if t["shortlist"]:
        assert agree >= 0.99
    plan = pkg.Plan(idx, nq_max=128, k_max=50, beta=0.1, shortlist=sl, tuning=t, graph=True)
    _same(pkg.detlsh_plan_query(plan, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0), got[:3])
    assert pkg.detlsh_plan_status(plan) == 0
    plan.destroy()
    idx.free()
