"""GPU tests of the continuous-batching server.

A query's result must not depend on the batch it runs in: the same query
submitted alone and among many others gives the same bits, equal to
detlsh_query's (itself checked against the oracle) and, on exact inputs, to
the oracle's. Admission, failure reporting and shutdown are exercised on
the host side (a failed batch is injected by the server's test hook, not by
a GPU fault).
"""

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EINVAL, ECUDA, EADMIT, PENDING = -1, -3, -5, 1
K, L, NR, MAX_LEAF, BETA = 16, 4, 16, 64, 0.05


@pytest.fixture(scope="module")
def index():
    import __graft_entry__ as g
    g.build()
    n, nq = 10_000, 400
    X, Q = make_workload("tiny", n=n, nq=nq, exact=True)
    A = gaussian_projection(L, K, 32, exact=True)
    ids = sample_ids(n, 1_000)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, NR, MAX_LEAF)
    gen = torch.Generator().manual_seed(9)
    ks = torch.tensor([1, 10, 20])[torch.randint(0, 3, (nq,), generator=gen)].to(torch.int32)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=gen)]
    want = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), 0.0, k_max=20, beta=BETA)
    yield dict(X=X, Q=Q, A=A, ids=ids, idx=idx, ks=ks, cs=cs, want=[t.cpu() for t in want[:3]])
    idx.free()


def _collect(srv, tickets):
    res = []
    for t in tickets:
        st, ids, dist, stats, lat = srv.poll(t, wait_us=5_000_000)
        assert st == 0, st
        assert lat is not None and lat >= 0
        res.append((ids, dist, stats))
    return res


def test_alone_equals_mixed_equals_direct_and_oracle(index):
    Q, ks, cs, want = index["Q"], index["ks"], index["cs"], index["want"]
    srv = pkg.Server(index["idx"], k_max=20, slots=64, pipelines=2, beta=BETA)
    q0 = 123
    alone = _collect(srv, [srv.submit(Q[q0], int(ks[q0]), float(cs[q0]))])[0]
    tickets = [srv.submit(Q[i], int(ks[i]), float(cs[i])) for i in range(Q.shape[0])]
    mixed = _collect(srv, tickets)
    for a, b in zip(alone, mixed[q0]):
        assert torch.equal(a, b)
    for i, (ids, dist, stats) in enumerate(mixed):
        assert torch.equal(ids, want[0][i]) and torch.equal(dist, want[1][i]) and torch.equal(stats, want[2][i]), i
    st = srv.stats()
    assert st["submitted"] == st["completed"] == Q.shape[0] + 1
    assert st["batches"] >= (Q.shape[0] + 63) // 64 and st["max_batch"] <= 64 and st["errors"] == 0
    srv.destroy()
    # the oracle on a few of them (exact inputs: bit-equal)
    ref = O.build_index(index["X"].numpy(), index["A"].numpy(), index["ids"].numpy(), K, L, NR, MAX_LEAF)
    eps = O.eps_from_lemma3(K, L)
    for i in (0, q0, 399):
        r = O.c2k_ann(ref, Q.numpy()[i], int(ks[i]), float(cs[i]), 0.0, eps, BETA, keep_candidates=False)
        kq = int(ks[i])
        assert np.array_equal(mixed[i][0][:kq].numpy(), r.ids[:kq])
        assert np.array_equal(mixed[i][1][:kq].numpy(), np.float32(r.dist[:kq]))


def test_replay_poisson_arrivals(index):
    Q, ks, cs, want = index["Q"], index["ks"], index["cs"], index["want"]
    srv = pkg.Server(index["idx"], k_max=20, slots=32, pipelines=2, max_delay_us=100, beta=BETA)
    gen = torch.Generator().manual_seed(4)
    rate = 20_000.0   # queries per second
    arrival = torch.cumsum(torch.empty(Q.shape[0], dtype=torch.float64).exponential_(rate / 1e6, generator=gen), 0)
    st, ids, dist, stats, lat = srv.replay(Q, ks, cs, 0.0, arrival)
    assert st == 0
    assert torch.equal(ids, want[0]) and torch.equal(dist, want[1]) and torch.equal(stats, want[2])
    assert (lat >= 0).all()
    s = srv.stats()
    assert s["completed"] == Q.shape[0] and s["errors"] == 0
    srv.destroy()


def test_admission_by_slots(index):
    Q, ks, cs = index["Q"], index["ks"], index["cs"]
    srv = pkg.Server(index["idx"], k_max=20, slots=4, pipelines=1, queue_cap=6, beta=BETA)
    tickets = [srv.submit(Q[i], int(ks[i]), float(cs[i])) for i in range(6)]
    with pytest.raises(pkg.DetlshError) as e:
        srv.submit(Q[6], int(ks[6]), float(cs[6]))
    assert e.value.status == EADMIT
    assert srv.stats()["rejected"] == 1
    _collect(srv, tickets[:1])
    t = srv.submit(Q[6], int(ks[6]), float(cs[6]))      # a slot is free again
    _collect(srv, tickets[1:] + [t])
    srv.destroy()


def test_memory_budget_admission(index):
    with pytest.raises(pkg.DetlshError) as e:
        pkg.Server(index["idx"], k_max=20, slots=4096, pipelines=2, mem_budget=1 << 20, beta=BETA)
    assert e.value.status == EADMIT
    srv = pkg.Server(index["idx"], k_max=20, pipelines=2, mem_budget=256 << 20, beta=BETA)
    slots = srv.stats()["slots"]
    assert 1 <= slots <= 4096 and slots & (slots - 1) == 0
    srv.destroy()


def test_failed_batch_is_reported_and_service_continues(index):
    Q, ks, cs, want = index["Q"], index["ks"], index["cs"], index["want"]
    srv = pkg.Server(index["idx"], k_max=20, slots=8, pipelines=1, beta=BETA, test_fail_batch=2)
    results = []
    for i in range(4):   # one request per batch: the second batch fails
        t = srv.submit(Q[i], int(ks[i]), float(cs[i]))
        results.append(srv.poll(t, wait_us=5_000_000))
    assert [r[0] for r in results] == [0, ECUDA, 0, 0]
    for i in (0, 2, 3):
        assert torch.equal(results[i][1], want[0][i])
    assert srv.stats()["errors"] == 1
    srv.destroy()


def test_bad_arguments_and_tickets(index):
    Q = index["Q"]
    srv = pkg.Server(index["idx"], k_max=20, slots=8, pipelines=1, beta=BETA)
    for k, c, r in ((0, 1.5, 0.0), (21, 1.5, 0.0), (5, 1.0, 0.0), (5, float("nan"), 0.0), (5, 1.5, float("inf"))):
        with pytest.raises(pkg.DetlshError) as e:
            srv.submit(Q[0], k, c, r)
        assert e.value.status == EINVAL
    t = srv.submit(Q[0], 5, 1.5)
    assert srv.poll(t, wait_us=5_000_000)[0] == 0
    assert srv.poll(t)[0] == EINVAL          # collected already
    assert srv.poll(12345)[0] == EINVAL
    srv.destroy()


def test_destroy_with_queued_requests(index):
    Q, ks, cs = index["Q"], index["ks"], index["cs"]
    srv = pkg.Server(index["idx"], k_max=20, slots=16, pipelines=2, beta=BETA)
    for i in range(100):                      # within the default pool of 4 * 16 * 2 slots
        srv.submit(Q[i], int(ks[i]), float(cs[i]))
    srv.destroy()                             # runs what is queued, then stops
