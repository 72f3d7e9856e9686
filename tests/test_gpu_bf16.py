"""GPU parity of the BF16 tensor-core projection mode (tcgen05, FP32 accumulation).

Its codes are exact for their BF16 inputs: on exact-arithmetic inputs (values
that BF16 represents exactly, with every FP32 partial sum exact) the whole
index and every query result must equal the oracle bit for bit; on general
FP32 inputs the projections must equal the FP64 projection of the
BF16-rounded inputs to FP32 accumulation accuracy.
"""

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O
from parity_helpers import (DEV, assert_trees_equal, gpu_codes, gpu_trees, oracle_queries,
                            proj_tolerance)
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu
BF16 = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float32)


@pytest.mark.parametrize("case", [
    # name, n, d, K, L, Nr, n_s, max_leaf
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256),
    ("tiny", 3_001, 32, 8, 2, 8, 333, 7),
    ("mid", 20_000, 128, 16, 4, 256, 2_000, 64),
    ("serving", 20_000, 128, 16, 4, 256, 2_000, 32),
    ("precision", 4_000, 960, 16, 4, 256, 400, 64),
    ("batching", 30_000, 96, 16, 4, 256, 3_000, 64),
])
def test_bf16_build_exact_bit_parity(case):
    name, n, d, K, L, Nr, n_s, max_leaf = case
    X, _ = make_workload(name, n=n, nq=1, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=BF16)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    Ps = pkg.detlsh_export(idx, "SAMPLE_PROJ").numpy().reshape(L * K, n_s).astype(np.float64)
    assert np.array_equal(Ps.T, ref.P[ids.numpy()])
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, Nr + 1).astype(np.float64)
    assert np.array_equal(E, ref.E)
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    idx.free()


@pytest.mark.parametrize("case", [
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256, 60, 10, 0.1),
    ("mid", 20_000, 128, 16, 4, 256, 2_000, 64, 20, 50, 0.1),
    ("precision", 6_000, 960, 16, 4, 256, 600, 64, 12, 100, 0.1),
    ("batching", 30_000, 96, 16, 4, 256, 3_000, 256, 16, 100, 0.01),
])
def test_bf16_query_exact_bit_parity(case):
    name, n, d, K, L, Nr, n_s, max_leaf, nq, k, beta = case
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    eps = O.eps_from_lemma3(K, L)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=BF16)
    ks = torch.full((nq,), k, dtype=torch.int32)
    cs = torch.full((nq,), 1.5)
    rm = torch.zeros(nq)
    oid, od, st, cand = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV), k_max=k,
                                         eps=eps, beta=beta, cand_cap=n)
    oid, od, st = oid.cpu().numpy(), od.cpu().numpy(), st.cpu().numpy()
    cand = cand.cpu().numpy().view(np.uint32)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    for qi, r in enumerate(oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), rm.numpy(), eps, beta)):
        assert (st[qi, 0], st[qi, 1], st[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        assert np.array_equal(np.sort(cand[qi, : st[qi, 0]].astype(np.int64)), r.cand), qi
        assert np.array_equal(oid[qi], r.ids), qi
        assert np.array_equal(od[qi], np.float32(r.dist)), qi
    idx.free()


@pytest.mark.parametrize("name,n,d,n_s", [("tiny", 3000, 32, 700), ("precision", 1000, 960, 300),
                                          ("batching", 5000, 96, 777)])
def test_bf16_projection_of_rounded_inputs(name, n, d, n_s):
    K, L, Nr = 16, 4, 16
    X, _ = make_workload(name, n=n, nq=1)
    A = gaussian_projection(L, K, d)
    ids = sample_ids(n, n_s)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, 64, proj_mode=BF16)
    Ps = pkg.detlsh_export(idx, "SAMPLE_PROJ").numpy().reshape(L * K, n_s).T.astype(np.float64)
    Xr, Ar = _bf16(X).numpy(), _bf16(A).numpy()
    ref = O.project(Ar, Xr[ids.numpy()])
    tol = proj_tolerance(Ar, Xr[ids.numpy()])
    assert (np.abs(Ps - ref) <= tol).all()
    idx.free()


@pytest.mark.parametrize("name,n,d,n_s,nq,k,shortlist", [("mid", 20_000, 128, 2_000, 20, 50, 512),
                                                         ("precision", 6_000, 960, 600, 12, 100, 4096)])
def test_shortlist_exact_inputs_match_the_oracle(name, n, d, n_s, nq, k, shortlist):
    """Values BF16 holds exactly (integer data; the 1/8 grid of the precision
    shape) make the coarse distances the exact ones, so the shortlist path
    must return the oracle's results."""
    K, L, Nr, max_leaf = 16, 4, 256, 64
    X, Q = make_workload(name, n=n, nq=nq, exact=True)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    eps = O.eps_from_lemma3(K, L)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=BF16)
    oid, od, st, _ = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, eps=eps, beta=0.1, shortlist=shortlist)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    oid, od, st = oid.cpu().numpy(), od.cpu().numpy(), st.cpu().numpy()
    for qi in range(nq):
        r = O.c2k_ann(ref, Q[qi].numpy(), k, 1.5, 0.0, eps, 0.1)
        assert (st[qi, 0], st[qi, 1], st[qi, 2]) == (r.n_cand, r.rounds, r.stop)
        assert np.array_equal(oid[qi], r.ids)
        assert np.array_equal(od[qi], np.float32(r.dist))
    idx.free()


def test_shortlist_float_inputs_recall_and_exact_distances():
    """FP32 data: the shortlist's distances are recomputed in FP32 (1e-5 of the
    FP64 value) and recall stays close to the plain FP32 path's."""
    n, d, K, L, Nr, n_s, nq, k = 8_000, 960, 16, 4, 64, 800, 16, 20
    X, Q = make_workload("precision", n=n, nq=nq)
    A = gaussian_projection(L, K, d)
    ids = sample_ids(n, n_s)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, 256, proj_mode=BF16)
    o1, d1, _, _ = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, beta=0.1)
    o2, d2, _, _ = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, beta=0.1, shortlist=1024)
    Xn, Qn = X.numpy().astype(np.float64), Q.numpy().astype(np.float64)
    o1, o2, d2 = o1.cpu().numpy(), o2.cpu().numpy(), d2.cpu().numpy()
    r1, r2 = [], []
    for qi in range(nq):
        e, _ = O.exact_knn(Xn, Qn[qi], k)
        r1.append(O.recall(o1[qi], e))
        r2.append(O.recall(o2[qi], e))
        true = np.sqrt(((Xn[o2[qi]] - Qn[qi]) ** 2).sum(axis=1))
        assert np.allclose(d2[qi], true, rtol=1e-5, atol=1e-6)
    assert np.mean(r2) >= np.mean(r1) - 0.02, (np.mean(r1), np.mean(r2))
    idx.free()


@pytest.mark.parametrize("name,n,d,K,L,Nr,n_s,max_leaf,nq,k,beta", [
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256, 40, 10, 0.1),       # d below one 64-coordinate stage
    ("batching", 30_000, 96, 16, 4, 256, 3_000, 256, 16, 100, 0.01),  # a partial second stage
    ("mid", 20_000, 128, 16, 4, 256, 2_000, 64, 20, 50, 0.1),
    ("tiny", 10_000, 32, 4, 4, 16, 1_000, 2_048, 12, 20, 0.5),      # leaves of several 224-point chunks
    ("precision", 6_000, 960, 16, 4, 256, 600, 64, 8, 100, 0.1),     # fifteen stages
])
def test_coarse_by_leaf_on_exact_inputs(name, n, d, K, L, Nr, n_s, max_leaf, nq, k, beta):
    """The shortlist mode's coarse distances by leaf on the tensor cores
    (||q||^2 + ||o||^2 - 2 q.o, BF16 operands, FP32 accumulation) are exact
    when BF16 holds the values and every sum is exact: the results equal the
    per-candidate gather's and the oracle's bit for bit, and the candidate
    sets are the oracle's."""
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    eps = O.eps_from_lemma3(K, L)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=BF16)
    g = torch.Generator().manual_seed(nq + d)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    rm = torch.zeros(nq)
    sl = min(4096, max(k, 256))
    outs = []
    for gather in (0, 1):
        outs.append(pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV), k_max=k, eps=eps,
                                     beta=beta, shortlist=sl, cand_cap=n, tuning={"coarse_gather": gather}))
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
    oid, od, st, cand = (t.cpu().numpy() for t in outs[0])
    cand = cand.view(np.uint32)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    for qi, r in enumerate(oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), rm.numpy(), eps, beta)):
        kq = int(ks[qi])
        assert (st[qi, 0], st[qi, 1], st[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        assert np.array_equal(np.sort(cand[qi, : st[qi, 0]].astype(np.int64)), r.cand), qi
        assert np.array_equal(oid[qi, :kq], r.ids[:kq]), qi
        assert np.array_equal(od[qi, :kq], np.float32(r.dist[:kq])), qi
    if name == "tiny" and K == 4:
        assert idx.info()["largest_leaf"] > 448     # some leaf spans three chunks
    idx.free()


def test_coarse_by_leaf_float_inputs_agree_with_the_gather():
    """FP32 inputs: the two coarse formulations round differently, so their
    shortlists may differ at the margin; the returned distances are exact FP32
    re-ranks either way and the top-k ids agree for nearly every query."""
    n, d, K, L, Nr, n_s, nq, k = 20_000, 128, 16, 4, 256, 2_000, 64, 20
    X, Q = make_workload("precision", n=n, nq=nq, d=d)
    A = gaussian_projection(L, K, d)
    ids = sample_ids(n, n_s)
    idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, 128, proj_mode=BF16)
    a = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, beta=0.1, shortlist=256)
    b = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, beta=0.1, shortlist=256,
                         tuning={"coarse_gather": 1})
    ia, ib = a[0].cpu().numpy(), b[0].cpu().numpy()
    agree = np.mean([len(set(ia[i]) & set(ib[i])) / k for i in range(nq)])
    assert agree >= 0.99, agree
    Xn, Qn = X.numpy().astype(np.float64), Q.numpy().astype(np.float64)
    da = a[1].cpu().numpy()
    for qi in range(nq):
        true = np.sqrt(((Xn[ia[qi]] - Qn[qi]) ** 2).sum(axis=1))
        assert np.allclose(da[qi], true, rtol=1e-5, atol=1e-6)
    idx.free()
