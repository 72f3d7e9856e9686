"""Parity at the full size of the mid workload (n = 1,000,000, d = 128, 10,000
queries, K = 16, L = 4, N_r = 256, n_s = 10,000, max_leaf = 256, c = 1.5,
k = 50, beta = 0.1), in the launch configuration the benchmark times.

The inputs are the exact-arithmetic variant of the workload (integer points,
projection vectors on a 1/16 grid), so every FP32 and BF16 sum on the GPU is
exact and the GPU must equal the FP64 oracle bit for bit: the whole index
(breakpoints, codes, leaf tables), and every output of sampled queries spread
over the query batches. The queries run as one 10,000-query call, the way the
benchmark issues them; the oracle answers only the sampled ones.
"""

import math

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O
from parity_helpers import DEV, assert_trees_equal, gpu_codes, gpu_trees
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu

N, D, NQ, K, L, NR, NS, MAX_LEAF, C, KK, BETA = 1_000_000, 128, 10_000, 16, 4, 256, 10_000, 256, 1.5, 50, 0.1
SAMPLED = (0, 1, 3333, 3334, 5000, 9999)


@pytest.fixture(scope="module")
def full():
    import __graft_entry__ as g
    g.build()
    X, Q = make_workload("mid", n=N, nq=NQ, exact=True)
    A = gaussian_projection(L, K, D, exact=True)
    ids = sample_ids(N, NS)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, NR, MAX_LEAF)
    return X, Q, A, ids, ref


def _check_index(idx, ref):
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, NR + 1).astype(np.float64)
    assert np.array_equal(E, ref.E)
    assert np.array_equal(gpu_codes(idx, N, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, N), ref.trees)


def _check_queries(out, Q, ref, eps, sampled=SAMPLED):
    ids, dist, stats = (t.cpu().numpy() for t in out[:3])
    for qi in sampled:
        r = O.c2k_ann(ref, Q.numpy()[qi], KK, C, 0.0, eps, BETA, keep_candidates=False)
        assert (stats[qi, 0], stats[qi, 1], stats[qi, 2], stats[qi, 3]) == (r.n_cand, r.rounds, r.stop, 0), qi
        assert np.array_equal(ids[qi], r.ids[:KK]), qi
        assert np.array_equal(dist[qi], np.float32(r.dist[:KK])), qi
    # properties of every query: k distinct ids sorted by (distance, id)
    assert (ids >= 0).all() and (ids < N).all()
    assert (np.diff(dist, axis=1) >= 0).all()
    assert all(len(set(row.tolist())) == KK for row in ids[:: max(1, NQ // 500)])


@pytest.mark.parametrize("proj_mode", [0, 1])
def test_mid_full_size_bit_parity(full, proj_mode):
    X, Q, A, ids, ref = full
    Xd, Qd = X.to(DEV), Q.to(DEV)
    idx = pkg.detlsh_build(Xd, A.to(DEV), ids.to(DEV), K, L, NR, MAX_LEAF, borrow=True, proj_mode=proj_mode)
    _check_index(idx, ref)
    eps = O.eps_from_lemma3(K, L)
    kk = torch.full((NQ,), KK, dtype=torch.int32, device=DEV)
    cc = torch.full((NQ,), C, dtype=torch.float32, device=DEV)
    rr = torch.zeros(NQ, dtype=torch.float32, device=DEV)
    out = pkg.detlsh_query(idx, Qd, kk, cc, rr, k_max=KK, eps=eps, beta=BETA)
    _check_queries(out, Q, ref, eps)
    if proj_mode == 1:
        # BF16 coarse distances are exact on these inputs: the shortlist path
        # gives the same bits
        out_sl = pkg.detlsh_query(idx, Qd, kk, cc, rr, k_max=KK, eps=eps, beta=BETA, shortlist=512)
        for a, b in zip(out_sl[:3], out[:3]):
            assert torch.equal(a, b)
    # a graph-captured plan of the sampled queries gives the same bits
    plan = pkg.Plan(idx, nq_max=4096, k_max=KK, eps=eps, beta=BETA, graph=True)
    sel = torch.tensor(SAMPLED, device=DEV)
    got = pkg.detlsh_plan_query(plan, Qd[sel], kk[sel], cc[sel], rr[sel])
    assert pkg.detlsh_plan_status(plan) == 0
    for a, b in zip(got, out[:3]):
        assert torch.equal(a, b[sel])
    plan.destroy()
    idx.free()


MIRROR_SAMPLED = (0, 1, 777, 2048, 3333, 3334, 4999, 5000, 6666, 8191, 8192, 9998, 9999)


def test_mid_full_size_fp32_mirror_candidate_sets():
    """The benchmark's own inputs (FP32 points with integer values, N(0,1)
    hash vectors, the benchmark's sample) and launch configuration (one
    10,000-query call): the oracle's FP32-mirror form, given the GPU's
    projected queries, breakpoints and codes, builds the same leaves and gives
    the same candidate sets, rounds, stop rules, ids and distances for sampled
    queries spread over the batches. The squared distances of these integer
    points (below 2^24) are exact in FP32, so the distance test decides as in
    FP64 and there is no tie band."""
    from parity_helpers import check_topk_up_to_ties, mirror_index
    X, Q = make_workload("mid", n=N, nq=NQ)
    A = gaussian_projection(L, K, D)
    ids = sample_ids(N, NS)
    Xd, Qd = X.to(DEV), Q.to(DEV)
    idx = pkg.detlsh_build(Xd, A.to(DEV), ids.to(DEV), K, L, NR, MAX_LEAF, borrow=True)
    ref = mirror_index(idx, X.numpy(), A.numpy(), K, L, NR, MAX_LEAF)
    eps = O.eps_from_lemma3(K, L)
    kk = torch.full((NQ,), KK, dtype=torch.int32, device=DEV)
    cc = torch.full((NQ,), C, dtype=torch.float32, device=DEV)
    rr = torch.zeros(NQ, dtype=torch.float32, device=DEV)
    qproj = torch.empty(NQ, L * K, dtype=torch.float32, device=DEV)
    cap = int(math.ceil(BETA * N + KK)) - 1 + idx.info()["largest_leaf"]
    out = pkg.detlsh_query(idx, Qd, kk, cc, rr, k_max=KK, eps=eps, beta=BETA, cand_cap=cap, qproj=qproj)
    sel = torch.tensor(MIRROR_SAMPLED, device=DEV)
    ids_o, dist_o, stats_o = (t[sel].cpu().numpy() for t in out[:3])
    cand = out[3][sel].cpu().numpy().view(np.uint32)
    qp = qproj[sel].cpu().numpy()
    X64 = X.numpy().astype(np.float64)
    for j, qi in enumerate(MIRROR_SAMPLED):
        q64 = Q.numpy()[qi].astype(np.float64)
        r = O.c2k_ann(ref, q64, KK, C, 0.0, eps, BETA, keep_candidates=True, qp32=qp[j])
        assert (stats_o[j, 0], stats_o[j, 1], stats_o[j, 2], stats_o[j, 3]) == (r.n_cand, r.rounds, r.stop, 0), qi
        assert np.array_equal(np.sort(cand[j, : stats_o[j, 0]].astype(np.int64)), r.cand), qi
        assert np.array_equal(ids_o[j], r.ids[:KK]), qi
        assert np.array_equal(dist_o[j], np.float32(r.dist[:KK])), qi
        check_topk_up_to_ties(ids_o[j], dist_o[j], r, X64, q64, KK, 1e-5)
    idx.free()
