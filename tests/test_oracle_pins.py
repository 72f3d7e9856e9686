"""Pins for the CPU oracle: each test checks it against something the paper or
the mathematics fixes independently of the oracle's own code (closed forms,
hand-worked examples, order-statistic counts, brute force, distribution laws).
"""

import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import detlsh_oracle as O
from workloads import gaussian_projection, make_workload, paa_projection, sample_ids

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ Lemma 3 / Eq. 2
def _chi2_sf_even(x, K):
    """Survival function of chi2 with even K in closed form (Poisson sum)."""
    m = K // 2
    h = x / 2.0
    term, tot = 1.0, 1.0
    for i in range(1, m):
        term *= h / i
        tot += term
    return math.exp(-h) * tot


def _bisect(f, lo, hi, it=200):
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("K,L", [(16, 4), (16, 1), (16, 8), (8, 4), (32, 2)])
def test_eps_matches_closed_form(K, L):
    alpha1 = math.exp(-1.0 / L)
    eps2 = _bisect(lambda x: _chi2_sf_even(x, K) - alpha1, 0.0, 400.0)
    assert abs(O.eps_from_lemma3(K, L) ** 2 - eps2) < 1e-9 * eps2


@pytest.mark.parametrize("L,c,beta", [(4, 1.2, 0.3734), (4, 1.5, 0.0380), (4, 2.0, 0.0010),
                                      (1, 1.5, 0.0843), (2, 1.5, 0.0553), (8, 1.5, 0.0275)])
def test_beta_matches_closed_form(L, c, beta):
    K = 16
    alpha1 = math.exp(-1.0 / L)
    eps2 = _bisect(lambda x: _chi2_sf_even(x, K) - alpha1, 0.0, 400.0)
    alpha2 = _chi2_sf_even(eps2 / (c * c), K)
    b = 2.0 - 2.0 * alpha2 ** L
    assert abs(O.beta_from_lemma3(K, L, c) - b) < 1e-9
    assert abs(b - beta) < 6e-5


def test_eps_default_value():
    # K=16, L=4 (the paper's defaults, Sec. 5.2): eps^2 = 11.4820...
    assert abs(O.eps_from_lemma3(16, 4) - 3.388514699) < 1e-8


# ------------------------------------------------------------------ Eq. 1 projection
def test_project_permutation_special_case():
    # L=1, K=d and A a scaled permutation: h_j(o) = 2 * o[perm[j]] exactly
    rng = np.random.default_rng(0)
    d = 12
    perm = rng.permutation(d)
    A = np.zeros((d, d))
    A[np.arange(d), perm] = 2.0
    X = rng.standard_normal((50, d))
    P = O.project(A, X)
    assert np.array_equal(P, 2.0 * X[:, perm])


def test_project_lemma1_chi2_law():
    """Lemma 1: s'^2 / s^2 ~ chi2(K) over the draws of the hash vectors."""
    from scipy.stats import chi2, kstest
    rng = np.random.default_rng(1)
    d, K = 40, 16
    o1 = rng.standard_normal(d)
    o2 = rng.standard_normal(d) * 3.0
    s2 = float(((o1 - o2) ** 2).sum())
    ratios = []
    for seed in range(300):
        A = gaussian_projection(1, K, d, seed=seed + 100).numpy()
        P = O.project(A, np.stack([o1, o2]))
        ratios.append(float(((P[0] - P[1]) ** 2).sum()) / s2)
    ratios = np.array(ratios)
    assert kstest(ratios, chi2(K).cdf).pvalue > 0.01
    assert abs(ratios.mean() - K) < 4 * math.sqrt(2 * K / len(ratios))


# ------------------------------------------------------------------ Alg. 1 breakpoints
@pytest.mark.parametrize("n_s,Nr", [(1000, 16), (10_000, 256), (257, 256), (64, 2)])
def test_breakpoints_are_rank_m_z_order_statistics(n_s, Nr):
    rng = np.random.default_rng(2)
    Ps = rng.standard_normal((n_s, 3)) * np.array([1.0, 50.0, 1e-3])
    E = O.select_breakpoints(Ps, Nr)
    m = n_s // Nr
    for r in range(3):
        col = Ps[:, r]
        assert E[r, 0] == col.min() and E[r, Nr] == col.max()
        for z in range(1, Nr):
            # exactly m*z sampled values lie strictly below interior edge z
            assert int((col < E[r, z]).sum()) == m * z
    # the sample's own codes fill regions 0..N_r-2 with m points each (Sec. 4.1)
    codes = O.encode(Ps, E)
    for r in range(3):
        counts = np.bincount(codes[:, r], minlength=Nr)
        assert (counts[:-1] == m).all()
        assert counts[-1] == n_s - m * (Nr - 1)


# ------------------------------------------------------------------ Alg. 2 encoding
def test_encode_bruteforce_and_ties():
    rng = np.random.default_rng(4)
    Nr = 8
    E = np.sort(rng.standard_normal((2, Nr + 1)), axis=1)
    P = np.concatenate([rng.standard_normal((200, 2)) * 2,
                        E[:, 1:-1].T,                  # exactly on interior edges
                        np.array([[-1e9, 1e9]])])      # outside the sampled range
    codes = O.encode(P, E)
    for o in range(P.shape[0]):
        for r in range(2):
            # brute force: the region b with e_b <= p < e_{b+1}, e_0=-inf, e_Nr=+inf
            b = 0
            for z in range(1, Nr):
                if P[o, r] >= E[r, z]:
                    b = z
            assert codes[o, r] == b
    # on an edge the value goes up into the region that starts there
    for z in range(1, Nr):
        assert codes[200 + z - 1, 0] == z
    assert codes[-1, 0] == 0 and codes[-1, 1] == Nr - 1


def test_encode_monotone():
    rng = np.random.default_rng(5)
    Ps = rng.standard_normal((500, 1))
    E = O.select_breakpoints(Ps, 32)
    p = np.sort(rng.standard_normal(3000) * 2)[:, None]
    c = O.encode(p, E)[:, 0]
    assert (np.diff(c.astype(int)) >= 0).all()
    assert c.min() == 0 and c.max() == 31


# ------------------------------------------------------------------ Alg. 3 DE-Tree
@pytest.mark.parametrize("fixture", ["split_example.json", "split_rule_hand.json", "split_tie_hand.json"])
def test_split_examples(fixture):
    g = _load(fixture)
    tree = O.build_tree(np.array(g["codes"], dtype=np.uint8), g["n_regions"], g["max_size"])
    assert tree.n_leaves == len(g["expected_leaves"])
    for leaf, exp in enumerate(g["expected_leaves"]):
        ids = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
        assert ids.tolist() == exp["ids"]
        assert tree.plen[leaf].tolist() == exp["plen"]
        assert tree.prefix[leaf].tolist() == exp["prefix"]


def _check_tree(tree, codes, Nr, max_size):
    n, K = codes.shape
    bits = int(math.log2(Nr))
    lo, hi = tree.box(bits)
    # the leaves partition the points
    assert sorted(tree.ids.tolist()) == list(range(n))
    keys_prev = None
    for leaf in range(tree.n_leaves):
        ids = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
        assert len(ids) > 0
        assert (np.diff(ids) > 0).all()                         # ascending ids
        cl = codes[ids].astype(np.int64)
        assert ((cl >= lo[leaf]) & (cl <= hi[leaf])).all()      # points lie in the box
        if len(ids) > max_size:                                 # oversized only if unsplittable
            assert (tree.plen[leaf] == bits).all()
        assert (tree.plen[leaf] >= 1).all()
        # depth-first order: boxes visited in ascending code order, dim 0 most significant
        key = tuple((lo[leaf] >> (bits - 1)).tolist())
        if keys_prev is not None:
            assert key >= keys_prev
        keys_prev = key
    # boxes are disjoint: every point's code vector falls in exactly one box
    inside = ((codes[:, None, :].astype(np.int64) >= lo[None]) &
              (codes[:, None, :].astype(np.int64) <= hi[None])).all(axis=2)
    assert (inside.sum(axis=1) == 1).all()


@pytest.mark.parametrize("Nr,max_size,K", [(16, 8, 4), (4, 3, 3), (256, 16, 2), (2, 1, 5)])
def test_tree_invariants_random(Nr, max_size, K):
    rng = np.random.default_rng(6)
    n = 600
    # skewed codes so that many splits happen, with duplicates
    codes = np.minimum(rng.geometric(0.3, size=(n, K)) - 1, Nr - 1).astype(np.uint8)
    tree = O.build_tree(codes, Nr, max_size)
    _check_tree(tree, codes, Nr, max_size)
    # the root has 2^K first-layer nodes: no leaf mixes two MSB vectors
    bits = int(math.log2(Nr))
    for leaf in range(tree.n_leaves):
        ids = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
        msb = codes[ids] >> (bits - 1)
        assert (msb == msb[0]).all()


def test_tree_no_split_equals_root_partition():
    # with max_size >= n there are no splits: the leaves are the 2^K root children
    rng = np.random.default_rng(7)
    codes = rng.integers(0, 16, size=(300, 3)).astype(np.uint8)
    tree = O.build_tree(codes, 16, 1000)
    keys = (codes >> 3).astype(int) @ np.array([4, 2, 1])
    assert tree.n_leaves == len(np.unique(keys))
    for leaf in range(tree.n_leaves):
        ids = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
        assert len(set(keys[ids].tolist())) == 1
        assert (tree.plen[leaf] == 1).all()


# ------------------------------------------------------------------ Alg. 5 lower bound
def test_lower_bound_vs_brute_force():
    rng = np.random.default_rng(8)
    K, Nr = 3, 8
    E32 = np.sort(rng.standard_normal((K, Nr + 1)), axis=1).astype(np.float32)
    lo = rng.integers(0, Nr, size=(200, K))
    hi = np.minimum(lo + rng.integers(0, 4, size=(200, K)), Nr - 1)
    for trial in range(20):
        q = (rng.standard_normal(K) * 1.5).astype(np.float32)
        lb2 = O.leaf_lb2_fp32(q, E32, lo, hi, Nr)
        for leaf in range(0, 200, 7):
            lower = np.where(lo[leaf] == 0, -np.inf, E32[np.arange(K), lo[leaf]]).astype(np.float64)
            upper = np.where(hi[leaf] == Nr - 1, np.inf,
                             E32[np.arange(K), np.minimum(hi[leaf] + 1, Nr)]).astype(np.float64)
            # random points of the box never come closer than the bound
            pts = rng.uniform(np.maximum(lower, -5), np.minimum(upper, 5), size=(64, K))
            d2 = ((pts - q.astype(np.float64)) ** 2).sum(axis=1)
            assert lb2[leaf] <= d2.min() * (1 + 1e-6) + 1e-12
            # and the box point nearest to q attains it
            nearest = np.clip(q.astype(np.float64), lower, upper)
            d2n = ((nearest - q.astype(np.float64)) ** 2).sum()
            assert abs(float(lb2[leaf]) - d2n) <= 1e-6 * max(d2n, 1e-30) + 1e-12


def test_lower_bound_zero_inside():
    E32 = np.array([[-3, -1, 0, 1, 3]], dtype=np.float32)
    lo = np.array([[0], [1], [2], [3], [1]])
    hi = np.array([[0], [1], [2], [3], [2]])
    lb = O.leaf_lb2_fp32(np.array([0.5], np.float32), E32, lo, hi, 4)
    assert lb.tolist() == [np.float32(1.5) ** 2, np.float32(0.5) ** 2, 0.0, np.float32(0.5) ** 2, 0.0]


# ------------------------------------------------------------------ Alg. 7 query
def _hand_index(g):
    X = np.array(g["X"], dtype=np.float64)[:, None]
    A = np.array([[1.0]])
    E = np.array([g["edges"]], dtype=np.float64)
    codes = O.encode(O.project(A, X), E)
    tree = O.build_tree(codes, 4, g["max_size"])
    return O.Index(X=X, A=A, E=E, trees=[tree], K=1, L=1, n_regions=4)


def test_query_hand_worked():
    g = _load("query_hand.json")
    idx = _hand_index(g)
    assert idx.trees[0].n_leaves == 4
    for case in g["cases"]:
        res = O.c2k_ann(idx, np.array([g["q"]]), case["k"], case["c"], case["r_min"],
                        g["eps"], case["beta"])
        exp_d = [np.inf if v == "inf" else v for v in case["dist"]]
        assert res.ids.tolist() == case["ids"], case["why"]
        assert res.dist.tolist() == exp_d, case["why"]
        assert (res.n_cand, res.rounds, res.stop) == (case["n_cand"], case["rounds"], case["stop"]), case["why"]


def _two_tree_index(g):
    X = np.array(g["X"], dtype=np.float64)
    A = np.eye(2)
    E = np.array(g["edges"], dtype=np.float64)
    codes = O.encode(O.project(A, X), E)
    return O.index_from_codes(X, A, E, codes, g["K"], g["L"], g["n_regions"], g["max_size"])


def test_query_hand_worked_two_trees():
    """Alg. 7 with L = 2, worked by hand: the order of the trees within a
    round, the lower-bound order of the leaves within a tree, the |S| test
    after every leaf and the duplicate-free count across trees each decide a
    case (tests/golden/query_hand_two_trees.json)."""
    g = _load("query_hand_two_trees.json")
    idx = _two_tree_index(g)
    assert [t.n_leaves for t in idx.trees] == [4, 4]
    assert idx.trees[0].ids.tolist() == [2, 4, 0, 1, 3, 5]
    assert idx.trees[1].ids.tolist() == [0, 5, 2, 3, 1, 4]
    for case in g["cases"]:
        res = O.c2k_ann(idx, np.array(g["q"]), case["k"], g["c"], g["r_min"], g["eps"], case["beta"],
                        keep_candidates=True)
        assert res.cand.tolist() == case["S"], case["why"]
        assert res.ids.tolist() == case["ids"], case["why"]
        assert res.dist.tolist() == [math.sqrt(v) for v in case["dist2"]], case["why"]
        assert (res.n_cand, res.rounds, res.stop) == (case["n_cand"], case["rounds"], case["stop"]), case["why"]


def test_query_tie_band_flag():
    """The tie band marks a round whose (c r)^2 lies within tie_rel of a
    candidate's squared distance: in the 1-d hand example ||q,o_3||^2 = 2^-6
    equals (c r_0)^2 exactly (flagged); with r_min = 1/2 no tested distance
    is near a threshold (not flagged)."""
    g = _load("query_hand.json")
    idx = _hand_index(g)
    q = np.array([g["q"]])
    hit = O.c2k_ann(idx, q, 1, 2.0, 0.0625, g["eps"], 1.0, tie_rel=1e-5)
    assert hit.tie_band and hit.stop == 2
    assert not O.c2k_ann(idx, q, 1, 2.0, 0.0625, g["eps"], 1.0).tie_band    # off unless asked
    miss = O.c2k_ann(idx, q, 2, 2.0, 0.5, g["eps"], 1.0, tie_rel=1e-5)
    assert not miss.tie_band


def test_mirror_form_with_own_values_is_the_plain_query():
    """index_from_codes over the oracle's own breakpoints and codes, queried
    with the FP32 rounding of the oracle's own projected query, is the plain
    c2k_ann: the mirror form adds no arithmetic of its own."""
    X, Q = make_workload("tiny", n=3000, nq=6)
    X, Q = X.numpy(), Q.numpy()
    A = gaussian_projection(4, 16, X.shape[1]).numpy()
    ref = O.build_index(X, A, sample_ids(3000, 300).numpy(), 16, 4, 16, 64)
    mir = O.index_from_codes(X, A, ref.E, ref.codes, 16, 4, 16, 64)
    for t_ref, t_mir in zip(ref.trees, mir.trees):
        assert np.array_equal(t_ref.ids, t_mir.ids) and np.array_equal(t_ref.offset, t_mir.offset)
    eps = O.eps_from_lemma3(16, 4)
    for q in Q:
        a = O.c2k_ann(ref, q, 10, 1.5, 0.0, eps, 0.1, keep_candidates=True)
        b = O.c2k_ann(mir, q, 10, 1.5, 0.0, eps, 0.1, keep_candidates=True,
                      qp32=O.project(A, q[None, :])[0].astype(np.float32))
        assert np.array_equal(a.cand, b.cand) and np.array_equal(a.ids, b.ids)
        assert (a.n_cand, a.rounds, a.stop) == (b.n_cand, b.rounds, b.stop)


def test_query_all_leaves_is_exact_knn():
    # beta*n + k >= n and a radius covering every leaf: S = D, so Alg. 7 returns the exact kNN
    X, Q = make_workload("tiny", n=2000, nq=10)
    X, Q = X.numpy(), Q.numpy()
    A = gaussian_projection(2, 8, X.shape[1]).numpy()
    idx = O.build_index(X, A, sample_ids(2000, 200).numpy(), 8, 2, 16, 32)
    for q in Q:
        res = O.c2k_ann(idx, q, 7, 1.5, 1e6, 3.0, 1.0, keep_candidates=True)
        ids, dist = O.exact_knn(X, q, 7)
        assert res.n_cand == 2000
        assert res.ids.tolist() == ids.tolist()
        assert np.allclose(res.dist, dist, rtol=0, atol=0)


def test_paa_projection_is_segment_means():
    """DET-ONLY's projection (Sec. 6.1): coordinate j of the reduced point is the
    mean of segment j of floor(d/K) coordinates; leftover coordinates are unused."""
    rng = np.random.default_rng(5)
    for K, d in ((16, 32), (16, 128), (5, 23), (1, 7)):
        A = paa_projection(K, d).numpy().astype(np.float64)
        x = rng.standard_normal(d)
        w = d // K
        want = np.array([x[j * w:(j + 1) * w].mean() for j in range(K)])
        assert np.allclose(A @ x, want, rtol=1e-6, atol=1e-7)
        assert (A[:, K * w:] == 0).all()


def test_det_only_all_leaves_is_exact_knn():
    """DET-ONLY (one DE-Tree over PAA, the same query) with S = D returns the exact kNN."""
    X, Q = make_workload("tiny", n=2000, nq=8)
    X, Q = X.numpy(), Q.numpy()
    A = paa_projection(16, X.shape[1]).numpy()
    idx = O.build_index(X, A, sample_ids(2000, 200).numpy(), 16, 1, 16, 32)
    for q in Q:
        res = O.c2k_ann(idx, q, 7, 1.5, 1e6, 3.0, 1.0, keep_candidates=True)
        ids, dist = O.exact_knn(X, q, 7)
        assert res.n_cand == 2000
        assert res.ids.tolist() == ids.tolist()
        assert np.allclose(res.dist, dist, rtol=0, atol=0)


def test_paa_reduce_hand():
    """DET-ONLY's reduction (Sec. 6.1) on hand-worked points: K=3 over d=7
    gives segments of w=2 coordinates and leaves the 7th out."""
    X = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 100.0], [0.0, -2.0, 8.0, 8.0, -1.0, 1.0, 3.0]])
    assert O.paa_reduce(X, 3).tolist() == [[1.5, 3.5, 5.5], [-1.0, 8.0, 0.0]]
    assert O.paa_reduce(X[:, :4], 1).tolist() == [[2.5], [3.5]]
    assert O.paa_reduce(X, 7).tolist() == X.tolist()


def test_det_only_index_reduces_x_itself():
    """The oracle's DET-ONLY index computes segment means from X (not from a
    projection matrix); with S = D its query returns the exact kNN."""
    X, Q = make_workload("tiny", n=2000, nq=6)
    X, Q = X.numpy(), Q.numpy()
    idx = O.build_index_det_only(X, sample_ids(2000, 200).numpy(), 16, 16, 32)
    assert idx.L == 1 and idx.reduction == "paa"
    assert np.array_equal(idx.P, O.paa_reduce(X, 16))
    for q in Q:
        res = O.c2k_ann(idx, q, 7, 1.5, 1e6, 3.0, 1.0, keep_candidates=True)
        ids, dist = O.exact_knn(X, q, 7)
        assert res.n_cand == 2000 and res.ids.tolist() == ids.tolist()


def _range_index(K=8, max_leaf=32):
    X, Q = make_workload("tiny", n=3000, nq=6)
    X, Q = X.numpy(), Q.numpy()
    A = gaussian_projection(2, K, X.shape[1]).numpy()
    idx = O.build_index(X, A, sample_ids(3000, 300).numpy(), K, 2, 16, max_leaf)
    return X, Q, idx


def test_leaf_bounds_bracket_every_point():
    """Alg. 4's bounds: lb^2 <= ||o' - q'||^2 <= ub^2 for every point of every leaf."""
    X, Q, idx = _range_index()
    K = idx.K
    for i in range(idx.L):
        t = idx.trees[i]
        P = idx.P[:, i * K:(i + 1) * K]
        for q in list(Q[:3]) + [X[7]]:
            qp = O.project(idx.A[i * K:(i + 1) * K], q[None, :])[0]
            lb2, ub2 = O.leaf_bounds2(idx, i, qp)
            d2 = ((P - qp[None, :]) ** 2).sum(1)
            for leaf in range(t.n_leaves):
                m = t.ids[t.offset[leaf]:t.offset[leaf + 1]]
                assert (lb2[leaf] <= d2[m] * (1 + 1e-12) + 1e-12).all()
                assert (d2[m] <= ub2[leaf] * (1 + 1e-12) + 1e-12).all()


def test_det_range_query_is_the_projected_ball():
    """Alg. 4/5 return exactly the points whose projection lies within r' of q'
    (brute force over all points), through all three leaf cases (small K and
    leaves so that some boxes lie inside the ball)."""
    X, Q, idx = _range_index(K=2, max_leaf=4)
    K = idx.K
    seen = dict(skipped=0, accepted=0, refined=0)
    for i in range(idx.L):
        P = idx.P[:, i * K:(i + 1) * K]
        # fresh queries, and one placed exactly on a point's projection (the
        # radius-0 ball then holds that point: the test is <=, not <)
        qps = [O.project(idx.A[i * K:(i + 1) * K], q[None, :])[0] for q in Q] + [P[7].copy()]
        for qp in qps:
            d = np.sqrt(((P - qp[None, :]) ** 2).sum(1))
            for r in (0.0, np.quantile(d, 0.01), np.quantile(d, 0.2), np.quantile(d, 0.9), d.max() * 2):
                st = {}
                got = O.det_range_query(idx, i, qp, r, stats=st)
                want = np.nonzero(d * d <= r * r)[0]
                assert np.array_equal(got, want), (i, r)
                for key in seen:
                    seen[key] += st[key]
    assert all(v > 0 for v in seen.values()), seen


def test_rc_ann_special_cases():
    """Alg. 6 in cases with a known answer: a radius covering everything gives
    the exact nearest neighbour (with or without the |S| exit); radius 0 gives
    nothing; a projected radius covering everything with c*r below the
    nearest distance and no |S| exit gives nothing."""
    X, Q, idx = _range_index()
    n = idx.n
    for q in Q:
        nn_id, nn_d = O.exact_knn(X, q, 1)
        r = O.rc_ann(idx, q, 1e9, 1.5, 1.0, beta=2.0)             # beta*n + 1 > n: no |S| exit
        assert (r.id, r.stop, r.n_cand, r.trees) == (int(nn_id[0]), 2, n, idx.L)
        assert r.dist == nn_d[0]
        r = O.rc_ann(idx, q, 1e9, 1.5, 1.0, beta=1.0 / n)         # exit after the first tree
        assert (r.id, r.stop, r.n_cand, r.trees) == (int(nn_id[0]), 1, n, 1)
        # |S| = n after the first tree, beta*n = n - 1/2: the bound beta*n + 1 is
        # not reached, so every tree is queried and the c*r test decides
        r = O.rc_ann(idx, q, 1e9, 1.5, 1.0, beta=(n - 0.5) / n)
        assert (r.id, r.stop, r.n_cand, r.trees) == (int(nn_id[0]), 2, n, idx.L)
        r = O.rc_ann(idx, q, 0.0, 1.5, 3.0, beta=0.1)
        assert (r.id, r.stop, r.n_cand) == (-1, 0, 0)
        tiny = nn_d[0] / 10.0
        r = O.rc_ann(idx, q, tiny, 1.5, 1e12 / tiny, beta=2.0)   # eps*r huge, c*r < nearest distance
        assert (r.id, r.stop, r.n_cand) == (-1, 0, n)


def test_insert_equals_building_from_all_points():
    """Inserting points whose arrival leaves the breakpoints unchanged (the
    sample lies among the first points) gives the index built from all points
    at once: codes, trees and query results; inserting nothing changes nothing."""
    X, Q = make_workload("tiny", n=3000, nq=4)
    X, Q = X.numpy(), Q.numpy()
    A = gaussian_projection(3, 8, X.shape[1]).numpy()
    ids = sample_ids(2000, 300).numpy()            # all among the first 2,000 points
    base = O.build_index(X[:2000], A, ids, 8, 3, 16, 24)
    grown = O.insert_points(O.insert_points(base, X[2000:2600]), X[2600:])
    full = O.build_index(X, A, ids, 8, 3, 16, 24)
    assert np.array_equal(grown.E, full.E)
    assert np.array_equal(grown.codes, full.codes)
    for a, b in zip(grown.trees, full.trees):
        assert np.array_equal(a.ids, b.ids) and np.array_equal(a.offset, b.offset)
        assert np.array_equal(a.plen, b.plen) and np.array_equal(a.prefix, b.prefix)
    eps = O.eps_from_lemma3(8, 3)
    for q in Q:
        ra = O.c2k_ann(grown, q, 5, 1.5, 0.0, eps, 0.1)
        rb = O.c2k_ann(full, q, 5, 1.5, 0.0, eps, 0.1)
        assert ra.ids.tolist() == rb.ids.tolist() and (ra.n_cand, ra.rounds, ra.stop) == (rb.n_cand, rb.rounds, rb.stop)
    same = O.insert_points(base, X[:0])
    assert np.array_equal(same.codes, base.codes)
    assert all(np.array_equal(a.ids, b.ids) for a, b in zip(same.trees, base.trees))


def test_tiny_config_quality():
    """Theorem 2 (statistical): on the tiny workload the result is a c^2-k-ANN for
    well over a (1/2 - 1/e) fraction of queries, and recall is high."""
    X, Q = make_workload("tiny")
    X, Q = X.numpy(), Q.numpy()
    A = gaussian_projection(4, 16, 32).numpy()
    idx = O.build_index(X, A, sample_ids(10_000, 1000).numpy(), 16, 4, 16, 256)
    eps = O.eps_from_lemma3(16, 4)
    recalls, ok = [], 0
    for q in Q[:40]:
        res = O.c2k_ann(idx, q, 10, 1.5, 0.0, eps, 0.1)
        ids, dist = O.exact_knn(X, q, 10)
        recalls.append(O.recall(res.ids, ids))
        if (res.dist <= 1.5 ** 2 * dist * (1 + 1e-12)).all():
            ok += 1
    assert ok / 40 >= 0.5 - 1 / math.e
    assert np.mean(recalls) >= 0.9


# ------------------------------------------------------------------ Sec. 6.1 measures
def test_recall_and_ratio_hand():
    assert O.recall(np.array([1, 2, 3, -1]), np.array([3, 2, 9, 8])) == 0.5
    assert O.overall_ratio(np.array([2.0, 1.0]), np.array([1.0, 2.0])) == 1.0
    assert abs(O.overall_ratio(np.array([1.0, 3.0]), np.array([1.0, 2.0])) - 1.25) < 1e-15
