"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

On exact-arithmetic inputs (values on a dyadic grid, so every FP32 sum and
product of the method is exact in any order) everything must be bit-exact:
projections, breakpoints, codes, DE-Tree leaves, candidate sets, round counts,
stop rules, top-k ids and distances. On general FP32 inputs the projections
match the FP64 oracle to 1e-5 of sum|a_t x_t|, codes match except where the
projected value lies within that tolerance of a breakpoint, and the leaves and
query results satisfy the method's invariants.
"""

import math

import numpy as np
import pytest
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O
from parity_helpers import (DEV, assert_trees_equal, check_tree_properties, gpu_build, gpu_codes,
                            gpu_trees, oracle_queries, proj_tolerance)
from workloads import gaussian_projection, make_workload, paa_projection, sample_ids
from workloads.synthetic import query_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    torch.cuda.init()


# ------------------------------------------------------------------ Eq. 1
@pytest.mark.parametrize("n,d,dtype", [(1007, 32, "f32"), (300, 33, "f32"), (129, 960, "f32"),
                                       (515, 128, "u8"), (64, 3, "u8"), (1, 1, "f32")])
def test_project_exact_inputs(n, d, dtype):
    g = torch.Generator().manual_seed(n + d)
    if dtype == "u8":
        X = torch.randint(0, 256, (n, d), generator=g, dtype=torch.uint8)
    else:
        X = torch.randint(-64, 64, (n, d), generator=g).float() / 4.0
    A = gaussian_projection(3, 16, d, seed=d, exact=True)
    P = pkg.detlsh_project(X.to(DEV), A.to(DEV)).cpu().numpy().astype(np.float64)
    ref = O.project(A.numpy(), X.numpy())
    assert np.array_equal(P, ref)


@pytest.mark.parametrize("name,n,d", [("tiny", 2000, 32), ("mid", 700, 128), ("precision", 300, 960),
                                      ("batching", 1500, 96)])
def test_project_float_inputs(name, n, d):
    X, _ = make_workload(name, n=n, nq=1)
    A = gaussian_projection(4, 16, d)
    P = pkg.detlsh_project(X.to(DEV), A.to(DEV)).cpu().numpy().astype(np.float64)
    ref = O.project(A.numpy(), X.numpy())
    tol = proj_tolerance(A.numpy(), X.numpy())
    assert (np.abs(P - ref) <= tol).all(), float((np.abs(P - ref) / tol).max())


# ------------------------------------------------------------------ Alg. 2
@pytest.mark.parametrize("Nr,LK,n", [(2, 1, 100), (16, 7, 3001), (256, 64, 5000), (8, 3, 1)])
def test_encode_values(Nr, LK, n):
    rng = np.random.default_rng(Nr * 31 + LK)
    E = np.sort(rng.standard_normal((LK, Nr + 1)).astype(np.float32), axis=1)
    E[:, 2:4] = E[:, 2:3]                      # repeated breakpoints (empty regions)
    P = (rng.standard_normal((n, LK)) * 1.5).astype(np.float32)
    m = min(n, Nr - 1)
    P[:m, 0] = E[0, 1:1 + m]                   # values exactly on breakpoints
    got = pkg.detlsh_encode_values(torch.from_numpy(P).to(DEV), torch.from_numpy(E).to(DEV), Nr)
    ref = O.encode(P.astype(np.float64), E.astype(np.float64))
    assert np.array_equal(got.cpu().numpy(), ref)


# ------------------------------------------------------------------ Alg. 1
@pytest.mark.parametrize("LK,n_s,Nr", [(64, 1000, 16), (64, 10_000, 256), (3, 257, 256), (1, 2, 2),
                                       (17, 4099, 32)])
def test_select_breakpoints(LK, n_s, Nr):
    rng = np.random.default_rng(LK * n_s)
    Ps = rng.standard_normal((LK, n_s)).astype(np.float32)
    Ps[:, : n_s // 3] = np.round(Ps[:, : n_s // 3] * 4) / 4   # ties
    Ps[0, 0] = -0.0
    got = pkg.detlsh_select_breakpoints(torch.from_numpy(Ps).to(DEV), Nr).cpu().numpy()
    ref = O.select_breakpoints(Ps.T.astype(np.float64), Nr)
    assert np.array_equal(got.astype(np.float64), ref)


# ------------------------------------------------------------------ build, exact inputs
BUILD_CASES = [
    # name, n, d, K, L, Nr, n_s, max_leaf
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256),
    ("tiny", 3_001, 32, 5, 3, 8, 333, 7),
    ("tiny", 500, 32, 16, 1, 2, 64, 1),
    ("tiny", 37, 32, 2, 2, 2, 2, 1),
    ("mid", 20_000, 128, 16, 4, 256, 2_000, 64),
    ("serving", 20_000, 128, 16, 4, 256, 2_000, 32),
    # the precision and batching shapes: d = 960 takes the CUDA-core encoder,
    # d = 96 the TF32 tensor-core one
    ("precision", 4_000, 960, 16, 4, 256, 400, 64),
    ("batching", 30_000, 96, 16, 4, 256, 3_000, 64),
]


def _exact_inputs(name, n, d, K, L, n_s, nq=0):
    X, Q = make_workload(name, n=n, nq=max(nq, 1), exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    return X, Q, A, ids


@pytest.mark.parametrize("case", BUILD_CASES)
def test_build_exact_bit_parity(case):
    name, n, d, K, L, Nr, n_s, max_leaf = case
    X, _, A, ids = _exact_inputs(name, n, d, K, L, n_s)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    assert np.array_equal(pkg.detlsh_export(idx, "A").numpy().reshape(L * K, d), A.numpy())
    Ps = pkg.detlsh_export(idx, "SAMPLE_PROJ").numpy().reshape(L * K, n_s).astype(np.float64)
    assert np.array_equal(Ps.T, ref.P[ids.numpy()])
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, Nr + 1).astype(np.float64)
    assert np.array_equal(E, ref.E)
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    info = idx.info()
    assert info["total_leaves"] == sum(t.n_leaves for t in ref.trees)
    assert info["largest_leaf"] == max(int(np.diff(t.offset).max()) for t in ref.trees)
    idx.free()


@pytest.mark.parametrize("name,d", [("tiny", 32), ("serving", 32), ("mid", 128)])
def test_build_from_misaligned_borrowed_points(name, d):
    """A borrowed device X whose base is not 16-byte aligned (a view one
    element into a buffer) takes the CUDA-core encoding instead of the TMA
    path and still gives the oracle's index (exact inputs)."""
    n, K, L, Nr, n_s, max_leaf = 3_000, 16, 4, 16, 300, 32
    X, _, A, ids = _exact_inputs(name, n, d, K, L, n_s)
    buf = torch.empty(n * d + 1, dtype=X.dtype, device=DEV)
    Xm = buf[1:].view(n, d)
    Xm.copy_(X.to(DEV))
    assert Xm.data_ptr() % 16 != 0
    idx = pkg.detlsh_build(Xm, A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, borrow=True)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    idx.free()


@pytest.mark.parametrize("kind", ["few_values", "narrow_offset"])
def test_build_degenerate_breakpoints_bit_parity(kind):
    """Breakpoints with many equal values (few distinct points) and breakpoints
    packed into a range narrow against their magnitude: the region search of
    the encoding must still give the oracle's codes (exact inputs)."""
    n, d, K, L, Nr, n_s, max_leaf = 2_000, 8, 4, 2, 16, 400, 16
    g = torch.Generator().manual_seed(11)
    if kind == "few_values":
        X = torch.randint(0, 2, (n, d), generator=g).to(torch.float32)
    else:
        X = 256.0 + torch.randint(0, 4, (n, d), generator=g).to(torch.float32) / 4.0
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, Nr + 1).astype(np.float64)
    assert np.array_equal(E, ref.E)
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    idx.free()
    if kind == "few_values":   # values BF16 holds exactly: the tensor-core path too
        idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, proj_mode=1)
        assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
        idx.free()


# ------------------------------------------------------------------ build from a seed (reading R15)
@pytest.mark.parametrize("name,n,d,sample_size,dtype_mode", [("tiny", 10_000, 32, 0, 0), ("mid", 20_000, 128, 2_000, 0),
                                                             ("serving", 30_000, 128, 0, 0), ("mid", 20_000, 128, 0, 1)])
def test_build_from_seed_alone(name, n, d, sample_size, dtype_mode):
    """detlsh_build with only the dataset, K, L, N_r and a seed: the library
    draws A and the sample itself, bit-equal to the oracle's generator, with
    n_s = ceil(0.1 n) by default (Sec. 6.1); the index equals one built from
    the same draws passed in explicitly."""
    K, L, Nr, max_leaf, seed = 16, 4, 256, 64, 2024
    X, _ = make_workload(name, n=n, nq=1)
    Xd = X.to(DEV)
    idx = pkg.detlsh_build(Xd, None, None, K, L, Nr, max_leaf, seed=seed, sample_size=sample_size,
                           proj_mode=dtype_mode)
    n_s = sample_size or O.default_sample_size(n)
    A_ref = O.draw_hashes(seed, L, K, d)
    ids_ref = O.draw_sample(seed, n, n_s)
    assert idx.info()["n_s"] == n_s
    assert np.array_equal(pkg.detlsh_export(idx, "A").numpy().reshape(L * K, d), A_ref)
    assert np.array_equal(pkg.detlsh_export(idx, "SAMPLE_IDS").numpy(), ids_ref)
    idx2 = pkg.detlsh_build(Xd, torch.from_numpy(A_ref).to(DEV), torch.from_numpy(ids_ref).to(DEV), K, L, Nr,
                            max_leaf, proj_mode=dtype_mode)
    for what in ("EDGES", "CODES", "LEAF_IDS", "LEAF_RANGE", "LEAF_PLEN", "LEAF_PREFIX"):
        assert torch.equal(pkg.detlsh_export(idx, what), pkg.detlsh_export(idx2, what)), what
    idx.free()
    idx2.free()


# ------------------------------------------------------------------ build, float inputs
@pytest.mark.parametrize("name,n,d,Nr,n_s", [("tiny", 10_000, 32, 16, 1_000),
                                             ("precision", 4_000, 960, 256, 400),
                                             ("batching", 20_000, 96, 256, 2_000),
                                             ("mid", 20_000, 128, 256, 2_000),
                                             ("serving", 20_000, 128, 256, 2_000)])
def test_build_float_within_tolerance(name, n, d, Nr, n_s):
    K, L, max_leaf = 16, 4, 128
    X, _ = make_workload(name, n=n, nq=1)
    A = gaussian_projection(L, K, d)
    ids = sample_ids(n, n_s)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    P64 = O.project(A.numpy(), X.numpy())
    tol = proj_tolerance(A.numpy(), X.numpy())
    Ps = pkg.detlsh_export(idx, "SAMPLE_PROJ").numpy().reshape(L * K, n_s).T.astype(np.float64)
    s = ids.numpy()
    assert (np.abs(Ps - P64[s]) <= tol[s]).all()
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, Nr + 1).astype(np.float64)
    E64 = O.select_breakpoints(P64[s], Nr)
    band = tol[s].max(axis=0)[:, None]
    assert (np.abs(E - E64) <= band).all()
    codes = gpu_codes(idx, n, K, L)
    ref_codes = O.encode(P64, E64)
    # away from a breakpoint the code is exact; near one it is one of the codes of p +- tol
    lo_codes = O.encode(P64 - tol - band.T, E64)
    hi_codes = O.encode(P64 + tol + band.T, E64)
    exact = lo_codes == hi_codes
    assert np.array_equal(codes[exact], ref_codes[exact])
    assert ((codes >= lo_codes) & (codes <= hi_codes)).all()
    # actual disagreement with the FP64 oracle is rare
    assert (codes != ref_codes).mean() < 1e-3
    for t, tree in enumerate(gpu_trees(idx, K, L, n)):
        check_tree_properties(tree, codes[:, t * K:(t + 1) * K], Nr, max_leaf)
    idx.free()


# ------------------------------------------------------------------ query, exact inputs
QUERY_CASES = [
    # name, n, d, K, L, Nr, n_s, max_leaf, nq, k, beta, r_min
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256, 100, 10, 0.1, 0.0),
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 64, 40, 10, 0.01, 0.0),
    ("tiny", 10_000, 32, 16, 4, 16, 1_000, 256, 30, 10, 0.1, 2.5),
    ("tiny", 3_001, 32, 5, 3, 8, 333, 7, 30, 7, 0.05, 0.0),
    ("tiny", 2_000, 32, 8, 2, 16, 200, 32, 20, 25, 2.0, 0.0),
    ("tiny", 500, 32, 16, 1, 2, 64, 1, 20, 3, 0.0, 0.0),
    ("mid", 20_000, 128, 16, 4, 256, 2_000, 64, 30, 50, 0.1, 0.0),
    ("serving", 20_000, 128, 16, 4, 256, 2_000, 32, 30, 10, 0.02, 0.0),
    # uint8 rows with d/16 lanes per row (2 and 32), and a d the integer
    # distance kernel does not take
    ("serving", 3_000, 32, 16, 4, 16, 300, 32, 12, 10, 0.1, 0.0),
    ("serving", 3_000, 512, 16, 4, 16, 300, 32, 12, 10, 0.1, 0.0),
    ("serving", 3_000, 48, 16, 4, 16, 300, 32, 12, 10, 0.1, 0.0),
    # the precision (d = 960) and batching (d = 96) shapes
    ("precision", 6_000, 960, 16, 4, 256, 600, 64, 16, 100, 0.1, 0.0),
    ("batching", 30_000, 96, 16, 4, 256, 3_000, 256, 24, 100, 0.01, 0.0),
]


@pytest.mark.parametrize("case", QUERY_CASES)
def test_query_exact_bit_parity(case):
    name, n, d, K, L, Nr, n_s, max_leaf, nq, k, beta, r_min = case
    X, Q, A, ids = _exact_inputs(name, n, d, K, L, n_s, nq=nq)
    eps = O.eps_from_lemma3(K, L)
    g = torch.Generator().manual_seed(nq)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    ks[0] = k
    rm = torch.full((nq,), r_min, dtype=torch.float32)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    cap = n
    out_ids, out_dist, stats, cand = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV),
                                                      k_max=k, eps=eps, beta=beta, cand_cap=cap)
    out_ids, out_dist = out_ids.cpu().numpy(), out_dist.cpu().numpy()
    stats, cand = stats.cpu().numpy(), cand.cpu().numpy().view(np.uint32)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    res = oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), rm.numpy(), eps, beta)
    for qi, r in enumerate(res):
        kq = int(ks[qi])
        assert (stats[qi, 0], stats[qi, 1], stats[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        got_S = np.sort(cand[qi, : stats[qi, 0]].astype(np.int64))
        assert np.array_equal(got_S, r.cand), qi
        assert np.array_equal(out_ids[qi, :kq], r.ids[:kq]), qi
        assert (out_ids[qi, kq:] == -1).all()
        exp = np.float32(r.dist[:kq])   # exact squared distances, so sqrt rounds alike
        assert np.array_equal(out_dist[qi, :kq], exp), qi
    idx.free()


@pytest.mark.parametrize("case", [QUERY_CASES[0], QUERY_CASES[3], QUERY_CASES[6], QUERY_CASES[7]])
def test_query_dedup_by_leaf_position_same_results(case):
    """The walk's duplicate test indexed by tree-0 leaf position (the layout
    large indexes get) gives the same candidates and results as by point id,
    and the oracle's on the first queries."""
    name, n, d, K, L, Nr, n_s, max_leaf, nq, k, beta, r_min = case
    X, Q, A, ids = _exact_inputs(name, n, d, K, L, n_s, nq=nq)
    eps = O.eps_from_lemma3(K, L)
    g = torch.Generator().manual_seed(nq + 1)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    rm = torch.full((nq,), r_min, dtype=torch.float32)
    outs = []
    for pos in (False, True):
        idx = pkg.detlsh_build(X.to(DEV), A.to(DEV), ids.to(DEV), K, L, Nr, max_leaf, dedup_pos=pos)
        o = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV), k_max=k, eps=eps, beta=beta,
                             cand_cap=n)
        outs.append([t.cpu() for t in o])
        idx.free()
    (i0, d0, s0, c0), (i1, d1, s1, c1) = outs
    assert torch.equal(i0, i1) and torch.equal(d0, d1) and torch.equal(s0, s1)
    for qi in range(nq):
        m = int(s0[qi, 0])
        assert torch.equal(torch.sort(c0[qi, :m])[0], torch.sort(c1[qi, :m])[0]), qi
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    res = oracle_queries(ref, Q.numpy()[:3], ks.numpy()[:3], cs.numpy()[:3], rm.numpy()[:3], eps, beta)
    for qi, r in enumerate(res):
        kq = int(ks[qi])
        assert np.array_equal(i1.numpy()[qi, :kq], r.ids[:kq]), qi
        assert int(s1[qi, 0]) == r.n_cand


@pytest.mark.parametrize("name,n,d,Nr,n_s,max_leaf,nq,k", [("tiny", 10_000, 32, 16, 1_000, 64, 30, 10),
                                                         ("mid", 20_000, 128, 256, 2_000, 64, 20, 50)])
def test_det_only_exact_bit_parity(name, n, d, Nr, n_s, max_leaf, nq, k):
    """DET-ONLY (Sec. 6.1): one DE-Tree over the PAA reduction and the same
    query. The library projects with the segment-mean matrix (exact here: 1/w
    with w a power of two); the oracle computes the segment means from X
    itself. Index and results equal the oracle's bit for bit."""
    K, L, beta = 16, 1, 0.1
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = paa_projection(K, d)
    ids = sample_ids(n, n_s)
    eps = O.eps_from_lemma3(K, L)
    g = torch.Generator().manual_seed(nq)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    rm = torch.zeros(nq, dtype=torch.float32)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    ref = O.build_index_det_only(X.numpy(), ids.numpy(), K, Nr, max_leaf)
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    out_ids, out_dist, stats, _ = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV), k_max=k,
                                                   eps=eps, beta=beta)
    out_ids, out_dist, stats = out_ids.cpu().numpy(), out_dist.cpu().numpy(), stats.cpu().numpy()
    res = oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), rm.numpy(), eps, beta, keep=False)
    for qi, r in enumerate(res):
        kq = int(ks[qi])
        assert (stats[qi, 0], stats[qi, 1], stats[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        assert np.array_equal(out_ids[qi, :kq], r.ids[:kq]), qi
        assert np.array_equal(out_dist[qi, :kq], np.float32(r.dist[:kq])), qi
    idx.free()


@pytest.mark.parametrize("name,d,K,L,Nr,max_leaf", [("tiny", 32, 8, 2, 16, 32), ("tiny", 32, 2, 2, 16, 4),
                                                    ("serving", 32, 8, 3, 16, 16)])
def test_rc_ann_exact_bit_parity(name, d, K, L, Nr, max_leaf):
    """Alg. 6 with the exact range query of Alg. 4/5: id, distance, |S|, trees
    queried and stop rule equal the oracle's bit for bit (exact inputs) over
    radii from nothing found to everything found, with and without the |S|
    exit."""
    n, n_s, nq = 3_000, 300, 8
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n, n_s)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    nn = np.array([O.exact_knn(X.numpy(), q, 1)[1][0] for q in Q.numpy()])
    for scale, c, eps, beta in ((0.0, 1.5, 3.0, 0.1), (0.5, 1.5, 3.0, 2.0), (1.0, 1.2, 1.0, 0.05),
                                (1.5, 2.0, 2.0, 2.0), (4.0, 1.5, 3.0, 0.01), (1e3, 1.5, 3.0, 2.0)):
        r = np.float32(nn * scale)
        got_id, got_d, got_st = (t.cpu().numpy() for t in
                                 pkg.detlsh_rc_ann(idx, Q.to(DEV), torch.from_numpy(r), c, eps, beta))
        for qi in range(nq):
            want = O.rc_ann(ref, Q.numpy()[qi], float(r[qi]), float(np.float32(c)), eps, beta)
            assert (int(got_id[qi]), float(got_d[qi])) == (want.id, want.dist), (scale, qi)
            assert tuple(got_st[qi]) == (want.n_cand, want.trees, want.stop), (scale, qi)
    idx.free()


@pytest.mark.parametrize("name,d", [("tiny", 32), ("serving", 32), ("mid", 128), ("tiny", 30)])
def test_insert_exact_bit_parity(name, d):
    """Insertion (reading R14): points added in two batches (device, then host
    memory) to an index of the first 2,000 get the oracle's codes, leaves and
    query results bit for bit (exact inputs), through the TF32, uint8 tensor-
    core and CUDA-core (d = 30) encodings."""
    n1, n, K, L, Nr, max_leaf, nq, k, beta = 2_000, 3_000, 16, 4, 16, 32, 12, 10, 0.1
    X, Q = make_workload(name, n=n, nq=nq, exact=True, d=d)
    A = gaussian_projection(L, K, d, exact=True)
    ids = sample_ids(n1, 300)
    idx = gpu_build(X[:n1], A, ids, K, L, Nr, max_leaf)
    pkg.detlsh_insert(idx, X[n1:2_600].to(DEV))
    pkg.detlsh_insert(idx, X[2_600:])
    assert idx.info()["n"] == n
    ref = O.build_index(X[:n1].numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    ref = O.insert_points(O.insert_points(ref, X[n1:2_600].numpy()), X[2_600:].numpy())
    assert np.array_equal(gpu_codes(idx, n, K, L), ref.codes)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    eps = O.eps_from_lemma3(K, L)
    g = torch.Generator().manual_seed(3)
    cs = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    ks = torch.randint(1, k + 1, (nq,), generator=g, dtype=torch.int32)
    rm = torch.zeros(nq, dtype=torch.float32)
    out_ids, out_dist, stats, _ = pkg.detlsh_query(idx, Q.to(DEV), ks.to(DEV), cs.to(DEV), rm.to(DEV), k_max=k,
                                                   eps=eps, beta=beta)
    out_ids, out_dist, stats = out_ids.cpu().numpy(), out_dist.cpu().numpy(), stats.cpu().numpy()
    res = oracle_queries(ref, Q.numpy(), ks.numpy(), cs.numpy(), rm.numpy(), eps, beta, keep=False)
    for qi, r in enumerate(res):
        kq = int(ks[qi])
        assert (stats[qi, 0], stats[qi, 1], stats[qi, 2]) == (r.n_cand, r.rounds, r.stop), qi
        assert np.array_equal(out_ids[qi, :kq], r.ids[:kq]), qi
        assert np.array_equal(out_dist[qi, :kq], np.float32(r.dist[:kq])), qi
    idx.free()


# ------------------------------------------------------------------ query, float inputs
@pytest.mark.parametrize("name,n,d,Nr,n_s,nq,k", [("tiny", 10_000, 32, 16, 1_000, 100, 10),
                                                  ("batching", 30_000, 96, 256, 3_000, 24, 50),
                                                  ("precision", 6_000, 960, 64, 600, 16, 20)])
def test_query_float_quality_and_distances(name, n, d, Nr, n_s, nq, k):
    """FP32 inputs: returned distances are the true ones to 1e-5, results are a
    c^2-k-ANN for the Theorem 2 fraction of queries, and recall matches the
    oracle's on the same inputs (the leaves may differ near breakpoints)."""
    K, L, max_leaf, beta = 16, 4, 256, 0.1
    X, Q = make_workload(name, n=n, nq=nq)
    A = gaussian_projection(L, K, d)
    ids = sample_ids(n, n_s)
    idx = gpu_build(X, A, ids, K, L, Nr, max_leaf)
    eps = O.eps_from_lemma3(K, L)
    out_ids, out_dist, stats, _ = pkg.detlsh_query(idx, Q.to(DEV), k, 1.5, 0.0, k_max=k, eps=eps, beta=beta)
    out_ids, out_dist = out_ids.cpu().numpy(), out_dist.cpu().numpy()
    Xn, Qn = X.numpy().astype(np.float64), Q.numpy().astype(np.float64)
    ref = O.build_index(X.numpy(), A.numpy(), ids.numpy(), K, L, Nr, max_leaf)
    rec_gpu, rec_ref, ok = [], [], 0
    for qi in range(nq):
        gids = out_ids[qi]
        assert (gids >= 0).all() and len(set(gids.tolist())) == k
        d64 = np.sqrt(((Xn[gids] - Qn[qi]) ** 2).sum(axis=1))
        assert np.allclose(out_dist[qi], d64, rtol=1e-5, atol=1e-6)
        assert (np.diff(out_dist[qi]) >= 0).all()
        eids, edist = O.exact_knn(Xn, Qn[qi], k)
        rec_gpu.append(O.recall(gids, eids))
        rec_ref.append(O.recall(O.c2k_ann(ref, Qn[qi], k, 1.5, 0.0, eps, beta).ids, eids))
        ok += (d64 <= 1.5 ** 2 * edist * (1 + 1e-6)).all()
    assert ok / nq >= 0.5 - 1 / math.e
    assert np.mean(rec_gpu) >= np.mean(rec_ref) - 0.05, (np.mean(rec_gpu), np.mean(rec_ref))
    if name == "tiny":
        assert np.mean(rec_gpu) >= 0.9
    idx.free()


# ------------------------------------------------------------------ edge cases
def test_query_empty_batch_and_padding():
    X, Q, A, ids = _exact_inputs("tiny", 50, 32, 8, 2, 8, nq=3)
    idx = gpu_build(X, A, ids, 8, 2, 8, 4)
    out = pkg.detlsh_query(idx, Q[:0].to(DEV), 5, 1.5, 0.0, k_max=5)
    assert out[0].shape == (0, 5)
    # k > n: every point returned, then -1 / +inf
    oid, od, st, _ = pkg.detlsh_query(idx, Q.to(DEV), 60, 1.5, 0.0, k_max=64, beta=0.0)
    oid, od = oid.cpu().numpy(), od.cpu().numpy()
    for qi in range(3):
        assert sorted(oid[qi, :50].tolist()) == list(range(50))
        assert (oid[qi, 50:] == -1).all() and np.isinf(od[qi, 50:]).all()
    idx.free()


def test_query_rejects_bad_device_arguments():
    X, Q, A, ids = _exact_inputs("tiny", 100, 32, 8, 2, 8, nq=2)
    idx = gpu_build(X, A, ids, 8, 2, 8, 4)
    with pytest.raises(pkg.DetlshError):
        pkg.detlsh_query(idx, Q.to(DEV), torch.tensor([3, 9], dtype=torch.int32), 1.5, 0.0, k_max=4)
    with pytest.raises(pkg.DetlshError):
        pkg.detlsh_query(idx, Q.to(DEV), 3, torch.tensor([1.5, 1.0]), 0.0, k_max=4)
    idx.free()


def test_build_rejects_out_of_range_sample_ids():
    X, _, A, ids = _exact_inputs("tiny", 100, 32, 8, 2, 8)
    bad = ids.clone()
    bad[3] = 100
    with pytest.raises(pkg.DetlshError):
        gpu_build(X, A, bad, 8, 2, 8, 4)


def test_host_and_device_memory_give_the_same_result():
    X, Q, A, ids = _exact_inputs("tiny", 2000, 32, 16, 2, 200, nq=8)
    idx_h = pkg.detlsh_build(X, A, ids, 16, 2, 16, 32)
    idx_d = gpu_build(X, A, ids, 16, 2, 16, 32)
    a = pkg.detlsh_query(idx_h, Q, 5, 1.5, 0.0, k_max=5)
    b = pkg.detlsh_query(idx_d, Q.to(DEV), 5, 1.5, 0.0, k_max=5)
    assert torch.equal(a[0], b[0].cpu()) and torch.equal(a[1], b[1].cpu()) and torch.equal(a[2], b[2].cpu())
    idx_h.free()
    idx_d.free()
