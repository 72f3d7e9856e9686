"""Shared helpers for the GPU parity tests (comparison glue, no method arithmetic)."""

import math

import numpy as np
import torch

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O

DEV = "cuda:0"


def gpu_build(X, A, ids, K, L, Nr, max_leaf, dev=DEV):
    return pkg.detlsh_build(X.to(dev), A.to(dev), ids.to(dev), K, L, Nr, max_leaf)


def gpu_trees(idx, K, L, n):
    """The GPU leaf table as oracle Trees (one per projected space)."""
    base = pkg.detlsh_export(idx, "LEAF_BASE").numpy()
    rng = pkg.detlsh_export(idx, "LEAF_RANGE").numpy().astype(np.int64).reshape(-1, 2)
    plen = pkg.detlsh_export(idx, "LEAF_PLEN").numpy().astype(np.int64).reshape(-1, K)
    pref = pkg.detlsh_export(idx, "LEAF_PREFIX").numpy().astype(np.int64).reshape(-1, K)
    lids = pkg.detlsh_export(idx, "LEAF_IDS").numpy().view(np.uint32).astype(np.int64).reshape(L, n)
    trees = []
    for t in range(L):
        a, b = int(base[t]), int(base[t + 1])
        starts = rng[a:b, 0]
        counts = rng[a:b, 1]
        offset = np.zeros(b - a + 1, dtype=np.int64)
        offset[1:] = np.cumsum(counts)
        assert (starts == offset[:-1]).all(), "leaves are not contiguous in leaf order"
        trees.append(O.Tree(ids=lids[t], offset=offset, plen=plen[a:b], prefix=pref[a:b]))
    return trees


def gpu_codes(idx, n, K, L):
    """GPU codes [L][n][K] -> oracle layout [n][L*K]."""
    c = pkg.detlsh_export(idx, "CODES").numpy().reshape(L, n, K)
    return np.ascontiguousarray(c.transpose(1, 0, 2).reshape(n, L * K))


def assert_trees_equal(got, ref):
    assert len(got) == len(ref)
    for t, (g, r) in enumerate(zip(got, ref)):
        assert g.n_leaves == r.n_leaves, f"tree {t}: {g.n_leaves} leaves vs {r.n_leaves}"
        assert np.array_equal(g.offset, r.offset), f"tree {t}: leaf sizes differ"
        assert np.array_equal(g.ids, r.ids), f"tree {t}: leaf-ordered ids differ"
        assert np.array_equal(g.plen, r.plen), f"tree {t}: prefix lengths differ"
        assert np.array_equal(g.prefix, r.prefix), f"tree {t}: prefixes differ"


def check_tree_properties(tree, codes, Nr, max_size):
    """Invariants any DE-Tree of the bulk-loaded reading satisfies for its own codes."""
    n, K = codes.shape
    bits = int(math.log2(Nr))
    lo, hi = tree.box(bits)
    assert np.array_equal(np.sort(tree.ids), np.arange(n))
    prev = None
    for leaf in range(tree.n_leaves):
        ids = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
        assert len(ids) > 0
        assert (np.diff(ids) > 0).all()
        cl = codes[ids].astype(np.int64)
        assert ((cl >= lo[leaf]) & (cl <= hi[leaf])).all()
        if len(ids) > max_size:
            assert (tree.plen[leaf] == bits).all()
        key = tuple((lo[leaf] >> (bits - 1)).tolist())
        if prev is not None:
            assert key >= prev
        prev = key


def proj_tolerance(A, X):
    """Scaled FP32 projection tolerance 1e-5 * sum_t |A[r,t] X[o,t]| (FP64)."""
    return 1e-5 * (np.abs(np.asarray(X, np.float64)) @ np.abs(np.asarray(A, np.float64)).T)


def oracle_queries(ref, Q, k, c, r_min, eps, beta, keep=True):
    res = []
    for qi in range(Q.shape[0]):
        res.append(O.c2k_ann(ref, Q[qi], int(k[qi]), float(c[qi]), float(r_min[qi]), eps, beta,
                             keep_candidates=keep))
    return res


def mirror_index(idx, X, A, K, L, Nr, max_leaf):
    """The FP32-mirror oracle index of a GPU index: the GPU's breakpoints and
    codes, the DE-Trees built from those codes by the oracle (which must equal
    the GPU's leaf tables)."""
    n = X.shape[0]
    E = pkg.detlsh_export(idx, "EDGES").numpy().reshape(L * K, Nr + 1).astype(np.float64)
    codes = gpu_codes(idx, n, K, L)
    ref = O.index_from_codes(np.asarray(X), np.asarray(A), E, codes, K, L, Nr, max_leaf)
    assert_trees_equal(gpu_trees(idx, K, L, n), ref.trees)
    return ref


def fp32_distance_band(d):
    """Relative bound on the error of an FP32 squared distance of d
    coordinates (a rounded difference, a rounded square and d rounded sums of
    non-negative terms: at most (d + 3) units of 2^-24), never below the 1e-5
    of the distance tolerance. Outside this band an FP32 comparison of the
    squared distance with an FP32 threshold decides as the FP64 one does."""
    return max(1e-5, (d + 3) * 2.0 ** -24)


def check_topk_up_to_ties(got_ids, got_dist, ref, X64, q64, k, band):
    """The GPU's top-k over the same candidate set as the oracle's: position
    by position the same ids, except a swap between candidates whose FP64
    distances agree within `band`; returned distances within 1e-5 of FP64."""
    got_ids = np.asarray(got_ids[:k])
    assert len(set(got_ids[got_ids >= 0].tolist())) == int((got_ids >= 0).sum())
    cand = set(ref.cand.tolist())
    for i in range(k):
        gi, ri = int(got_ids[i]), int(ref.ids[i])
        if ri < 0:
            assert gi == -1 and np.isinf(got_dist[i])
            continue
        assert gi in cand
        d_true = math.sqrt(float(((X64[gi] - q64) ** 2).sum()))
        assert abs(float(got_dist[i]) - d_true) <= 1e-5 * d_true + 1e-30
        if gi != ri:
            assert abs(d_true ** 2 - float(ref.dist[i]) ** 2) <= band * float(ref.dist[i]) ** 2, (i, gi, ri)
