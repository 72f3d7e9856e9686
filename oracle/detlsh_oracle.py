"""CPU oracle for DET-LSH (Wei et al., PVLDB 17(9), 2024) -- TEST INFRASTRUCTURE.

This module is a plain, slow, deliberately unoptimised restatement of what the
paper's method computes. It exists only to check the CUDA library: it may be
imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``, and by nothing else. It shares no code with the CUDA path.

Precision: FP64 throughout, except where floating point decides an integer
(a leaf's activation round): there the lower bound is evaluated in FP32 with a
fixed operation order, the precision the GPU path decides in (see
``leaf_lb2_fp32``).

Readings of passages that are silent or ambiguous (numbered as in the design
notes):
 R1  breakpoints: interior edge z (1-based, z=1..N_r-1) is the element of
     0-based rank floor(n_s/N_r)*z of the sorted sample (Sec. 4.1 formula for
     B_ij, indices read 0-based, n replaced by the sample size n_s of Alg. 1).
 R2  encoding: regions are half-open [e_z, e_{z+1}); a value equal to an edge
     goes up; values outside the sample range clamp to region 0 / N_r-1.
 R3  DE-Tree: bulk-loaded, insertion-order-free version of Alg. 3: a node
     holding more than max_size points splits by one more bit of the dimension
     whose next bit divides its points most evenly (ties to the lowest
     dimension); bit-0 child first; empty children dropped; a node whose codes
     are fully resolved stays an (oversized) leaf.
 R4  leaf box in the lower bound uses -inf/+inf for the outermost edges.
 R5  query (Alg. 7 + the optimised range query of Sec. 6.2.2): a leaf is taken
     whole in the first round whose projected radius covers its lower bound;
     within a round trees go in order 1..L and leaves by (lower bound, leaf
     number); the |S| >= beta*n+k test runs after every leaf; the
     ">= k within c*r" test after every round; the loop also ends once every
     leaf is active (S cannot grow further, so the result is unchanged).
 R6  thresholds: r_0 = r_min, r_{t+1} = r_t * c in FP64; the projected-radius
     threshold (eps*r_t)^2 and the exact-distance threshold (c*r_t)^2 are
     formed in FP64 and rounded once to FP32; from round ROUND_CAP-1 on both
     are +inf.
 R7  r_min <= 0 selects sqrt(min positive leaf lower bound^2)/eps (the paper's
     "magic" r_min of Sec. 5.2 is defined only through the search itself);
     with no positive lower bound r_min = 1.
 R8  eps = sqrt(chi2 upper alpha1-quantile with K degrees of freedom),
     alpha1 = exp(-1/L) (Lemma 3, Eq. 2).
 R11 exact range query (Alg. 4/5): the upper bound of a leaf box also takes
     -inf/+inf for the outermost edges (a point can lie beyond the sample's
     range), so leaves on the outside are always checked point by point.
 R12 range tests compare squared distances in FP64.
 R13 (r,c)-ANN (Alg. 6): |S| >= beta*n + 1 compared as real numbers; a
     query that returns nothing reports id -1.
 R14 insertion: new points are encoded against the existing breakpoints and
     the trees of all points are those of R3 (order-free), not the result of
     Alg. 3's on-line splits in arrival order.
 R15 random draws (the paper names no generator): splitmix64 feeding
     Box-Muller for the N(0,1) hash vectors and a partial Fisher-Yates
     shuffle for the sample (``draw_hashes``, ``draw_sample``).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

ROUND_CAP = 256


# ---------------------------------------------------------------- random draws
# The paper draws the hash vectors from N(0,1) (Eq. 1) and samples the points
# for Alg. 1 without fixing a generator. Reading R15: one splitmix64 stream
# (Steele, Lea and Flood, OOPSLA 2014) feeds the Box-Muller transform for the
# hash vectors (state = seed) and a partial Fisher-Yates shuffle for the sample
# (state = seed XOR 0x5A).
_MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """The splitmix64 output sequence from an initial 64-bit state: the state
    advances by 0x9E3779B97F4A7C15 and each output is the new state mixed by
    two xor-shift-multiply steps and a final xor-shift."""
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        yield z ^ (z >> 31)


def draw_hashes(seed: int, L: int, K: int, d: int) -> np.ndarray:
    """The L*K hash vectors of Eq. 1 as A [L*K, d] FP32 (row r = i*K + j),
    entries N(0,1) by Box-Muller (Box and Muller, 1958) in FP64: two outputs
    give u1 in (0, 1] and u2 in [0, 1) (53 bits each), rho = sqrt(-2 ln u1),
    theta = 2 pi u2, and the next two entries in row-major order are
    rho cos theta and rho sin theta, each rounded to FP32 (reading R15)."""
    count = L * K * d
    out = np.empty(count, dtype=np.float32)
    g = splitmix64(int(seed) & _MASK64)
    for e in range(0, count, 2):
        u1 = float((next(g) >> 11) + 1) * 2.0 ** -53
        u2 = float(next(g) >> 11) * 2.0 ** -53
        rho = math.sqrt(-2.0 * math.log(u1))
        theta = 2.0 * math.pi * u2
        out[e] = np.float32(rho * math.cos(theta))
        if e + 1 < count:
            out[e + 1] = np.float32(rho * math.sin(theta))
    return out.reshape(L * K, d)


def draw_sample(seed: int, n: int, n_s: int) -> np.ndarray:
    """The sample of Alg. 1: n_s distinct ids of [0, n), ascending, from a
    partial Fisher-Yates shuffle of the positions 0..n-1 where step i swaps
    position i with i + floor(z (n - i) / 2^64), z the next output (reading
    R15)."""
    if not 1 <= n_s <= n:
        raise ValueError("need 1 <= n_s <= n")
    g = splitmix64((int(seed) ^ 0x5A) & _MASK64)
    moved = {}
    out = np.empty(n_s, dtype=np.int64)
    for i in range(n_s):
        j = i + ((next(g) * (n - i)) >> 64)
        vi, vj = moved.get(i, i), moved.get(j, j)
        moved[i], moved[j] = vj, vi
        out[i] = vj
    return np.sort(out)


def default_sample_size(n: int) -> int:
    """Sec. 6.1 sets n_s = 0.1 n; as an integer, ceil(0.1 n)."""
    return (int(n) + 9) // 10


# ---------------------------------------------------------------- parameters
def eps_from_lemma3(K: int, L: int) -> float:
    """epsilon of Lemma 3 / Eq. 2: eps^2 = chi2_{alpha1}(K), alpha1 = exp(-1/L).

    L = -1/ln(alpha1) in Lemma 3 is inverted for alpha1 (reading R8).
    """
    from scipy.stats import chi2
    alpha1 = math.exp(-1.0 / L)
    return math.sqrt(chi2.isf(alpha1, K))


def beta_from_lemma3(K: int, L: int, c: float) -> float:
    """Theoretical beta of Lemma 3: beta = 2 - 2 * alpha2^L with
    chi2_{alpha2}(K) = eps^2 / c^2 (Eq. 2)."""
    from scipy.stats import chi2
    eps2 = eps_from_lemma3(K, L) ** 2
    alpha2 = chi2.sf(eps2 / (c * c), K)
    return 2.0 - 2.0 * alpha2 ** L


# ---------------------------------------------------------------- encoding phase
def project(A: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Eq. 1, h(o) = a . o for all L*K hash vectors: P[o, r] = sum_t A[r,t] X[o,t].

    A is [L*K, d] (row r = i*K + j), X is [n, d]; returns FP64 [n, L*K].
    """
    return np.asarray(X, dtype=np.float64) @ np.asarray(A, dtype=np.float64).T


def paa_reduce(X: np.ndarray, K: int) -> np.ndarray:
    """DET-ONLY's reduction (Sec. 6.1): the Piecewise Aggregate Approximation
    of each point to K dimensions, coordinate j the mean of the j-th segment
    of w = floor(d/K) consecutive coordinates (the last d - K*w coordinates
    belong to no segment). Returns FP64 [n, K]."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    w = d // K
    if w < 1:
        raise ValueError("need K <= d")
    out = np.empty((n, K), dtype=np.float64)
    for j in range(K):
        out[:, j] = X[:, j * w:(j + 1) * w].sum(axis=1) / w
    return out


def select_breakpoints(Ps: np.ndarray, n_regions: int) -> np.ndarray:
    """Alg. 1 / Sec. 4.1: N_r+1 breakpoints per projected dimension from the sample.

    Ps is [n_s, L*K] (projections of the sampled points). For each column the
    values are sorted ascending (the QuickSelect rounds of Alg. 1 find the
    same order statistics); B(1) is the minimum, B(N_r+1) the maximum and the
    interior breakpoint z (z=1..N_r-1) is the element of rank
    floor(n_s/N_r)*z (reading R1). Returns FP64 [L*K, N_r+1].
    """
    n_s, LK = Ps.shape
    m = n_s // n_regions
    E = np.empty((LK, n_regions + 1), dtype=np.float64)
    for r in range(LK):
        srt = np.sort(np.asarray(Ps[:, r], dtype=np.float64))
        E[r, 0] = srt[0]
        for z in range(1, n_regions):
            E[r, z] = srt[m * z]
        E[r, n_regions] = srt[n_s - 1]
    return E


def encode(P: np.ndarray, E: np.ndarray) -> np.ndarray:
    """Alg. 2: region symbol of every projected coordinate.

    code = number of interior breakpoints e_z (z=1..N_r-1) with e_z <= p,
    i.e. the b of B(b) <= h < B(b+1) with half-open regions (reading R2).
    P is [n, L*K]; returns uint8 [n, L*K].
    """
    n, LK = P.shape
    out = np.empty((n, LK), dtype=np.uint8)
    for r in range(LK):
        interior = E[r, 1:-1]
        out[:, r] = np.searchsorted(interior, P[:, r], side="right")
    return out


# ---------------------------------------------------------------- indexing phase
@dataclass
class Tree:
    """One DE-Tree as its leaves in depth-first order.

    ids:      point ids in leaf order (leaf by leaf, ascending id within a leaf)
    offset:   [n_leaves+1] start of each leaf in ``ids``
    plen:     [n_leaves, K] prefix length (bits) of each dimension
    prefix:   [n_leaves, K] prefix value of each dimension
    """
    ids: np.ndarray
    offset: np.ndarray
    plen: np.ndarray
    prefix: np.ndarray

    @property
    def n_leaves(self) -> int:
        return len(self.offset) - 1

    def box(self, bits: int):
        """Code range [lo, hi] of every leaf in every dimension."""
        shift = bits - self.plen.astype(np.int64)
        lo = self.prefix.astype(np.int64) << shift
        hi = ((self.prefix.astype(np.int64) + 1) << shift) - 1
        return lo, hi


def build_tree(codes: np.ndarray, n_regions: int, max_size: int) -> Tree:
    """Alg. 3 with the split rule of Sec. 4.2, bulk-loaded (reading R3).

    codes is uint8 [n, K] (one projected space). The root has 2^K first-layer
    nodes, one per vector of the K most significant code bits (dimension 0 is
    the most significant bit of the node key). A node holding more than
    max_size points is split on the dimension whose next bit divides it most
    evenly, bit-0 child first.
    """
    codes = np.asarray(codes, dtype=np.int64)
    n, K = codes.shape
    bits = int(round(math.log2(n_regions)))
    assert 1 << bits == n_regions
    leaves_ids: List[np.ndarray] = []
    leaves_plen: List[np.ndarray] = []
    leaves_prefix: List[np.ndarray] = []

    def split(members: np.ndarray, plen: np.ndarray, prefix: np.ndarray):
        count = len(members)
        splittable = np.nonzero(plen < bits)[0]
        if count <= max_size or len(splittable) == 0:
            leaves_ids.append(members)
            leaves_plen.append(plen.copy())
            leaves_prefix.append(prefix.copy())
            return
        best_j, best_gap, best_bit = -1, None, None
        for j in splittable:
            nb = (codes[members, j] >> (bits - 1 - plen[j])) & 1
            ones = int(nb.sum())
            gap = abs(2 * ones - count)
            if best_gap is None or gap < best_gap:
                best_j, best_gap, best_bit = j, gap, nb
        for bit in (0, 1):
            child = members[best_bit == bit]
            if len(child) == 0:
                continue
            cplen = plen.copy()
            cprefix = prefix.copy()
            cplen[best_j] += 1
            cprefix[best_j] = prefix[best_j] * 2 + bit
            split(child, cplen, cprefix)

    msb = (codes >> (bits - 1)) & 1
    key = np.zeros(n, dtype=np.int64)
    for j in range(K):
        key = key * 2 + msb[:, j]
    order = np.argsort(key, kind="stable")
    skey = key[order]
    starts = np.nonzero(np.r_[True, skey[1:] != skey[:-1]])[0]
    ends = np.r_[starts[1:], n]
    for s, e in zip(starts, ends):
        members = order[s:e]
        plen = np.ones(K, dtype=np.int64)
        prefix = msb[members[0]].astype(np.int64)
        split(members, plen, prefix)

    offset = np.zeros(len(leaves_ids) + 1, dtype=np.int64)
    offset[1:] = np.cumsum([len(x) for x in leaves_ids])
    ids = np.concatenate(leaves_ids) if leaves_ids else np.zeros(0, np.int64)
    return Tree(ids=ids.astype(np.int64), offset=offset,
                plen=np.array(leaves_plen, dtype=np.int64).reshape(-1, K),
                prefix=np.array(leaves_prefix, dtype=np.int64).reshape(-1, K))


@dataclass
class Index:
    """Everything the query phase reads: data, hash vectors, breakpoints, L trees."""
    X: np.ndarray
    A: np.ndarray
    E: np.ndarray          # FP64 [L*K, N_r+1]
    trees: List[Tree]
    K: int
    L: int
    n_regions: int
    P: Optional[np.ndarray] = None       # FP64 projections [n, L*K] (kept for tests)
    codes: Optional[np.ndarray] = None   # uint8 [n, L*K]
    max_size: int = 0                    # max_size of Alg. 3
    reduction: str = "hash"              # "hash": Eq. 1 with A; "paa": DET-ONLY's segment means

    @property
    def n(self) -> int:
        return self.X.shape[0]

    def project(self, X) -> np.ndarray:
        """The projected points the index encodes (FP64 [m, L*K])."""
        if self.reduction == "paa":
            return paa_reduce(X, self.K)
        return project(self.A, X)


def build_index(X, A, sample, K: int, L: int, n_regions: int, max_size: int) -> Index:
    """Encoding phase (Alg. 1, Alg. 2) followed by the indexing phase (Alg. 3)."""
    X = np.asarray(X)
    A = np.asarray(A)
    sample = np.asarray(sample, dtype=np.int64)
    P = project(A, X)
    E = select_breakpoints(P[sample], n_regions)
    codes = encode(P, E)
    trees = [build_tree(codes[:, i * K:(i + 1) * K], n_regions, max_size) for i in range(L)]
    return Index(X=X, A=A, E=E, trees=trees, K=K, L=L, n_regions=n_regions, P=P, codes=codes, max_size=max_size)


def build_index_det_only(X, sample, K: int, n_regions: int, max_size: int) -> Index:
    """DET-ONLY (Sec. 6.1): the encoding and indexing phases of DET-LSH with
    one projected space (L = 1) given by the PAA reduction of the points
    instead of Gaussian projections."""
    X = np.asarray(X)
    sample = np.asarray(sample, dtype=np.int64)
    P = paa_reduce(X, K)
    E = select_breakpoints(P[sample], n_regions)
    codes = encode(P, E)
    trees = [build_tree(codes, n_regions, max_size)]
    return Index(X=X, A=np.zeros((K, X.shape[1])), E=E, trees=trees, K=K, L=1, n_regions=n_regions, P=P,
                 codes=codes, max_size=max_size, reduction="paa")


def index_from_codes(X, A, E, codes, K: int, L: int, n_regions: int, max_size: int) -> Index:
    """The indexing phase (Alg. 3, reading R3) over given breakpoints E
    [L*K, N_r+1] and region codes [n, L*K], e.g. those another implementation
    computed from its own FP32 projections. With the projected queries passed
    to c2k_ann as well (its qp32 argument), the query phase then runs on
    exactly that implementation's FP32 inputs: the FP32-mirror form of the
    oracle."""
    codes = np.asarray(codes, dtype=np.uint8)
    trees = [build_tree(codes[:, i * K:(i + 1) * K], n_regions, max_size) for i in range(L)]
    return Index(X=np.asarray(X), A=np.asarray(A), E=np.asarray(E, dtype=np.float64), trees=trees, K=K, L=L,
                 n_regions=n_regions, codes=codes, max_size=max_size)


def insert_points(index: Index, X_new) -> Index:
    """Insertion of new points (ids n, n+1, ...) into an index (reading R14):
    their codes by Alg. 2 against the index's breakpoints (Alg. 1 is not run
    again), then the DE-Trees of all points as Alg. 3 builds them under
    reading R3 (bulk-loaded, so the result does not depend on the order in
    which points arrive)."""
    X_new = np.asarray(X_new)
    X = np.concatenate([index.X, X_new.astype(index.X.dtype)], axis=0)
    P = np.concatenate([index.P, index.project(X_new)], axis=0)
    codes = np.concatenate([index.codes, encode(P[index.n:], index.E)], axis=0)
    K, L = index.K, index.L
    trees = [build_tree(codes[:, i * K:(i + 1) * K], index.n_regions, index.max_size) for i in range(L)]
    return Index(X=X, A=index.A, E=index.E, trees=trees, K=K, L=L, n_regions=index.n_regions, P=P, codes=codes,
                 max_size=index.max_size)


# ---------------------------------------------------------------- query phase
def leaf_lb2_fp32(qp32: np.ndarray, E32: np.ndarray, lo: np.ndarray, hi: np.ndarray,
                  n_regions: int) -> np.ndarray:
    """Squared lower-bound distance between q' and each leaf box (Alg. 5, first step).

    For one projected space: qp32 [K] fp32, E32 [K, N_r+1] fp32 breakpoints,
    lo/hi [n_leaves, K] code ranges. A leaf covers [e_lo, e_{hi+1}) in every
    dimension, with e_0 = -inf and e_{N_r} = +inf (reading R4). Per dimension
    delta = max(e_lo - x, x - e_{hi+1}, 0) in FP32; the squares are added in
    FP32 in dimension order 0..K-1 (the decision precision of the GPU path).
    """
    nl, K = lo.shape
    acc = np.zeros(nl, dtype=np.float32)
    inf = np.float32(np.inf)
    for j in range(K):
        x = np.float32(qp32[j])
        el = np.where(lo[:, j] == 0, -inf, E32[j, lo[:, j]]).astype(np.float32)
        eh = np.where(hi[:, j] == n_regions - 1, inf,
                      E32[j, np.minimum(hi[:, j] + 1, n_regions)]).astype(np.float32)
        a = (el - x).astype(np.float32)
        b = (x - eh).astype(np.float32)
        delta = np.maximum(np.maximum(a, b), np.float32(0.0))
        sq = (delta * delta).astype(np.float32)
        acc = (acc + sq).astype(np.float32)
    return acc


def round_thresholds(r_min: float, c: float, eps: float):
    """Per-round thresholds of Alg. 7 (r <- c*r), reading R6.

    Returns (thr_proj, thr_exact): FP32 arrays of length ROUND_CAP holding
    (eps*r_t)^2 and (c*r_t)^2.
    """
    thr_p = np.empty(ROUND_CAP, dtype=np.float32)
    thr_c = np.empty(ROUND_CAP, dtype=np.float32)
    r = float(r_min)
    c = float(np.float32(c))
    with np.errstate(over="ignore"):
        for t in range(ROUND_CAP):
            if t == ROUND_CAP - 1:
                thr_p[t] = np.inf
                thr_c[t] = np.inf
                break
            er = eps * r
            cr = c * r
            thr_p[t] = np.float32(er * er)
            thr_c[t] = np.float32(cr * cr)
            r = r * c
    return thr_p, thr_c


@dataclass
class QueryResult:
    ids: np.ndarray          # int64 [k], -1 padded
    dist: np.ndarray         # FP64 [k] Euclidean distance, +inf padded
    n_cand: int              # |S| at termination
    rounds: int              # rounds started (t* + 1)
    stop: int                # 1: |S| >= beta n + k; 2: >= k within c r; 3: all leaves active
    cand: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))  # sorted S
    tie_band: bool = False   # some tested distance lay within tie_rel of its round's (c r)^2


def c2k_ann(index: Index, q: np.ndarray, k: int, c: float, r_min: float, eps: float,
            beta: float, keep_candidates: bool = False, qp32: Optional[np.ndarray] = None,
            tie_rel: float = 0.0) -> QueryResult:
    """Alg. 7 (c^2-k-ANN) with the optimised range query of Sec. 6.2.2 (readings R5-R7).

    qp32 (FP32 [L*K]) replaces the projected query H(q) (FP64, rounded to FP32
    for the lower bounds) by given values: with index_from_codes this is the
    FP32-mirror form. tie_rel > 0 flags the query (``tie_band``) when, in a
    round whose ">= k within c*r" test ran, some candidate's FP64 squared
    distance lies within tie_rel (relative) of (c*r_t)^2, where an FP32
    distance could decide that test the other way.
    """
    X = index.X
    n = X.shape[0]
    K, L, Nr = index.K, index.L, index.n_regions
    bits = int(round(math.log2(Nr)))
    T = math.ceil(float(beta) * float(n) + float(k))

    q64 = np.asarray(q, dtype=np.float64)
    if qp32 is None:
        qp = index.project(q64[None, :])[0]              # Alg. 7: H_i(q), hoisted out of the loop
        qp32 = qp.astype(np.float32)
    qp32 = np.asarray(qp32, dtype=np.float32)
    E32 = index.E.astype(np.float32)

    lb2 = []
    for i, tree in enumerate(index.trees):
        lo, hi = tree.box(bits)
        lb2.append(leaf_lb2_fp32(qp32[i * K:(i + 1) * K], E32[i * K:(i + 1) * K], lo, hi, Nr))

    if r_min <= 0:                                       # reading R7
        pos = [x[x > 0] for x in lb2]
        pos = np.concatenate(pos) if pos else np.zeros(0, np.float32)
        r_min = math.sqrt(float(pos.min())) / eps if pos.size else 1.0
    thr_p, thr_c = round_thresholds(r_min, c, eps)

    # first round in which each leaf's lower bound is covered
    first_round = [np.searchsorted(thr_p, x, side="left") for x in lb2]

    in_S = np.zeros(n, dtype=bool)
    tie_band = False
    S_order: List[np.ndarray] = []
    dist2_of = {}
    n_S = 0
    stop = 0
    t = 0
    for t in range(ROUND_CAP):
        for i, tree in enumerate(index.trees):
            new_leaves = np.nonzero(first_round[i] == t)[0]
            order = np.lexsort((new_leaves, lb2[i][new_leaves]))
            for leaf in new_leaves[order]:
                pts = tree.ids[tree.offset[leaf]:tree.offset[leaf + 1]]
                fresh = pts[~in_S[pts]]
                in_S[fresh] = True
                if len(fresh):
                    S_order.append(fresh)
                    diff = X[fresh].astype(np.float64) - q64[None, :]
                    d2 = np.einsum("ij,ij->i", diff, diff)
                    for o, v in zip(fresh.tolist(), d2.tolist()):
                        dist2_of[o] = v
                n_S += len(fresh)
                if n_S >= T:
                    stop = 1
                    break
            if stop:
                break
        if stop:
            break
        thr = float(thr_c[t])
        within = sum(1 for v in dist2_of.values() if v <= thr)
        if tie_rel > 0 and any(abs(v - thr) <= tie_rel * thr for v in dist2_of.values()):
            tie_band = True
        if within >= k:
            stop = 2
            break
        if all((fr <= t).all() for fr in first_round):
            stop = 3
            break

    cand = np.concatenate(S_order) if S_order else np.zeros(0, np.int64)
    d2 = np.array([dist2_of[o] for o in cand.tolist()], dtype=np.float64)
    order = np.lexsort((cand, d2))[:k]
    ids = np.full(k, -1, dtype=np.int64)
    dist = np.full(k, np.inf, dtype=np.float64)
    ids[:len(order)] = cand[order]
    dist[:len(order)] = np.sqrt(d2[order])
    return QueryResult(ids=ids, dist=dist, n_cand=int(n_S), rounds=t + 1, stop=stop,
                       cand=np.sort(cand) if keep_candidates else np.zeros(0, np.int64), tie_band=tie_band)


# ---------------------------------------------------------------- exact range query and (r,c)-ANN
def leaf_bounds2(index: Index, i: int, qp: np.ndarray):
    """Squared lower and upper bound distances (FP64) between the projected
    query qp [K] and every leaf box of tree i (the bounds Alg. 4 asks for).

    A leaf covers [e_lo, e_{hi+1}] in every dimension, with the outermost
    edges -inf / +inf (reading R4, and R11 for the upper bound: a box that
    reaches an outer region has an infinite upper bound, so its points are
    always checked one by one). Per dimension the lower bound takes
    max(e_lo - x, x - e_{hi+1}, 0) and the upper bound max(|x - e_lo|,
    |x - e_{hi+1}|); both are squared and summed.
    """
    K, Nr = index.K, index.n_regions
    t = index.trees[i]
    lo, hi = t.box(int(round(math.log2(Nr))))
    lb2 = np.zeros(t.n_leaves)
    ub2 = np.zeros(t.n_leaves)
    for j in range(K):
        e = index.E[i * K + j]
        x = float(qp[j])
        el = np.where(lo[:, j] == 0, -np.inf, e[lo[:, j]])
        eh = np.where(hi[:, j] == Nr - 1, np.inf, e[np.minimum(hi[:, j] + 1, Nr)])
        delta = np.maximum(np.maximum(el - x, x - eh), 0.0)
        far = np.maximum(np.abs(x - el), np.abs(x - eh))
        lb2 += delta * delta
        ub2 += far * far
    return lb2, ub2


def det_range_query(index: Index, i: int, qp: np.ndarray, r_proj: float, stats: Optional[dict] = None):
    """Alg. 4 (DET range query) with Alg. 5 (traverse subtree) in tree i: the
    ids of the points whose projection lies within r_proj of qp, ascending.

    A leaf whose lower bound exceeds r_proj is skipped; a leaf whose upper
    bound is at most r_proj gives all its points; any other leaf gives the
    points whose projected distance is at most r_proj. An internal node's box
    contains its leaves' boxes, so its lower bound is not above theirs and
    pruning it never drops a leaf the leaf test keeps: visiting the leaves
    one by one gives the same set as the recursion. Distances are compared
    squared (FP64). stats, if given, counts the leaves of each kind.
    """
    K = index.K
    t = index.trees[i]
    lb2, ub2 = leaf_bounds2(index, i, qp)
    r2 = float(r_proj) * float(r_proj)
    P = index.P[:, i * K:(i + 1) * K]
    out = []
    n_skip = n_all = n_ref = 0
    for leaf in range(t.n_leaves):
        members = t.ids[t.offset[leaf]:t.offset[leaf + 1]]
        if lb2[leaf] > r2:
            n_skip += 1
        elif ub2[leaf] <= r2:
            n_all += 1
            out.append(members)
        else:
            n_ref += 1
            diff = P[members] - np.asarray(qp, dtype=np.float64)[None, :]
            d2 = np.einsum("ij,ij->i", diff, diff)
            out.append(members[d2 <= r2])
    if stats is not None:
        stats.update(skipped=n_skip, accepted=n_all, refined=n_ref)
    return np.sort(np.concatenate(out)) if out else np.zeros(0, np.int64)


@dataclass
class RCResult:
    id: int                  # the returned point, or -1 (nothing returned)
    dist: float              # its distance to q (+inf when nothing is returned)
    n_cand: int              # |S| when the query ended
    trees: int               # trees range-queried
    stop: int                # 1: |S| >= beta n + 1; 2: a point of S within c r; 0: nothing returned


def rc_ann(index: Index, q: np.ndarray, r: float, c: float, eps: float, beta: float) -> RCResult:
    """Alg. 6, the (r,c)-ANN query: range-query the trees in order with the
    projected radius eps*r, adding each result to S; once |S| >= beta*n + 1
    (reading R13: the real-valued bound) return the point of S closest to q;
    after all L trees return it if some point of S lies within c*r of q, else
    nothing. Closest by (distance, id), distances in FP64.
    """
    q = np.asarray(q, dtype=np.float64)
    K = index.K
    S = np.zeros(0, np.int64)
    bound = beta * index.n + 1.0

    def closest(ids):
        diff = np.asarray(index.X, dtype=np.float64)[ids] - q[None, :]
        d2 = np.einsum("ij,ij->i", diff, diff)
        o = np.lexsort((ids, d2))[0]
        return int(ids[o]), float(np.sqrt(d2[o]))

    for i in range(index.L):
        qp = project(index.A[i * K:(i + 1) * K], q[None, :])[0]
        S = np.union1d(S, det_range_query(index, i, qp, eps * r))
        if len(S) >= bound:
            o, dist = closest(S)
            return RCResult(id=o, dist=dist, n_cand=len(S), trees=i + 1, stop=1)
    if len(S):
        o, dist = closest(S)
        if dist <= c * r:
            return RCResult(id=o, dist=dist, n_cand=len(S), trees=index.L, stop=2)
    return RCResult(id=-1, dist=math.inf, n_cand=len(S), trees=index.L, stop=0)


# ---------------------------------------------------------------- evaluation measures
def exact_knn(X: np.ndarray, q: np.ndarray, k: int):
    """The exact k nearest points o*_1..o*_k of Def. 2 by a full scan (FP64), ties by id."""
    diff = np.asarray(X, dtype=np.float64) - np.asarray(q, dtype=np.float64)[None, :]
    d2 = np.einsum("ij,ij->i", diff, diff)
    order = np.lexsort((np.arange(len(d2)), d2))[:k]
    return order.astype(np.int64), np.sqrt(d2[order])


def recall(result_ids: np.ndarray, exact_ids: np.ndarray) -> float:
    """Sec. 6.1: |R intersect R*| / k."""
    k = len(exact_ids)
    return len(set(int(x) for x in result_ids if x >= 0) & set(int(x) for x in exact_ids)) / k


def overall_ratio(result_dist: np.ndarray, exact_dist: np.ndarray) -> float:
    """Sec. 6.1: (1/k) sum_i ||q,o_i|| / ||q,o*_i||, both lists ascending."""
    rd = np.sort(np.asarray(result_dist, dtype=np.float64))
    ed = np.sort(np.asarray(exact_dist, dtype=np.float64))
    ratios = []
    for a, b in zip(rd, ed):
        if b == 0.0:
            ratios.append(1.0 if a == 0.0 else np.inf)
        else:
            ratios.append(a / b)
    return float(np.mean(ratios))
