"""Seeded synthetic workloads shaped like the paper's experiments (Sec. 6.1).

The paper measures on real datasets (Table 2: Msong, Deep1M, Sift10M/100M, ...)
that are not available here; these Gaussian-mixture stand-ins take their
shapes instead:

* ``tiny``      n=1e4, d=32,  10 clusters, centres N(0,4I), points centre+N(0,I), fp32
* ``mid``       n=1e6, d=128, 1000 clusters, integer values 0..255 stored as fp32
                (Sift-like): centres clip(N(64,48^2)), points round(clip(centre+N(0,20^2)))
* ``precision`` n=1e6, d=960, 500 anisotropic clusters: centres N(0,I), per-cluster
                per-dimension sigma log-uniform in [0.1, 1]
* ``batching``  n=1e7, d=96, 10,000 clusters on the unit sphere (Deep-like):
                centres normalise(N(0,I)), points normalise(centre + 0.5 N(0,I)/sqrt(d))
* ``serving``   n=1e8, d=128, as ``mid`` but stored as uint8

Queries are fresh draws from the same mixture (same centres, another seed),
the synthetic counterpart of the paper's held-out queries (Sec. 6.1).

``exact=True`` returns a variant on a dyadic grid (``tiny``: multiples of 1/4;
``precision``: multiples of 1/8 clipped to +-63/8; ``batching``: multiples of
1/256, which keeps |x| <= 1) so that every FP32 sum and product of the method
is exact with hash vectors from ``gaussian_projection(exact=True)`` (N(0,1)
draws on a 1/16 grid, at most 7 significant bits): at d = 960 a projection
is at most 960 * 127 * 63 < 2^24 units of 2^-7 and a squared distance at
most 960 * 126^2 < 2^24 units of 2^-6; at d = 96 a squared distance between
points of norm about 1 is at most about 4 * 2^16 units of 2^-16. BF16 holds
every such value. ``mid``/``serving`` are integer-valued already.

Generation uses ``torch.Generator`` on the requested device; the same seed
gives different numbers on CPU and CUDA, so a test that compares two sides
always hands both the same tensors.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import torch


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    nq: int
    dtype: str          # "f32" or "u8"
    K: int = 16
    L: int = 4
    n_regions: int = 256
    sample_size: int = 0    # n_s
    c: float = 1.5
    k: int = 50
    beta: float = 0.1
    max_leaf: int = 256


WORKLOADS = {
    "tiny": Workload("tiny", 10_000, 32, 100, "f32", n_regions=16,
                     sample_size=1_000, c=1.5, k=10),
    "mid": Workload("mid", 1_000_000, 128, 10_000, "f32",
                    sample_size=10_000, c=1.5, k=50),
    "precision": Workload("precision", 1_000_000, 960, 10_000, "f32",
                          sample_size=10_000, c=1.5, k=100),
    "batching": Workload("batching", 10_000_000, 96, 100_000, "f32",
                         sample_size=100_000, c=1.5, k=100),
    "serving": Workload("serving", 100_000_000, 128, 100_000, "u8",
                        sample_size=1_000_000, c=1.5, k=10),
}


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _mixture_params(name: str, d: int, seed: int, device):
    g = _gen(seed * 7919 + 17, device)
    if name == "tiny":
        m = 10
        centres = 2.0 * torch.randn(m, d, generator=g, device=device)
        return {"centres": centres}
    if name in ("mid", "serving"):
        m = 1000
        centres = (64.0 + 48.0 * torch.randn(m, d, generator=g, device=device)).clamp_(0, 255)
        return {"centres": centres}
    if name == "precision":
        m = 500
        centres = torch.randn(m, d, generator=g, device=device)
        u = torch.rand(m, d, generator=g, device=device)
        sigma = torch.exp(math.log(0.1) + u * (math.log(1.0) - math.log(0.1)))
        return {"centres": centres, "sigma": sigma}
    if name == "batching":
        m = 10_000
        centres = torch.randn(m, d, generator=g, device=device)
        centres = centres / centres.norm(dim=1, keepdim=True)
        return {"centres": centres}
    raise ValueError(f"unknown workload {name!r}")


def _draw(name: str, params, count: int, d: int, g: torch.Generator, device,
          chunk: int = 1 << 20):
    """Draw ``count`` mixture points (fp32 [count, d]) in chunks."""
    centres = params["centres"]
    m = centres.shape[0]
    out = torch.empty(count, d, dtype=torch.float32, device=device)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        lab = torch.randint(0, m, (e - s,), generator=g, device=device)
        z = torch.randn(e - s, d, generator=g, device=device)
        mu = centres[lab]
        if name == "tiny":
            x = mu + z
        elif name in ("mid", "serving"):
            x = (mu + 20.0 * z).clamp_(0, 255).round_()
        elif name == "precision":
            x = mu + params["sigma"][lab] * z
        elif name == "batching":
            x = mu + (0.5 / math.sqrt(d)) * z
            x = x / x.norm(dim=1, keepdim=True)
        else:
            raise ValueError(name)
        out[s:e] = x
    return out


def make_workload(name: str, n: Optional[int] = None, nq: Optional[int] = None,
                  seed_data: int = 1, seed_query: int = 2, device="cpu",
                  exact: bool = False, d: Optional[int] = None):
    """Return ``(X, Q)`` for a named workload (fp32 tensors, or uint8 for serving).

    ``n``/``nq``/``d`` override the configured sizes (smaller parity cases).
    Data and queries share the mixture's centres (seeded by ``seed_data``).
    """
    w = WORKLOADS[name]
    n = w.n if n is None else int(n)
    nq = w.nq if nq is None else int(nq)
    d = w.d if d is None else int(d)
    params = _mixture_params(name, d, seed_data, device)
    X = _draw(name, params, n, d, _gen(seed_data, device), device)
    Q = _draw(name, params, nq, d, _gen(seed_query, device), device)
    if exact:
        if name == "tiny":
            X = (X * 4.0).round_() / 4.0
            Q = (Q * 4.0).round_() / 4.0
        elif name == "precision":
            X = (X * 8.0).round_().clamp_(-63, 63) / 8.0
            Q = (Q * 8.0).round_().clamp_(-63, 63) / 8.0
        elif name == "batching":
            X = (X * 256.0).round_() / 256.0
            Q = (Q * 256.0).round_() / 256.0
        elif name not in ("mid", "serving"):
            raise ValueError(f"no exact-arithmetic variant of {name!r}")
    if w.dtype == "u8":
        X = X.to(torch.uint8)
        Q = Q.to(torch.uint8)
    return X, Q


def gaussian_projection(L: int, K: int, d: int, seed: int = 3, device="cpu",
                        exact: bool = False) -> torch.Tensor:
    """The L*K hash vectors of Eq. 1 as one fp32 matrix A [L*K, d], entries N(0,1).

    Row r = i*K + j holds a_ij, the j-th hash of the i-th projected space.
    ``exact=True`` rounds each draw to a multiple of 1/16 and clips it to
    +-127/16, so every entry has at most 7 significant bits.
    """
    g = _gen(seed, device)
    A = torch.randn(L * K, d, generator=g, device=device, dtype=torch.float32)
    if exact:
        A = ((A * 16.0).round_().clamp_(-127, 127)) / 16.0
    return A


def paa_projection(K: int, d: int, device="cpu") -> torch.Tensor:
    """The Piecewise Aggregate Approximation of DET-ONLY (the paper's single-tree
    baseline, Sec. 6.1) as a projection matrix [K, d]: row j averages the
    coordinates of segment j, w = floor(d/K) consecutive coordinates from j*w
    (the last d - K*w coordinates belong to no segment). Entries 1/w: exact
    in FP32 when w is a power of two."""
    if not 1 <= K <= d:
        raise ValueError("need 1 <= K <= d")
    w = d // K
    A = torch.zeros(K, d, dtype=torch.float32, device=device)
    for j in range(K):
        A[j, j * w:(j + 1) * w] = 1.0 / w
    return A


def sample_ids(n: int, n_s: int, seed: int = 3, device="cpu") -> torch.Tensor:
    """n_s distinct point ids drawn uniformly from [0, n), ascending (int64)."""
    if not 0 < n_s <= n:
        raise ValueError("need 0 < n_s <= n")
    g = _gen(seed * 31 + 5, device)
    ids = torch.randperm(n, generator=g, device=device)[:n_s]
    return torch.sort(ids).values


def query_params(name: str, nq: int, seed: int = 4, device="cpu"):
    """Per-query (k, c) arrays. ``batching`` mixes k ~ U[1,100] and c in {1.2,1.5,2.0}."""
    w = WORKLOADS[name]
    if name == "batching":
        g = _gen(seed, device)
        k = torch.randint(1, 101, (nq,), generator=g, device=device, dtype=torch.int64).to(torch.int32)
        cs = torch.tensor([1.2, 1.5, 2.0], device=device, dtype=torch.float32)
        c = cs[torch.randint(0, 3, (nq,), generator=g, device=device)]
        return k, c
    k = torch.full((nq,), w.k, dtype=torch.int32, device=device)
    c = torch.full((nq,), w.c, dtype=torch.float32, device=device)
    return k, c
