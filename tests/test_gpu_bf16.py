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
