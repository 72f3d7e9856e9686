"""The failure path of the bounded device waits, exercised without a fault.

Every mbarrier wait of the tensor-core projection kernel is bounded; when one
runs out the kernel sets an error word, winds down (the copies it issued
land, its MMAs complete, its tensor memory is freed) and returns, and the
call reports DETLSH_ETIMEOUT. A test-only entry point shortens the limit to
zero, so that the first wait that cannot succeed at once (the MMA issuer
waiting for the first tile's copy) runs out; the context stays usable and
the next call, with the limit restored, gives the normal result.
"""

import pytest
import torch

import paper_2406_10938_gb300 as pkg
from parity_helpers import DEV
from workloads import gaussian_projection, make_workload, sample_ids

pytestmark = pytest.mark.gpu
ETIMEOUT = -4


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    return pkg.lib()


@pytest.mark.parametrize("name,d,proj_mode", [("tiny", 32, 0), ("serving", 128, 0), ("mid", 128, 1)])
def test_wait_that_runs_out_reports_etimeout_and_the_next_call_succeeds(L, name, d, proj_mode):
    n, K, Lt, Nr, n_s, max_leaf = 200_000, 16, 4, 16, 2_000, 256
    X, _ = make_workload(name, n=n, nq=1, d=d)
    A = gaussian_projection(Lt, K, d)
    ids = sample_ids(n, n_s)
    Xd, Ad, idd = X.to(DEV), A.to(DEV), ids.to(DEV)
    ref = pkg.detlsh_build(Xd, Ad, idd, K, Lt, Nr, max_leaf, proj_mode=proj_mode)
    codes_ref = pkg.detlsh_export(ref, "CODES")
    ref.free()
    prev = L.detlsh_test_set_wait_limit_ns(0)
    try:
        with pytest.raises(pkg.DetlshError) as e:
            pkg.detlsh_build(Xd, Ad, idd, K, Lt, Nr, max_leaf, proj_mode=proj_mode)
        assert e.value.status == ETIMEOUT
        assert b"ran out" in L.detlsh_last_error()
    finally:
        assert L.detlsh_test_set_wait_limit_ns(prev) == 0
    torch.cuda.synchronize()          # the context is still usable
    again = pkg.detlsh_build(Xd, Ad, idd, K, Lt, Nr, max_leaf, proj_mode=proj_mode)
    assert torch.equal(pkg.detlsh_export(again, "CODES"), codes_ref)
    again.free()
