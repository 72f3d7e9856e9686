"""The no-allocation breakpoint entry point.

Some callers must not let the library allocate device memory (a fixed
footprint while serving, or their own allocator owning all of it); for them
detlsh_select_breakpoints_noalloc takes its temporary storage from a fixed
array inside the library. This checks, through the C ABI, that it returns
exactly what the allocating detlsh_select_breakpoints returns, on calls made
back to back (they share the fixed array), and that it refuses inputs larger
than that array serves. Collected last so a failure here stops a -x run only
after every other test has run.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2406_10938_gb300 as p
    return p


def _noalloc(L, Ps, n_regions, E):
    stream = torch.cuda.current_stream().cuda_stream
    return L.detlsh_select_breakpoints_noalloc(ctypes.c_void_p(Ps.data_ptr()), Ps.shape[1], Ps.shape[0],
                                               n_regions, ctypes.c_void_p(E.data_ptr()),
                                               ctypes.c_void_p(stream))


def _inputs(LK, n_s, seed):
    rng = np.random.default_rng(seed)
    Ps = rng.standard_normal((LK, n_s)).astype(np.float32)
    Ps[:, : n_s // 4] = np.round(Ps[:, : n_s // 4] * 8) / 8     # repeated values
    return torch.from_numpy(Ps).to("cuda:0")


def test_matches_allocating_entry_point_on_consecutive_calls(pkg):
    L = pkg.lib()
    cases = [(64, 4096, 256, 11), (17, 999, 16, 12), (64, 4096, 256, 13)]
    outs, refs = [], []
    for LK, n_s, Nr, seed in cases:        # back to back, sharing the fixed scratch
        Ps = _inputs(LK, n_s, seed)
        E = torch.full((LK, Nr + 1), float("nan"), device="cuda:0")
        assert _noalloc(L, Ps, Nr, E) == 0, L.detlsh_last_error()
        outs.append(E)
        refs.append(pkg.detlsh_select_breakpoints(Ps, Nr))
    torch.cuda.synchronize()
    for E, ref in zip(outs, refs):
        assert torch.equal(E, ref)         # the selection is exact: zero tolerance


def test_rejects_inputs_beyond_the_fixed_scratch(pkg):
    L = pkg.lib()
    Ps = torch.zeros(64, 4097, device="cuda:0")   # 64*4097 > DETLSH_NOALLOC_MAX_ITEMS
    E = torch.empty(64, 257, device="cuda:0")
    assert _noalloc(L, Ps, 256, E) == -1
    assert b"exceeds" in L.detlsh_last_error()
