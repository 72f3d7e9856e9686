"""The no-allocation breakpoint entry point.

Some callers must not let the library allocate device memory (a fixed
footprint while serving, or their own allocator owning all of it); for them
detlsh_select_breakpoints_noalloc takes its temporary storage from a fixed
array inside the library. This checks, through the C ABI, that it returns
exactly what the allocating detlsh_select_breakpoints returns, on calls made
back to back (they share the fixed array); that those calls raise neither the
library pool's nor the device pool's high-water mark (while the allocating
entry point does raise the library pool's); that it refuses inputs larger
than the fixed array serves; and that it refuses a host buffer before any
device work. Collected last so a failure here stops a -x run only after every
other test has run.
"""

import ctypes
import gc

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


def _pool_stats(L, reset):
    out = (ctypes.c_int64 * 4)()
    assert L.detlsh_memory_stats(1 if reset else 0, out, 4) == 4, L.detlsh_last_error()
    return list(out)


def _inputs(LK, n_s, seed):
    rng = np.random.default_rng(seed)
    Ps = rng.standard_normal((LK, n_s)).astype(np.float32)
    Ps[:, : n_s // 4] = np.round(Ps[:, : n_s // 4] * 8) / 8     # repeated values
    return torch.from_numpy(Ps).to("cuda:0")


def test_matches_allocating_entry_point_on_consecutive_calls(pkg):
    L = pkg.lib()
    cases = [(64, 4096, 256, 11), (17, 999, 16, 12), (64, 4096, 256, 13)]
    ins = [(_inputs(LK, n_s, seed), Nr) for LK, n_s, Nr, seed in cases]
    outs = [torch.full((Ps.shape[0], Nr + 1), float("nan"), device="cuda:0") for Ps, Nr in ins]
    # first call on the device (looks up the fixed array), then measure
    assert _noalloc(L, ins[0][0], ins[0][1], outs[0]) == 0, L.detlsh_last_error()
    # tensors of earlier tests held in reference cycles are freed now, not
    # during the measurement
    gc.collect()
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    before = _pool_stats(L, reset=True)
    for (Ps, Nr), E in zip(ins, outs):     # back to back, sharing the fixed scratch
        assert _noalloc(L, Ps, Nr, E) == 0, L.detlsh_last_error()
    torch.cuda.synchronize()
    after = _pool_stats(L, reset=False)
    assert after[1] == before[0], "the library pool's high-water mark rose: something was allocated"
    assert after[3] == before[2], "the device pool's high-water mark rose: something was allocated"
    assert torch.cuda.memory_allocated() == torch_before
    refs = [pkg.detlsh_select_breakpoints(Ps, Nr) for Ps, Nr in ins]
    torch.cuda.synchronize()
    # the measurement sees allocations: the allocating entry point raised the peak
    assert _pool_stats(L, reset=False)[1] > before[0]
    for E, ref in zip(outs, refs):
        assert torch.equal(E, ref)         # the selection is exact: zero tolerance


def test_rejects_inputs_beyond_the_fixed_scratch(pkg):
    L = pkg.lib()
    Ps = torch.zeros(64, 4097, device="cuda:0")   # 64*4097 > DETLSH_NOALLOC_MAX_ITEMS
    E = torch.empty(64, 257, device="cuda:0")
    assert _noalloc(L, Ps, 256, E) == -1
    assert b"exceeds" in L.detlsh_last_error()


def test_rejects_host_buffers_before_device_work(pkg):
    L = pkg.lib()
    Ps = np.zeros((16, 512), dtype=np.float32)
    E = np.zeros((16, 17), dtype=np.float32)
    st = L.detlsh_select_breakpoints_noalloc(Ps.ctypes.data_as(ctypes.c_void_p), 512, 16, 16,
                                             E.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(0))
    assert st == -1
    assert b"device" in L.detlsh_last_error()
    # a later successful call clears the message
    Pd = _inputs(16, 512, 3)
    Ed = torch.empty(16, 17, device="cuda:0")
    assert _noalloc(L, Pd, 16, Ed) == 0
    assert L.detlsh_last_error() == b""
