"""Host-side checks of the C ABI: the library loads and exports every entry
point include/detlsh.h declares; host-only logic (argument checks, the chi2
solver for eps) behaves. No GPU work is launched here."""

import ctypes
import math
import os
import re

import pytest

import paper_2406_10938_gb300 as pkg
from paper_2406_10938_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "detlsh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(detlsh_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return pkg.lib()


def test_header_declarations_match_binding():
    assert _declared() == sorted(binding.SYMBOLS)


def test_every_declared_symbol_is_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_normal_build_reports_no_device_checks(L):
    # the index checks exist only in the DETLSH_CHECKED build; the normal
    # library says so without touching a GPU
    import ctypes
    out = (ctypes.c_uint32 * 4)(7, 7, 7, 7)
    assert L.detlsh_check_status(out, 4) == 0
    assert list(out) == [7, 7, 7, 7]


def test_eps_solver_matches_scipy(L):
    from scipy.stats import chi2
    for K in (1, 2, 8, 16, 31, 32):
        for Lx in (1, 2, 4, 8):
            ref = math.sqrt(chi2.isf(math.exp(-1.0 / Lx), K))
            got = L.detlsh_eps_lemma3(K, Lx)
            assert abs(got - ref) <= 1e-9 * ref, (K, Lx, got, ref)
    assert L.detlsh_eps_lemma3(0, 4) < 0


def test_strerror_texts(L):
    for st in range(0, -7, -1):
        assert L.detlsh_strerror(st)


def test_build_rejects_bad_arguments_before_any_device_work(L):
    out = ctypes.c_void_p(0)
    x = (ctypes.c_float * 64)()
    a = (ctypes.c_float * 64)()
    ids = (ctypes.c_int64 * 4)(0, 1, 2, 3)
    bad = [dict(K=0), dict(K=17), dict(L=0), dict(n_regions=3), dict(n_regions=512),
           dict(max_leaf=0), dict(sample_size=2), dict(sample_size=-1), dict(proj_mode=7), dict(flags=4), dict(flags=-1)]
    for change in bad:
        p = dict(K=4, L=1, n_regions=4, max_leaf=4, sample_size=4, proj_mode=0, flags=0)
        p.update(change)
        st = L.detlsh_build(x, 16, 4, 0, a, ids, ctypes.byref(binding.Params(**p)), 0, None,
                            ctypes.byref(out))
        assert st == -1, change
        assert out.value is None
        assert L.detlsh_last_error()


def test_insert_and_rc_ann_reject_bad_arguments(L):
    assert L.detlsh_insert(None, None, 5, 0, 1, None) == -1
    assert L.detlsh_last_error()
    assert L.detlsh_rc_ann(None, None, 4, 0, None, None, 3.0, 0.1, None, None, None, None) == -1
    assert L.detlsh_last_error()


def test_query_rejects_null_index(L):
    st = L.detlsh_query(None, None, 0, 0, None, None, None, 1, None, None, None, None, 0, None)
    assert st == -1
