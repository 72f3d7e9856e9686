"""GB300 (sm_103a) implementation of DET-LSH's encode/index/query hot path.

The computation lives in ``libdetlsh.so`` (CUDA kernels behind the C ABI of
``include/detlsh.h``); ``binding`` exposes the same entry points to Python.
"""

from .binding import (  # noqa: F401
    DetlshError,
    Index,
    Plan,
    Server,
    Tuning,
    detlsh_autotune,
    detlsh_plan_query,
    detlsh_plan_status,
    detlsh_build,
    detlsh_check_status,
    detlsh_draw_hashes,
    detlsh_draw_sample,
    detlsh_memory_stats,
    detlsh_encode_values,
    detlsh_eps_lemma3,
    detlsh_export,
    detlsh_info,
    detlsh_insert,
    detlsh_launch_count,
    detlsh_project,
    detlsh_query,
    detlsh_rc_ann,
    detlsh_select_breakpoints,
    detlsh_trace_enable,
    detlsh_trace_get,
    lib,
)
from .build_lib import LIB, build  # noqa: F401
