"""ctypes binding of libdetlsh (include/detlsh.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: torch tensors supply pointers (all CPU -> host memory,
all CUDA -> device memory on torch's current stream) and receive the outputs.
If the library has not been built, loading it raises; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

from .build_lib import LIB

F32, U8 = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
BORROW_X = 1
DEDUP_POS = 2
EXPORT = {"A": 0, "EDGES": 1, "CODES": 2, "LEAF_IDS": 3, "LEAF_BASE": 4, "LEAF_RANGE": 5,
          "LEAF_PLEN": 6, "LEAF_PREFIX": 7, "SAMPLE_PROJ": 8, "SAMPLE_IDS": 9}
_EXPORT_DTYPE = {"A": torch.float32, "EDGES": torch.float32, "CODES": torch.uint8,
                 "LEAF_IDS": torch.int32, "LEAF_BASE": torch.int64, "LEAF_RANGE": torch.int32,
                 "LEAF_PLEN": torch.uint8, "LEAF_PREFIX": torch.uint8, "SAMPLE_PROJ": torch.float32,
                 "SAMPLE_IDS": torch.int64}

# every symbol declared in include/detlsh.h
SYMBOLS = ("detlsh_build", "detlsh_query", "detlsh_free", "detlsh_export_size", "detlsh_export",
           "detlsh_info", "detlsh_project", "detlsh_encode_values", "detlsh_select_breakpoints",
           "detlsh_eps_lemma3", "detlsh_strerror", "detlsh_last_error", "detlsh_trace_enable",
           "detlsh_trace_get", "detlsh_launch_count", "detlsh_select_breakpoints_noalloc",
           "detlsh_plan_create", "detlsh_plan_query", "detlsh_plan_status", "detlsh_plan_info",
           "detlsh_plan_destroy", "detlsh_autotune", "detlsh_server_create", "detlsh_server_submit",
           "detlsh_server_poll", "detlsh_server_replay", "detlsh_server_stats", "detlsh_server_destroy",
           "detlsh_rc_ann", "detlsh_insert", "detlsh_memory_stats", "detlsh_draw_hashes",
           "detlsh_draw_sample", "detlsh_test_set_wait_limit_ns", "detlsh_check_status")
PENDING, EADMIT = 1, -5
PLAN_GRAPH = 1
TRACE_KEYS = ("sample_proj_ms", "breakpoints_ms", "encode_ms", "leaves_ms", "query_proj_ms", "lb_ms",
              "dist_ms", "dist_launches", "lb_launches", "build_ms", "query_ms", "walk_ms", "finalize_ms",
              "bucket_ms", "leaf_root_ms", "leaf_gather_ms", "leaf_levels_ms", "leaf_iterations", "group_ms")


class DetlshError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("L", ctypes.c_int32), ("n_regions", ctypes.c_int32),
                ("max_leaf", ctypes.c_int32), ("sample_size", ctypes.c_int64), ("proj_mode", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("walk_ctas_per_sm", ctypes.c_int32),
                ("dist_rows", ctypes.c_int32), ("dist_ctas_per_sm", ctypes.c_int32),
                ("shortlist", ctypes.c_int32), ("streams", ctypes.c_int32), ("coarse_gather", ctypes.c_int32),
                ("id_bucket_log2", ctypes.c_int32)]

    def as_dict(self):
        return {"batch": self.batch, "walk_ctas_per_sm": self.walk_ctas_per_sm, "dist_rows": self.dist_rows,
                "dist_ctas_per_sm": self.dist_ctas_per_sm, "shortlist": self.shortlist, "streams": self.streams,
                "coarse_gather": self.coarse_gather, "id_bucket_log2": self.id_bucket_log2}


def _tuning(t) -> Optional[Tuning]:
    if t is None or isinstance(t, Tuning):
        return t
    return Tuning(batch=t.get("batch", 0), walk_ctas_per_sm=t.get("walk_ctas_per_sm", 0),
                  dist_rows=t.get("dist_rows", 0), dist_ctas_per_sm=t.get("dist_ctas_per_sm", 0),
                  shortlist=t.get("shortlist", 0), streams=t.get("streams", 0),
                  coarse_gather=t.get("coarse_gather", 0), id_bucket_log2=t.get("id_bucket_log2", 0))


class ServerConfig(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("slots", ctypes.c_int32), ("pipelines", ctypes.c_int32),
                ("queue_cap", ctypes.c_int32), ("max_delay_us", ctypes.c_int32), ("shortlist", ctypes.c_int32),
                ("eps", ctypes.c_double), ("beta", ctypes.c_double), ("mem_budget", ctypes.c_int64),
                ("tuning", ctypes.POINTER(Tuning)), ("test_fail_batch", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class QueryParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("beta", ctypes.c_double),
                ("cand_ids", ctypes.c_void_p), ("cand_cap", ctypes.c_int64),
                ("shortlist", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tuning", ctypes.POINTER(Tuning)), ("qproj", ctypes.c_void_p)]


_lib = None


def lib(path: Optional[str] = None):
    """Load libdetlsh.so (raises if it is missing). With DETLSH_CHECKED=1 in the
    environment the checked build (device index checks) is built if needed and
    loaded instead."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if path is None and os.environ.get("DETLSH_CHECKED") == "1":
        from .build_lib import build as _build
        p = _build(checked=True)
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.detlsh_build.argtypes = [vp, i64, i32, i32, vp, vp, ctypes.POINTER(Params), i32, vp,
                               ctypes.POINTER(vp)]
    L.detlsh_build.restype = ctypes.c_int
    L.detlsh_query.argtypes = [vp, vp, i64, i32, vp, vp, vp, i32, ctypes.POINTER(QueryParams), vp,
                               vp, vp, i32, vp]
    L.detlsh_query.restype = ctypes.c_int
    L.detlsh_free.argtypes = [vp]
    L.detlsh_free.restype = None
    L.detlsh_export_size.argtypes = [vp, i32]
    L.detlsh_export_size.restype = i64
    L.detlsh_export.argtypes = [vp, i32, vp, i64, i32, vp]
    L.detlsh_export.restype = ctypes.c_int
    L.detlsh_info.argtypes = [vp, ctypes.POINTER(i64), i32]
    L.detlsh_info.restype = ctypes.c_int
    L.detlsh_project.argtypes = [vp, i64, i32, i32, vp, i32, vp, i32, vp]
    L.detlsh_project.restype = ctypes.c_int
    L.detlsh_encode_values.argtypes = [vp, i64, i32, vp, i32, vp, i32, vp]
    L.detlsh_encode_values.restype = ctypes.c_int
    L.detlsh_select_breakpoints.argtypes = [vp, i64, i32, i32, vp, i32, vp]
    L.detlsh_select_breakpoints.restype = ctypes.c_int
    L.detlsh_eps_lemma3.argtypes = [i32, i32]
    L.detlsh_eps_lemma3.restype = dbl
    L.detlsh_strerror.argtypes = [ctypes.c_int]
    L.detlsh_strerror.restype = ctypes.c_char_p
    L.detlsh_last_error.argtypes = []
    L.detlsh_last_error.restype = ctypes.c_char_p
    L.detlsh_trace_enable.argtypes = [i32]
    L.detlsh_trace_enable.restype = ctypes.c_int
    L.detlsh_trace_get.argtypes = [ctypes.POINTER(dbl), i32]
    L.detlsh_trace_get.restype = ctypes.c_int
    L.detlsh_launch_count.argtypes = []
    L.detlsh_launch_count.restype = i64
    L.detlsh_check_status.argtypes = [ctypes.POINTER(ctypes.c_uint32), i32]
    L.detlsh_check_status.restype = ctypes.c_int
    L.detlsh_rc_ann.argtypes = [vp, vp, i64, i32, vp, vp, dbl, dbl, vp, vp, vp, vp]
    L.detlsh_rc_ann.restype = ctypes.c_int
    L.detlsh_insert.argtypes = [vp, vp, i64, i32, i32, vp]
    L.detlsh_insert.restype = ctypes.c_int
    L.detlsh_draw_hashes.argtypes = [ctypes.c_uint64, i32, i32, vp]
    L.detlsh_draw_hashes.restype = ctypes.c_int
    L.detlsh_draw_sample.argtypes = [ctypes.c_uint64, i64, i64, vp]
    L.detlsh_draw_sample.restype = ctypes.c_int
    L.detlsh_test_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
    L.detlsh_test_set_wait_limit_ns.restype = ctypes.c_uint64
    L.detlsh_memory_stats.argtypes = [i32, ctypes.POINTER(i64), i32]
    L.detlsh_memory_stats.restype = ctypes.c_int
    L.detlsh_select_breakpoints_noalloc.argtypes = [vp, i64, i32, i32, vp, vp]
    L.detlsh_select_breakpoints_noalloc.restype = ctypes.c_int
    L.detlsh_plan_create.argtypes = [vp, i64, i32, ctypes.POINTER(QueryParams), i32, vp, ctypes.POINTER(vp)]
    L.detlsh_plan_create.restype = ctypes.c_int
    L.detlsh_plan_query.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, i32, vp]
    L.detlsh_plan_query.restype = ctypes.c_int
    L.detlsh_plan_status.argtypes = [vp, vp]
    L.detlsh_plan_status.restype = ctypes.c_int
    L.detlsh_plan_info.argtypes = [vp, ctypes.POINTER(i64)]
    L.detlsh_plan_info.restype = ctypes.c_int
    L.detlsh_plan_destroy.argtypes = [vp]
    L.detlsh_plan_destroy.restype = None
    L.detlsh_autotune.argtypes = [vp, vp, i64, i32, vp, vp, vp, i32, ctypes.POINTER(QueryParams), dbl, i32,
                                  vp, ctypes.POINTER(Tuning)]
    L.detlsh_autotune.restype = ctypes.c_int
    L.detlsh_server_create.argtypes = [vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.detlsh_server_create.restype = ctypes.c_int
    L.detlsh_server_submit.argtypes = [vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_uint64)]
    L.detlsh_server_submit.restype = ctypes.c_int
    L.detlsh_server_poll.argtypes = [vp, ctypes.c_uint64, i32, vp, vp, vp, ctypes.POINTER(dbl)]
    L.detlsh_server_poll.restype = ctypes.c_int
    L.detlsh_server_replay.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.detlsh_server_replay.restype = ctypes.c_int
    L.detlsh_server_stats.argtypes = [vp, ctypes.POINTER(i64)]
    L.detlsh_server_stats.restype = ctypes.c_int
    L.detlsh_server_destroy.argtypes = [vp]
    L.detlsh_server_destroy.restype = None
    if path is None:
        _lib = L
    return L


def _check(st: int, where: str):
    if st != 0:
        L = lib()
        raise DetlshError(st, where, f"{L.detlsh_strerror(st).decode()} -- {L.detlsh_last_error().decode()}")


def _mem_of(*ts):
    devs = {t.device.type for t in ts if t is not None}
    if len(devs) != 1:
        raise ValueError("all tensors of one call must be on the CPU or all on the GPU")
    return MEM_DEVICE if devs.pop() == "cuda" else MEM_HOST


def _stream(mem):
    if mem == MEM_DEVICE:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype_code(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.uint8:
        return U8
    raise TypeError(f"unsupported dtype {t.dtype}")


class Index:
    """Owner of a detlsh_index*; freed by ``free()`` or on garbage collection."""

    def __init__(self, handle: int, keep=None):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep      # a borrowed X must outlive the index

    def free(self):
        if self.handle:
            lib().detlsh_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        return detlsh_info(self)


PROJ_FP32, PROJ_BF16 = 0, 1


def detlsh_build(X: torch.Tensor, A: Optional[torch.Tensor], sample_ids: Optional[torch.Tensor], K: int, L: int,
                 n_regions: int, max_leaf: int, borrow: bool = False, proj_mode: int = 0,
                 dedup_pos: bool = False, seed: int = 0, sample_size: int = 0) -> Index:
    """A or sample_ids None: the library draws them from ``seed``
    (detlsh_draw_hashes / detlsh_draw_sample), the sample of ``sample_size``
    points (0: ceil(0.1 n))."""
    X = X.contiguous()
    A = A.contiguous().to(torch.float32) if A is not None else None
    sample_ids = sample_ids.contiguous().to(torch.int64) if sample_ids is not None else None
    mem = _mem_of(X, A, sample_ids)
    n_s = sample_ids.numel() if sample_ids is not None else int(sample_size)
    p = Params(K=K, L=L, n_regions=n_regions, max_leaf=max_leaf, sample_size=n_s, proj_mode=proj_mode,
               flags=(BORROW_X if (borrow and mem == MEM_DEVICE) else 0) | (DEDUP_POS if dedup_pos else 0),
               seed=int(seed) & 0xFFFFFFFFFFFFFFFF)
    out = ctypes.c_void_p(0)
    st = lib().detlsh_build(_ptr(X), X.shape[0], X.shape[1], _dtype_code(X), _ptr(A), _ptr(sample_ids),
                            ctypes.byref(p), mem, _stream(mem), ctypes.byref(out))
    _check(st, "detlsh_build")
    return Index(out.value, keep=X if p.flags & BORROW_X else None)


def _per_query(v, nq, dtype, dev):
    if not torch.is_tensor(v) or v.dim() == 0:
        return torch.as_tensor(v, dtype=dtype, device=dev).expand(nq).contiguous()
    return v.to(dev, dtype).contiguous()


def _query_args(Q, k, c, r_min):
    Q = Q.contiguous()
    nq, dev = Q.shape[0], Q.device
    k = _per_query(k, nq, torch.int32, dev)
    c = _per_query(c, nq, torch.float32, dev)
    r_min = _per_query(0.0 if r_min is None else r_min, nq, torch.float32, dev)
    return Q, k, c, r_min


def detlsh_insert(index: Index, X: torch.Tensor) -> None:
    """Add the rows of X (host or device, the index's dtype) as points
    n, n+1, ...: codes against the index's breakpoints, then the leaves of all
    points rebuilt (the index then owns a copy of every point)."""
    X = X.contiguous()
    mem = MEM_DEVICE if X.is_cuda else MEM_HOST
    st = lib().detlsh_insert(index.handle, _ptr(X), X.shape[0], _dtype_code(X), mem, _stream(mem))
    _check(st, "detlsh_insert")


def detlsh_rc_ann(index: Index, Q: torch.Tensor, r, c, eps: float, beta: float):
    """The (r,c)-ANN query of Alg. 6 (exact range query of Alg. 4/5 per tree,
    FP64). Q [nq, d] on the GPU in the index's dtype; r, c scalars or [nq].
    Returns (ids int64 [nq], -1 for nothing; distances float64 [nq];
    stats int32 [nq, 3]: |S|, trees queried, stop rule)."""
    Q = Q.contiguous()
    if not Q.is_cuda:
        raise DetlshError(-1, "detlsh_rc_ann", "takes device tensors")
    nq = Q.shape[0]
    dev = Q.device
    r = torch.as_tensor(r, dtype=torch.float32, device=dev).expand(nq).contiguous()
    c = torch.as_tensor(c, dtype=torch.float32, device=dev).expand(nq).contiguous()
    ids = torch.empty(nq, dtype=torch.int64, device=dev)
    dist = torch.empty(nq, dtype=torch.float64, device=dev)
    stats = torch.empty(nq, 3, dtype=torch.int32, device=dev)
    st = lib().detlsh_rc_ann(index.handle, _ptr(Q), nq, _dtype_code(Q), _ptr(r), _ptr(c), float(eps), float(beta),
                             _ptr(ids), _ptr(dist), _ptr(stats), _stream(MEM_DEVICE))
    _check(st, "detlsh_rc_ann")
    return ids, dist, stats


def detlsh_query(index: Index, Q: torch.Tensor, k, c, r_min=None, k_max: Optional[int] = None,
                 eps: float = 0.0, beta: float = 0.1, cand_cap: int = 0,
                 out=None, shortlist: int = 0, tuning=None, qproj: Optional[torch.Tensor] = None):
    """Returns (ids int64 [nq,k_max], dist fp32 [nq,k_max], stats int32 [nq,4], cand or None).

    ``k``, ``c``, ``r_min`` are per-query tensors (or scalars, broadcast).
    ``out`` optionally supplies preallocated (ids, dist, stats) tensors;
    ``tuning`` is a ``Tuning`` or a dict of its fields (launch shapes);
    ``qproj`` (fp32 [nq, L*K], on Q's device) receives the projected queries.
    """
    Q, k, c, r_min = _query_args(Q, k, c, r_min)
    nq, dev = Q.shape[0], Q.device
    if k_max is None:
        k_max = int(k.max().item()) if nq else 1
    mem = _mem_of(Q, k, c, r_min)
    tu = _tuning(tuning)
    if out is None:
        ids = torch.empty(nq, k_max, dtype=torch.int64, device=dev)
        dist = torch.empty(nq, k_max, dtype=torch.float32, device=dev)
        stats = torch.empty(nq, 4, dtype=torch.int32, device=dev)
    else:
        ids, dist, stats = out
    cand = torch.empty(nq, cand_cap, dtype=torch.int32, device=dev) if cand_cap > 0 else None
    qp = QueryParams(eps=eps, beta=beta, cand_ids=cand.data_ptr() if cand is not None else None,
                     cand_cap=cand_cap, shortlist=shortlist, reserved=0,
                     tuning=ctypes.pointer(tu) if tu is not None else None,
                     qproj=qproj.data_ptr() if qproj is not None else None)
    if qproj is not None and (qproj.device != dev or qproj.dtype != torch.float32 or not qproj.is_contiguous()):
        raise ValueError("qproj must be a contiguous fp32 tensor on the queries' device")
    st = lib().detlsh_query(index.handle, _ptr(Q), nq, _dtype_code(Q), _ptr(k), _ptr(c), _ptr(r_min),
                            k_max, ctypes.byref(qp), _ptr(ids), _ptr(dist), _ptr(stats), mem, _stream(mem))
    _check(st, "detlsh_query")
    return ids, dist, stats, cand


class Plan:
    """Owner of a detlsh_plan* (preallocated batch buffers, optional CUDA graph)."""

    def __init__(self, index: Index, nq_max: int, k_max: int, eps: float = 0.0, beta: float = 0.1,
                 shortlist: int = 0, tuning=None, graph: bool = True):
        self.index = index          # the plan refers to the index
        self.k_max = k_max
        self._tuning = _tuning(tuning)
        qp = QueryParams(eps=eps, beta=beta, cand_ids=None, cand_cap=0, shortlist=shortlist, reserved=0,
                         tuning=ctypes.pointer(self._tuning) if self._tuning is not None else None)
        out = ctypes.c_void_p(0)
        st = lib().detlsh_plan_create(index.handle, nq_max, k_max, ctypes.byref(qp), PLAN_GRAPH if graph else 0,
                                      _stream(MEM_DEVICE), ctypes.byref(out))
        _check(st, "detlsh_plan_create")
        self.handle = ctypes.c_void_p(out.value)

    def destroy(self):
        if self.handle:
            lib().detlsh_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def info(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        _check(lib().detlsh_plan_info(self.handle, out), "detlsh_plan_info")
        return {"batch": out[0], "scratch_bytes": out[1], "graph_launches": out[2], "batches": out[3],
                "graph_kernels": out[4]}


def detlsh_plan_query(plan: Plan, Q: torch.Tensor, k, c, r_min=None, out=None):
    """Returns (ids, dist, stats) like detlsh_query, through the plan."""
    Q, k, c, r_min = _query_args(Q, k, c, r_min)
    nq, dev = Q.shape[0], Q.device
    mem = _mem_of(Q, k, c, r_min)
    if out is None:
        ids = torch.empty(nq, plan.k_max, dtype=torch.int64, device=dev)
        dist = torch.empty(nq, plan.k_max, dtype=torch.float32, device=dev)
        stats = torch.empty(nq, 4, dtype=torch.int32, device=dev)
    else:
        ids, dist, stats = out
    st = lib().detlsh_plan_query(plan.handle, _ptr(Q), nq, _ptr(k), _ptr(c), _ptr(r_min), _ptr(ids), _ptr(dist),
                                 _ptr(stats), mem, _stream(mem))
    _check(st, "detlsh_plan_query")
    return ids, dist, stats


def detlsh_plan_status(plan: Plan) -> int:
    """Synchronizes torch's current stream; returns the plan's status code."""
    return lib().detlsh_plan_status(plan.handle, _stream(MEM_DEVICE))


def detlsh_autotune(index: Index, Q: torch.Tensor, k, c, r_min=None, k_max: Optional[int] = None,
                    eps: float = 0.0, beta: float = 0.1, shortlist: int = 0, min_agreement: float = 0.0,
                    tuning=None) -> dict:
    """Launch shapes (and, for a BF16 index, a shortlist) timed on the sample Q."""
    Q, k, c, r_min = _query_args(Q, k, c, r_min)
    if k_max is None:
        k_max = int(k.max().item())
    mem = _mem_of(Q, k, c, r_min)
    tu = _tuning(tuning)
    qp = QueryParams(eps=eps, beta=beta, cand_ids=None, cand_cap=0, shortlist=shortlist, reserved=0,
                     tuning=ctypes.pointer(tu) if tu is not None else None)
    res = Tuning()
    st = lib().detlsh_autotune(index.handle, _ptr(Q), Q.shape[0], _dtype_code(Q), _ptr(k), _ptr(c), _ptr(r_min),
                               k_max, ctypes.byref(qp), float(min_agreement), mem, _stream(mem), ctypes.byref(res))
    _check(st, "detlsh_autotune")
    return res.as_dict()


class Server:
    """Owner of a detlsh_server* (continuous batching over a resident index).

    Queries and results live in host memory (CPU tensors)."""

    def __init__(self, index: Index, k_max: int, slots: int = 0, pipelines: int = 0, queue_cap: int = 0,
                 max_delay_us: int = 0, eps: float = 0.0, beta: float = 0.1, shortlist: int = 0,
                 mem_budget: int = 0, tuning=None, test_fail_batch: int = 0):
        self.index = index
        self.k_max = k_max
        self._tuning = _tuning(tuning)
        cfg = ServerConfig(k_max=k_max, slots=slots, pipelines=pipelines, queue_cap=queue_cap,
                           max_delay_us=max_delay_us, shortlist=shortlist, eps=eps, beta=beta,
                           mem_budget=mem_budget,
                           tuning=ctypes.pointer(self._tuning) if self._tuning is not None else None,
                           test_fail_batch=test_fail_batch, reserved=0)
        out = ctypes.c_void_p(0)
        _check(lib().detlsh_server_create(index.handle, ctypes.byref(cfg), ctypes.byref(out)),
               "detlsh_server_create")
        self.handle = ctypes.c_void_p(out.value)

    def submit(self, q: torch.Tensor, k: int, c: float, r_min: float = 0.0) -> int:
        """Queues one query (a CPU tensor of d values); returns its ticket.
        Raises DetlshError (status EADMIT when every slot is in use)."""
        q = q.contiguous()
        if q.device.type != "cpu":
            raise ValueError("server queries are host tensors")
        t = ctypes.c_uint64(0)
        _check(lib().detlsh_server_submit(self.handle, _ptr(q), int(k), float(c), float(r_min), ctypes.byref(t)),
               "detlsh_server_submit")
        return t.value

    def poll(self, ticket: int, wait_us: int = 0):
        """(status, ids, dist, stats, latency_us); ids/dist/stats are None unless status is 0."""
        ids = torch.empty(self.k_max, dtype=torch.int64)
        dist = torch.empty(self.k_max, dtype=torch.float32)
        stats = torch.empty(4, dtype=torch.int32)
        lat = ctypes.c_double(0.0)
        st = lib().detlsh_server_poll(self.handle, ctypes.c_uint64(ticket), int(wait_us), _ptr(ids), _ptr(dist),
                                      _ptr(stats), ctypes.byref(lat))
        if st != 0:
            return st, None, None, None, (lat.value if st != PENDING else None)
        return st, ids, dist, stats, lat.value

    def replay(self, Q: torch.Tensor, k, c, r_min, arrival_us: torch.Tensor):
        """Open-loop load: returns (status, ids, dist, stats, latency_us) for all queries."""
        Q, k, c, r_min = _query_args(Q, k, c, r_min)
        nq = Q.shape[0]
        arr = arrival_us.to(torch.float64).contiguous()
        ids = torch.empty(nq, self.k_max, dtype=torch.int64)
        dist = torch.empty(nq, self.k_max, dtype=torch.float32)
        stats = torch.empty(nq, 4, dtype=torch.int32)
        lat = torch.empty(nq, dtype=torch.float64)
        st = lib().detlsh_server_replay(self.handle, _ptr(Q), nq, _ptr(k), _ptr(c), _ptr(r_min), _ptr(arr), _ptr(ids),
                                        _ptr(dist), _ptr(stats), _ptr(lat))
        return st, ids, dist, stats, lat

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 8)()
        _check(lib().detlsh_server_stats(self.handle, out), "detlsh_server_stats")
        keys = ("submitted", "completed", "rejected", "batches", "batched_queries", "max_batch", "errors", "slots")
        return dict(zip(keys, list(out)))

    def destroy(self):
        if self.handle:
            lib().detlsh_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def detlsh_export(index: Index, what: str, device="cpu") -> torch.Tensor:
    L = lib()
    code = EXPORT[what]
    nbytes = L.detlsh_export_size(index.handle, code)
    if nbytes < 0:
        _check(int(nbytes), "detlsh_export_size")
    dt = _EXPORT_DTYPE[what]
    out = torch.empty(nbytes // torch.empty(0, dtype=dt).element_size(), dtype=dt, device=device)
    mem = _mem_of(out)
    _check(L.detlsh_export(index.handle, code, _ptr(out), nbytes, mem, _stream(mem)), "detlsh_export")
    return out


def detlsh_info(index: Index) -> dict:
    buf = (ctypes.c_int64 * 10)()
    m = lib().detlsh_info(index.handle, buf, 10)
    if m < 0:
        _check(m, "detlsh_info")
    keys = ("n", "d", "dtype", "K", "L", "n_regions", "max_leaf", "n_s", "total_leaves", "largest_leaf")
    return {k: int(buf[i]) for i, k in enumerate(keys[:m])}


def detlsh_project(X: torch.Tensor, A: torch.Tensor) -> torch.Tensor:
    X = X.contiguous()
    A = A.contiguous().to(torch.float32)
    mem = _mem_of(X, A)
    P = torch.empty(X.shape[0], A.shape[0], dtype=torch.float32, device=X.device)
    _check(lib().detlsh_project(_ptr(X), X.shape[0], X.shape[1], _dtype_code(X), _ptr(A), A.shape[0],
                                _ptr(P), mem, _stream(mem)), "detlsh_project")
    return P


def detlsh_encode_values(P: torch.Tensor, E: torch.Tensor, n_regions: int) -> torch.Tensor:
    P = P.contiguous().to(torch.float32)
    E = E.contiguous().to(torch.float32)
    mem = _mem_of(P, E)
    codes = torch.empty(P.shape, dtype=torch.uint8, device=P.device)
    _check(lib().detlsh_encode_values(_ptr(P), P.shape[0], P.shape[1], _ptr(E), n_regions, _ptr(codes),
                                      mem, _stream(mem)), "detlsh_encode_values")
    return codes


def detlsh_select_breakpoints(Ps: torch.Tensor, n_regions: int) -> torch.Tensor:
    """Ps [LK, n_s] -> E [LK, n_regions+1]."""
    Ps = Ps.contiguous().to(torch.float32)
    mem = _mem_of(Ps)
    E = torch.empty(Ps.shape[0], n_regions + 1, dtype=torch.float32, device=Ps.device)
    _check(lib().detlsh_select_breakpoints(_ptr(Ps), Ps.shape[1], Ps.shape[0], n_regions, _ptr(E), mem,
                                           _stream(mem)), "detlsh_select_breakpoints")
    return E


def detlsh_select_breakpoints_noalloc(Ps: torch.Tensor, n_regions: int, E: torch.Tensor) -> None:
    """Same as detlsh_select_breakpoints into a preallocated device E, allocating
    nothing on the device (for callers that must not allocate); asynchronous on
    torch's current stream."""
    if Ps.device.type != "cuda" or E.device.type != "cuda":
        raise ValueError("detlsh_select_breakpoints_noalloc takes device tensors only")
    Ps = Ps.contiguous()
    _check(lib().detlsh_select_breakpoints_noalloc(_ptr(Ps), Ps.shape[1], Ps.shape[0], n_regions, _ptr(E),
                                                   _stream(MEM_DEVICE)), "detlsh_select_breakpoints_noalloc")


def detlsh_draw_hashes(seed: int, LK: int, d: int) -> torch.Tensor:
    """The library's hash vectors of Eq. 1 for ``seed`` (host, no GPU): fp32 [LK, d]."""
    A = torch.empty(LK, d, dtype=torch.float32)
    _check(lib().detlsh_draw_hashes(int(seed) & 0xFFFFFFFFFFFFFFFF, LK, d, _ptr(A)), "detlsh_draw_hashes")
    return A


def detlsh_draw_sample(seed: int, n: int, n_s: int) -> torch.Tensor:
    """The library's Alg. 1 sample for ``seed`` (host, no GPU): int64 [n_s], ascending."""
    ids = torch.empty(n_s, dtype=torch.int64)
    _check(lib().detlsh_draw_sample(int(seed) & 0xFFFFFFFFFFFFFFFF, n, n_s, _ptr(ids)), "detlsh_draw_sample")
    return ids


def detlsh_memory_stats(reset_peak: bool = False) -> dict:
    """Stream-ordered device memory in use (library pool, device default pool) and high-water marks."""
    out = (ctypes.c_int64 * 4)()
    m = lib().detlsh_memory_stats(1 if reset_peak else 0, out, 4)
    if m < 0:
        _check(m, "detlsh_memory_stats")
    return {"lib_used": out[0], "lib_peak": out[1], "default_used": out[2], "default_peak": out[3]}


def detlsh_eps_lemma3(K: int, L: int) -> float:
    return float(lib().detlsh_eps_lemma3(K, L))


def detlsh_trace_enable(on: bool) -> bool:
    return bool(lib().detlsh_trace_enable(1 if on else 0))


def detlsh_trace_get() -> dict:
    buf = (ctypes.c_double * len(TRACE_KEYS))()
    m = lib().detlsh_trace_get(buf, len(TRACE_KEYS))
    return {k: float(buf[i]) for i, k in enumerate(TRACE_KEYS[:m])}


def detlsh_launch_count() -> int:
    return int(lib().detlsh_launch_count())


def detlsh_check_status():
    """None for the normal build; for the checked build (failed checks since
    the last call, site of the first, its index), the record then cleared."""
    out = (ctypes.c_uint32 * 4)()
    r = lib().detlsh_check_status(out, 4)
    if r < 0:
        _check(r, "detlsh_check_status")
    if r == 0:
        return None
    return int(out[0]), int(out[1]), int(out[2]) | (int(out[3]) << 32)
