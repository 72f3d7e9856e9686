"""Benchmark of the DET-LSH hot path on GB300.

The headline step is the mid workload: build the index over n points already
resident in HBM (projection, breakpoints, encoding, DE-Tree leaves) and
answer a batch of c^2-k-ANN queries (Alg. 7) against it. The default run
also measures the other parts of the metric, each on its own workload and
reported under "workloads" of the same JSON line: serving (n = 1e8 uint8,
Poisson arrivals through the continuous-batching server: p50/p99 latency and
QPS at recall@10 >= 0.9), precision (d = 960: the BF16 tensor-core path
against the plain FP32 path at equal recall@100) and batching (n = 1e7,
100,000 mixed queries per step through a graph-captured plan).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload mid|batching|serving|precision] [--no-extra]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank runs an
independent replica on its own GPU with its own query batch (weak scaling);
the value is the queries of all ranks over the slowest rank's time.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "index Mpts/s; QPS@recall≥0.9 vs plain FP32 GPU; p99 latency; % HBM peak"
WORKLOAD = dict(name="mid", n=1_000_000, d=128, nq=10_000, K=16, L=4, n_regions=256, n_s=10_000,
                max_leaf=256, c=1.5, k=50, beta=0.1)


def workload_desc():
    if WORKLOAD.get("method") == "det-only":
        return ("mid, DET-ONLY: n=1,000,000 d=128 fp32 integer 0-255 Gaussian mixture of 1,000 clusters, "
                f"{WORKLOAD['nq']:,} queries from the same mixture; one DE-Tree over the PAA reduction "
                "(K=16 segment means of 8 coordinates), N_r=256 n_s=1% c=1.5 k=50 beta=0.1 max_leaf=256")
    return ("mid: n=1,000,000 d=128 fp32 integer 0-255 Gaussian mixture of 1,000 clusters, "
            f"{WORKLOAD['nq']:,} queries from the same mixture; K=16 L=4 N_r=256 n_s=1% c=1.5 k=50 "
            "beta=0.1 max_leaf=256")


def projection_for(w, device="cpu"):
    """The index's projection matrix: L*K Gaussian hash vectors (DET-LSH, Eq. 1),
    or the PAA segment means of DET-ONLY (L = 1)."""
    from workloads import gaussian_projection, paa_projection
    if w.get("method") == "det-only":
        return paa_projection(w["K"], w["d"], device=device)
    return gaussian_projection(w["L"], w["K"], w["d"], device=device)


def build_bytes_per_point(d, s_in, K, L):
    """Algorithmic bytes of the build per point: read the point, write its L*K
    codes, read them again to group the leaves, write L leaf-ordered ids."""
    return d * s_in + K * L + K * L + 4 * L


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _src_sha1(relpath):
    with open(os.path.join(ROOT, relpath), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def _ncu_traffic_per_unit(kernel, workload="mid"):
    """DRAM bytes per processed unit of `kernel` from its committed ncu summary,
    if the kernel's source file is unchanged since that capture; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_unit:"):
                _, val, _unit, src, sha = line.split()
                if _src_sha1(src) == sha:
                    return float(val)
    except (OSError, ValueError):
        pass
    return None


def gather_kernel(d, shortlist):
    """The distance kernel the library launches for FP32 rows of d coordinates."""
    if shortlist:
        return "k_dist_bf16"
    return "k_dist_g8" if d % 4 == 0 and d <= 128 else "k_dist"


def roofline_obj(kernel, algo_bytes_per_launch, avg_launch_ms, launches, traffic=None, source=None):
    peak, peak_kind = _peaks()
    achieved = algo_bytes_per_launch / (avg_launch_ms / 1000.0) / 1e9
    out = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
           "algorithmic_bytes_per_launch": algo_bytes_per_launch, "launches_per_step": launches,
           "avg_launch_ms": avg_launch_ms}
    if source:
        out["source"] = source
    return out


def tensor_roofline_obj(kernel, flops_per_launch, avg_launch_ms, launches, source=None):
    """A contraction on the tensor cores against the measured dense BF16 rate
    (the sustained figure: the kernel runs inside a long step)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        peak, kind = 1700.0, "fallback (sustained)"
    achieved = flops_per_launch / (avg_launch_ms / 1000.0) / 1e12
    out = {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "peak_kind": kind, "traffic": None,
           "algorithmic_flops_per_launch": flops_per_launch, "launches_per_step": launches,
           "avg_launch_ms": avg_launch_ms}
    if source:
        out["source"] = source
    return out


def build_roofline_obj(n, bytes_per_point, build_ms, phases=None):
    peak, peak_kind = _peaks()
    achieved = n * bytes_per_point / (build_ms / 1000.0) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_kind": peak_kind, "bytes_per_point": bytes_per_point, "build_ms": build_ms,
           "mpts_per_s": n / (build_ms / 1000.0) / 1e6}
    if phases:
        out["phase_ms"] = phases
    return out


# ------------------------------------------------------------------ replicas
def max_over_ranks(x, world, device="cpu"):
    """The largest x over the ranks (each replica's time; the job ends with the slowest)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed units_per_rank
    in at most `seconds` (weak scaling)."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_worker(spec):
    """Times the FP64 oracle as it stands on this host's cores (run in a child
    process with no GPU visible). spec: workload, number of queries, workers.

    workers == 1: the oracle's own build_index, then the queries one by one.
    workers > 1: the same oracle functions spread over the cores without
    changing their arithmetic: the projection in row blocks and the encoding
    in column blocks on threads, the L trees and the queries on forked
    processes (forked from this process, which never touches a GPU)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np

    from oracle import detlsh_oracle as O
    from workloads import gaussian_projection, make_workload, sample_ids

    w, nqs, workers, reps = spec["w"], int(spec["nqs"]), int(spec["workers"]), int(spec.get("reps", 1))
    det_only = w.get("method") == "det-only"
    X, Q = make_workload(w["name"], n=w["n"], nq=max(nqs, 1), seed_query=2)
    A = None if det_only else gaussian_projection(w["L"], w["K"], w["d"]).numpy()
    ids = sample_ids(w["n"], w["n_s"]).numpy()
    Xn, Qn = X.numpy(), Q.numpy()
    K, L, Nr, ml = w["K"], w["L"], w["n_regions"], w["max_leaf"]
    eps = O.eps_from_lemma3(K, L)
    runs = []
    for _ in range(reps):
        runs.append(_cpu_oracle_step(O, np, cf, mp, Xn, Qn, A, ids, w, nqs, workers, det_only, eps))
    return runs


def _cpu_oracle_step(O, np, cf, mp, Xn, Qn, A, ids, w, nqs, workers, det_only, eps):
    """One timed CPU step: a full index build, then nqs queries."""
    K, L, Nr, ml = w["K"], w["L"], w["n_regions"], w["max_leaf"]
    t0 = time.perf_counter()
    if workers == 1:
        idx = (O.build_index_det_only(Xn, ids, K, Nr, ml) if det_only
               else O.build_index(Xn, A, ids, K, L, Nr, ml))
    else:
        rows = np.array_split(np.arange(Xn.shape[0]), workers)
        with cf.ThreadPoolExecutor(workers) as ex:
            if det_only:
                P = np.concatenate(list(ex.map(lambda r: O.paa_reduce(Xn[r], K), rows)))
            else:
                P = np.concatenate(list(ex.map(lambda r: O.project(A, Xn[r]), rows)))
            E = O.select_breakpoints(P[ids], Nr)
            cols = np.array_split(np.arange(P.shape[1]), min(workers, P.shape[1]))
            codes = np.concatenate(list(ex.map(lambda c: O.encode(P[:, c], E[c]), cols)), axis=1)
        with mp.get_context("fork").Pool(min(workers, L)) as pool:
            trees = pool.starmap(O.build_tree, [(codes[:, i * K:(i + 1) * K], Nr, ml) for i in range(L)])
        idx = O.Index(X=Xn, A=(np.zeros((K, Xn.shape[1])) if det_only else A), E=E, trees=trees, K=K, L=L,
                      n_regions=Nr, P=P, codes=codes, max_size=ml, reduction="paa" if det_only else "hash")
    build_s = time.perf_counter() - t0
    global _CPU_IDX, _CPU_Q, _CPU_ARGS
    _CPU_IDX, _CPU_Q, _CPU_ARGS = idx, Qn, (w["k"], w["c"], eps, w["beta"])
    t0 = time.perf_counter()
    if workers == 1:
        for i in range(nqs):
            _cpu_query(i)
    else:
        with mp.get_context("fork").Pool(workers) as pool:
            pool.map(_cpu_query, range(nqs), chunksize=1)
    query_wall = time.perf_counter() - t0
    return {"build_s": build_s, "query_wall_s": query_wall, "queries": nqs, "workers": workers}


_CPU_IDX = _CPU_Q = _CPU_ARGS = None


def _cpu_query(i):
    from oracle import detlsh_oracle as O
    k, c, eps, beta = _CPU_ARGS
    O.c2k_ann(_CPU_IDX, _CPU_Q[i], k, c, 0.0, eps, beta)
    return i


def run_cpu_oracle(nqs, workers, reps=1):
    """reps timed CPU steps (a build and nqs queries each) in a child process."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    spec = json.dumps({"w": WORKLOAD, "nqs": nqs, "workers": workers, "reps": reps})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-oracle-worker", spec],
                       capture_output=True, text=True, env=env, timeout=1500)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_step_seconds(res, nq):
    """One step of the workload on the CPU: the build, plus nq queries at the
    measured wall time per query (queries run in parallel when workers > 1)."""
    return res["build_s"] + nq * res["query_wall_s"] / res["queries"]


def cpu_baseline_obj(all_core, single, nq):
    step = cpu_step_seconds(all_core, nq)
    out = {"value": nq / step, "unit": "queries/s", "cores": all_core["workers"], "kind": "oracle",
           "host_cores": os.cpu_count(),
           "sample": (f"FP64 oracle on {all_core['workers']} host cores: one full {WORKLOAD['n']:,}-point index "
                      f"build ({all_core['build_s']:.2f} s; projection and encoding on threads, the {WORKLOAD['L']} "
                      f"trees on processes) + {all_core['queries']} of the {nq:,} queries on processes "
                      f"({all_core['query_wall_s']:.2f} s wall); step time = build + {nq:,} x wall per query "
                      "(extrapolated)")}
    if single is not None:
        s1 = cpu_step_seconds(single, nq)
        out["single_thread"] = {
            "value": nq / s1, "unit": "queries/s", "cores": 1,
            "sample": (f"FP64 oracle, 1 thread: full index build ({single['build_s']:.2f} s) + "
                       f"{single['queries']} queries ({single['query_wall_s'] / single['queries']:.3f} s each); "
                       f"step time = build + {nq:,} x mean query (extrapolated)")}
    return out


def reference_arm(args, rank, world):
    """The oracle as the reference arm: each timed step is one full index build
    plus a bounded sample of the step's queries on all host cores, and the
    step time is extrapolated to the workload's query count (labelled)."""
    if rank != 0:
        return 0
    nq = WORKLOAD["nq"]
    workers = max(1, os.cpu_count() or 1)
    per_step_q = 2 * workers
    t_all = time.perf_counter()
    steps = run_cpu_oracle(per_step_q, workers, reps=args.steps)
    wall = time.perf_counter() - t_all
    step_s = statistics.mean(cpu_step_seconds(r, nq) for r in steps)
    value = nq / step_s
    cb = cpu_baseline_obj(steps[-1], None, nq)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": 0, "ms_per_step": step_s * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(), **WORKLOAD},
            "measured": {"steps_run": args.steps, "builds_timed": args.steps,
                         "queries_timed_per_step": per_step_q, "wall_s": wall,
                         "extrapolated": (f"each step's time = its measured build + {nq:,} x its measured wall "
                                          f"time per query over {per_step_q} queries"),
                         "warmup": "none: a CPU program needs no warm-up"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU helpers
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_steps(step, steps, warmup, world, dev, barrier):
    """Warm-up, then `steps` timed steps between a barrier and a synchronize
    on both sides (CUDA events on the current stream); ms per step (max over
    ranks) and the clocks seen during the timed region."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0).start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = _events()
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    return max_over_ranks(e0.elapsed_time(e1), world, dev) / steps, clk


def _recall_exact_topk(X, Q, ids_out, k, rows=200, chunk=8):
    """recall@k of ids_out against an exact FP32 scan of X (evaluation only)."""
    import torch
    nqr = min(rows, Q.shape[0])
    hits = 0
    for i0 in range(0, nqr, chunk):
        qs = Q[i0:min(nqr, i0 + chunk)].float()
        d = torch.cdist(qs, X.float() if X.dtype != torch.float32 else X,
                        compute_mode="donot_use_mm_for_euclid_dist")
        top = torch.topk(d, k, largest=False).indices.cpu()
        got = ids_out[i0:i0 + qs.shape[0]].cpu()
        for j in range(qs.shape[0]):
            hits += len(set(top[j].tolist()) & set(got[j, :k].tolist()))
    return hits / (nqr * k)


# ------------------------------------------------------------------ mid (headline)
def mid_leg(args, rank, world, local_rank, barrier):
    import torch

    import paper_2406_10938_gb300 as pkg
    from workloads import make_workload, sample_ids

    proj_mode = 1 if args.proj == "bf16" else 0
    dev = torch.device("cuda", local_rank)
    w = WORKLOAD
    X, Q = make_workload(w["name"], n=w["n"], nq=w["nq"], seed_query=2 + rank, device=dev)
    A = projection_for(w, device=dev)
    ids = sample_ids(w["n"], w["n_s"], device=dev)
    nq = w["nq"]
    kk = torch.full((nq,), w["k"], dtype=torch.int32, device=dev)
    cc = torch.full((nq,), w["c"], dtype=torch.float32, device=dev)
    rr = torch.zeros(nq, dtype=torch.float32, device=dev)
    eps = pkg.detlsh_eps_lemma3(w["K"], w["L"])
    out = (torch.empty(nq, w["k"], dtype=torch.int64, device=dev),
           torch.empty(nq, w["k"], dtype=torch.float32, device=dev),
           torch.empty(nq, 4, dtype=torch.int32, device=dev))
    traces = []

    def step():
        idx = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True,
                               proj_mode=proj_mode)
        pkg.detlsh_query(idx, Q, kk, cc, rr, k_max=w["k"], eps=eps, beta=w["beta"], out=out,
                         shortlist=args.shortlist)
        traces.append((pkg.detlsh_trace_get(), idx.info()))
        idx.free()

    pkg.detlsh_trace_enable(True)
    for _ in range(args.warmup):
        step()
    traces.clear()
    torch.cuda.synchronize()
    launches0 = pkg.detlsh_launch_count()
    ms_per_step, clk = _time_steps(step, args.steps, 0, world, dev, barrier)
    launches = pkg.detlsh_launch_count() - launches0
    value = job_throughput(nq, world, ms_per_step / 1000.0)

    ph = {k: statistics.mean(tr[k] for tr, _ in traces) for k in traces[0][0]}
    info = traces[-1][1]
    stats = out[2].cpu().numpy()
    n_cand = float(stats[:, 0].astype("float64").sum())
    s_in = 4
    total_leaves = info["total_leaves"]
    enc_bytes = w["n"] * (w["d"] * (2 if proj_mode else s_in) + w["K"] * w["L"])
    cand = {
        gather_kernel(w["d"], args.shortlist): (
            n_cand * (w["d"] * (2 if args.shortlist else s_in) + 4 + 4), ph["dist_ms"], ph["dist_launches"]),
        "k_walk": (nq * total_leaves * 4.0 + n_cand * 8, ph["walk_ms"], ph["dist_launches"]),
        "k_finalize": (n_cand * 8.0, ph["finalize_ms"], ph["dist_launches"]),
        ("k_project_tc" if proj_mode else "k_project_encode"): (enc_bytes, ph["encode_ms"], 1.0),
        "k_leaf_lb": (nq * total_leaves * 4.0 + ph["lb_launches"] * total_leaves * (2 * w["K"] + 10.0),
                      ph["lb_ms"], ph["lb_launches"]),
    }
    dom = max(cand, key=lambda k_: cand[k_][1])
    b, ms, nl = cand[dom]
    per_unit = _ncu_traffic_per_unit(dom.split("<")[0])
    traffic = per_unit * (n_cand / nl) if (per_unit is not None and dom in ("k_dist", "k_dist_g8")) else None
    roofline = roofline_obj(dom, b / nl, ms / nl, nl, traffic=traffic,
                            source="CUDA events around the kernel on the query's stream, timed steps")
    bpp = build_bytes_per_point(w["d"], s_in, w["K"], w["L"])
    build_roof = build_roofline_obj(w["n"], bpp, ph["build_ms"],
                                    {k_: round(ph[k_], 4) for k_ in ("sample_proj_ms", "breakpoints_ms",
                                                                     "encode_ms", "leaves_ms")})
    build_roof["encode_kernel"] = roofline_obj("k_project_tc (TF32 split)" if not proj_mode else "k_project_tc",
                                               enc_bytes, ph["encode_ms"], 1)
    recall = _recall_exact_topk(X, Q, out[0], w["k"])

    # the mixed-precision path on the same steps: BF16 tensor-core build, BF16
    # coarse candidate distances, FP32 re-rank of a shortlist autotuned on a
    # held-out query draw (seed 1000 + rank) that is never scored
    mixed = None
    if proj_mode == 0 and not args.no_mixed:
        pkg.detlsh_trace_enable(False)
        idx_m = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True, proj_mode=1)
        # as many held-out queries as the scored step: the tuned batch size
        # and stream count are chosen for this query count
        ns = nq
        _, Q_tune = make_workload(w["name"], n=1, nq=ns, seed_query=1000 + rank, device=dev)
        tune = pkg.detlsh_autotune(idx_m, Q_tune, kk[:ns], cc[:ns], rr[:ns], k_max=w["k"], eps=eps,
                                   beta=w["beta"], min_agreement=0.995)
        idx_m.free()
        sl = tune["shortlist"]
        out_m = (torch.empty_like(out[0]), torch.empty_like(out[1]), torch.empty_like(out[2]))

        def step_m():
            im = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True, proj_mode=1)
            pkg.detlsh_query(im, Q, kk, cc, rr, k_max=w["k"], eps=eps, beta=w["beta"], out=out_m, shortlist=sl,
                             tuning=tune)
            im.free()

        ms_m, clk_m = _time_steps(step_m, args.steps, args.warmup, world, dev, barrier)
        mixed = {"value": job_throughput(nq, world, ms_m / 1000.0), "unit": "queries/s", "ms_per_step": ms_m,
                 "recall_at_k": _recall_exact_topk(X, Q, out_m[0], w["k"]), "shortlist": sl, "tuning": tune,
                 "tuned_on": f"{ns} held-out queries (another draw of the mixture), not the scored ones",
                 "projection": "bf16 tcgen05 (FP32 accumulation)",
                 "distances": "bf16 coarse (FP32 accumulation), FP32 re-rank of the shortlist",
                 "vs_plain_fp32": (ms_per_step / ms_m), "clocks": clk_m}

    # end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 3))
    Xh = X.cpu().pin_memory()
    Qh = Q.cpu().pin_memory()
    Ah, idh = A.cpu().pin_memory(), ids.cpu().pin_memory()
    kh, ch, rh = kk.cpu(), cc.cpu(), rr.cpu()
    outh = (torch.empty(nq, w["k"], dtype=torch.int64).pin_memory(),
            torch.empty(nq, w["k"], dtype=torch.float32).pin_memory(),
            torch.empty(nq, 4, dtype=torch.int32).pin_memory())
    pkg.detlsh_trace_enable(False)

    def step_host():
        idx = pkg.detlsh_build(Xh, Ah, idh, w["K"], w["L"], w["n_regions"], w["max_leaf"], proj_mode=proj_mode)
        pkg.detlsh_query(idx, Qh, kh, ch, rh, k_max=w["k"], eps=eps, beta=w["beta"], out=outh,
                         shortlist=args.shortlist)
        idx.free()

    step_host()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    h2d = X.numel() * 4 + Q.numel() * 4 + A.numel() * 4 + ids.numel() * 8 + nq * 12
    d2h = nq * w["k"] * 12 + nq * 16

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            workers = max(1, os.cpu_count() or 1)
            cpu_base = cpu_baseline_obj(run_cpu_oracle(2 * workers, workers)[0],
                                        run_cpu_oracle(args.cpu_queries, 1)[0], nq)
        except Exception as e:  # reported, not fatal
            cpu_base = {"value": None, "error": str(e)[-300:]}

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(), **w, "projection": args.proj,
                       "shortlist": args.shortlist,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (X is 512 MB)"},
            "clocks": clk,
            "e2e": {"value": job_throughput(nq, world, e2e_s), "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "build_roofline": build_roof,
            "cpu_baseline": cpu_base,
            "build_mpts_per_s": w["n"] / (ph["build_ms"] / 1000.0) / 1e6,
            "query_qps": nq / (ph["query_ms"] / 1000.0),
            "recall_at_k": recall,
            "mixed_precision": mixed,
            "mean_candidates": n_cand / nq,
            "phase_ms": {k_: round(v, 4) for k_, v in ph.items()}}
    del X, Q, Xh, Qh
    torch.cuda.empty_cache()
    return line


# ------------------------------------------------------------------ batching workload
BATCHING = dict(name="batching", n=10_000_000, d=96, nq=100_000, K=16, L=4, n_regions=256, n_s=100_000,
                max_leaf=1024, beta=0.01, k_max=100)


def batching_desc():
    return ("batching: n=10,000,000 d=96 fp32 unit vectors, 10,000 clusters on the sphere (Deep-like), "
            f"{BATCHING['nq']:,} queries per step with k~U[1,100] and c in {{1.2,1.5,2.0}}; K=16 L=4 N_r=256 "
            "n_s=1% max_leaf=1024 beta=0.01 (recall@k >= 0.9); index built once before the timed steps")


def batching_leg(args, rank, world, local_rank, barrier, steps, warmup):
    """Query throughput on the batching workload through one of three routes:
    detlsh_query (per-call scratch, direct launches), a plan with direct
    launches, or a plan replaying its captured CUDA graph per batch."""
    import torch

    import paper_2406_10938_gb300 as pkg
    from workloads import gaussian_projection, make_workload, sample_ids

    dev = torch.device("cuda", local_rank)
    w = BATCHING
    nq, km = w["nq"], w["k_max"]
    X, Q = make_workload("batching", n=w["n"], nq=nq, seed_query=2 + rank, device=dev)
    A = gaussian_projection(w["L"], w["K"], w["d"], device=dev)
    ids = sample_ids(w["n"], w["n_s"], device=dev)
    g = torch.Generator().manual_seed(17 + rank)
    kk = torch.randint(1, km + 1, (nq,), generator=g, dtype=torch.int32).to(dev)
    cc = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)].to(dev)
    rr = torch.zeros(nq, dtype=torch.float32, device=dev)
    proj_mode = 1 if args.proj == "bf16" else 0
    pkg.detlsh_trace_enable(True)
    idx = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True,
                           proj_mode=proj_mode)
    idx.free()
    idx = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True,
                           proj_mode=proj_mode)
    trb = pkg.detlsh_trace_get()
    build_ms = trb["build_ms"]
    info = idx.info()
    out = (torch.empty(nq, km, dtype=torch.int64, device=dev), torch.empty(nq, km, dtype=torch.float32, device=dev),
           torch.empty(nq, 4, dtype=torch.int32, device=dev))
    plan = None
    if args.route != "query":
        plan = pkg.Plan(idx, nq_max=args.plan_batch, k_max=km, beta=w["beta"], shortlist=args.shortlist,
                        graph=args.route == "graph")

    def step():
        if plan is None:
            pkg.detlsh_query(idx, Q, kk, cc, rr, k_max=km, beta=w["beta"], out=out, shortlist=args.shortlist)
        else:
            pkg.detlsh_plan_query(plan, Q, kk, cc, rr, out=out)

    # phase times of the same batch through detlsh_query (graph replays cannot be traced per kernel)
    pkg.detlsh_query(idx, Q, kk, cc, rr, k_max=km, beta=w["beta"], out=out, shortlist=args.shortlist)
    ph = pkg.detlsh_trace_get()
    pkg.detlsh_trace_enable(False)
    l0 = pkg.detlsh_launch_count()
    g0 = plan.info()["graph_launches"] if plan is not None else 0
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    l0 = pkg.detlsh_launch_count()
    g0 = plan.info()["graph_launches"] if plan is not None else 0
    ms_per_step, clk = _time_steps(step, steps, 0, world, dev, barrier)
    launches = pkg.detlsh_launch_count() - l0
    if plan is not None:
        pi = plan.info()
        launches += (pi["graph_launches"] - g0) * pi["graph_kernels"]
    value = job_throughput(nq, world, ms_per_step / 1000.0)

    stats = out[2].cpu().numpy()
    n_cand = float(stats[:, 0].astype("float64").sum())
    # per-k recall on 400 sampled queries against an exact scan (untimed)
    sel = torch.linspace(0, nq - 1, 400).long()
    rec, kq_all = [], kk.cpu()
    for i0 in range(0, len(sel), 8):
        qs = sel[i0:i0 + 8]
        d = torch.cdist(Q[qs.to(dev)], X, compute_mode="donot_use_mm_for_euclid_dist")
        top = torch.topk(d, km, largest=False).indices.cpu()
        got = out[0][qs.to(dev)].cpu()
        for j, qi in enumerate(qs.tolist()):
            kq = int(kq_all[qi])
            rec.append((kq, len(set(top[j, :kq].tolist()) & set(got[j, :kq].tolist())) / kq))
    by_k = {}
    for lo, hi in ((1, 25), (26, 50), (51, 75), (76, 100)):
        v = [r for kq, r in rec if lo <= kq <= hi]
        by_k[f"k{lo}-{hi}"] = round(sum(v) / max(1, len(v)), 4)
    recall = sum(r for _, r in rec) / len(rec)

    dbytes = w["d"] * (2 if args.shortlist else 4) + 8
    cand = {gather_kernel(w["d"], args.shortlist): (n_cand * dbytes, ph["dist_ms"], ph["dist_launches"]),
            "k_walk": (nq * info["total_leaves"] * 4.0 + n_cand * 8, ph["walk_ms"], ph["dist_launches"]),
            "k_leaf_lb": (nq * info["total_leaves"] * 4.0, ph["lb_ms"], ph["lb_launches"])}
    dom = max(cand, key=lambda k_: cand[k_][1])
    b, ms, nl = cand[dom]
    roofline = roofline_obj(dom, b / nl, ms / nl, nl,
                            source="CUDA events around each kernel in a traced detlsh_query of the same batch")

    # end to end with host buffers through the same route
    Qh = Q.cpu().pin_memory()
    kh, ch, rh = kk.cpu(), cc.cpu(), rr.cpu()
    outh = (torch.empty(nq, km, dtype=torch.int64).pin_memory(), torch.empty(nq, km).pin_memory(),
            torch.empty(nq, 4, dtype=torch.int32).pin_memory())

    def step_host():
        if plan is None:
            pkg.detlsh_query(idx, Qh, kh, ch, rh, k_max=km, beta=w["beta"], out=outh, shortlist=args.shortlist)
        else:
            pkg.detlsh_plan_query(plan, Qh, kh, ch, rh, out=outh)

    step_host()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(steps, 3))
    for _ in range(e2e_steps):
        step_host()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if plan is not None:
        plan.destroy()
    idx.free()
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": batching_desc(), **w, "route": args.route, "plan_batch": args.plan_batch,
                       "projection": args.proj, "shortlist": args.shortlist,
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (X is 3.84 GB)"},
            "clocks": clk,
            "e2e": {"value": job_throughput(nq, world, max_over_ranks(e2e_s, world, dev)), "unit": "queries/s",
                    "h2d_bytes_per_step": nq * (w["d"] * 4 + 12),
                    "d2h_bytes_per_step": nq * (km * 12 + 16)},
            "gpu_launches": int(launches), "roofline": roofline,
            "build_roofline": build_roofline_obj(w["n"], build_bytes_per_point(w["d"], 4, w["K"], w["L"]), build_ms,
                                                 {k_: round(trb[k_], 4) for k_ in ("sample_proj_ms", "breakpoints_ms",
                                                                                   "encode_ms", "leaves_ms")}),
            "build_mpts_per_s": w["n"] / (build_ms / 1000.0) / 1e6, "recall_at_k": round(recall, 4),
            "recall_by_k": by_k, "mean_candidates": n_cand / nq,
            "phase_ms": {k_: round(v, 4) for k_, v in ph.items()}}
    del X, Q, Qh
    torch.cuda.empty_cache()
    return line


# ------------------------------------------------------------------ precision workload
PRECISION = dict(name="precision", n=1_000_000, d=960, nq=10_000, K=16, L=4, n_regions=256, n_s=10_000,
                 max_leaf=256, c=1.5, k=100, beta=0.1, shortlist=4096)


def precision_desc():
    return ("precision: n=1,000,000 d=960 fp32 Gaussian mixture of 500 anisotropic clusters (per-dimension "
            "sigma log-uniform in [0.1,1]), 10,000 queries; K=16 L=4 N_r=256 n_s=1% c=1.5 k=100 beta=0.1; "
            "FP32 path vs BF16 path (tcgen05 projection, BF16 coarse distances, FP32 re-rank of a 4,096 "
            "shortlist); recall@100 against an exact scan and distance error against FP64")


def precision_leg(args, rank, world, local_rank, barrier, steps, warmup):
    """Both paths on the precision workload: QPS (build + queries per step),
    recall@100 and the relative error of the returned distances against FP64."""
    import torch

    import paper_2406_10938_gb300 as pkg
    from workloads import gaussian_projection, make_workload, sample_ids

    dev = torch.device("cuda", local_rank)
    w = PRECISION
    n, d, nq, k = w["n"], w["d"], w["nq"], w["k"]
    X, Q = make_workload("precision", n=n, nq=nq, seed_query=2 + rank, device=dev)
    A = gaussian_projection(w["L"], w["K"], d, device=dev)
    ids = sample_ids(n, w["n_s"], device=dev)
    kk = torch.full((nq,), k, dtype=torch.int32, device=dev)
    cc = torch.full((nq,), w["c"], dtype=torch.float32, device=dev)
    rr = torch.zeros(nq, dtype=torch.float32, device=dev)
    eps = pkg.detlsh_eps_lemma3(w["K"], w["L"])
    # exact neighbours of sampled queries (FP32 scan without the matmul shortcut)
    nqr = 300
    sel = torch.linspace(0, nq - 1, nqr).long().to(dev)
    gt = []
    for i0 in range(0, nqr, 10):
        qs = Q[sel[i0:i0 + 10]]
        dd = torch.cdist(qs, X, compute_mode="donot_use_mm_for_euclid_dist")
        gt.append(torch.topk(dd, k, largest=False).indices)
    gt = torch.cat(gt)

    def run(proj_mode, shortlist):
        out = (torch.empty(nq, k, dtype=torch.int64, device=dev), torch.empty(nq, k, device=dev),
               torch.empty(nq, 4, dtype=torch.int32, device=dev))

        def step():
            idx = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True,
                                   proj_mode=proj_mode)
            pkg.detlsh_query(idx, Q, kk, cc, rr, k_max=k, eps=eps, beta=w["beta"], out=out, shortlist=shortlist)
            idx.free()

        pkg.detlsh_trace_enable(False)
        l0 = pkg.detlsh_launch_count()
        ms, clk = _time_steps(step, steps, warmup, world, dev, barrier)
        launches = (pkg.detlsh_launch_count() - l0) * steps / (steps + warmup)
        pkg.detlsh_trace_enable(True)
        step()
        ph = pkg.detlsh_trace_get()
        pkg.detlsh_trace_enable(False)
        got = out[0][sel]
        rec = sum(len(set(got[i].tolist()) & set(gt[i].tolist())) for i in range(nqr)) / (nqr * k)
        rows = got.reshape(-1)
        d64 = ((X[rows].double() - Q[sel].double().repeat_interleave(k, 0)) ** 2).sum(1).sqrt()
        g32 = out[1][sel].reshape(-1).double()
        rel = ((g32 - d64).abs() / d64.clamp_min(1e-30))
        n_cand = float(out[2][:, 0].double().sum())
        if shortlist:
            # the coarse distances by leaf on the tensor cores: the algorithmic
            # work is one d-long dot product (2d flops) per coarse candidate
            roof = tensor_roofline_obj(
                "k_dist_lm (BF16 tcgen05, by leaf chunk)", n_cand * 2.0 * d / ph["dist_launches"],
                ph["dist_ms"] / ph["dist_launches"], ph["dist_launches"],
                source="CUDA events around the coarse-distance stage (record sort + kernel) in a traced step")
        else:
            roof = roofline_obj("k_dist", n_cand * (4 * d + 8) / ph["dist_launches"],
                                ph["dist_ms"] / ph["dist_launches"], ph["dist_launches"],
                                source="CUDA events around the kernel in a traced step")
        bpp = build_bytes_per_point(d, 2 if proj_mode else 4, w["K"], w["L"])
        return {"qps": job_throughput(nq, world, ms / 1000.0), "ms_per_step": ms, "recall_at_100": rec,
                "dist_rel_err_max": float(rel.max()), "dist_rel_err_mean": float(rel.mean()),
                "mean_candidates": n_cand / nq, "clocks": clk, "roofline": roof, "gpu_launches": int(launches),
                "build_roofline": build_roofline_obj(n, bpp, ph["build_ms"]),
                "phase_ms": {k_: round(v, 4) for k_, v in ph.items()}}

    fp32 = run(0, 0)
    bf16 = run(1, w["shortlist"])
    line = {"metric": METRIC, "value": bf16["qps"], "unit": "queries/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": bf16["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 inputs, f32 accumulation, f32 re-rank",
            "data": "synthetic",
            "config": {"workload": precision_desc(), **w, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (X is 3.84 GB)"},
            "clocks": bf16["clocks"], "roofline": bf16["roofline"], "gpu_launches": bf16["gpu_launches"],
            "bf16_path": bf16, "fp32_path": fp32, "bf16_vs_fp32_qps": bf16["qps"] / fp32["qps"],
            "recall_sample": f"{nqr} queries, exact neighbours by an FP32 scan without the matmul shortcut",
            "e2e": None, "cpu_baseline": None}
    del X, Q
    torch.cuda.empty_cache()
    return line


# ------------------------------------------------------------------ serving workload
SERVING = dict(name="serving", n=100_000_000, d=128, nq=20_000, K=16, L=4, n_regions=256, n_s=1_000_000,
               max_leaf=1024, k_max=100, betas=(1e-3, 1.5e-3, 2e-3, 2.5e-3, 3e-3, 4e-3, 5e-3, 1e-2, 2e-2, 5e-2),
               rates=(5_000, 20_000, 50_000, 100_000, 200_000))


def serving_desc():
    return ("serving: n=100,000,000 d=128 uint8 Gaussian mixture of 1,000 clusters (12.8 GB, widened in the "
            "kernels), Poisson arrivals through the continuous-batching server, k in {1,10,100}, c in "
            "{1.2,1.5,2.0}; K=16 L=4 N_r=256 n_s=1% max_leaf=1024; beta = the smallest of "
            f"{SERVING['betas']} with recall@10 >= 0.9 on 200 queries")


def serving_leg(args, rank, world, local_rank, barrier):
    """Open-loop Poisson load through the server at several offered rates;
    value = the highest achieved throughput, with p50/p99 latency per rate."""
    import torch

    import paper_2406_10938_gb300 as pkg
    from workloads import gaussian_projection, make_workload, sample_ids

    dev = torch.device("cuda", local_rank)
    torch.backends.cuda.matmul.allow_tf32 = False
    w = SERVING
    n, d, nq, km = w["n"], w["d"], w["nq"], w["k_max"]
    X, Q = make_workload("serving", n=n, nq=nq, seed_query=2 + rank, device=dev)
    A = gaussian_projection(w["L"], w["K"], d, device=dev)
    ids = sample_ids(n, w["n_s"], device=dev)
    proj_mode = 1 if args.proj == "bf16" else 0
    pkg.detlsh_trace_enable(True)
    idx = pkg.detlsh_build(X, A, ids, w["K"], w["L"], w["n_regions"], w["max_leaf"], borrow=True,
                           proj_mode=proj_mode)
    trb = pkg.detlsh_trace_get()
    build_ms = trb["build_ms"]
    pkg.detlsh_trace_enable(False)
    # exact top-10 of 200 queries (integer data: FP32 GEMM distances are exact)
    nqr = 200
    Qf = Q[:nqr].float()
    qn = (Qf * Qf).sum(1, keepdim=True)
    best_d = torch.full((nqr, 10), float("inf"), device=dev)
    best_i = torch.zeros((nqr, 10), dtype=torch.int64, device=dev)
    for c0 in range(0, n, 10_000_000):
        Xc = X[c0:c0 + 10_000_000].float()
        dd = qn - 2 * Qf @ Xc.T + (Xc * Xc).sum(1)[None, :]
        v, i = torch.topk(dd, 10, largest=False)
        cd, ci = torch.cat([best_d, v], 1), torch.cat([best_i, i + c0], 1)
        o = torch.sort(cd, dim=1, stable=True).indices[:, :10]
        best_d, best_i = torch.gather(cd, 1, o), torch.gather(ci, 1, o)
        del Xc, dd
    gt = best_i.cpu()
    k10 = torch.full((nqr,), 10, dtype=torch.int32, device=dev)
    c15 = torch.full((nqr,), 1.5, device=dev)
    sweep, beta = [], None
    for b in w["betas"]:
        got = pkg.detlsh_query(idx, Q[:nqr], k10, c15, 0.0, k_max=10, beta=b, shortlist=args.shortlist)[0].cpu()
        rec = sum(len(set(got[i].tolist()) & set(gt[i].tolist())) for i in range(nqr)) / (10.0 * nqr)
        sweep.append({"beta": b, "recall_at_10": round(rec, 4)})
        if rec >= 0.9:
            beta = b
            break
    if beta is None:
        beta = w["betas"][-1]
    del Qf, qn
    torch.cuda.empty_cache()
    g = torch.Generator().manual_seed(23 + rank)
    kq = torch.tensor([1, 10, 100], dtype=torch.int32)[torch.randint(0, 3, (nq,), generator=g)]
    cq = torch.tensor([1.2, 1.5, 2.0])[torch.randint(0, 3, (nq,), generator=g)]
    # kernel roofline of a 2,048-query batch of the same mix (traced detlsh_query)
    nb = 2048
    pkg.detlsh_trace_enable(True)
    ob = pkg.detlsh_query(idx, Q[:nb], kq[:nb].to(dev), cq[:nb].to(dev), 0.0, k_max=km, beta=beta,
                          shortlist=args.shortlist)
    ph = pkg.detlsh_trace_get()
    pkg.detlsh_trace_enable(False)
    n_cand = float(ob[2][:, 0].double().sum())
    roofline = roofline_obj("k_dist_u8", n_cand * (d + 8) / ph["dist_launches"], ph["dist_ms"] / ph["dist_launches"],
                            ph["dist_launches"],
                            source="CUDA events around the kernel in a traced 2,048-query detlsh_query of the mix")
    Qh = Q.cpu()
    srv = pkg.Server(idx, k_max=km, pipelines=2, beta=beta, shortlist=args.shortlist, mem_budget=48 << 30,
                     max_delay_us=200)
    slots = srv.stats()["slots"]
    # warm-up: one pass at a moderate rate
    warm = min(nq, 2000)
    arr = torch.cumsum(torch.empty(warm, dtype=torch.float64).exponential_(20_000 / 1e6, generator=g), 0)
    srv.replay(Qh[:warm], kq[:warm], cq[:warm], 0.0, arr)
    rates = []
    l0 = pkg.detlsh_launch_count()
    clocks = ClockSampler(local_rank).start()
    for rate in w["rates"]:
        m = int(min(nq, max(2000, rate * 1.0)))
        arr = torch.cumsum(torch.empty(m, dtype=torch.float64).exponential_(rate / 1e6, generator=g), 0)
        b0 = srv.stats()
        t0 = time.perf_counter()
        st, _ids, _dist, _stats, lat = srv.replay(Qh[:m], kq[:m], cq[:m], 0.0, arr)
        wall = time.perf_counter() - t0
        b1 = srv.stats()
        ok = lat[lat >= 0]
        rates.append({"offered_qps": rate, "queries": m, "achieved_qps": round(m / wall, 1), "status": st,
                      "p50_us": round(float(ok.quantile(0.5)), 1), "p99_us": round(float(ok.quantile(0.99)), 1),
                      "mean_batch": round((b1["batched_queries"] - b0["batched_queries"]) /
                                          max(1, b1["batches"] - b0["batches"]), 1)})
    clk = clocks.stop()
    launches = pkg.detlsh_launch_count() - l0
    srv.destroy()
    idx.free()
    best = max(rates, key=lambda r: r["achieved_qps"])
    # the highest offered rate the server keeps up with (achieved >= 95% of offered)
    kept = [r for r in rates if r["achieved_qps"] >= 0.95 * r["offered_qps"]]
    sustained = max(kept, key=lambda r: r["offered_qps"]) if kept else None
    line = {"metric": METRIC, "value": best["achieved_qps"], "unit": "queries/s", "n_gpus": world,
            "steps": len(rates), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8 data, f32 arithmetic", "data": "synthetic",
            "config": {"workload": serving_desc(), **{k_: v for k_, v in w.items() if k_ not in ("betas", "rates")},
                       "beta": beta, "slots": slots, "pipelines": 2, "projection": args.proj,
                       "shortlist": args.shortlist, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (X is 12.8 GB)"},
            "clocks": clk, "latency_by_rate": rates, "beta_sweep": sweep,
            "p50_us_at_best": best["p50_us"], "p99_us_at_best": best["p99_us"],
            "sustained": ({"offered_qps": sustained["offered_qps"], "achieved_qps": sustained["achieved_qps"],
                           "p50_us": sustained["p50_us"], "p99_us": sustained["p99_us"]} if sustained else None),
            "build_mpts_per_s": n / (build_ms / 1000.0) / 1e6,
            "build_roofline": build_roofline_obj(n, build_bytes_per_point(d, 1, w["K"], w["L"]), build_ms,
                                                 {k_: round(trb[k_], 4) for k_ in ("sample_proj_ms", "breakpoints_ms",
                                                                                   "encode_ms", "leaves_ms")}),
            "e2e": {"value": best["achieved_qps"], "unit": "queries/s", "h2d_bytes_per_step": None,
                    "d2h_bytes_per_step": None, "note": "requests and results in host memory through the server"},
            "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": None,
            "batch_phase_ms": {k_: round(v, 4) for k_, v in ph.items()}}
    del X, Q
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-queries", type=int, default=8, help="queries of the single-thread oracle baseline")
    ap.add_argument("--nq", type=int, default=None,
                    help="queries per step (default: the workload's; applies to the workload run alone)")
    ap.add_argument("--method", default="det-lsh", choices=["det-lsh", "det-only"],
                    help="mid workload: DET-LSH (L Gaussian projections) or DET-ONLY (one tree over PAA)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--proj", default="fp32", choices=["fp32", "bf16"],
                    help="projection arithmetic of the build (bf16: tensor cores)")
    ap.add_argument("--shortlist", type=int, default=0,
                    help="with --proj bf16: coarse BF16 candidate distances, FP32 re-rank of this many")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison of the mid step")
    ap.add_argument("--no-extra", action="store_true",
                    help="mid workload only (skip the serving, precision and batching legs)")
    ap.add_argument("--workload", default="mid", choices=["mid", "batching", "serving", "precision"],
                    help="mid: build + 10,000 queries per step (default, with the other legs attached); "
                         "another name runs that leg alone")
    ap.add_argument("--route", default="graph", choices=["query", "plan", "graph"],
                    help="batching workload: detlsh_query, a plan with direct launches, or a plan replaying "
                         "its CUDA graph")
    ap.add_argument("--plan-batch", type=int, default=8192, help="queries per plan batch")
    ap.add_argument("--cpu-oracle-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_oracle_worker is not None:
        print(json.dumps(cpu_oracle_worker(json.loads(args.cpu_oracle_worker))), flush=True)
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.nq is not None:
        {"mid": WORKLOAD, "batching": BATCHING, "precision": PRECISION, "serving": SERVING}[args.workload]["nq"] = args.nq
    if args.method == "det-only":
        WORKLOAD["method"] = "det-only"
        WORKLOAD["L"] = 1
    if args.impl == "reference" and args.workload != "mid":
        ap.error("the reference arm times the mid workload")
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.shortlist and args.proj != "bf16":
        ap.error("--shortlist needs --proj bf16")
    import torch
    import paper_2406_10938_gb300 as pkg
    pkg.build()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sub_steps, sub_warm = max(1, min(args.steps, 5)), max(3, min(args.warmup, 3))
    try:
        if args.workload == "batching":
            line = batching_leg(args, rank, world, local_rank, barrier, args.steps, args.warmup)
        elif args.workload == "serving":
            line = serving_leg(args, rank, world, local_rank, barrier)
        elif args.workload == "precision":
            line = precision_leg(args, rank, world, local_rank, barrier, args.steps, args.warmup)
        else:
            line = mid_leg(args, rank, world, local_rank, barrier)
            if not args.no_extra and args.method == "det-lsh":
                legs = {}
                for name, fn in (("batching", lambda: batching_leg(args, rank, world, local_rank, barrier,
                                                                   sub_steps, sub_warm)),
                                 ("precision", lambda: precision_leg(args, rank, world, local_rank, barrier,
                                                                     sub_steps, sub_warm)),
                                 ("serving", lambda: serving_leg(args, rank, world, local_rank, barrier))):
                    t0 = time.perf_counter()
                    try:
                        legs[name] = fn()
                        legs[name]["leg_wall_s"] = round(time.perf_counter() - t0, 1)
                    except Exception as e:  # reported in the line, the headline stands
                        legs[name] = {"error": f"{type(e).__name__}: {str(e)[-400:]}"}
                    torch.cuda.empty_cache()
                line["workloads"] = legs
        if rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
