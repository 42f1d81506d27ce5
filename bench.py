#!/usr/bin/env python
"""Benchmark of the GB300 CD-ADC hot path; prints one JSON line.

Workload (default): EA-ADC(2)+x(3) with x = 0.5, nocc = 40, nvir = 200,
naux = 1200, complex128 Cholesky vectors (synthetic, seeded), 8 lowest roots.
A step is one complete Davidson solve of those roots with tensor-core (BF16x3)
sigma products refined by FP64-accurate sigma products until every residual
norm of those is below tol; the setup of the operators (adc_init) is timed
separately. The refinement products are, by default, the sliced tensor-core
product (integer BF16 digits summed exactly in FP32, combined in FP64, about
1e-12 relative); --refine fp64 uses the FP64 CUDA-core product instead.

Metric: Davidson seconds per root (lower is better); the line also carries
the sigma TFLOP/s of the mixed and FP64 products, the FP64 Davidson s/root,
the eigenvalue difference between the two, a live roofline of the dominant
kernel, clocks, an end-to-end number through the public API with host
buffers, the number of library kernels launched, and the CPU oracle timed on
a bounded sample of the same workload.

--impl reference times the CPU oracle (the only reference there is) on the
same workload and prints the same metric for it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import (BATCH_CONFIGS, CONFIGS, batch_problems, batch_sizes, config_problem,  # noqa: E402
                       random_hermitian_direction,
                       random_vectors)

METRIC = "Davidson s/root and sigma TFLOP/s: mixed vs FP64 on GPU at 1e-6 Eh error"


def log(*a):
    print(f"[bench {time.strftime('%H:%M:%S')}]", *a, file=sys.stderr, flush=True)


def nvtx_range(name, push):
    """Marks the timed region for a profiler's launch filter (a no-op without one attached)."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


THREE_M = ("zgemm", "gram", "combine")  # FP64 kernels whose complex products take 3 real products
# k_gram<32, 8, 4, 2, 32> on 32 x 8 vectors of n = 796200 (one launch, ncu): 510,109,184 B read +
# 4,893,696 B written against (32 + 8) * 796200 * 16 + 32 * 8 * 16 = 509,572,096 algorithmic bytes
GRAM_DRAM_RATIO = (510109184 + 4893696) / ((32 + 8) * 796200 * 16 + 32 * 8 * 16)
# k_combine<8>, 32 inputs to 8 outputs of n = 796200 (one launch, ncu): 407,728,128 B read + 82,273,792 B
# written against (32 + 8) * 796200 * 16 algorithmic bytes
COMBINE_DRAM_RATIO = (407728128 + 82273792) / ((32 + 8) * 796200 * 16)


def fp64_peak(adcgpu):
    """FP64 FMA peak of this GPU, measured now by the library's FMA probe
    (TFLOP/s), with the nominal figure from the unit counts and clocks."""
    try:
        best = max(adcgpu.diag_fp64_peak(152 * b, 1 << 14)[0] for b in (4, 8))
        return best, "measured (FP64 FMA probe, 16 independent chains per thread, this run)"
    except Exception as exc:  # the probe reports, it never stops the run
        log("fp64 probe failed", exc)
        return 1.25, "nominal: 152 SMs x 2.07 GHz x 2 FP64 FMA/clk x 2"


def alu_row(name, e, peak64, peak_kind):
    """Roofline entry of an FP64 CUDA-core kernel: algorithmic rate (8 flops
    per complex multiply-add) and the rate of the FP64 work it executes (6 per
    complex multiply-add for the 3M products)."""
    avg = e["total_ms"] / e["launches"]
    alg = e["flops"] / e["launches"]
    ach = alg / (avg * 1e-3) / 1e12
    ex = 0.75 if name.split("/")[0].split("_")[0] in THREE_M else 1.0
    return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
            "frac": ach / peak64, "traffic": None, "peak_kind": f"fp64 FMA {peak64:.3f} TFLOP/s, {peak_kind}; "
            "3M complex products execute 6 of the 8 algorithmic flops, so frac can reach 4/3",
            "executed_frac": ex * ach / peak64, "flops_per_launch": alg, "avg_launch_ms": avg,
            "algorithmic_bytes_per_launch": e.get("bytes", 0.0) / e["launches"], "launches": e["launches"]}


def attach_traffic(roof, config):
    """roof["traffic"]: DRAM bytes per launch of the dominant kernel from an ncu
    capture. A capture of the same launch shape is kept only for the kernel and
    workload it was taken on; for kernels whose launches differ in shape the
    captured launch's DRAM bytes over its algorithmic bytes scale this run's
    algorithmic bytes per launch."""
    measured_traffic = {("ea2x3_o40_v200_q1200", "zgemm_fp64/ladder"): 7.795e9}
    key = (config, roof["kernel"])
    if key in measured_traffic:
        roof["traffic"] = measured_traffic[key]
        roof["traffic_note"] = "one ncu capture of the 320 x 19900 x 19900 FP64 ladder GEMM"
    traffic_ratio = {"gram_fp64": (GRAM_DRAM_RATIO, "ncu capture of one k_gram launch, 32 x 8 vectors of "
                                                    "n = 796200: DRAM bytes / algorithmic bytes"),
                     "combine_fp64": (COMBINE_DRAM_RATIO, "ncu capture of one k_combine launch, 32 to 8 vectors "
                                                          "of n = 796200: DRAM bytes / algorithmic bytes")}
    base = roof["kernel"].split("/")[0]
    if roof.get("traffic") is None and base in traffic_ratio and roof.get("algorithmic_bytes_per_launch"):
        ratio, note = traffic_ratio[base]
        roof["traffic"] = ratio * roof["algorithmic_bytes_per_launch"]
        roof["traffic_note"] = f"{note} = {ratio:.3f}, scaled to this run's launches"
    return roof


def reduce_across(values, op):
    """All-reduce numbers over the process group of the replicas: "max" (the
    slowest replica's times) or "sum" (counts of all replicas). NCCL takes
    device tensors, gloo host ones. Returns a list of floats."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return [float(a) for a in t.tolist()]


def sigma_flops_formula(o, v, Q, k):
    """Algorithmic flops of one EA sigma block of k vectors as the library forms it
    (8 per complex multiply-add): coupling both ways (2 v n2 k), ladder over packed
    pairs (Pv^2 o k), ring over (k, c) (o v * o v * v k)."""
    pv = v * (v - 1) // 2
    n2 = o * pv
    cmac = 2 * v * n2 * k + pv * pv * o * k + (o * v) * (o * v) * (v * k) + v * v * k
    return 8.0 * cmac


def _pair(p, q, n):
    return p * n - p * (p + 1) // 2 + (q - p - 1)


# Sigma vectors per root that scale both oracle legs' seconds per sigma row to
# seconds per root (one number per workload for both legs), with where it comes
# from: the FP64 block Davidson (the oracle's algorithm, run on the GPU in FP64)
# where it was measured, else the closest measured count, else an assumption.
ORACLE_SIGMA_VECTORS_PER_ROOT = {
    "ea2x3_o40_v200_q1200": (41.625, "FP64 Davidson count of this workload at its tolerance "
                                     "(333 sigma vectors for 8 roots)"),
    "ee2x3_o30_v150_q900": (110.0, "mixed Davidson count of this workload (440 sigma vectors for 4 roots, "
                                   "residual 1e-6); its FP64 Davidson was not run to the end"),
    "ee3_o60_v300_q1800": (40.0, "assumed: no solve of this workload has run to the end"),
}


def sigma_vectors_per_root(cfgname, default=None):
    """(sigma vectors per root, where the number comes from) for a workload,
    or `default` (a pair, or None) when none is recorded."""
    return ORACLE_SIGMA_VECTORS_PER_ROOT.get(cfgname, default)


def pick_rows(kind, o, v, n_rows, seed):
    """Seeded satellite (IP/EA) or doubles (EE) rows: (row tuples, packed indices in S)."""
    rng = np.random.default_rng(seed)
    rows, idx = [], []
    for _ in range(n_rows):
        if kind == "EA":
            k = int(rng.integers(o))
            d, e = sorted(rng.choice(v, 2, replace=False))
            rows.append((k, int(d), int(e)))
            idx.append(v + k * (v * (v - 1) // 2) + _pair(int(d), int(e), v))
        elif kind == "IP":
            i, j = sorted(rng.choice(o, 2, replace=False))
            a = int(rng.integers(v))
            rows.append((int(i), int(j), a))
            idx.append(o + _pair(int(i), int(j), o) * v + a)
        else:
            k, l = sorted(int(a) for a in rng.choice(o, 2, replace=False))
            c, d = sorted(int(a) for a in rng.choice(v, 2, replace=False))
            rows.append((k, l, c, d))
            idx.append(o * v + _pair(k, l, o) * (v * (v - 1) // 2) + _pair(c, d, v))
    return rows, idx


def _dim(kind, o, v):
    if kind == "EA":
        return v + o * v * (v - 1) // 2
    if kind == "IP":
        return o + o * (o - 1) // 2 * v
    return o * v + (o * (o - 1) // 2) * (v * (v - 1) // 2)


def cpu_oracle_sample(p, x, n_rows=6, seed=5, kind="EA", want_rows=False, X=None):
    """Seconds per satellite sigma row (one vector) of the oracle on this
    workload, in this process. With want_rows, also (X, packed indices of the
    rows in S, the rows' values); X [1][N] may be given, else it is drawn."""
    from oracle.rows import ea_satellite_rows, ip_satellite_rows
    o, v = p.nocc, p.nvir
    N = _dim(kind, o, v)
    X = random_vectors(N, 1, seed=seed) if X is None else np.asarray(X).reshape(1, N)
    rows, idx = pick_rows(kind, o, v, n_rows, seed)
    fn = ea_satellite_rows if kind == "EA" else ip_satellite_rows
    t0 = time.perf_counter()
    R = fn(p.B, p.eps_occ, p.eps_vir, 3, x, X, rows)
    t = time.perf_counter() - t0
    what = f"{n_rows} satellite rows of S = M X for one vector, each row from Eq. 43 integrals"
    if want_rows:
        return t / n_rows, what, (X, idx, R)
    return t / n_rows, what


# ---- the oracle on the host cores: one process per core (spawn start, so
# that no process forks from one that has touched the GPU), one row per task
_POOL = {}


def _spec_problem(spec):
    if spec[0] == "batch":
        return batch_problems(spec[1], select=[spec[2]])[0]
    return config_problem(spec[1])


def _pool_init(spec, xseed):
    p = _spec_problem(spec)
    _POOL.update(p=p, X=random_vectors(_dim(p.kind, p.nocc, p.nvir), 1, seed=xseed))


def _pool_row(task):
    from oracle.rows import ea_satellite_rows, ee_doubles_rows, ip_satellite_rows
    kind, order, x, dd_order, row = task
    p, X = _POOL["p"], _POOL["X"]
    t0 = time.perf_counter()
    if kind == "EE":
        R = ee_doubles_rows(p.B, p.eps_occ, p.eps_vir, order, x, X, [row], dd_order=dd_order)
    else:
        fn = ea_satellite_rows if kind == "EA" else ip_satellite_rows
        R = fn(p.B, p.eps_occ, p.eps_vir, order, x, X, [row])
    return np.asarray(R)[0, 0], time.perf_counter() - t0


def _mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def _blas_name():
    try:
        cfg = np.show_config(mode="dicts")
        b = cfg["Build Dependencies"]["blas"]
        return f"{b.get('name')} {b.get('version')}"
    except Exception:
        return "unknown"


def oracle_rows_pool(spec, kind, order, x, dd_order, n_rows, seed=5, xseed=5, workers=None):
    """The oracle's sigma rows of one seeded vector on the host cores.

    Worker processes (spawn) each rebuild the seeded problem and vector, then
    compute rows, one single-threaded row per task (the row oracle is numpy
    einsum loops; BLAS is held to one thread per process). Returns the sample:
    X, packed row indices, row values [1][n_rows], the pool's wall time for the
    rows, the mean seconds of one row inside a worker, and the worker count."""
    import multiprocessing as mp
    p_sizes = _spec_problem(spec) if spec[0] == "batch" else CONFIGS[spec[1]]
    o = p_sizes.nocc if spec[0] == "batch" else p_sizes["nocc"]
    v = p_sizes.nvir if spec[0] == "batch" else p_sizes["nvir"]
    q = p_sizes.naux if spec[0] == "batch" else p_sizes["naux"]
    cores = os.cpu_count() or 1
    bytes_b = 16.0 * q * (o + v) ** 2
    avail = _mem_available()
    cap = cores if avail is None else max(1, int(avail // (4.0 * bytes_b)))
    workers = max(1, min(workers or cores, cores, cap, n_rows))
    rows, idx = pick_rows(kind, o, v, n_rows, seed)
    env_keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_pool_init, initargs=(spec, xseed)) as pool:
            # every worker has built its problem before the rows are timed
            pool.map(time.sleep, [0.0] * workers, chunksize=1)
            t0 = time.perf_counter()
            res = pool.map(_pool_row, [(kind, order, x, dd_order, r) for r in rows], chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, val in saved.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val
    X = random_vectors(_dim(kind, o, v), 1, seed=xseed)
    R = np.array([[r[0] for r in res]])
    return {"X": X, "idx": idx, "R": R, "wall_s": wall, "row_s": float(np.mean([r[1] for r in res])),
            "workers": workers, "rows": n_rows}


def cpu_baseline_of(sample, N, spr, spr_note, kind):
    """cpu_baseline object: seconds per root of the oracle on the host cores,
    from the pool's rows per second, N rows per sigma vector and spr sigma
    vectors per root."""
    per_row = sample["wall_s"] / sample["rows"]
    what = ("doubles rows (the oracle's term tables with the row's indices fixed)" if kind == "EE"
            else "satellite rows (integrals of each row from Eq. 43)")
    return {"value": per_row * N * spr, "unit": "s/root", "cores": sample["workers"], "kind": "oracle",
            "sample": (f"{sample['rows']} {what} of S = M X for one seeded vector, one single-threaded row per "
                       f"process on {sample['workers']} processes, {sample['wall_s']:.1f} s wall; seconds per row "
                       f"x N={N} rows x {spr:.2f} sigma vectors per root ({spr_note})"),
            "row_s_one_thread": sample["row_s"], "threads_per_process": 1, "host_cores": os.cpu_count(),
            "blas": _blas_name()}


ORACLE_SOLVE_MAX_N = 5000  # the oracle's whole Davidson runs on workloads up to this dimension


def oracle_solve_feasible(cfgname):
    c = CONFIGS.get(cfgname)
    return c is not None and _dim(c["kind"], c["nocc"], c["nvir"]) <= ORACLE_SOLVE_MAX_N


def oracle_davidson_baseline(cfgname):
    """The oracle's whole FP64 solve of a small workload, in this process, not
    extrapolated: its ground-state amplitudes and exact diagonal, then its
    block Davidson (FP64 sigma_ref products) to the workload's residual
    tolerance. Seconds per root of that wall time; the threads are numpy's
    defaults (BLAS on every host core, the einsum contractions on one), and
    the process CPU time over the wall time says how many were busy."""
    from oracle import adc, adc_ee
    from oracle.davidson import davidson
    c = CONFIGS[cfgname]
    p = config_problem(cfgname)
    kind, order, x, nroots, tol = c["kind"], c["order"], c["x"], c["nroots"], c.get("tol", 1e-8)
    dd = c.get("dd_order", 1)
    calls = [0]
    w0, c0 = time.perf_counter(), time.process_time()
    if kind == "EE":
        T = adc_ee.Tensors(p.B, p.eps_occ, p.eps_vir)
        diag = adc_ee.diagonal_ref(order, x, p.B, p.eps_occ, p.eps_vir, dd_order=dd, T=T)

        def sig(V):
            calls[0] += V.shape[0]
            return adc_ee.sigma_ref(order, x, p.B, p.eps_occ, p.eps_vir, V, dd_order=dd, T=T)
    else:
        amp = adc.Amplitudes(p.B, p.eps_occ, p.eps_vir, second_order=(order == 3))
        diag = adc.diagonal_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, amp=amp)

        def sig(V):
            calls[0] += V.shape[0]
            return adc.sigma_ref(kind, order, x, p.B, p.eps_occ, p.eps_vir, V, amp=amp)
    w, _, rn, it = davidson(sig, diag, diag.shape[0], nroots, tol=tol, max_iter=300)
    wall, cpu_s = time.perf_counter() - w0, time.process_time() - c0
    cores = os.cpu_count() or 1
    return {"value": wall / nroots, "unit": "s/root", "cores": cores, "kind": "oracle",
            "sample": (f"the whole workload: the oracle's FP64 block Davidson (sigma_ref products, exact "
                       f"diagonal) for {nroots} roots to a residual of {tol:g}, {it} iterations, {calls[0]} "
                       f"sigma vectors, {wall:.1f} s wall including its amplitudes; not extrapolated"),
            "wall_s": wall, "effective_threads": cpu_s / max(wall, 1e-9), "host_cores": cores,
            "blas": _blas_name(), "iterations": it, "sigma_vectors": calls[0],
            "omega": [float(a) for a in w], "max_residual": float(np.max(rn))}


def sampled_parity(ctx, sample, precisions):
    """The GPU sigma of the sampled vector, in each precision, at the rows the
    oracle computed: largest absolute difference and that over the largest
    oracle row value."""
    X, idx, R = sample
    scale = float(np.abs(R).max())
    out = {"rows": len(idx), "oracle_row_max": scale}
    for prec in precisions:
        S = np.asarray(ctx.sigma(X, prec))
        err = float(np.abs(S[:, idx] - R).max())
        out[prec] = {"max_abs_err": err, "rel": err / max(scale, 1e-300)}
    return out


def run_batch(args, cfgname):
    """Batched IP/EA workload: the problems are planned into waves that fit the
    device memory; each wave is initialised, its batched split-precision sigma
    is timed (graph replays, and the grouped tensor-core kernel alone), and it
    is solved with the batched Davidson after --warmup warm-up solves. value =
    Davidson seconds per root over all problems; e2e is the adc_init calls
    (host inputs copied inside) plus the first solve of each wave."""
    import torch
    import paper_2511_21640_gb300 as adcgpu
    c = BATCH_CONFIGS[cfgname]
    nroots = c["nroots"]
    tol = args.tol if args.tol is not None else c["tol"]
    sizes = batch_sizes(cfgname)
    free = torch.cuda.mem_get_info()[0]
    nw, order, wave, mem, cost = adcgpu.batch_plan(sizes, nroots, int(0.85 * free))
    log(f"{len(sizes)} problems in {nw} waves")
    tot = dict(init_s=0.0, solve_s=0.0, first_solve_s=0.0, sig_ms=0.0, sig_flops=0.0, g_ms=0.0, g_flops=0.0, g_launch=0,
               batches=0, graph_launches=0, sigma_calls=0, sigma_calls_fp64=0, iters=[])
    omegas, errs, status_all = {}, {}, {}
    batch_parity = []
    clocks = Clocks()
    clocks.start()
    for w in range(nw):
        ids = [int(i) for i in order if wave[i] == w]
        probs = batch_problems(cfgname, select=ids)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the sliced setup; the batched solves refine in FP64 (the planner's waves
        # leave no room for every problem's sliced operator copies)
        ctxs = [adcgpu.Context(p.B, p.eps_occ, p.eps_vir, kind=p.kind, order=p.order, x=p.x, setup=args.e2e_setup)
                for p in probs]
        for cx in ctxs:
            cx.sync()
        tot["init_s"] += time.perf_counter() - t0
        log(f"wave {w}: {len(ids)} problems initialised in {time.perf_counter() - t0:.1f} s")
        with adcgpu.Batch(ctxs) as b:
            Xs = [torch.from_numpy(random_vectors(cx.N, nroots, seed=900 + i)).cuda() for i, cx in zip(ids, ctxs)]
            Ss = [torch.empty_like(X) for X in Xs]
            # grouped tensor-core kernel alone (batches enqueued without a graph)
            b.use_graphs(False)
            b.sigma(Xs, "bf16x3", outs=Ss)
            if w == 0 and args.cpu_rows > 0:
                # one problem of each kind: its batched product against oracle rows of the same vector
                seen = set()
                for j, pr in enumerate(probs):
                    if pr.kind in seen:
                        continue
                    seen.add(pr.kind)
                    try:
                        X0 = Xs[j][:1].cpu().numpy()
                        S0 = Ss[j][:1].cpu().numpy()
                        _, _, (_, idx, R) = cpu_oracle_sample(pr, pr.x, n_rows=min(args.cpu_rows, 4), kind=pr.kind,
                                                              want_rows=True, X=X0)
                        err = float(np.abs(S0[:, idx] - R).max())
                        scale = float(np.abs(R).max())
                        batch_parity.append({"problem": ids[j], "kind": pr.kind, "nocc": pr.nocc, "nvir": pr.nvir,
                                             "rows": len(idx), "bf16x3_max_abs_err": err,
                                             "rel": err / max(scale, 1e-300)})
                    except Exception as exc:  # the check reports, it never stops the run
                        batch_parity.append({"problem": ids[j], "error": str(exc)[:200]})
                log("batched sampled parity", batch_parity)
            i0 = b.info()
            for _ in range(3):
                b.sigma(Xs, "bf16x3", outs=Ss)
            i1 = b.info()
            tot["g_ms"] += i1["grouped_ms"] - i0["grouped_ms"]
            tot["g_flops"] += i1["grouped_flops"] - i0["grouped_flops"]
            tot["g_launch"] += i1["grouped_launches"] - i0["grouped_launches"]
            # whole batched product, CUDA graph replays
            b.use_graphs(True)
            for _ in range(max(args.warmup, 2)):
                b.sigma(Xs, "bf16x3", outs=Ss)
            i2 = b.info()
            for _ in range(5):
                b.sigma(Xs, "bf16x3", outs=Ss)
            i3 = b.info()
            tot["sig_ms"] += i3["batch_ms"] - i2["batch_ms"]
            tot["sig_flops"] += i3["tc_flops"] - i2["tc_flops"]
            del Xs, Ss
            # warm-up solves of the wave (each starts from scratch); the first one
            # closes the end-to-end figure
            first = None
            for _ in range(args.warmup):
                tw = time.perf_counter()
                b.davidson(nroots, tol=tol, max_iter=300, precision="bf16x3")
                first = time.perf_counter() - tw if first is None else first
            i2 = b.info()
            torch.cuda.synchronize()
            l0 = adcgpu.launch_count()
            t1 = time.perf_counter()
            om, e64, st_codes, sts, rc = b.davidson(nroots, tol=tol, max_iter=300, precision="bf16x3")
            dt = time.perf_counter() - t1
            tot["solve_s"] += dt
            tot["first_solve_s"] += dt if first is None else first
            tot["launches"] = tot.get("launches", 0) + adcgpu.launch_count() - l0
            i3 = b.info()
            tot["batches"] += i3["batches"] - i2["batches"]
            tot["graph_launches"] += i3["graph_launches"] - i2["graph_launches"]
            log(f"wave {w}: solved in {time.perf_counter() - t1:.1f} s, rc {rc}")
            for j, i in enumerate(ids):
                omegas[i] = om[j].tolist()
                errs[i] = float(e64[j].max())
                status_all[i] = int(st_codes[j])
                tot["sigma_calls"] += sts[j]["sigma_calls"]
                tot["sigma_calls_fp64"] += sts[j]["sigma_calls_fp64"]
                tot["iters"].append(sts[j]["iterations"])
        for cx in ctxs:
            cx.close()
    clk = clocks.stop()
    nprob = len(sizes)
    roots = nprob * nroots
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    g_ach = 3.0 * tot["g_flops"] / (tot["g_ms"] * 1e-3) / 1e12 if tot["g_ms"] > 0 else None
    line = {
        "metric": METRIC, "value": tot["solve_s"] / roots, "unit": "s/root", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot["solve_s"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f64", "data": "synthetic",
        "config": {"workload": cfgname, "problems": nprob, "nroots": nroots, "tol_fp64_residual": tol,
                   "waves": nw, "sizes": "nocc U[10,40], nvir U[50,250], naux 6 nvir, IP even / EA odd, x 0.5",
                   "l2": "operators larger than L2"},
        "clocks": clk, "sampled_parity": batch_parity,
        "roofline": {"bound": "tensor", "kernel": "k_tc_grouped (all problems' coupling, ladder, ring jobs)",
                     "achieved": g_ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": (g_ach / peak) if g_ach else None, "traffic": None,
                     "peak_kind": f"bf16 dense sustained ({pk_kind}); achieved counts 3 BF16 products per "
                                  "split-precision product", "launches_timed": tot["g_launch"],
                     "avg_launch_ms": tot["g_ms"] / max(1, tot["g_launch"])},
        "batched_sigma": {"tflops_algorithmic": tot["sig_flops"] / (tot["sig_ms"] * 1e-3) / 1e12,
                          "ms_per_batch": tot["sig_ms"] / (5 * nw), "vectors_per_problem": nroots,
                          "includes": "FP64 main block, operand packing, grouped tensor-core launch, epilogues "
                                      "(CUDA graph replays)"},
        "davidson": {"iterations_max": max(tot["iters"]), "iterations_mean": float(np.mean(tot["iters"])),
                     "sigma_calls": tot["sigma_calls"], "sigma_calls_fp64": tot["sigma_calls_fp64"],
                     "batched_products": tot["batches"], "graph_replays": tot["graph_launches"],
                     "max_err64": max(errs.values()), "status_nonzero": [i for i, s in status_all.items() if s]},
        "init_s": tot["init_s"],
        "e2e": {"value": (tot["init_s"] + tot["first_solve_s"]) / roots, "unit": "s/root",
                "h2d_bytes_per_step": int(sum(16 * d["naux"] * (d["nocc"] + d["nvir"]) ** 2 for d in sizes)),
                "d2h_bytes_per_step": int(16 * roots),
                "includes": f"adc_init of every problem (H2D copy + {args.e2e_setup} operator setup) + the first "
                            "batched Davidson of each wave"},
        "gpu_launches": int(tot.get("launches", 0)), "cpu_baseline": None,
    }
    print(json.dumps(line))


def run_ee(args, cfgname):
    """EE-ADC workload: mixed-precision Davidson seconds per root (FP64
    residuals) after --warmup warm-up solves, the end-to-end time of setup
    and first solve from host inputs, the FP64 Davidson for comparison
    (unless --no-fp64-davidson), one sigma block in each precision, and the
    gradients of the roots (adjoint) with a central-difference check along
    one random direction (dB Hermitian, deps, dx), h = 1e-5, from two more
    mixed-precision solves."""
    import torch
    import paper_2511_21640_gb300 as adcgpu
    cfg = dict(CONFIGS[cfgname])
    nroots, x = cfg["nroots"], cfg["x"]
    tol = args.tol if args.tol is not None else cfg["tol"]
    p = config_problem(cfgname)
    o, v, Q = p.nocc, p.nvir, p.naux
    t0 = time.perf_counter()
    dd_order, block = cfg.get("dd_order", 1), cfg.get("block", 0)
    setup = cfg.get("setup", "fp64")
    ctx = adcgpu.Context(p.B, p.eps_occ, p.eps_vir, kind="EE", order=cfg["order"], x=x, refine=args.refine,
                         dd_order=dd_order, block=block, setup=setup)
    init_s = time.perf_counter() - t0
    mem_init = ctx.memory()
    log(f"init {init_s:.1f} s, N = {ctx.N}, device memory after init {mem_init['in_use'] / 2**30:.1f} GiB "
        f"(peak {mem_init['peak'] / 2**30:.1f} GiB)")
    tp = time.perf_counter()
    ctx.sigma(random_vectors(ctx.N, 1, seed=3), args.mixed)  # builds the split-precision operators
    prep_s = time.perf_counter() - tp
    # warm-up solves; the first one closes the end-to-end figure (host inputs,
    # setup, operators, one solve with its eigenvalues and residuals read back)
    first_s = None
    for _ in range(args.warmup):
        tw = time.perf_counter()
        _, _, _, stw, _ = ctx.davidson(nroots, tol=tol, max_iter=400, precision=args.mixed, want_vectors=False)
        first_s = time.perf_counter() - tw if first_s is None else first_s
        log("warmup solve", stw)
    clocks = Clocks()
    clocks.start()
    ctx.profile(True)
    l0 = adcgpu.launch_count()
    t1 = time.perf_counter()
    om, Y, e64, st, rc = ctx.davidson(nroots, tol=tol, max_iter=400, precision=args.mixed)
    solve_s = time.perf_counter() - t1
    launches = adcgpu.launch_count() - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    mem_solve = ctx.memory()
    log(f"mixed davidson {solve_s:.1f} s, peak device memory {mem_solve['peak'] / 2**30:.1f} GiB", st)
    first_s = solve_s if first_s is None else first_s
    e2e = {"value": (init_s + prep_s + first_s) / nroots, "unit": "s/root",
           "h2d_bytes_per_step": int(p.B.nbytes + 8 * (o + v)), "d2h_bytes_per_step": int(16 * nroots),
           "includes": "adc_init from host inputs (H2D copy + operator setup), the split-precision operators "
                       "and the first mixed-precision solve (eigenvalues and residuals read back)",
           "init_s": init_s, "operators_s": prep_s, "first_solve_s": first_s, "setup": setup}
    fp64 = None
    if not args.no_fp64_davidson and cfg.get("fp64_davidson", True):
        t2 = time.perf_counter()
        om64, _, e6, st6, rc6 = ctx.davidson(nroots, tol=tol, max_iter=400, precision="fp64", want_vectors=False)
        t64 = time.perf_counter() - t2
        log(f"fp64 davidson {t64:.1f} s", st6)
        fp64 = {"s_per_root": t64 / nroots, "iterations": st6["iterations"], "sigma_calls": st6["sigma_calls"],
                "max_eig_diff_vs_mixed": float(np.abs(om64 - om).max()), "rc": int(rc6)}
    nsig = nroots if ctx.N < 20_000_000 else 1
    Xs = random_vectors(ctx.N, nsig, seed=7)
    sig = {}
    for prec in (args.mixed, "sliced", "fp64"):
        ctx.sigma(Xs, prec)
        ctx.profile(True)
        t2 = time.perf_counter()
        ctx.sigma(Xs, prec)
        ts = time.perf_counter() - t2
        sp = ctx.profile_read()
        ctx.profile(False)
        sig[prec] = {"ms": 1e3 * ts, "flops_timed_kernels": sum(e["flops"] for e in sp.values())}
    cpu, parity = None, None
    if args.cpu_rows > 0:
        smp = oracle_rows_pool(("config", cfgname), "EE", cfg["order"], x, dd_order, args.cpu_rows)
        try:
            parity = sampled_parity(ctx, (smp["X"], smp["idx"], smp["R"]), ("fp64", args.mixed, "sliced"))
        except Exception as exc:  # the check reports, it never stops the run
            parity = {"error": str(exc)[:200]}
        log("sampled parity", parity)
        spr, note = sigma_vectors_per_root(cfgname, (st["sigma_calls"] / nroots, "this run's mixed solve"))
        cpu = cpu_baseline_of(smp, ctx.N, spr, note, "EE")
    fns = None
    if cfg.get("fns_eta") is not None:
        ctx.profile(True)
        t4 = time.perf_counter()
        n_keep = ctx.fns_density(cfg["fns_eta"])["n_keep"]
        fns_s = time.perf_counter() - t4
        ctx.profile(False)
        fns = {"s": fns_s, "eta_crit": cfg["fns_eta"], "n_keep": int(n_keep), "nvir": v}
        log(f"fns density {fns_s:.2f} s, keep {n_keep} of {v}")
    grad = None
    if args.no_gradient or not cfg.get("gradient", True):
        ctx.close()
    else:
        rng = np.random.default_rng(11)
        wts = rng.standard_normal(nroots)
        ctx.profile(True)
        t3 = time.perf_counter()
        gB, geo, gev, gx = ctx.sigma_adjoint(Y, wts)
        adj_s = time.perf_counter() - t3
        adj_prof = ctx.profile_read()
        ctx.profile(False)
        adj_stages = {k[6:]: round(e["total_ms"], 1) for k, e in adj_prof.items() if k.startswith("stage:")}
        log(f"adjoint {adj_s:.1f} s", adj_stages)
        ctx.close()
        D = (random_hermitian_direction(p.B.shape, 12), rng.standard_normal(o), rng.standard_normal(v), 0.7)
        # derivative along D that the gradients predict
        pred = float(np.real(np.vdot(gB, D[0]))) + float(np.dot(geo, D[1])) + float(np.dot(gev, D[2])) \
            + float(gx) * D[3]
        h = 1e-5
        ws = []
        for sgn in (1, -1):
            with adcgpu.Context(p.B + sgn * h * D[0], p.eps_occ + sgn * h * D[1], p.eps_vir + sgn * h * D[2],
                                kind="EE", order=cfg["order"], x=x + sgn * h * D[3], refine=args.refine) as c2:
                w, _, _, _, rcf = c2.davidson(nroots, tol=min(tol, 1e-8), max_iter=400, precision=args.mixed,
                                              want_vectors=False)
                ws.append(w)
        fd = float(np.dot(wts, (ws[0] - ws[1]) / (2 * h)))
        log(f"gradient check: adjoint {pred:.10e} fd {fd:.10e}")
        grad = {"adjoint_s": adj_s, "adjoint_stages_ms": adj_stages, "directional_adjoint": pred, "directional_fd": fd,
                "rel_diff": abs(pred - fd) / max(1.0, abs(fd)), "fd_step": h, "weights": [float(w) for w in wts]}
    by = sorted(((k, e) for k, e in prof.items() if e["launches"] > 0), key=lambda t: -t[1]["total_ms"])
    pk, pk_kind = peaks()
    peak64, peak64_kind = fp64_peak(adcgpu)

    def roof(name, e):
        avg = e["total_ms"] / e["launches"]
        alg = e["flops"] / e["launches"]
        if name.startswith("tc_"):
            mma = (1.0 if name.startswith("tc_sliced") else 6.0 if "bf16x6" in name else 3.0) * alg
            peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
            ach = mma / (avg * 1e-3) / 1e12
            return {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "peak_kind": f"bf16 dense sustained ({pk_kind})",
                    "launches": e["launches"], "avg_launch_ms": avg}
        return alu_row(name, e, peak64, peak64_kind)

    by_kernel = [roof(k, e) for k, e in by]
    line = {
        "metric": METRIC, "value": solve_s / nroots, "unit": "s/root", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": 1e3 * solve_s, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{args.mixed}+" + ("f64 from exact bf16 digit products" if args.refine == "sliced" else "f64"),
        "data": "synthetic",
        "config": {"workload": cfgname, "kind": "EE", "order": cfg["order"], "x": x, "nocc": o, "nvir": v,
                   "naux": Q, "nroots": nroots, "tol_fp64_residual": tol, "N": int(Y.shape[1]),
                   "dd_order": dd_order, "block": block, "setup": setup,
                   "l2": "operators larger than L2"},
        "clocks": clk, "gpu_launches": int(launches), "roofline": by_kernel[0], "roofline_by_kernel": by_kernel,
        "mixed_davidson": {"iterations": st["iterations"], "sigma_calls": st["sigma_calls"],
                           "sigma_calls_fp64": st["sigma_calls_fp64"], "sigma_calls_mid": st["sigma_calls_mid"],
                           "rc": int(rc),
                           "omega": [float(w) for w in om], "err64": [float(e) for e in e64]},
        "fp64_davidson": fp64,
        "fns": fns,
        "memory_gib": {"after_init": mem_init["in_use"] / 2**30, "peak_init": mem_init["peak"] / 2**30,
                       "peak_through_solve": mem_solve["peak"] / 2**30},
        "sigma": {"vectors": nsig, "mixed": args.mixed, "mixed_ms": sig[args.mixed]["ms"],
                  "sliced_ms": sig["sliced"]["ms"], "fp64_ms": sig["fp64"]["ms"],
                  "speedup": sig["fp64"]["ms"] / sig[args.mixed]["ms"],
                  "speedup_sliced": sig["fp64"]["ms"] / sig["sliced"]["ms"]},
        "refine": args.refine,
        "gradient": grad,
        "init_s": init_s, "e2e": e2e, "cpu_baseline": cpu, "sampled_parity": parity,
    }
    print(json.dumps(line))


def run_reference(args, cfgname):
    """CPU oracle arm: sigma rows of the workload on the host cores (one
    single-threaded row per process, as in the CPU baseline of the GPU arm),
    scaled to seconds per root with the same factor. The rows of all timed
    steps run together on the pool; a step's time is the pool's wall time per
    row times the rows of one step."""
    if cfgname in BATCH_CONFIGS:
        # one EA problem of the batch stands for all of them
        spec = ("batch", cfgname, 1)
        p = batch_problems(cfgname, select=[1])[0]
        c = dict(kind="EA", order=3, x=BATCH_CONFIGS[cfgname]["x"], nroots=BATCH_CONFIGS[cfgname]["nroots"])
        o, v, q = p.nocc, p.nvir, p.naux
    else:
        spec = ("config", cfgname)
        c = CONFIGS[cfgname]
        o, v, q = c["nocc"], c["nvir"], c["naux"]
    kind, dd_order = c["kind"], c.get("dd_order", 1)
    N = _dim(kind, o, v)
    if spec[0] == "config" and oracle_solve_feasible(cfgname):
        # small enough for the oracle's whole solve: every step is one solve
        for _ in range(args.warmup):
            import oracle.davidson  # noqa: F401
        runs = [oracle_davidson_baseline(cfgname) for _ in range(max(args.steps, 1))]
        cpu = dict(runs[-1])
        cpu["value"] = float(np.mean([r["value"] for r in runs]))
        cpu["sample"] = f"{len(runs)} x " + cpu["sample"]
        value = cpu["value"]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/root", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * float(np.mean([r["wall_s"] for r in runs])),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": cfgname, "nocc": o, "nvir": v, "naux": q,
                                                "kind": kind, "order": c["order"], "x": c["x"],
                                                "nroots": c["nroots"]},
                "cpu_baseline": cpu,
                "e2e": {"value": value, "unit": "s/root", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    spr, note = sigma_vectors_per_root(cfgname, (40.0, "assumed 40"))
    cores = os.cpu_count() or 1
    # warm-up: the oracle modules imported, no timing
    for _ in range(args.warmup):
        import oracle.rows  # noqa: F401
    rows = max(args.steps, 1) * max(args.ref_rows, 1)
    workers = min(cores, rows)
    rows = -(-rows // workers) * workers  # whole rounds of the pool
    smp = oracle_rows_pool(spec, kind, c["order"], c["x"], dd_order, rows, seed=10)
    cpu = cpu_baseline_of(smp, N, spr, note, kind)
    value = cpu["value"]
    per_step_s = smp["wall_s"] / rows * max(args.ref_rows, 1)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/root", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_step_s,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfgname, "nocc": o, "nvir": v, "naux": q,
                                            "kind": kind, "order": c["order"], "x": c["x"],
                                            "nroots": c["nroots"]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "s/root", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_init_profile(args, name):
    """adc_init of the workload from host buffers (the e2e leg's setup) with the
    library's profile on from the start: wall time, the device time of each
    setup stage and of the GEMMs inside (one JSON line)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2511_21640_gb300 as adcgpu
    cfg = dict(CONFIGS[name])
    p = config_problem(name)
    Bh = torch.from_numpy(p.B).pin_memory()
    eoh, evh = torch.from_numpy(p.eps_occ), torch.from_numpy(p.eps_vir)
    torch.cuda.synchronize()
    nvtx_range("init", True)
    t0 = time.perf_counter()
    ctx = adcgpu.Context(Bh, eoh, evh, kind=cfg["kind"], order=cfg["order"], x=cfg["x"], setup=args.e2e_setup,
                         dd_order=cfg.get("dd_order", 1), profile=True)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    nvtx_range("init", False)
    prof = ctx.profile_read()
    stages = {k[6:]: round(v["total_ms"], 3) for k, v in prof.items() if k.startswith("stage:")}
    gemms = sorted(((k, v) for k, v in prof.items() if not k.startswith("stage:")), key=lambda kv: -kv[1]["total_ms"])
    out = {"config": name, "setup": args.e2e_setup, "init_s": init_s, "stages_ms": stages,
           "gemm_ms_total": round(sum(v["total_ms"] for _, v in gemms), 3),
           "gemms": [{"name": k, "launches": v["launches"], "ms": round(v["total_ms"], 3),
                      "tflops": (v["flops"] / (v["total_ms"] * 1e-3) / 1e12) if v["total_ms"] > 0 else None}
                     for k, v in gemms[:30]],
           "mem_peak_gib": ctx.memory()["peak"] / 2**30, "setup_routes": ctx.setup_routes()}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_sigma_only(args, name):
    """One sigma block of the workload (nroots seeded vectors, device buffers) in one
    precision, after three warm-up blocks (tile widths tuned, operands packed), inside
    the NVTX range 'sigma': its CUDA-event time and algorithmic rate (one JSON line)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2511_21640_gb300 as adcgpu
    cfg = dict(CONFIGS[name])
    p = config_problem(name)
    torch.cuda.set_stream(torch.cuda.Stream())
    ctx = adcgpu.Context(p.B, p.eps_occ, p.eps_vir, kind=cfg["kind"], order=cfg["order"], x=cfg["x"],
                         setup=args.e2e_setup, dd_order=cfg.get("dd_order", 1), stream="torch")
    X = torch.from_numpy(random_vectors(ctx.N, cfg["nroots"], seed=7)).cuda()
    for _ in range(3):
        ctx.sigma(X, args.sigma_only)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    nvtx_range("sigma", True)
    a.record(torch.cuda.current_stream())
    ctx.sigma(X, args.sigma_only)
    b.record(torch.cuda.current_stream())
    nvtx_range("sigma", False)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = a.elapsed_time(b)
    fl = sum(e["flops"] for e in prof.values() if not e.get("name", "").startswith("stage:"))
    print(json.dumps({"config": name, "precision": args.sigma_only, "vectors": cfg["nroots"], "ms": ms,
                      "algorithmic_tflops": fl / (ms * 1e-3) / 1e12,
                      "kernels": {k: {"launches": e["launches"], "ms": round(e["total_ms"], 3)}
                                  for k, e in prof.items()}}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="ea2x3_o40_v200_q1200")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--no-fp64-davidson", action="store_true")
    ap.add_argument("--no-gradient", action="store_true", help="EE workloads: skip the adjoint and its check")
    ap.add_argument("--mixed", default="bf16x3", choices=["bf16x3", "bf16x6"],
                    help="split precision of the mixed Davidson")
    ap.add_argument("--refine", default="sliced", choices=["sliced", "fp64"],
                    help="product of the Davidson refinement (both FP64-accurate)")
    ap.add_argument("--e2e-setup", default="sliced", choices=["sliced", "fp64"],
                    help="IP/EA/EE: adc_init contractions of the end-to-end run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-subspace", type=int, default=0, help="Davidson subspace limit (0: the library's default)")
    ap.add_argument("--block", type=int, default=0, help="Davidson block size (0: the number of roots)")
    ap.add_argument("--correction", default="davidson", choices=["davidson", "olsen"],
                    help="Davidson correction vectors (preconditioned residuals, or Olsen's)")
    ap.add_argument("--ref-rows", type=int, default=1,
                    help="reference arm: oracle rows per step (about 30 s of one core each)")
    ap.add_argument("--cpu-rows", type=int, default=16,
                    help="CPU baseline: oracle rows, run one per host core (about 30 s each)")
    ap.add_argument("--init-only", action="store_true",
                    help="time adc_init alone (host inputs, the e2e setup) and print its stage and GEMM profile")
    ap.add_argument("--sigma-only", default=None, choices=["bf16x3", "sliced", "sliced24", "fp64"],
                    help="one sigma block of nroots vectors in this precision after three warm-up blocks, "
                         "inside the NVTX range 'sigma' (for a capture of its kernels)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, args.config)
        return

    if args.init_only:
        if rank == 0:
            run_init_profile(args, args.config)
        return
    if args.sigma_only:
        if rank == 0:
            run_sigma_only(args, args.config)
        return
    if args.config in CONFIGS and CONFIGS[args.config]["kind"] == "EE":
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            run_ee(args, args.config)
        return
    if args.config in BATCH_CONFIGS:
        if rank == 0:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            run_batch(args, args.config)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # a dedicated stream shared with the library, so CUDA events on it bracket the library's kernels
    torch.cuda.set_stream(torch.cuda.Stream())
    import paper_2511_21640_gb300 as adcgpu

    cfg = dict(CONFIGS[args.config])
    kind, order, x, nroots = cfg["kind"], cfg["order"], cfg["x"], cfg["nroots"]
    tol = args.tol if args.tol is not None else cfg.get("tol", 1e-5)
    p = config_problem(args.config)
    o, v, Q = p.nocc, p.nvir, p.naux
    # replicas: every rank solves its own instance of the workload
    B = torch.from_numpy(p.B).cuda()
    eo = torch.from_numpy(p.eps_occ).cuda()
    ev = torch.from_numpy(p.eps_vir).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = adcgpu.Context(B, eo, ev, kind=kind, order=order, x=x, stream="torch", refine=args.refine,
                         max_subspace=args.max_subspace, block=args.block, correction=args.correction)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    log(f"init {init_s:.1f} s, N = {ctx.N}")
    stream = torch.cuda.current_stream()

    def solve(prec, t=tol):
        return ctx.davidson(nroots, tol=t, max_iter=300, precision=prec, want_vectors=False)

    for _ in range(args.warmup):
        om, _, e64, st, rc = solve(args.mixed)
        log("warmup solve", st)
    # ---- timed region
    clocks = Clocks()
    clocks.start()
    ctx.profile(True)
    l0 = adcgpu.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    nvtx_range("timed", True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        om, _, e64, st, rc = solve(args.mixed)
        stats.append(st)
    ev1.record(stream)
    nvtx_range("timed", False)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = adcgpu.launch_count() - l0
    if dist:
        # whole job: the slowest replica's time, the kernels of all replicas
        ms = reduce_across([ms], "max")[0]
        launches = int(reduce_across([launches], "sum")[0])
    log(f"timed {ms:.1f} ms for {args.steps} steps")
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    ms_per_step = ms / args.steps
    value = ms_per_step / 1e3 / (nroots * world)

    pk, pk_kind = peaks()
    peak64, peak64_kind = fp64_peak(adcgpu)

    def roofline_of(name, e):
        avg_ms = e["total_ms"] / e["launches"]
        alg = e["flops"] / e["launches"]
        if name.startswith("tc_"):
            # MMA work: the split products per complex product (3 or 6); the sliced digit
            # pairs are recorded as MMA work already
            mma = (1.0 if name.startswith("tc_sliced") else 6.0 if "bf16x6" in name else 3.0) * alg
            ach = mma / (avg_ms * 1e-3) / 1e12
            peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
            return {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "peak_kind": f"bf16 dense sustained ({pk_kind})",
                    "flops_per_launch": mma, "avg_launch_ms": avg_ms, "launches": e["launches"]}
        return alu_row(name, e, peak64, peak64_kind)

    by_kernel = sorted((roofline_of(k, e) for k, e in prof.items() if e["launches"] > 0),
                       key=lambda r: -r["avg_launch_ms"] * r["launches"])
    roof = by_kernel[0]
    attach_traffic(roof, args.config)
    tc_rows = [r for r in by_kernel if r["kernel"].startswith("tc_")]
    roof_tc = tc_rows[0] if tc_rows else None

    # ---- sigma TFLOP/s, mixed vs FP64 (one block of nroots vectors each)
    Xs = torch.from_numpy(random_vectors(ctx.N, nroots, seed=7)).cuda()
    sig = {}
    sig_precs = (args.mixed, "sliced", "fp64") if kind in ("IP", "EA") else (args.mixed, "fp64")
    for prec in sig_precs:
        ctx.sigma(Xs, prec)
        torch.cuda.synchronize()
        ctx.profile(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        reps = 3 if prec != "fp64" else 1
        for _ in range(reps):
            ctx.sigma(Xs, prec)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / reps
        pr = ctx.profile_read()
        ctx.profile(False)
        fl = sum(e["flops"] for e in pr.values()) / reps
        sig[prec] = {"ms": t, "tflops": fl / (t * 1e-3) / 1e12, "flops": fl}
    log("sigma", sig)
    # the whole mixed sigma block (packing, FP64 main block, epilogues included) against the
    # BF16 tensor peak: counted as 3M BF16x3 (9 BF16 real MACs per complex MAC) and as executed
    # (the real embedding: 12 per complex MAC)
    peak_tc = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    alg_tf = sig[args.mixed]["tflops"]
    tensor_share = {"algorithmic_tflops": alg_tf, "tflops_3m_count": alg_tf * 18 / 8,
                    "frac_3m_count": alg_tf * 18 / 8 / peak_tc, "tflops_mma_executed": alg_tf * 24 / 8,
                    "frac_mma_executed": alg_tf * 24 / 8 / peak_tc, "peak_tflops": peak_tc,
                    "peak_kind": f"bf16 dense sustained ({pk_kind})"}
    S64 = ctx.sigma(Xs, "fp64")

    def rel_to_fp64(S):
        return float(((S - S64).abs().pow(2).sum(1).sqrt() / S64.abs().pow(2).sum(1).sqrt()).max().item())

    sig_rel = rel_to_fp64(ctx.sigma(Xs, args.mixed))
    sig_rel_sliced = rel_to_fp64(ctx.sigma(Xs, "sliced")) if "sliced" in sig else None

    # ---- the residuals of the timed solve's roots recomputed with the FP64 sigma
    # (the solve itself checks them with the sliced product by default)
    om_v, Yv, e_v, _, _ = ctx.davidson(nroots, tol=tol, max_iter=300, precision=args.mixed, want_vectors=True)
    Yt = torch.from_numpy(Yv).cuda()
    R64 = ctx.sigma(Yt, "fp64") - torch.from_numpy(np.asarray(om_v)).cuda()[:, None] * Yt
    resid_fp64 = [float(r) for r in R64.abs().pow(2).sum(1).sqrt().cpu().numpy()]
    del Yt, R64

    # ---- FP64 Davidson for the comparison and the 1e-6 Eh check
    fp64 = None
    if not args.no_fp64_davidson and cfg.get("fp64_davidson", True):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        om64, _, e6, st6, rc6 = ctx.davidson(nroots, tol=tol, max_iter=300, precision="fp64", want_vectors=False)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t1
        log(f"fp64 davidson {t64:.1f} s", st6)
        fp64 = {"s_per_root": t64 / nroots, "iterations": st6["iterations"], "sigma_calls": st6["sigma_calls"],
                "max_eig_diff_vs_mixed": float(np.abs(om64 - om).max()),
                "eig_diff_vs_mixed": [float(d) for d in np.asarray(om) - np.asarray(om64)],
                "err64": [float(e) for e in e6], "rc": rc6}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        Bh = torch.from_numpy(p.B).pin_memory()
        eoh, evh = torch.from_numpy(p.eps_occ), torch.from_numpy(p.eps_vir)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        with adcgpu.Context(Bh, eoh, evh, kind=kind, order=order, x=x, refine=args.refine,
                            setup=args.e2e_setup, max_subspace=args.max_subspace, block=args.block,
                            correction=args.correction) as c2:
            t3 = time.perf_counter()
            om2, _, e2, st2, rc2 = c2.davidson(nroots, tol=tol, max_iter=300, precision=args.mixed,
                                               want_vectors=False)
        te2e, ti2e = time.perf_counter() - t2, t3 - t2
        if dist:
            # whole job: the slowest replica's time for the roots of all replicas
            te2e, ti2e = reduce_across([te2e, ti2e], "max")
        log(f"e2e {te2e:.1f} s (init {ti2e:.1f} s)")
        ref_om = om64 if fp64 is not None else om
        e2e = {"value": te2e / (nroots * world), "unit": "s/root",
               "h2d_bytes_per_step": int(world * (p.B.nbytes + 8 * (o + v))),
               "d2h_bytes_per_step": int(world * 16 * nroots),
               "includes": "adc_init (H2D copy + operator setup) + adc_davidson" +
                           (f", on each of {world} replicas (slowest replica's time)" if world > 1 else ""),
               "setup": args.e2e_setup, "init_s": ti2e, "rc": int(rc2),
               "max_eig_diff_vs_" + ("fp64_davidson" if fp64 is not None else "timed_solve"):
                   float(np.abs(np.asarray(om2) - np.asarray(ref_om)).max()),
               "eig_diff": [float(d) for d in np.asarray(om2) - np.asarray(ref_om)],
               "err64": [float(e) for e in e2], "sigma_calls": st2["sigma_calls"],
               "sigma_calls_fp64": st2["sigma_calls_fp64"], "sigma_calls_mid": st2["sigma_calls_mid"]}

    cpu = None
    parity = None
    if rank == 0 and world == 1 and args.cpu_rows > 0 and oracle_solve_feasible(args.config):
        # the oracle's whole solve of the same workload: its time and its eigenvalues
        cpu = oracle_davidson_baseline(args.config)
        ref_w = np.asarray(cpu["omega"])
        parity = {"oracle_eigenvalues": cpu["omega"],
                  "max_abs_diff_mixed_davidson": float(np.abs(np.asarray(om) - ref_w).max()),
                  "max_abs_diff_fp64_davidson": (float(np.abs(np.asarray(om64) - ref_w).max())
                                                 if fp64 is not None else None)}
        log("oracle solve", parity)
    elif rank == 0 and world == 1 and args.cpu_rows > 0:
        smp = oracle_rows_pool(("config", args.config), kind, order, x, 1, args.cpu_rows)
        try:
            parity = sampled_parity(ctx, (smp["X"], smp["idx"], smp["R"]), ("fp64", args.mixed, "sliced"))
        except Exception as exc:  # the check reports, it never stops the run
            parity = {"error": str(exc)[:200]}
        log("sampled parity", parity)
        spr, note = sigma_vectors_per_root(
            args.config, (np.mean([s["sigma_calls"] for s in stats]) / nroots, "this run's mixed solve"))
        cpu = cpu_baseline_of(smp, ctx.N, spr, note, kind)
        cpu["gpu_mixed_sigma_vectors_per_root"] = float(np.mean([s["sigma_calls"] for s in stats]) / nroots)

    last = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "s/root", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{args.mixed}+" + ("f64 from exact bf16 digit products" if args.refine == "sliced" else "f64"),
        "data": "synthetic",
        "config": {"workload": args.config, "kind": kind, "order": order, "x": x, "nocc": o, "nvir": v, "naux": Q,
                   "nroots": nroots, "tol_fp64_residual": tol, "N": ctx.N, "replicas": world,
                   "max_subspace": args.max_subspace, "block": args.block, "correction": args.correction,
                   "l2": "operators larger than L2 (packed <ab||cd> 6.3 GB FP64, 3.2 GB per BF16 plane)"},
        "clocks": clk, "gpu_launches": int(launches), "roofline": roof, "roofline_tensor_core": roof_tc,
        "roofline_by_kernel": by_kernel,
        "sigma": {**sig, "speedup": sig["fp64"]["ms"] / sig[args.mixed]["ms"],
                  "rel_diff_mixed_vs_fp64": sig_rel, "rel_diff_sliced_vs_fp64": sig_rel_sliced,
                  "speedup_sliced": (sig["fp64"]["ms"] / sig["sliced"]["ms"]) if "sliced" in sig else None,
                  "vectors": nroots, "tensor_roofline": tensor_share},
        "sampled_parity": parity,
        "refine": args.refine,
        "fp64_davidson": fp64,
        "mixed_davidson": {"omega": [float(w) for w in om], "err64": [float(e) for e in e64],
                           "err64_source": "sliced product" if args.refine == "sliced" else "fp64 product",
                           "residual_fp64_recomputed": resid_fp64,
                           "iterations": last["iterations"], "sigma_calls": last["sigma_calls"],
                           "sigma_calls_fp64": last["sigma_calls_fp64"], "sigma_calls_mid": last["sigma_calls_mid"],
                           "rc": int(rc)},
        "init_s": init_s, "e2e": e2e, "cpu_baseline": cpu,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
