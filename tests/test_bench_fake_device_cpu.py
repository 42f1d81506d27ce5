"""bench.py's GPU leg run against a stand-in for the device library (no GPU).

The stand-in answers the calls the bench makes (context, Davidson, sigma,
profile, launch counter, FP64 probe) with the explicit matrix of the small
IP-ADC(3) workload, or with a diagonal matrix of a larger workload's
dimension (the default EA workload, a small EE one), and torch's CUDA entry
points are replaced by host no-ops. Nothing here measures anything: the test checks that the bench's
orchestration runs to the end and that its JSON line carries every key of
the benchmark contract with consistent types and values.
"""
import io
import json
import os
import sys
import time
import types
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synthetic import CONFIGS, config_problem  # noqa: E402

CFG = "ip3_o8_v24_q96"


def _fake_library(cfg=CFG):
    """Stand-in library: the explicit matrix of the small workload, or for a
    large one a diagonal matrix of the right dimension (the bench only needs
    answers of the right shape there)."""
    from oracle import adc
    c = CONFIGS[cfg]
    if cfg == CFG:
        p = config_problem(cfg)
        M = adc.explicit_matrix(c["kind"], c["order"], c["x"], p.B, p.eps_occ, p.eps_vir)
        w, V = np.linalg.eigh(M)
        apply = lambda X: X @ M.T  # noqa: E731
    else:
        n = bench._dim(c["kind"], c["nocc"], c["nvir"])
        d = np.linspace(0.5, 9.0, n)
        w, V = d, None
        apply = lambda X: X * d[None, :]  # noqa: E731
    lib = types.ModuleType("paper_2511_21640_gb300")
    lib.apply = apply
    lib.launches = 0

    class Context:
        def __init__(self, B, eo, ev, kind="IP", order=3, x=1.0, **opts):
            # (the gradient check's contexts move x by a finite-difference step)
            assert (kind, order) == (c["kind"], c["order"]) and abs(x - c["x"]) < 1e-3
            self.N = w.shape[0]
            self.prof = False
            self.stats = {}

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            self.close()

        def close(self):
            pass

        def _record(self, name, flops, nbytes=0.0):
            lib.launches += 1
            if self.prof:
                e = self.stats.setdefault(name, {"name": name, "launches": 0, "total_ms": 0.0, "flops": 0.0,
                                                 "bytes": 0.0})
                e["launches"] += 1
                e["total_ms"] += 0.5
                e["flops"] += flops
                e["bytes"] += nbytes

        def sigma(self, X, precision="fp64"):
            Xn = X.numpy() if torch.is_tensor(X) else np.asarray(X)
            k = Xn.shape[0]
            name = {"fp64": "zgemm_fp64/main", "bf16x3": "tc_bf16x3/sigma",
                    "sliced": "tc_sliced/sigma"}.get(precision, "other")
            self._record(name, 8.0 * k * self.N * self.N, 16.0 * k * self.N)
            return torch.from_numpy(apply(Xn))

        def davidson(self, nroots, tol=1e-8, max_iter=200, precision="fp64", want_vectors=True, **kw):
            self._record("gram_fp64/extend", 8.0 * 40 * nroots * self.N, 16.0 * 48 * self.N)
            self._record("combine_fp64", 8.0 * 40 * nroots * self.N, 16.0 * 48 * self.N)
            st = {"iterations": 12, "sigma_calls": 4 * nroots, "sigma_calls_fp64": nroots,
                  "sigma_calls_mid": 0, "iterations_fp64": 3}
            if not want_vectors:
                Y = None
            elif V is not None:
                Y = np.ascontiguousarray(V[:, :nroots].T)
            else:
                Y = np.zeros((nroots, self.N), np.complex128)
                Y[np.arange(nroots), np.arange(nroots)] = 1.0
            return w[:nroots].copy(), Y, np.full(nroots, 1e-10), st, 0

        def profile(self, on=True):
            self.prof = bool(on)
            if on:
                self.stats = {}

        def profile_read(self):
            return {k: dict(e) for k, e in self.stats.items()}

        def memory(self):
            return {"in_use": 1 << 30, "peak": 2 << 30}

        def sigma_adjoint(self, Y, wts):
            self._record("adjoint_fp64", 1.0)
            p = config_problem(cfg)
            return np.zeros_like(p.B), np.zeros(p.nocc), np.zeros(p.nvir), 0.0

    lib.Context = Context
    lib.launch_count = lambda: lib.launches
    lib.diag_fp64_peak = lambda blocks, iters: (1.26, 1.0)
    return lib


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return 1e3 * (other.t - self.t)


def _patch_device(monkeypatch, lib):
    monkeypatch.setitem(sys.modules, "paper_2511_21640_gb300", lib)
    for name, val in {"set_device": lambda *a, **k: None, "set_stream": lambda *a, **k: None,
                      "Stream": lambda *a, **k: object(), "synchronize": lambda *a, **k: None,
                      "current_stream": lambda *a, **k: object(), "Event": _Event}.items():
        monkeypatch.setattr(torch.cuda, name, val, raising=False)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(bench, "nvtx_range", lambda *a, **k: None)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)


def _run_main(monkeypatch, argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    return json.loads([ln for ln in buf.getvalue().splitlines() if ln.startswith("{")][-1])


def _check_contract(d):
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "clocks", "gpu_launches", "roofline",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["metric"] == bench.METRIC and d["unit"] == "s/root" and d["higher_is_better"] is False
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    r = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r, key
    assert r["bound"] in ("hbm", "tensor", "alu") and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    cb = d["cpu_baseline"]
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in cb, key
    assert cb["kind"] == "oracle" and cb["unit"] == "s/root" and cb["value"] > 0
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in d["e2e"], key


def test_bench_gpu_leg_line_against_a_stand_in(monkeypatch):
    _patch_device(monkeypatch, _fake_library())
    d = _run_main(monkeypatch, ["--config", CFG, "--steps", "2", "--warmup", "3"])
    _check_contract(d)

    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["config"]["workload"] == CFG
    assert d["value"] > 0 and abs(d["value"] - d["ms_per_step"] / 1e3 / CONFIGS[CFG]["nroots"]) < 1e-12
    assert d["gpu_launches"] == 2 * 2  # two solves in the timed region, two recorded launches each
    e = d["e2e"]
    p = config_problem(CFG)
    assert e["h2d_bytes_per_step"] == p.B.nbytes + 8 * (p.nocc + p.nvir)
    assert e["d2h_bytes_per_step"] == 16 * CONFIGS[CFG]["nroots"]
    # the small workload's oracle solve: its eigenvalues against the stand-in's (the explicit matrix)
    assert d["sampled_parity"]["max_abs_diff_mixed_davidson"] < 1e-10
    assert d["sigma"]["rel_diff_mixed_vs_fp64"] == 0.0


def test_bench_default_workload_line_against_a_stand_in(monkeypatch):
    """The default workload (EA-ADC(2)+x(3), o=40, v=200, Q=1200) takes the
    oracle-rows branch of the CPU baseline; the rows come from the stand-in
    here, so only the orchestration and the line are checked."""
    cfg = "ea2x3_o40_v200_q1200"
    lib = _fake_library(cfg)
    _patch_device(monkeypatch, lib)

    def rows_pool(spec, kind, order, x, dd_order, n_rows, seed=5, xseed=5, workers=None):
        c = CONFIGS[cfg]
        rows, idx = bench.pick_rows(kind, c["nocc"], c["nvir"], n_rows, seed)
        X = bench.random_vectors(bench._dim(kind, c["nocc"], c["nvir"]), 1, seed=xseed)
        R = lib.apply(X)[:, idx]
        return {"X": X, "idx": idx, "R": R, "wall_s": 2.0, "row_s": 2.0, "workers": 2, "rows": n_rows}

    monkeypatch.setattr(bench, "oracle_rows_pool", rows_pool)
    d = _run_main(monkeypatch, ["--steps", "1", "--warmup", "3", "--cpu-rows", "4"])
    _check_contract(d)
    assert d["config"]["workload"] == cfg and d["config"]["N"] == 796200
    cb = d["cpu_baseline"]
    spr, _ = bench.sigma_vectors_per_root(cfg)
    assert abs(cb["value"] - 2.0 / 4 * 796200 * spr) < 1e-6 * cb["value"]
    assert d["sampled_parity"]["fp64"]["max_abs_err"] == 0.0
    assert d["e2e"]["h2d_bytes_per_step"] == 16 * 1200 * 240 ** 2 + 8 * 240


def _replica_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK="0")
    mp_ = pytest.MonkeyPatch()
    try:
        _patch_device(mp_, _fake_library())
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(world))  # _patch_device cleared them
        init = dist.init_process_group
        mp_.setattr(dist, "init_process_group", lambda backend, *a, **k: init("gloo", *a, **k))
        mp_.setattr(sys, "argv", ["bench.py", "--config", CFG, "--steps", "2", "--warmup", "3"])
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.main()
        out[rank] = buf.getvalue()
    finally:
        mp_.undo()


def test_bench_replicas_on_gloo_ranks():
    """Two replicas (torchrun's environment, gloo standing in for NCCL): only
    rank 0 prints, the line is whole-job (n_gpus 2, the launches of both
    replicas, s/root over both replicas' roots) and carries no CPU baseline
    (that one runs at one GPU only)."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_replica_rank, args=(2, port, out), nprocs=2, join=True)
    lines0 = [ln for ln in out[0].splitlines() if ln.startswith("{")]
    assert len(lines0) == 1 and not [ln for ln in out[1].splitlines() if ln.startswith("{")]
    d = json.loads(lines0[0])
    assert d["n_gpus"] == 2 and d["config"]["replicas"] == 2
    assert d["gpu_launches"] == 2 * 2 * 2  # two replicas, two solves each, two recorded launches each
    assert abs(d["value"] - d["ms_per_step"] / 1e3 / (2 * CONFIGS[CFG]["nroots"])) < 1e-12
    assert d["cpu_baseline"] is None
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 2 * (config_problem(CFG).B.nbytes + 8 * 32)
    assert "replicas" in e["includes"]


def test_bench_ee_leg_line_against_a_stand_in(monkeypatch):
    """The EE leg (EE-ADC(2)+x(3), o=12, v=60, Q=360) with warm-up solves, the
    gradient check and the oracle-rows baseline (rows from the stand-in)."""
    cfg = "ee2x3_o12_v60_q360"
    lib = _fake_library(cfg)
    _patch_device(monkeypatch, lib)

    def rows_pool(spec, kind, order, x, dd_order, n_rows, seed=5, xseed=5, workers=None):
        c = CONFIGS[cfg]
        rows, idx = bench.pick_rows(kind, c["nocc"], c["nvir"], n_rows, seed)
        X = bench.random_vectors(bench._dim(kind, c["nocc"], c["nvir"]), 1, seed=xseed)
        return {"X": X, "idx": idx, "R": lib.apply(X)[:, idx], "wall_s": 1.0, "row_s": 1.0, "workers": 2,
                "rows": n_rows}

    monkeypatch.setattr(bench, "oracle_rows_pool", rows_pool)
    d = _run_main(monkeypatch, ["--config", cfg, "--warmup", "3", "--cpu-rows", "4"])
    _check_contract(d)
    assert d["warmup"] == 3 and d["config"]["workload"] == cfg
    e = d["e2e"]
    p = config_problem(cfg)
    assert e["h2d_bytes_per_step"] == p.B.nbytes + 8 * (p.nocc + p.nvir)
    assert abs(e["value"] - (e["init_s"] + e["operators_s"] + e["first_solve_s"]) / 4) < 1e-12
    assert d["gradient"]["fd_step"] == 1e-5 and d["sampled_parity"]["fp64"]["max_abs_err"] == 0.0


def test_bench_batched_leg_line_against_a_stand_in(monkeypatch):
    """The batched leg over four small problems (two waves) with a stand-in
    batch: warm-up solves, one timed solve per wave, the line's keys."""
    from synthetic import make_problem
    sizes = [dict(kind="IP" if i % 2 == 0 else "EA", nocc=3 + i, nvir=8 + i, naux=6 * (8 + i), order=3, x=0.5,
                  seed=i) for i in range(4)]
    monkeypatch.setattr(bench, "batch_sizes", lambda name, n=None: sizes)
    monkeypatch.setattr(bench, "batch_problems", lambda name, n=None, select=None: [
        make_problem(sizes[i]["nocc"], sizes[i]["nvir"], sizes[i]["naux"], seed=i, kind=sizes[i]["kind"], x=0.5)
        for i in (range(len(sizes)) if select is None else select)])
    lib = types.ModuleType("paper_2511_21640_gb300")
    lib.launches = 0
    solves = []

    class Context:
        def __init__(self, B, eo, ev, kind="IP", order=3, x=1.0, **opts):
            self.N = bench._dim(kind, len(eo), len(ev))
            self.d = np.linspace(0.5, 5.0, self.N)

        def sync(self):
            pass

        def close(self):
            pass

    class Batch:
        def __init__(self, ctxs):
            self.ctxs = ctxs
            self.i = dict(grouped_ms=0.0, grouped_flops=0.0, grouped_launches=0, batch_ms=0.0, tc_flops=0.0,
                          batches=0, graph_launches=0)

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            pass

        def use_graphs(self, on=True):
            pass

        def sigma(self, Xs, precision="bf16x3", outs=None):
            for c, X, S in zip(self.ctxs, Xs, outs):
                S.copy_(torch.from_numpy(X.numpy() * c.d[None, :]))
            for k, dv in (("grouped_ms", 1.0), ("grouped_flops", 1e12), ("grouped_launches", 1),
                          ("batch_ms", 1.5), ("tc_flops", 1e12), ("batches", 1), ("graph_launches", 1)):
                self.i[k] += dv
            lib.launches += 1

        def davidson(self, nroots, tol=1e-8, max_iter=200, precision="bf16x3"):
            solves.append(len(self.ctxs))
            lib.launches += 2
            n = len(self.ctxs)
            om = np.array([c.d[:nroots] for c in self.ctxs])
            sts = [{"iterations": 10, "sigma_calls": 3 * nroots, "sigma_calls_fp64": nroots}] * n
            return om, np.full((n, nroots), 1e-6), np.zeros(n, int), sts, 0

        def info(self):
            return dict(self.i)

    lib.Context = Context
    lib.Batch = Batch
    lib.launch_count = lambda: lib.launches
    lib.batch_plan = lambda sz, nroots, budget: (2, np.arange(len(sz)), np.array([0, 0, 1, 1]), None, None)
    _patch_device(monkeypatch, lib)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (64 << 30, 80 << 30), raising=False)
    d = _run_main(monkeypatch, ["--config", "batch64_ipea", "--warmup", "3", "--cpu-rows", "0"])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "clocks", "gpu_launches", "roofline", "e2e"):
        assert key in d, key
    assert solves == [2, 2, 2, 2, 2, 2, 2, 2]  # per wave: three warm-up solves and the timed one
    assert d["warmup"] == 3 and d["config"]["problems"] == 4 and d["config"]["waves"] == 2
    assert d["gpu_launches"] == 2 * 2  # the two timed solves' launches only
    assert d["e2e"]["value"] > 0 and "first batched Davidson" in d["e2e"]["includes"]
