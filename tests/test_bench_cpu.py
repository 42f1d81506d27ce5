"""Host-side pieces of bench.py, without a GPU: the FP64 roofline rows, the
DRAM traffic attached to the dominant kernel, the algorithmic sigma flop
count, the reference arm's JSON line (the CPU oracle on the small IP-ADC(3)
workload), and the reductions that turn several replicas' figures into
whole-job ones (gloo ranks on CPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _entry(name, launches, ms, flops, nbytes):
    return {"name": name, "launches": launches, "total_ms": ms, "flops": flops, "bytes": nbytes}


def test_alu_row_rates_and_bytes():
    # 10 launches of 1 ms, 1.2e9 algorithmic flops each: 1.2 TFLOP/s
    e = _entry("combine_fp64", 10, 10.0, 1.2e10, 5.0e9)
    r = bench.alu_row("combine_fp64", e, 1.25, "test")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 1.2) < 1e-12
    assert abs(r["frac"] - 1.2 / 1.25) < 1e-12
    # 3M products execute 6 of the 8 algorithmic flops
    assert abs(r["executed_frac"] - 0.75 * 1.2 / 1.25) < 1e-12
    assert abs(r["algorithmic_bytes_per_launch"] - 5.0e8) < 1e-3
    # a kernel outside the 3M set executes what it counts
    r2 = bench.alu_row("other_fp64", e, 1.25, "test")
    assert abs(r2["executed_frac"] - r2["frac"]) < 1e-15


@pytest.mark.parametrize("kernel,ratio", [("combine_fp64", bench.COMBINE_DRAM_RATIO),
                                          ("gram_fp64/extend", bench.GRAM_DRAM_RATIO)])
def test_traffic_scaled_from_the_captured_ratio(kernel, ratio):
    roof = {"kernel": kernel, "traffic": None, "algorithmic_bytes_per_launch": 4.0e8}
    bench.attach_traffic(roof, "ea2x3_o40_v200_q1200")
    assert abs(roof["traffic"] - ratio * 4.0e8) < 1e-3
    assert "scaled" in roof["traffic_note"]
    # the captured launches read each operand byte about once
    assert 0.9 < ratio < 1.1


def test_traffic_kept_only_where_captured():
    roof = {"kernel": "zgemm_fp64/ladder", "traffic": None, "algorithmic_bytes_per_launch": 1.0}
    bench.attach_traffic(roof, "ea2x3_o40_v200_q1200")
    assert roof["traffic"] == 7.795e9
    other = {"kernel": "zgemm_fp64/ladder", "traffic": None, "algorithmic_bytes_per_launch": 1.0}
    bench.attach_traffic(other, "ee2x3_o30_v150_q900")
    assert other["traffic"] is None
    tc = {"kernel": "tc_grouped_bf16x3/grouped", "traffic": None, "algorithmic_bytes_per_launch": 1.0}
    bench.attach_traffic(tc, "ea2x3_o40_v200_q1200")
    assert tc["traffic"] is None


def test_sigma_flops_formula_terms():
    o, v, k = 40, 200, 8
    pv = v * (v - 1) // 2
    n2 = o * pv
    expect = 8.0 * (2 * v * n2 * k + pv * pv * o * k + (o * v) ** 2 * v * k + v * v * k)
    assert bench.sigma_flops_formula(o, v, 1200, k) == expect
    # the bench workload's block of 8 vectors, as reported by the GPU runs
    assert abs(bench.sigma_flops_formula(o, v, 1200, k) - 1.853e12) / 1.853e12 < 1e-3


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--config", "ip3_o8_v24_q96", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["higher_is_better"] is False and d["unit"] == "s/root"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "ip3_o8_v24_q96"
    # small enough for the oracle's whole solve: timed, not extrapolated, and
    # its eigenvalues are the lowest of the explicit matrix
    cb = d["cpu_baseline"]
    assert "not extrapolated" in cb["sample"] and cb["iterations"] > 0 and cb["max_residual"] <= 1e-8
    assert abs(d["value"] - cb["wall_s"] / 4) < 1e-9 * d["value"]
    import numpy as np
    from oracle import adc
    from synthetic import config_problem
    p = config_problem("ip3_o8_v24_q96")
    w = np.linalg.eigvalsh(adc.explicit_matrix("IP", 3, 1.0, p.B, p.eps_occ, p.eps_vir))[:4]
    assert np.abs(np.asarray(cb["omega"]) - w).max() < 1e-10


def test_reference_arm_rows_line():
    """A workload too large for the oracle's whole solve (one EA problem of the
    batched workload): oracle rows on the host cores, scaled to s/root."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--config", "batch64_ipea", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    cb = d["cpu_baseline"]
    assert d["impl"] == "reference" and d["value"] == cb["value"] > 0
    assert cb["threads_per_process"] == 1 and cb["cores"] >= 1 and "rows" in cb["sample"]
    assert d["config"]["kind"] == "EA"


def _reduce_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica's step time, launch count and end-to-end times
        mx = bench.reduce_across([10.0 + rank, 3.5 * (world - rank)], "max")
        sm = bench.reduce_across([100 + rank], "sum")
        out[rank] = (mx, sm)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_reduce_across_replicas_on_gloo(world):
    """The whole-job figures of several replicas: the slowest replica's times
    and the sum of their kernel launches, the same on every rank."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_reduce_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        mx, sm = out[r]
        assert mx == [10.0 + world - 1, 3.5 * world]
        assert sm == [float(sum(100 + q for q in range(world)))]


def test_sigma_vectors_per_root_sources():
    """Each recorded scale names where it comes from; unknown workloads take the default."""
    spr, note = bench.sigma_vectors_per_root("ea2x3_o40_v200_q1200")
    assert abs(spr - 333 / 8) < 1e-12 and "FP64 Davidson" in note
    spr, note = bench.sigma_vectors_per_root("ee2x3_o30_v150_q900")
    assert abs(spr - 440 / 4) < 1e-12 and "mixed" in note
    assert "assumed" in bench.sigma_vectors_per_root("ee3_o60_v300_q1800")[1]
    assert bench.sigma_vectors_per_root("nope", (7.0, "x")) == (7.0, "x")
    assert bench.sigma_vectors_per_root("nope") is None


def test_launch_list_summary(tmp_path):
    """ncu_launches.py: per-kernel launch counts and device-time totals of an
    ncu CSV launch list, units converted to ms, namespaces stripped, other
    metrics and non-CSV lines ignored."""
    import ncu_launches
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = ['"1","adc::(anonymous namespace)::k_gram<32, 8>(const double2 *)","gpu__time_duration.sum","us","1,500"\n',
            '"2","adc::(anonymous namespace)::k_gram<32, 8>(const double2 *)","gpu__time_duration.sum","ms","2.5"\n',
            '"3","k_tc_grouped(int)","gpu__time_duration.sum","ns","250000"\n',
            '"3","k_tc_grouped(int)","dram__bytes_read.sum","byte","7"\n',
            '"4","void adc::<unnamed>::k_combine<8>(const double2 *)","gpu__time_duration.sum","ms","1.0"\n']
    f = tmp_path / "launches.csv"
    f.write_text("==PROF== Connected to process\n" + hdr + "".join(rows))
    agg = ncu_launches.summarise(str(f))
    assert set(agg) == {"k_gram<32, 8>", "k_tc_grouped", "void k_combine<8>"}
    assert agg["k_gram<32, 8>"][0] == 2 and abs(agg["k_gram<32, 8>"][1] - 4.0) < 1e-12
    assert agg["k_tc_grouped"][0] == 1 and abs(agg["k_tc_grouped"][1] - 0.25) < 1e-12
