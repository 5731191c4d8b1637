"""Host logic of bench.py on the CPU.

Each GPU of a multi-GPU run factors its own replica (no collective on the
data path); the bench reports the slowest rank's time and counts the units
of every rank.  These tests run that reduction with two gloo ranks, the
reference arm's rules (rank 0 only, the GPU arm's config), the roofline and
kernel-table arithmetic, the traffic record's validity rule and the clock
summary.
"""
import json
import multiprocessing as mp
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        ms = bench._max_over_ranks(10.0 + 5.0 * rank, "cpu")   # rank 1 is the slow one
        q.put((rank, ms, bench._job_rate(1000, ws, ms), bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_units():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [g[0] for g in got] == [0, 1]
    for rank, ms, rate, dist_env in got:
        assert ms == 15.0                              # max over ranks, seen by both
        assert rate == pytest.approx(2 * 1000 / 0.015)  # both ranks' units over the slowest time
        assert dist_env == (2, rank, rank)


def test_job_rate_of_one_rank_is_units_over_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench._job_rate(65536, 1, 1000.0) == pytest.approx(65536.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""   # no work and no line on the other ranks


def test_traffic_record_follows_the_captured_kernel_only():
    """The ncu traffic of a kernel stays valid while that kernel's source (and
    its helpers') is unchanged, whatever else changes in its file."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = "int a;\n__global__ void k(int x) {\n  x += 1;\n}\nint b;\n"
    base = bench._kernel_source_sha(src, ["__global__ void k("])
    assert bench._kernel_source_sha(src.replace("int b;", "int c;"), ["__global__ void k("]) == base
    assert bench._kernel_source_sha(src.replace("x += 1", "x += 2"), ["__global__ void k("]) != base
    assert bench._kernel_source_sha(src, ["missing("]) is None
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    text = open(os.path.join(ROOT, "paper_2603_09381_gb300", "csrc", rec["dense_matvec64"]["source"])).read()
    for a in rec["dense_matvec64"]["anchors"]:
        assert a in text


def test_reference_arm_reports_the_block_it_ran(monkeypatch, capsys):
    """The reference arm's config names the block the oracle actually timed (a
    4 x 4 block of the recipe, N = 4,096), says which workload it is a block of,
    and declares that it is not the GPU arm's config."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda nx, reps=1: (2 * 128 * nx * nx, [2.0] * reps))

    class Args:
        steps, warmup, gpus, workload, precision = 2, 1, 1, "star16", "mixed"

    assert bench.run_reference(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    cfg = dict(line["config"])
    assert cfg.pop("block_of") == bench._workload_config(16, 65536, 4, "mixed", 1)["workload"]
    assert cfg == bench._workload_config(4, 4096, 2, "fp64", 1)
    assert line["same_config_as_gpu_arm"] is False
    assert line["value"] == pytest.approx(4096 / 2.0)
    assert line["cpu_baseline"]["kind"] == "oracle" and "4x4 block" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_roofline_of_the_dominant_kernel():
    """The roofline object names the kernel with the largest time and divides
    its algorithmic work by its summed event time; FP64 kernels against the
    nominal FP64 peak, the byte-counted FP32 CPQR against the copy bandwidth."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    steps = 2
    prof = {"dense_matvec64": {"launches": 2, "ms": 400.0, "work": 2 * 2.75e11},
            "qr_panel32": {"launches": 120, "ms": 150.0, "work": 0.0}}
    r = bench._roofline(prof, steps)
    assert r["kernel"] == "dense_matvec64" and r["launches_per_step"] == 1 and r["kernel_ms_per_step"] == 200.0
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(2.75e11 / 0.2 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_NOMINAL_TFLOPS)
    # with measured FMA peaks the fraction is taken against them
    rm = bench._roofline(prof, steps, {"fp64_tflops": 1.2, "fp32_tflops": 70.0})
    assert rm["peak"] == 1.2 and rm["frac"] == pytest.approx(rm["achieved"] / 1.2) and "measured" in rm["peak_source"]
    r32 = bench._roofline({"qr_update32": {"launches": 3, "ms": 10.0, "work": 3.5e11}}, 1, {"fp64_tflops": None,
                                                                                          "fp32_tflops": 70.0})
    assert r32["peak"] == 70.0 and r32["achieved"] == pytest.approx(35.0)
    assert r["traffic"] == json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))[
        "dense_matvec64"]["bytes_per_launch"]
    r = bench._roofline({"cpqr_step32": {"launches": 10, "ms": 50.0, "work": 1e11}}, 1)
    peak, _ = bench._peaks()
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(1e11 / 0.05 / 1e9) and r["frac"] == pytest.approx(r["achieved"] / peak)
    t = bench._kernel_table(prof, steps)
    assert list(t) == ["dense_matvec64", "qr_panel32"] and t["qr_panel32"] == {"launches": 60, "ms": 75.0}


def test_clock_summary_parses_samples():
    """Median SM clock under load, the maximum clock and every throttle reason
    seen active in the nvidia-smi samples."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line", "0, [N/A], 2070, 0, 0x0, a, b, c, d"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = []
    assert c.summary()["sm_mhz"] is None
