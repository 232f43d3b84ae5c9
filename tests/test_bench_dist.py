"""bench.py's multi-rank path on CPU: two gloo ranks, barrier and max-over-ranks timing."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        bench.barrier(ws, cuda=False)
        ms = bench.barrier_max(10.0 + 5.0 * rank, ws, device="cpu")
        q.put((rank, ms, bench.whole_job_mlups(1000, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]
    # whole job: 2 ranks x 1000 updates in 15 ms
    assert abs(got[0][2] - 2 * 1000 / 15e-3 / 1e6) < 1e-12


def test_clock_sampler_windows_and_reasons():
    """The clock record of a bench line: samples inside each timed region only (by nvidia-smi's own
    timestamps), the median SM clock, and every throttle reason seen in them."""
    import datetime

    import bench

    clk = bench.ClockSampler(0, interval_ms=20)
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = lambda k: t0 + datetime.timedelta(milliseconds=k)  # noqa: E731
    clk.samples = [(ms(0), 1500.0, 2070.0, set()), (ms(20), 2070.0, 2070.0, set()),
                   (ms(40), 2070.0, 2070.0, {"sw_power_cap"}), (ms(60), 1800.0, 2070.0, {"hw_slowdown"}),
                   (ms(80), 2070.0, 2070.0, set())]
    one = clk.summary(ms(10), ms(45))
    assert one["samples"] == 2 and one["sm_mhz"] == 2070.0 and one["reasons"] == ["sw_power_cap"]
    assert abs(one["window_s"] - 0.035) < 1e-12
    clk.windows = [(ms(10), ms(25)), (ms(55), ms(85))]
    both = clk.summary_windows()
    assert both["samples"] == 3 and both["windows"] == 2 and both["reasons"] == ["hw_slowdown"]
    assert both["sm_mhz"] == 2070.0
    assert clk.summary()["samples"] == 5


def test_profiled_traffic_needs_the_sources_the_counters_were_taken_on(tmp_path):
    """The roofline's `traffic` comes from the committed ncu summary only while the kernel's sources
    hash to the value recorded beside the counters; a changed source, a missing or malformed summary
    give null."""
    import sys

    sys.path.insert(0, ROOT)
    import bench

    srcs = []
    for i, text in enumerate(("kernel a\n", "header b\n")):
        f = tmp_path / ("src%d.cu" % i)
        f.write_text(text)
        srcs.append(str(f))
    h = bench.kernel_sources_hash(srcs)
    assert len(h) == 16 and h != bench.kernel_sources_hash(srcs[::-1])
    prof = tmp_path / "prof.md"
    prof.write_text("# k\n\nsource_sha256_16: %s\ndram_bytes_per_launch: 5042171904\n" % h)
    assert bench.profiled_traffic(srcs, str(prof)) == 5042171904.0
    (tmp_path / "src1.cu").write_text("header b, changed\n")
    assert bench.profiled_traffic(srcs, str(prof)) is None
    assert bench.profiled_traffic(srcs, str(tmp_path / "missing.md")) is None
    prof.write_text("no counters here\n")
    assert bench.profiled_traffic(srcs, str(prof)) is None


def test_reference_arm_prints_its_line_on_the_host():
    """`bench.py --impl reference` times the CPU oracle on the host cores (a tiny sample here) and
    prints one JSON line with the contract's keys: impl, the metric of the GPU arm, a cpu_baseline
    describing the run, and an e2e entry without copies."""
    import json
    import subprocess
    import sys

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-n", "8"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    import bench

    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "MLUPS"
    assert line["steps"] == 2 and line["warmup"] >= 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
