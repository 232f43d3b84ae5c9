#!/usr/bin/env python
"""Throughput of the fourth-order BGK lattice Boltzmann hot path on D3Q19 256^3 (periodic).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 256]

One benchmark step is one pass of the hot path over the workload: one FP64 lattice update at each
relaxation time tau in {0.6, 0.8, 1.2}, one update of the FP32-deviation path and one adjoint update
(FP32-deviation adjoint with the dL/dR accumulation) at tau = 0.8, each a fused stream+collide kernel
over all 256^3 nodes. `value` is the FP64 path's MLUPS (million lattice-node updates per second,
whole job over N GPUs) over the three tau; every form is reported under "forms", with tau = 1/2 (the
s = 2 collision) as an extra line. Inputs are resident in HBM and each population buffer (2.5 GB)
exceeds the 126 MB L2, so no L2 flush is needed between iterations. `e2e` times the FP64 metric
through the public API with host buffers: upload of phi0 and grad phi0 from pinned memory, init,
1000 steps at tau = 0.8 (the workload's run length), macro and download of phi, per job, over
--e2e-steps consecutive jobs whose copies run on a second stream alongside the neighbouring jobs'
steps (the first upload and the last download of the timed region overlap nothing).

Under torchrun (N > 1) every rank runs the workload on its own GPU (independent replicas: the path
has no data exchange between boxes of one replica), timing is bracketed by a barrier and CUDA
synchronisation on both sides, and rank 0 reports the max over ranks.

--impl reference times the FP64 CPU oracle (the reference implementation of this paper-only
repository) on the host cores: per benchmark step, one oracle step at each tau on a 128^3 sample of
the workload (--ref-n).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM GB/s (% of peak), D3Q19 256^3: FP64 vs FP32-mixed vs adjoint"
UNIT = "MLUPS"
U = (0.1, 0.1, 0.1)
NMODES, SEED = 8, 2
TAUS = (0.6, 0.8, 1.2)
TAU_DEV = 0.8
BYTES_PER_SITE = {"fp64": 2 * 19 * 8, "fp32dev": 2 * 19 * 4 + 16, "adjoint": 2 * 19 * 4 + 16 + 16}
E2E_STEPS = 1000


def workload(n):
    return {"workload": "D3Q19 %d^3 periodic, 8 seeded Fourier modes (k in 1..3), u=(0.1,0.1,0.1), "
                        "tau in {0.6, 0.8, 1.2}, R=0" % n,
            "lattice": "D3Q19", "n": n, "sites": n ** 3, "tau": list(TAUS), "u": list(U), "modes": NMODES,
            "step": "one fp64 update at each tau, one fp32dev update and one adjoint(fp32dev, with dL/dR) "
                    "update at tau=%g" % TAU_DEV,
            "l2": "inputs larger than L2 (population buffers 2.5 GB / 1.3 GB)",
            "e2e_job": "H2D phi0+grad (pinned), init, %d fp64 steps at tau=%g, macro, D2H phi" % (E2E_STEPS, TAU_DEV)}


# the sources that define k_step_fp64: its translation unit and the device headers it inlines
FP64_KERNEL_SOURCES = [os.path.join(ROOT, "paper_2410_13165_gb300", "csrc", f)
                       for f in ("lhe_step_fp64.cu", "lhe_device.cuh", "lhe_sites.cuh", "lhe_internal.h")]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sources_hash(paths) -> str:
    """First 16 hex digits of the SHA-256 of the given source files, concatenated in order."""
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_srcs, path=None):
    """DRAM bytes per launch of the FP64 step kernel from the committed ncu summary, if the kernel's
    sources (its translation unit and the device headers it inlines) are unchanged since the capture
    (the summary records their hash)."""
    path = path or os.path.join(ROOT, "profiles", "fp64_step_d3q19_256.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    h = kernel_sources_hash(kernel_srcs)
    want = None
    for line in txt.splitlines():
        if line.startswith("source_sha256_16:"):
            want = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].strip())
            return val if want == h else None
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, each with nvidia-smi's own timestamp, taken
    every `interval_ms` for as long as the sampler runs; summary(t0, t1) keeps the samples inside a
    timed region (wall-clock datetimes of its start and end)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.gpu, self.interval, self.samples, self.proc = gpu_index, interval_ms, [], None
        self.windows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        import datetime

        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                sm, mx = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.REASONS, parts[6:10]) if v.lower() == "active"}
            self.samples.append((ts, sm, mx, reasons))

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    @staticmethod
    def now():
        import datetime

        return datetime.datetime.now()

    def mark(self):
        """Context manager recording a timed region's window (see summary_windows)."""
        import contextlib

        @contextlib.contextmanager
        def cm():
            t0 = self.now()
            try:
                yield
            finally:
                self.windows.append((t0, self.now()))
        return cm()

    def summary_windows(self, windows=None):
        """Clocks over the samples that fall inside any of the windows (default: every window marked)."""
        ws = list(self.windows if windows is None else windows)
        sel = [x for x in list(self.samples) if any(a <= x[0] <= b for a, b in ws)]
        reasons = set()
        for x in sel:
            reasons |= x[3]
        return {"sm_mhz": float(np.median([x[1] for x in sel])) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "reasons": sorted(reasons), "samples": len(sel),
                "interval_ms": self.interval, "windows": len(ws),
                "window_s": float(sum((b - a).total_seconds() for a, b in ws))}

    def summary(self, t0=None, t1=None):
        """Median SM clock, max clock, every throttle reason seen and the sample count in [t0, t1]
        (all samples when no window is given)."""
        sel = [x for x in list(self.samples) if (t0 is None or x[0] >= t0) and (t1 is None or x[0] <= t1)]
        reasons = set()
        for x in sel:
            reasons |= x[3]
        out = {"sm_mhz": float(np.median([x[1] for x in sel])) if sel else None,
               "sm_max_mhz": sel[-1][2] if sel else None, "reasons": sorted(reasons), "samples": len(sel),
               "interval_ms": self.interval}
        if t0 is not None and t1 is not None:
            out["window_s"] = (t1 - t0).total_seconds()
        return out


def dist_setup():
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier_max(x: float, ws: int, device: str = "cuda") -> float:
    """Maximum of x over the ranks (the slowest rank decides a timed region)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int, cuda: bool = True):
    """CUDA synchronisation and a process-group barrier on both sides of a timed region."""
    import torch

    if cuda:
        torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def whole_job_mlups(sites_per_rank: int, ws: int, ms_max: float) -> float:
    """Whole-job throughput: lattice updates of all ranks divided by the slowest rank's time."""
    return ws * sites_per_rank / (ms_max * 1e-3) / 1e6


def cpu_oracle_mlups(n: int, steps: int, threads: int):
    """The FP64 oracle on the host cores: `steps` steps at each tau of the workload on n^3 nodes."""
    from oracle import oracle as O
    from paper_2410_13165_gb300 import workloads as W

    O.set_threads(threads)
    phi0, grad, _, _ = W.periodic_problem(3, n, NMODES, SEED)
    dt = 0.0
    for tau in TAUS:
        m = O.Model(3, n, 0.0, 1.0, U, tau=tau)
        f = m.step(m.init(phi0, grad, 3), 0, 1)
        t0 = time.perf_counter()
        m.step(f, 1, steps)
        dt += time.perf_counter() - t0
    return len(TAUS) * n ** 3 * steps / dt / 1e6, dt


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    from oracle import oracle as O
    from paper_2410_13165_gb300 import workloads as W

    threads = os.cpu_count() or 1
    O.set_threads(threads)
    n = args.ref_n
    phi0, grad, _, _ = W.periodic_problem(3, n, NMODES, SEED)
    models, states = [], []
    for tau in TAUS:
        m = O.Model(3, n, 0.0, 1.0, U, tau=tau)
        models.append(m)
        states.append(m.step(m.init(phi0, grad, 3), 0, args.warmup))
    t0 = time.perf_counter()
    for i, m in enumerate(models):
        states[i] = m.step(states[i], args.warmup, args.steps)
    dt = time.perf_counter() - t0
    mlups = len(TAUS) * n ** 3 * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": mlups, "unit": UNIT, "impl": "reference", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(args.n),
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "FP64 CPU oracle; per benchmark step one oracle step at each tau in "
                                       "{0.6, 0.8, 1.2} on a D3Q19 %d^3 sample of the workload" % n},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        return _run_ours(args, clk)


def _run_ours(args, clk):
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    ws, rank, local = dist_setup()
    if ws == 1:
        torch.cuda.set_device(0)
    build.build()
    n = args.n
    S = n ** 3
    phi0_np, grad_np, F, X = W.periodic_problem(3, n, NMODES, SEED)
    dev = torch.device("cuda", torch.cuda.current_device())
    phi0 = torch.from_numpy(phi0_np).to(dev)
    grad = torch.from_numpy(np.ascontiguousarray(grad_np).ravel()).to(dev)
    del X

    fp64_names = ["fp64_tau%g" % t for t in TAUS]
    sims = {name: LBM(3, n, u=U, tau=t) for name, t in zip(fp64_names, TAUS)}
    sims["fp32dev"] = LBM(3, n, u=U, tau=TAU_DEV, precision="fp32dev")
    adj = LBM(3, n, u=U, tau=TAU_DEV, precision="fp32dev")
    for s in sims.values():
        s.init(phi0, grad)
    adj.init(phi0, grad)
    adj.step(1)
    adj.adjoint_seed(adj.macro())
    stream = torch.cuda.current_stream()
    order = fp64_names + ["fp32dev"]

    def one_pass(ev=None):
        for i, name in enumerate(order):
            if ev:
                ev[i].record(stream)
            sims[name].step(1)
        if ev:
            ev[len(order)].record(stream)
        adj.adjoint_step(1)
        if ev:
            ev[len(order) + 1].record(stream)

    for _ in range(max(args.warmup, 3)):
        one_pass()
    K = args.steps
    nev = len(order) + 2
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(K)]
    barrier(ws)
    with clk.mark():
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(K):
            one_pass(evs[k])
        t_end.record(stream)
        barrier(ws)
    timed_window = clk.windows[-1]
    total_ms = t_start.elapsed_time(t_end)
    names = order + ["adjoint"]
    per = {name: 0.0 for name in names}
    for k in range(K):
        for i, name in enumerate(names):
            per[name] += evs[k][i].elapsed_time(evs[k][i + 1])
    per = {k: barrier_max(v / K, ws) for k, v in per.items()}
    per["fp64"] = sum(per[nm] for nm in fp64_names) / len(fp64_names)  # mean update time over the tau set
    total_ms = barrier_max(total_ms, ws)
    peak, peak_kind = measured_peaks()
    forms = {}
    for name, ms in per.items():
        bps = BYTES_PER_SITE["fp64" if name.startswith("fp64") else name]
        gbs = bps * S / (ms * 1e-3) / 1e9
        forms[name] = {"mlups": whole_job_mlups(S, ws, ms), "ms_per_lb_step": ms, "gbs_per_gpu": gbs,
                       "frac_of_hbm": gbs / peak, "bytes_per_site": bps}
    forms["fp64"]["tau"] = list(TAUS)
    forms["fp32dev"]["tau"] = forms["adjoint"]["tau"] = TAU_DEV
    # the s = 2 collision (tau = 1/2) outside the timed pass, for reference
    half = LBM(3, n, u=U, tau=0.5)
    half.init(phi0, grad)
    ms_half = barrier_max(_timed(lambda: half.step(1), 50, clk=clk), ws)
    half.close()
    gbs = BYTES_PER_SITE["fp64"] * S / (ms_half * 1e-3) / 1e9
    forms["fp64_tau0.5"] = {"mlups": whole_job_mlups(S, ws, ms_half), "ms_per_lb_step": ms_half, "gbs_per_gpu": gbs,
                            "frac_of_hbm": gbs / peak, "bytes_per_site": BYTES_PER_SITE["fp64"],
                            "note": "s = 2 collision, timed separately (50 steps)"}
    # the precision form at 128^3 (the precision workload's grid), where a step is ~0.1 ms and fixed
    # costs per launch weigh most: FP32 deviations vs FP64 in calls of one step and of 50 steps
    if args.extra_forms:
        forms["precision_128"] = precision_ratio_128(W, LBM, clk, ws)
        # the differentiation workload (D3Q19 128^3, FP32 deviations, T = 1024 through torch.autograd)
        forms["differentiation_128"] = differentiation_workload(clk)
        # the Dirichlet box of Example 3 (D4Q33 64^4, full-way, order 4)
        forms["dirichlet_d4q33_64"] = dirichlet_box_form(clk, ws)
    fp64 = forms["fp64"]
    traffic = profiled_traffic(FP64_KERNEL_SOURCES)

    # e2e through the public API with host buffers (FP64 path, whole job). Consecutive jobs are
    # pipelined as a serving loop would run them: a job's inputs are uploaded on a copy stream into one
    # of two device buffers while the job before it steps, and its result is downloaded on the copy
    # stream while the next job steps. Every job's copies lie inside the timed region (the first upload
    # and the last download are not overlapped with anything).
    e2e = None
    if args.e2e_steps > 0:
        h_phi0 = torch.from_numpy(phi0_np).pin_memory()
        h_grad = torch.from_numpy(np.ascontiguousarray(grad_np).ravel()).pin_memory()
        h_out = [torch.empty(S, dtype=torch.float64).pin_memory() for _ in range(2)]
        d_in = [(torch.empty_like(phi0), torch.empty_like(grad)) for _ in range(2)]
        sim = sims["fp64_tau%g" % TAU_DEV]
        cstream = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]    # the buffer's inputs are on the device
        ev_used = [torch.cuda.Event() for _ in range(2)]  # the job's init has read the buffer
        ev_res = [torch.cuda.Event() for _ in range(2)]   # the job's result is ready
        # phases of the last job: upload (copy stream), init, steps, macro, download (copy stream)
        ph = [torch.cuda.Event(enable_timing=True) for _ in range(8)]

        def upload(j):
            bi = j % 2
            cstream.wait_event(ev_used[bi])
            ph[0].record(cstream)
            with torch.cuda.stream(cstream):
                d_in[bi][0].copy_(h_phi0, non_blocking=True)
                d_in[bi][1].copy_(h_grad, non_blocking=True)
            ph[1].record(cstream)
            ev_in[bi].record(cstream)

        def run(j):
            bi = j % 2
            stream.wait_event(ev_in[bi])
            ph[2].record(stream)
            sim.init(d_in[bi][0], d_in[bi][1])
            ev_used[bi].record(stream)
            ph[3].record(stream)
            sim.step(E2E_STEPS)
            ph[4].record(stream)
            m = sim.macro()
            ph[5].record(stream)
            ev_res[bi].record(stream)
            cstream.wait_event(ev_res[bi])
            m.record_stream(cstream)
            ph[6].record(cstream)
            with torch.cuda.stream(cstream):
                h_out[bi].copy_(m, non_blocking=True)
            ph[7].record(cstream)

        def jobs(count):
            upload(0)
            for j in range(count):
                if j + 1 < count:
                    upload(j + 1)
                run(j)

        for bi in range(2):
            ev_used[bi].record(stream)
        jobs(2)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cstream.wait_event(a)
        jobs(args.e2e_steps)
        stream.wait_stream(cstream)
        b.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        e2e_ms = barrier_max(a.elapsed_time(b) / args.e2e_steps, ws)
        e2e = {"value": whole_job_mlups(S * E2E_STEPS, ws, e2e_ms), "unit": UNIT, "ms_per_job": e2e_ms,
               "h2d_bytes_per_step": (h_phi0.numel() + h_grad.numel()) * 8, "d2h_bytes_per_step": h_out[0].numel() * 8,
               "lb_steps_per_job": E2E_STEPS, "jobs": args.e2e_steps,
               "pipelining": "each job's upload overlaps the previous job's steps, its download the next job's",
               "last_job_phases_ms": {"h2d": ph[0].elapsed_time(ph[1]), "init": ph[2].elapsed_time(ph[3]),
                                      "steps": ph[3].elapsed_time(ph[4]), "macro": ph[4].elapsed_time(ph[5]),
                                      "d2h": ph[6].elapsed_time(ph[7])}}

    cpu = None
    if rank == 0 and args.cpu_baseline:
        threads = os.cpu_count() or 1
        mlups, secs = cpu_oracle_mlups(args.cpu_n, args.cpu_steps, threads)
        cpu = {"value": mlups, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "FP64 CPU oracle, D3Q19 %d^3 sample of the workload, %d steps at each tau in "
                         "{0.6, 0.8, 1.2} (%.1f s)" % (args.cpu_n, args.cpu_steps, secs)}

    if rank == 0:
        line = {"metric": METRIC, "value": fp64["mlups"], "unit": UNIT, "n_gpus": ws, "steps": K,
                "warmup": max(args.warmup, 3), "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload(n), parallelism="replicas" if ws > 1 else "single GPU"),
                "forms": forms,
                "roofline": {"bound": "hbm", "kernel": "k_step_fp64<3,fwd,periodic,scaled> (tau in {0.6, 0.8, 1.2}; "
                                                      "1 launch in 49..218 is the renormalising general form)",
                             "achieved": fp64["gbs_per_gpu"], "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                             "frac": fp64["gbs_per_gpu"] / peak, "traffic": traffic,
                             "algorithmic_bytes_per_launch": BYTES_PER_SITE["fp64"] * S},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": (len(order) + 1) * K,
                "clocks": clk.summary(*timed_window),
                "clocks_all_timed_regions": clk.summary_windows()}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def precision_ratio_128(W, LBM, clk, ws, n=128):
    """FP32-deviation vs FP64 step time on D3Q19 n^3 (periodic, the workload's modes and u) at tau = 1/2
    (the precision workload) and 0.8, in calls of one step and of 50 steps."""
    import torch

    phi0_np, grad_np, _, _ = W.periodic_problem(3, n, NMODES, SEED)
    phi0 = torch.from_numpy(phi0_np).cuda()
    grad = torch.from_numpy(np.ascontiguousarray(grad_np).ravel()).cuda()
    peak, _ = measured_peaks()
    out = {"n": n}
    for tau in (0.5, TAU_DEV):
        ms = {}
        for prec in ("fp64", "fp32dev"):
            sim = LBM(3, n, u=U, tau=tau, precision=prec)
            sim.init(phi0, grad)
            one = barrier_max(_timed(lambda: sim.step(1), 200, clk=clk), ws)
            many = barrier_max(_timed(lambda: sim.step(50), 4, clk=clk), ws) / 50
            sim.close()
            bps = BYTES_PER_SITE[prec]
            ms[prec] = {"ms_one_step_calls": one, "ms_50_step_calls": many,
                        "frac_of_hbm_one_step_calls": bps * n ** 3 / (one * 1e-3) / 1e9 / peak,
                        "frac_of_hbm_50_step_calls": bps * n ** 3 / (many * 1e-3) / 1e9 / peak}
        out["tau%g" % tau] = dict(ms, ratio_one_step_calls=ms["fp64"]["ms_one_step_calls"] / ms["fp32dev"]["ms_one_step_calls"],
                                  ratio_50_step_calls=ms["fp64"]["ms_50_step_calls"] / ms["fp32dev"]["ms_50_step_calls"])
    return out


def dirichlet_box_form(clk, ws, n=64, steps=20):
    """Example 3's box [-1, 1]^4 (n^4 nodes, D4Q33), phi = sin(pi sum_i (x_i - u_i t)), full-way order-4
    boundaries, u = (0.05, 0.2, 0.08, 0.1), K = 3: time per step (boundary data included) and the fraction
    of the roofline of an interior node (528 B per node and step)."""
    import torch

    from paper_2410_13165_gb300 import LBM
    from paper_2410_13165_gb300 import workloads as W

    u = (0.05, 0.2, 0.08, 0.1)
    X = W.node_coords(4, n, -1.0, 2.0 / (n - 1))
    arg = np.pi * X.sum(axis=0)
    del X
    phi0 = torch.from_numpy(np.sin(arg)).cuda()
    grad = torch.from_numpy(np.repeat((np.pi * np.cos(arg))[None, :], 4, axis=0).ravel()).cuda()
    del arg
    sim = LBM(4, n, -1.0, 1.0, u=u, bc="fullway")
    sim.init(phi0, grad)
    del phi0, grad
    sim.set_boundary_wave([1.0], [[np.pi] * 4], [0.0])
    ms = barrier_max(_timed(lambda: sim.step(1), steps, clk=clk), ws)
    sim.close()
    peak, _ = measured_peaks()
    return {"n": n, "bc": "fullway", "order": 4, "ms_per_step": ms, "mlups": n ** 4 / (ms * 1e-3) / 1e6,
            "frac_of_interior_roofline": 528 * n ** 4 / (ms * 1e-3) / 1e9 / peak, "boundary_nodes": sim.n_boundary}


def differentiation_workload(clk, n=128, T=1024, reps=3):
    """D3Q19 n^3, FP32-deviation forward of T steps, loss 1/2 |phi(T) - target|^2, gradients w.r.t.
    phi0 and R(x) through torch.autograd (the backward pass is T adjoint steps: the scheme is affine
    in the state, so nothing is recomputed). Returns forward / backward times and their ratio."""
    import torch

    from paper_2410_13165_gb300 import LBM
    from paper_2410_13165_gb300 import workloads as W
    from paper_2410_13165_gb300.autograd import lbm_loss

    X = W.node_coords(3, n, 0.0, 1.0 / n)
    phi0 = torch.from_numpy(W.fourier_field(3, NMODES, SEED).value(X)).cuda()
    R = torch.from_numpy(0.1 * W.fourier_field(3, 4, SEED + 10).value(X)).cuda()
    target = torch.from_numpy(W.fourier_field(3, 8, SEED + 11).value(X)).cuda()
    del X
    sim = LBM(3, n, u=U, precision="fp32dev")
    times = {"forward": [], "backward": []}
    for rep in range(reps + 1):
        p, r = phi0.clone().requires_grad_(True), R.clone().requires_grad_(True)
        torch.cuda.synchronize()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        with (clk.mark() if rep else _null()):
            a.record()
            loss = lbm_loss(p, r, sim, T, target)
            b.record()
            loss.backward()
            c.record()
            torch.cuda.synchronize()
        if rep:
            times["forward"].append(a.elapsed_time(b))
            times["backward"].append(b.elapsed_time(c))
    sim.close()
    fw, bw = float(np.mean(times["forward"])), float(np.mean(times["backward"]))
    return {"T": T, "forward_ms": fw, "backward_ms": bw, "backward_over_forward": bw / fw, "loss": float(loss),
            "note": "no recomputation: the backward pass is T adjoint steps from dL/dphi_T"}


def _null():
    import contextlib

    return contextlib.nullcontext()


# ------------------------------------------------------------------------------------------------
# Other workloads of the same path (each prints one JSON line; the default is the line above).

def _timed(fn, steps, warmup=3, clk=None):
    """Mean milliseconds per call of fn over `steps` calls after `warmup` calls (CUDA events on the
    current stream); the timed region's window is recorded on the clock sampler when one is given."""
    import contextlib

    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with (clk.mark() if clk is not None else contextlib.nullcontext()):
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_d4q33_dirichlet(args, clk):
    """Example 3's 4D box [-1, 1]^4 (64^4 nodes), phi = sin(pi sum_i (x_i - u_i t)): full-way at
    u = (0.05, 0.2, 0.08, 0.1) and half-way at u = 1e-3 (1,1,1,1), order-4 boundaries, K = 3 init; then
    the same boxes with the manufactured solution exp(-t) prod_i sin(pi x_i) and its source."""
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()
    n = args.n if args.n != 256 else 64
    out = {"metric": "MLUPS, D4Q33 %d^4 Dirichlet box" % n, "unit": UNIT, "dtype": "f64", "data": "synthetic"}
    for bc, u in (("fullway", (0.05, 0.2, 0.08, 0.1)), ("halfway", (1e-3,) * 4)):
        dx = 2.0 / ((n - 1) if bc == "fullway" else n)
        X = W.node_coords(4, n, -1.0, dx, halfway=(bc == "halfway"))
        arg = np.pi * X.sum(axis=0)
        phi0 = torch.from_numpy(np.sin(arg)).cuda()
        grad = torch.from_numpy(np.repeat((np.pi * np.cos(arg))[None, :], 4, axis=0).ravel()).cuda()
        sim = LBM(4, n, -1.0, 1.0, u=u, bc=bc)
        sim.init(phi0, grad)
        sim.set_boundary_wave([1.0], [[np.pi] * 4], [0.0])
        ms = _timed(lambda: sim.step(1), args.steps, clk=clk)
        T = sim.step_index * sim.dt
        exact = np.sin(np.pi * (X - np.asarray(u)[:, None] * T).sum(axis=0))
        err = float(np.sqrt(np.mean((sim.macro().cpu().numpy() - exact) ** 2)))
        out[bc] = {"mlups": n ** 4 / (ms * 1e-3) / 1e6, "ms_per_step": ms, "boundary_nodes": sim.n_boundary,
                   "boundary_fraction": sim.n_boundary / n ** 4, "steps_run": sim.step_index, "t_final": T,
                   "rmse_vs_exact": err,
                   "gbs_interior_equiv": 528 * n ** 4 / (ms * 1e-3) / 1e9}
        sim.close()
        del phi0, grad
    # the manufactured solution exp(-t) prod_i sin(pi x_i) with its source R = phi_t + u.grad phi
    # (varying in x and t), data and source formed on the device (lhe_lbm_set_boundary_sine_product)
    for bc, u in (("fullway", (0.05, 0.2, 0.08, 0.1)), ("halfway", (1e-3,) * 4)):
        dx = 2.0 / ((n - 1) if bc == "fullway" else n)
        X = W.node_coords(4, n, -1.0, dx, halfway=(bc == "halfway"))
        sim = LBM(4, n, -1.0, 1.0, u=u, bc=bc)
        sim.init(torch.from_numpy(W.sine_product_value(X, 0.0)).cuda(),
                 torch.from_numpy(W.sine_product_grad(X, 0.0).ravel()).cuda(),
                 torch.from_numpy(W.sine_product_source(X, 0.0, u)).cuda())
        sim.set_boundary_sine_product()
        ms = _timed(lambda: sim.step(1), args.steps, clk=clk)
        T = sim.step_index * sim.dt
        exact = W.sine_product_value(X, T)
        err = float(np.sqrt(np.mean((sim.macro().cpu().numpy() - exact) ** 2)))
        out[bc + "_sine_product"] = {"mlups": n ** 4 / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps_run": sim.step_index,
                                     "t_final": T, "rmse_vs_exact": err, "max_abs_exact": float(np.max(np.abs(exact))),
                                     "data": "exp(-t) prod_i sin(pi x_i), source phi_t + u.grad phi, device-formed"}
        sim.close()
        del X, exact
    out["clocks"] = clk.summary_windows()
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def run_d5q51_fp32dev(args, clk):
    """D5Q51 24^5 periodic (7.96 M nodes), tau = 1/2: FP32-deviation vs FP64 MLUPS, and the error of
    both against the FP64 CPU oracle: on the 24^5 box after --oracle-steps steps (the oracle's run
    time bounds that count) and on a 12^5 box after --error-steps steps (the workload's 2000)."""
    import torch

    from oracle import oracle as O
    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()
    O.set_threads(os.cpu_count() or 1)
    n = args.n if args.n != 256 else 24
    u = (0.02, 0.04, 0.06, 0.08, 0.1)

    def problem(nn):
        X = W.node_coords(5, nn, 0.0, 1.0 / nn)
        F = W.fourier_field(5, NMODES, SEED + 3)
        return F.value(X), np.ascontiguousarray(F.grad(X))

    phi0_np, grad_np = problem(n)
    phi0 = torch.from_numpy(phi0_np).cuda()
    grad = torch.from_numpy(grad_np.ravel()).cuda()
    res = {}
    for prec, bps in (("fp64", 816), ("fp32dev", 424)):
        sim = LBM(5, n, u=u, precision=prec)
        sim.init(phi0, grad)
        # at least 200 steps (0.1-0.2 s), so that the clock sampler sees the timed region several times
        ms = _timed(lambda: sim.step(1), max(args.steps, 200), clk=clk)
        res[prec] = {"mlups": n ** 5 / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                     "gbs": bps * n ** 5 / (ms * 1e-3) / 1e9, "bytes_per_site": bps}
        sim.close()
    peak, _ = measured_peaks()
    for v in res.values():
        v["frac_of_hbm"] = v["gbs"] / peak

    def errors(nn, steps, phi0_np, grad_np):
        m = O.Model(5, nn, 0.0, 1.0, u)
        t0 = time.perf_counter()
        ref = m.phi(m.step(m.init(phi0_np, grad_np, 3), 0, steps))
        secs = time.perf_counter() - t0
        out = {"grid": "%d^5" % nn, "steps": steps, "oracle_seconds": secs}
        for prec in ("fp64", "fp32dev"):
            sim = LBM(5, nn, u=u, precision=prec)
            sim.init(torch.from_numpy(phi0_np).cuda(), torch.from_numpy(grad_np.ravel()).cuda())
            sim.step(steps)
            out["rel_maxnorm_err_%s_vs_oracle" % prec] = float(
                np.max(np.abs(sim.macro().cpu().numpy() - ref)) / np.max(np.abs(ref)))
            sim.close()
        return out

    errs = [errors(n, args.oracle_steps, phi0_np, grad_np)]
    if args.error_steps > 0:
        errs.append(errors(12, args.error_steps, *problem(12)))
    print(json.dumps({"metric": "MLUPS, D5Q51 %d^5 periodic: FP64 vs FP32-deviation" % n, "unit": UNIT,
                      "forms": res, "ratio_fp32dev_over_fp64": res["fp32dev"]["mlups"] / res["fp64"]["mlups"],
                      "errors_vs_oracle": errs, "clocks": clk.summary_windows()}))
    return 0


def run_adjoint_ratio(args, clk):
    """The differentiation workload: D3Q19 128^3, FP32-deviation forward, T = 1024, loss
    1/2 |phi(T) - target|^2, gradients w.r.t. phi0 and R(x) through torch.autograd."""
    from paper_2410_13165_gb300 import build

    build.build()
    r = differentiation_workload(clk)
    print(json.dumps({"metric": "adjoint/forward time ratio, D3Q19 128^3 FP32-deviation, T=1024", "unit": "ratio",
                      "value": r["backward_over_forward"], **r, "clocks": clk.summary_windows()}))
    return 0


def run_convergence(args, clk):
    """Convergence slopes on the GPU at tau = 1/2 (periodic, K = 3): D2Q9 N = 16..128 (4 modes) and
    D3Q19 N = 32..256 (8 modes), FP64 and FP32-deviation; T = 1 (steps = N)."""
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()
    out = {"metric": "RMSE and convergence slopes vs the exact solution, tau = 1/2, T = 1", "unit": "rate"}
    for d, Ns, u, modes in ((2, (16, 32, 64, 128), (0.1, 0.2), 4), (3, (32, 64, 128, 256), U, NMODES)):
        for prec in ("fp64", "fp32dev"):
            errs = []
            for N in Ns:
                X = W.node_coords(d, N, 0.0, 1.0 / N)
                F = W.fourier_field(d, modes, SEED + 20 + d)
                sim = LBM(d, N, u=u, precision=prec)
                sim.init(torch.from_numpy(F.value(X)).cuda(), torch.from_numpy(np.ascontiguousarray(F.grad(X)).ravel()).cuda())
                sim.step(N)
                exact = F.value(X, shift=np.asarray(u) * 1.0)
                errs.append(float(np.sqrt(np.mean((sim.macro().cpu().numpy() - exact) ** 2))))
                sim.close()
            out["D%dQ%d_%s" % (d, 2 * d * d + 1, prec)] = {
                "N": list(Ns), "rmse": errs, "slopes": [float(np.log2(a / b)) for a, b in zip(errs, errs[1:])]}
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def run_fp32_floor(args, clk):
    """Where the FP32-deviation form stops converging at fourth order: periodic, tau = 1/2, K = 3,
    T = 1 (steps = N), RMSE against the exact solution for FP64 and FP32 deviations, D2Q9 N = 64..2048
    (4 modes) and D3Q19 N = 64..512 (8 modes). Fields of the large grids are generated on the host in
    slabs of the slowest axis."""
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()
    out = {"metric": "RMSE vs the exact solution and slopes, FP64 vs FP32 deviations, tau = 1/2, T = 1", "unit": "rate"}

    def slabs(d, N, rows=None):
        rows = rows or max(1, (1 << 22) // N ** (d - 1))
        for z0 in range(0, N, rows):
            z1 = min(N, z0 + rows)
            axes = [np.arange(N) / N] * (d - 1) + [np.arange(z0, z1) / N]
            grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
            yield z0, z1, np.stack([g.ravel() for g in grids])

    for d, Ns, u, modes in ((2, (64, 128, 256, 512, 1024, 2048), (0.1, 0.2), 4), (3, (64, 128, 256, 512), U, NMODES)):
        F = W.fourier_field(d, modes, SEED + 30 + d)
        res = {}
        for prec in ("fp64", "fp32dev"):
            errs = []
            for N in Ns:
                S, plane = N ** d, N ** (d - 1)
                phi0 = torch.empty(S, dtype=torch.float64, device="cuda")
                grad = torch.empty(d, S, dtype=torch.float64, device="cuda")
                for z0, z1, X in slabs(d, N):
                    phi0[z0 * plane:z1 * plane] = torch.from_numpy(F.value(X))
                    grad[:, z0 * plane:z1 * plane] = torch.from_numpy(F.grad(X))
                sim = LBM(d, N, u=u, precision=prec)
                sim.init(phi0, grad.reshape(-1))
                del phi0, grad
                sim.step(N)
                phi = sim.macro()
                sim.close()
                se = 0.0
                for z0, z1, X in slabs(d, N):
                    diff = phi[z0 * plane:z1 * plane].cpu().numpy() - F.value(X, shift=np.asarray(u) * 1.0)
                    se += float(np.sum(diff * diff))
                del phi
                torch.cuda.empty_cache()
                errs.append((se / S) ** 0.5)
            res[prec] = {"N": list(Ns), "rmse": errs, "slopes": [float(np.log2(a / b)) for a, b in zip(errs, errs[1:])]}
        ratio = [b / a for a, b in zip(res["fp64"]["rmse"], res["fp32dev"]["rmse"])]
        res["fp32dev_over_fp64"] = ratio
        out["D%dQ%d" % (d, 2 * d * d + 1)] = res
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def run_order_law(args, clk):
    """Eq. (cr-estimation) on the GPU: convergence rates of the Dirichlet schemes against the boundary
    order P and the initialisation order K (2D, Example 1's setting with R = 5 and exact solutions of
    the wave family, T = 2; full-way at u = (0.1, 0.1), half-way at u = (0.01, 0.01); N = 20, 40, 80)."""
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()
    wave = dict(a=[1.0, 0.5], kappa=[(np.pi, np.pi), (2.0, -1.0)], theta=[0.3, 1.1], b=0.2)

    def rmse(bc, P, K, N, u):
        n = N + 1 if bc == "fullway" else N
        X = W.node_coords(2, n, 0.0, 1.0 / N, halfway=(bc == "halfway"))
        phi0, grad = W.wave_solution(X, 0.0, u, 5.0, **wave)
        sim = LBM(2, n, u=u, R=5.0, bc=bc, bc_order=P, init_order=K)
        sim.init(torch.from_numpy(phi0).cuda(), torch.from_numpy(np.ascontiguousarray(grad).ravel()).cuda())
        sim.set_boundary_wave(wave["a"], wave["kappa"], wave["theta"], wave["b"])
        steps = int(round(2.0 / sim.dt))
        sim.step(steps)
        ex, _ = W.wave_solution(X, steps * sim.dt, u, 5.0, **wave)
        e = float(np.sqrt(np.mean((sim.macro().cpu().numpy() - ex) ** 2)))
        sim.close()
        return e

    out = {"metric": "convergence rate vs boundary order P and init order K (Eq. (cr-estimation))", "unit": "rate",
           "grids": [20, 40, 80]}
    for bc, u, Ps in (("fullway", (0.1, 0.1), (1, 3, 4)), ("halfway", (0.01, 0.01), (1, 2, 3, 4))):
        for P in Ps:
            for K in (1, 3):
                errs = [rmse(bc, P, K, N, u) for N in (20, 40, 80)]
                out["%s_P%d_K%d" % (bc, P, K)] = {
                    "rmse": errs, "rates": [float(np.log2(a / b)) for a, b in zip(errs, errs[1:])],
                    "law_min_K+1_P": min(K + 1, P)}
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def run_examples(args, clk):
    """Example 2 (tanh bubble, periodic, 2D on [-1, 1]^2 and 3D on [-1/2, 1/2]^3) and Example 3's
    periodic 4D box: the total kinetic entropy sum_x sum_k f_k^2 / (2 omega_k) over time (conserved
    when every omega_k > 0, not for u = 0.4 (1, 1, 1, 1) in 4D), and the RMSE convergence rates at
    T = 1 for the first- and third-order initialisations (Tables 2 and 3 report ~2 and ~4)."""
    import torch

    from paper_2410_13165_gb300 import LBM, build
    from paper_2410_13165_gb300 import workloads as W

    build.build()

    def t_(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()

    def bubble(d, N, u, K, T, every=None, unstable=False):
        lo, hi = (d - 4) / 2.0, (4 - d) / 2.0
        dx = (hi - lo) / N
        X = W.node_coords(d, N, lo, dx)
        v, g = W.tanh_bubble(X, 0.0, u, lo, hi)
        sim = LBM(d, N, lo, hi, u=u, init_order=K, allow_unstable=unstable)
        sim.init(t_(v), t_(g))
        steps = int(round(T / sim.dt))
        series = []
        if every:
            for n in range(0, steps + 1, every):
                if n:
                    sim.step(every)
                series.append([n * sim.dt, sim.diagnostics()["entropy"]])
        else:
            sim.step(steps)
        ex, _ = W.tanh_bubble(X, steps * sim.dt, u, lo, hi)
        err = float(np.sqrt(np.mean((sim.macro().cpu().numpy() - ex) ** 2)))
        sim.close()
        return err, series

    out = {"metric": "kinetic entropy over time and RMSE rates, Examples 2 and 3", "unit": "rate"}
    ent = {}
    for d, N, us in ((2, 200, [(0.1, 0.2), (0.45, 0.45)]), (3, 100, [(0.1, 0.1, 0.1), (0.05, 0.1, 0.08)])):
        for u in us:
            _, ser = bubble(d, N, u, 3, 1.0, every=max(1, N // 10))
            e0 = ser[0][1]
            ent["D%d_u%s" % (d, ",".join("%g" % x for x in u))] = {
                "t": [x[0] for x in ser], "entropy_rel_change": [x[1] / e0 - 1.0 for x in ser]}
    # Example 3, periodic 4D: sin(pi sum_i (x_i - u_i t)) on [-1, 1]^4, 24^4 nodes
    for uu in (0.05, 0.1, 0.2, 0.4):
        N, u = 24, (uu,) * 4
        X = W.node_coords(4, N, -1.0, 2.0 / N)
        v, g = W.wave_solution(X, 0.0, u, 0.0, a=[1.0], kappa=[(np.pi,) * 4], theta=[0.0])
        sim = LBM(4, N, -1.0, 1.0, u=u, allow_unstable=True)
        sim.init(t_(v), t_(g))
        ser = []
        for n in range(0, 5 * N + 1, N // 2):
            if n:
                sim.step(N // 2)
            e = sim.diagnostics()["entropy"]
            ser.append([n * sim.dt, e if np.isfinite(e) else None])
        ent["D4_u%g" % uu] = {"t": [x[0] for x in ser],
                              "entropy_rel_change": [None if x[1] is None else x[1] / ser[0][1] - 1.0 for x in ser],
                              "min_omega": min(sim.omega)}
        sim.close()
    out["entropy"] = ent
    rates = {}
    for d, Ns, u in ((2, (200, 400, 800, 1600), (0.1, 0.2)), (2, (200, 400, 800, 1600), (0.45, 0.45)),
                     (3, (150, 180, 210, 240, 270, 300), (0.1, 0.1, 0.1))):
        for K in (1, 3):
            errs = [bubble(d, N, u, K, 1.0)[0] for N in Ns]
            rates["D%d_u%s_K%d" % (d, ",".join("%g" % x for x in u), K)] = {
                "N": list(Ns), "rmse": errs,
                "rates": [float(np.log(a / b) / np.log(n2 / n1)) for a, b, n1, n2 in zip(errs, errs[1:], Ns, Ns[1:])]}
    out["rates"] = rates
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def run_stability_map(args, clk):
    """Stability maps (Sec. 4) on the GPU: per velocity the smallest EDF weight (entropy conditions,
    Prop. 1) and the largest spectral radius of Eq. (G) over a xi grid (L2 conditions); the two
    regions are compared away from the boundary min omega = 0, as the paper states they coincide."""
    from paper_2410_13165_gb300 import build, stability_map

    build.build()
    out = {"metric": "stability maps: agreement of the entropy and L2 regions; matrices per second", "unit": "count"}
    cases = [("D2Q9", 2, np.round(np.linspace(-0.8, 0.8, 161), 12), [None], 32),
             ("D3Q19", 3, np.round(np.linspace(-0.6, 0.6, 81), 12), [0.0, 0.2, 0.4], 12),
             ("D4Q33", 4, np.round(np.linspace(-0.4, 0.4, 41), 12), [(0.0, 0.0), (0.1, 0.2)], 6)]
    for name, d, g, extra, nxi in cases:
        for x in extra:
            pts = []
            for a in g:
                for b in g:
                    pts.append((a, b) if d == 2 else ((a, b, x) if d == 3 else (a, b) + tuple(x)))
            S = np.array(pts)
            t0 = time.perf_counter()
            rho, omin = stability_map(d, S, nxi)
            dt = time.perf_counter() - t0
            away = np.abs(omin) > 1e-12
            agree = (omin[away] > 0) == (rho[away] <= 1.0 + 1e-9)
            key = name if x is None else "%s_slice%s" % (name, x)
            out[key] = {"points": len(S), "xi_per_point": nxi ** d, "entropy_stable": int(np.sum(omin > 0)),
                        "l2_stable": int(np.sum(rho <= 1.0 + 1e-9)), "on_boundary": int(np.sum(~away)),
                        "agree_away_from_boundary": int(agree.sum()), "disagree": int((~agree).sum()),
                        "max_rho": float(np.max(rho)), "seconds": dt,
                        "matrices_per_second": len(S) * nxi ** d / dt}
    out.setdefault("clocks", clk.summary())
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--cpu-n", type=int, default=128)
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--ref-n", type=int, default=128)
    ap.add_argument("--error-steps", type=int, default=2000)
    ap.add_argument("--oracle-steps", type=int, default=50)
    ap.add_argument("--extra-forms", type=int, default=1,
                    help="default line: also measure the precision form and the differentiation workload at 128^3 "
                         "and the D4Q33 64^4 Dirichlet box")
    ap.add_argument("--workload", default="d3q19_256",
                    choices=["d3q19_256", "d4q33_dirichlet", "d5q51_fp32dev", "adjoint", "convergence",
                             "order_law", "examples", "stability_map", "fp32_floor"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    others = {"d4q33_dirichlet": run_d4q33_dirichlet, "d5q51_fp32dev": run_d5q51_fp32dev,
              "adjoint": run_adjoint_ratio, "convergence": run_convergence, "order_law": run_order_law,
              "examples": run_examples, "stability_map": run_stability_map, "fp32_floor": run_fp32_floor}
    if args.workload in others:
        if args.steps == 400:
            args.steps = 50
        with ClockSampler(0) as clk:
            return others[args.workload](args, clk)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
