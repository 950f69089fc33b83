"""Benchmark: k.q pairs/s of the electron linewidth (Eq. linewidthel) on one GB300.

Headline workload (the largest single-GPU configuration): diamond lattice with a
two-atom basis, nw = 8 Wannier functions, 6 modes (masses 1 and 1.2), 249 Re =
Rp vectors (whole shells), 2000 k-points near the band edges x (60^3 uniform
grid + 10^5 random q = 316,000 q), sigma = 10 meV, T = 300 K: 6.32e8 (k,q)
pairs per step.  A step is one epw_linewidth call: q-side phases and phonons,
k-side bands and vertex, the per-pair interpolation, eigensolve, rotation and
reduction (the wide-shape tensor-core kernels E and G), and the final sum.

The line also carries the fcc nw=4 configuration (1000 k x 40^3 q, the fused
single-kernel form) under "c2", the hexagonal nw=5 configuration (20^3 k x 40^3 q)
with its adjoint under "c5", the other split form and the plain FP64 GPU form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision auto|bf16x3|tf32x3|fp32|fp64]
  python bench.py --impl reference     # the FP64 CPU oracle on a bounded sample of the workload
  python bench.py --workload fcc_nw4|hex_nw5|batch   # another configuration as the line

Under torchrun the k list of the one problem is split into contiguous shards,
one per rank (strong scaling: the total work is fixed); no collective runs in
the timed region, and the shards' Im Sigma are gathered after it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "diamond_nw8"
METRIC = "k·q pairs/s for ImΣ_nk on 1 GB300 (and % roofline) at stated error vs FP64 oracle"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# The split form that meets the 1e-4 relative target against the oracle on each workload
# (tests/test_tcw_gpu.py, tests/test_parity_gpu.py: sampled k at the full q lists).
AUTO_PRECISION = {"diamond_nw8": "bf16x3", "hex_nw5": "bf16x3", "fcc_nw4": "bf16x3"}
DESCR = {
    "diamond_nw8": "diamond nw=8 nat=2 (6 modes, M=1,1.2), 249 Re=Rp, 2000 k (band edges) x (60^3 + 1e5 random) q, "
                   "sigma=10 meV, T=300 K",
    "fcc_nw4": "fcc nw=4 nat=1, 135 Re=Rp, 1000 k (0.2 eV window of E_F) x 40^3 q, sigma=20 meV, T=300 K",
    "hex_nw5": "hexagonal nw=5 nat=3 (9 modes), ~300 Re=Rp, 20^3 k x 40^3 q, sigma=15 meV, T=50 K",
}
CPU_SAMPLE = {"diamond_nw8": (32, 8192), "fcc_nw4": (1000, 2560), "hex_nw5": (64, 16384)}
WIDE_PROFILE = os.path.join(ROOT, "profiles", "k_tcwf_diamond_nw8.md")
WIDE_SOURCE = os.path.join(ROOT, "paper_1604_03525_gb300", "csrc", "epw_tcw.cu")
TC_PROFILE = os.path.join(ROOT, "profiles", "k_tc_linewidth_fcc_nw4.md")
TC_SOURCE = os.path.join(ROOT, "paper_1604_03525_gb300", "csrc", "epw_tc.cu")


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def flops_per_pair(m):
    """Algorithmic contraction flops per (k,q) pair (complex MAC = 8 flops).

    H(k+q): 8 nRe nw^2 (kernel E of the wide form); g(k,q) U_k: 8 nRp 3nat nw^2 (kernel G);
    U_k+q^+ rotation and mode projection, dense: 8 3nat nw^3 + 8 (3nat)^2 nw^2 (CUDA cores;
    the wide form evaluates only the terms whose Gaussians do not underflow).  Eigensolve
    steps, deltas and occupations are not counted.
    """
    nw, nm = m.nw, 3 * m.nat
    h = 8 * nw * nw * len(m.Re)
    g = 8 * nw * nw * nm * len(m.Rp)
    rot = 8 * nm * nw ** 3 + 8 * nm * nm * nw * nw
    return h, g, rot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm_, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm_)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled(path, source, key, form):
    """A figure recorded in a committed ncu summary for this kernel source.

    The summary holds lines `<key> <form> <value> source-sha256 <hash>`; a value is
    used only while the kernel source still has that hash (otherwise the counters
    describe an older kernel and null is reported).
    """
    try:
        sha = hashlib.sha256(open(source, "rb").read()).hexdigest()
        for line in open(path):
            parts = line.strip().strip("`").split()
            if len(parts) == 5 and parts[0] == key and parts[1] == form and parts[3] == "source-sha256":
                if parts[4] == sha:
                    return float(parts[2]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, " + \
                        os.path.relpath(path, ROOT)
                return None, "kernel changed since the ncu capture"
    except OSError:
        pass
    return None, "no ncu capture recorded"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = {}
        for ln in out.splitlines():
            if ":" in ln:
                a, b = ln.split(":", 1)
                info[a.strip()] = b.strip()
        name = info.get("Model name") or info.get("BIOS Model name") or platform.processor()
        return f"{name} ({info.get('Architecture', platform.machine())}, {os.cpu_count()} logical CPUs)"
    except (OSError, subprocess.SubprocessError):
        return f"{platform.machine()}, {os.cpu_count()} logical CPUs"


def oracle_sample(wl_name, nk_s, nq_s):
    import workloads as W
    wl = W.make_workload(wl_name, nq_sub=nq_s)
    k = wl.k[::max(1, len(wl.k) // nk_s)][:nk_s]
    return wl, k


def cpu_baseline(wl_name, nk_s, nq_s):
    """The FP64 oracle (as it stands) on a bounded sample of the workload."""
    import oracle
    wl, k = oracle_sample(wl_name, nk_s, nq_s)
    t0 = time.perf_counter()
    oracle.linewidth(wl.model, k, wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
    dt = time.perf_counter() - t0
    pairs = len(k) * len(wl.q)
    return {"value": pairs / dt, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{len(k)} of the {wl_name} k x {len(wl.q)} q (seeded subsample of its q list), "
                      f"{pairs} pairs, {dt:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    nk_s, nq_s = (16, 2048) if args.workload == "diamond_nw8" else (64, 2048)
    wl, k = oracle_sample(args.workload, nk_s, nq_s)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.linewidth(wl.model, k, wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    pairs = len(k) * len(wl.q)
    ms = 1e3 * float(np.mean(times))
    val = pairs / (ms / 1e3)
    sample = f"{len(k)} k x {len(wl.q)} q per step (seeded subsample of the {args.workload} lists), {pairs} pairs"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": DESCR[args.workload], "sample_per_step": sample},
        "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args):
    """Uneven systems (the seeded 64-system draw at its stated sizes) through one captured CUDA graph.

    Each system draws nw from {1, 2, 4, 5, 8, 12, 18}, nat 1..6, Re and Rp shell targets
    27..400 each, nk 50..5000 (log-uniform) and a q grid N^3 with N in 16..48; the draw is
    redrawn until the vertices take at most 64 GB as complex64.  All jobs run split-BF16 (the
    fused kernel where the shape has one, else the wide or staged tensor-core form); jobs
    whose k-side buffers would pass 8 GiB run their k list in passes.  A step is one graph
    replay; the L2 is flushed between steps.
    """
    import torch
    import paper_1604_03525_gb300 as epw
    import workloads as W
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = W.models.batch_specs(64)
    jobs, pairs, tfl = [], 0, 0.0
    t0 = time.perf_counter()

    def note(msg):
        print(f"[batch {time.perf_counter() - t0:8.1f} s] {msg}", file=sys.stderr, flush=True)

    for sp in specs:
        wm, k, q = W.models.batch_system(sp)
        m = epw.Model(wm)
        jobs.append(dict(model=m, k=torch.tensor(k, device=dev), q=torch.tensor(q, device=dev), wq=None, T=300.0,
                         EF=0.0, sigma=0.05, precision=epw.BF16X3))
        pairs += len(k) * len(q)
        h, g, _ = flops_per_pair(wm)
        tfl += (h + g) * len(k) * len(q)
        del wm
    t_models = time.perf_counter() - t0
    note(f"{len(jobs)} models built and loaded, {pairs:.3e} pairs per replay")
    tc = time.perf_counter()
    b = epw.Batch(jobs)  # autotunes, captures the graph and runs every job once
    t_create = time.perf_counter() - tc
    note(f"batch created (autotune, eager pass, candidate graphs): {t_create:.1f} s")
    for _ in range(args.warmup):
        b.run()
        torch.cuda.synchronize()
        note("warm-up replay done")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    l0 = epw.launch_count()
    with ClockSampler(local) as clk:
        for e0, e1 in evs:
            flush.zero_()
            e0.record()
            b.run()
            e1.record()
        torch.cuda.synchronize()
    launches = epw.launch_count() - l0
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs]))
    peaks, peak_src = measured_peaks()
    ach = tfl / (ms / 1e3) / 1e12
    info = b.info()
    print(json.dumps({
        "metric": METRIC, "value": pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32+f64", "data": "synthetic",
        "config": {"workload": f"uneven batch: the {len(jobs)}-system draw (nw in "
                               f"{sorted({sp.nw for sp in specs})}, nat in {sorted({sp.nat for sp in specs})}, "
                               "Re and Rp shell targets 27..400, nk 50..5000, q 16^3..48^3), one CUDA graph "
                               "replay per step",
                   "pairs_per_step": pairs, "precision": "bf16x3",
                   "systems": [[sp.lattice, sp.nw, sp.nat, sp.nRe, sp.nRp, sp.nk, sp.nq_grid] for sp in specs],
                   "graph": {"branches": info[0], "workspace_bytes": info[1], "kernel_nodes": info[2]},
                   "host_model_build_s": t_models, "batch_create_s": t_create,
                   "l2": "flushed between timed steps (256 MB write)"},
        "clocks": clk.summary(), "gpu_launches": int(launches + info[2] * args.steps),
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_tflops"], "traffic": None,
                     "peak_source": f"{peak_src} bf16_tflops (burst)",
                     "work": f"{tfl:.3e} algorithmic contraction flops per replay (all systems)"},
        "e2e": None, "cpu_baseline": None,
    }))
    b.close()


class Runner:
    """One workload on this rank's k shard, device buffers, L2 flushed between timed steps."""

    def __init__(self, epw, torch, name, rank, world, dev, nk=0):
        import dataclasses

        import workloads as W
        self.epw, self.torch, self.name, self.dev = epw, torch, name, dev
        self.wl = W.make_workload(name)
        if nk > 0:  # the first nk of the k list (small profiling cases)
            self.wl = dataclasses.replace(self.wl, k=self.wl.k[:nk])
        from paper_1604_03525_gb300.shard import shard_bounds
        self.lo, self.hi = shard_bounds(len(self.wl.k), rank, world)
        self.m = epw.Model(self.wl.model)
        self.k = torch.tensor(self.wl.k[self.lo:self.hi], device=dev)
        self.q = torch.tensor(self.wl.q, device=dev)
        self.wq = torch.tensor(self.wl.wq, device=dev)
        self.out = torch.empty((self.hi - self.lo, self.wl.model.nw), dtype=torch.float64, device=dev)
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.pairs = (self.hi - self.lo) * len(self.wl.q)
        self.pairs_total = len(self.wl.k) * len(self.wl.q)

    def kw(self, prec):
        return dict(T=self.wl.T, EF=self.wl.EF, sigma=self.wl.sigma, precision=prec)

    def timed(self, nsteps, nwarm, prec, barrier=None, k=None):
        torch, m = self.torch, self.m
        k = self.k if k is None else k
        for _ in range(nwarm):
            m.linewidth(k, self.q, self.wq, out=self.out[:len(k)], **self.kw(prec))
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        (barrier or torch.cuda.synchronize)()
        m.timing(True)
        l0 = self.epw.launch_count()
        for e0, e1 in evs:
            self.flush.zero_()  # evict L2 between timed steps (outside the timed events)
            e0.record(stream)
            m.linewidth(k, self.q, self.wq, out=self.out[:len(k)], **self.kw(prec))
            e1.record(stream)
        (barrier or torch.cuda.synchronize)()
        launches = self.epw.launch_count() - l0
        (g_ms, g_n), (e_ms, e_n) = m.timing_read_tags()
        m.timing(False)
        m.sync()
        step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        return {"step_ms": step_ms, "kern": (g_ms / nsteps, g_n // max(nsteps, 1)),
                "eig": (e_ms / nsteps, e_n // max(nsteps, 1)), "launches": launches}

    def e2e(self, prec, n):
        torch = self.torch
        kh = torch.tensor(self.wl.k[self.lo:self.hi]).pin_memory()
        qh = torch.tensor(self.wl.q).pin_memory()
        wh = torch.tensor(self.wl.wq).pin_memory()
        oh = torch.empty((self.hi - self.lo, self.wl.model.nw), dtype=torch.float64).pin_memory()
        self.m.linewidth(kh, qh, wh, out=oh, **self.kw(prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            self.m.linewidth(kh, qh, wh, out=oh, **self.kw(prec))
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n
        return {"value": self.pairs / dt, "unit": "pairs/s", "h2d_bytes_per_step": int(kh.nbytes + qh.nbytes + wh.nbytes),
                "d2h_bytes_per_step": int(oh.nbytes)}


def roofline(wl_model, prec_name, r, pairs, peaks, peak_src, fused):
    """Tensor roofline of the path's contraction kernels against the burst bf16 peak
    (these kernels run for milliseconds to seconds at the boost clock; tf32 = bf16 x 1.1/2.25)."""
    h, g, rot = flops_per_pair(wl_model)
    ratio = 1.0 if prec_name == "bf16x3" else 1.1 / 2.25
    peak = peaks["bf16_tflops"] * ratio
    src = f"{peak_src} bf16_tflops (burst)" + ("" if ratio == 1.0 else " x 1.1/2.25 (tf32)")
    g_ms, g_n = r["kern"]
    e_ms, e_n = r["eig"]
    if fused:
        ach = (h + g) * pairs / (g_ms / 1e3) / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "peak_source": src, "kernel": "k_tc_linewidth (fused: contraction, eigensolve, rotation, deltas)",
               "work": f"{h + g} algorithmic contraction flops/pair x {pairs} pairs per step",
               "kernel_ms": g_ms, "kernel_launches": g_n}
    elif e_n == 0:
        ach = (h + g) * pairs / (g_ms / 1e3) / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "peak_source": src,
               "kernel": "k_tcwf (wide shapes, one persistent kernel: H(k+q) contraction and per-pair "
                         "eigensolve beside the vertex contraction, rotation and deltas of the reachable terms)",
               "work": f"{h + g} algorithmic contraction flops/pair ({h} H(k+q), {g} vertex) x {pairs} pairs "
                       "per step",
               "kernel_ms": g_ms, "kernel_launches": g_n}
    else:
        tot = e_ms + g_ms
        ach = (h + g) * pairs / (tot / 1e3) / 1e12
        out = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "peak_source": src,
               "kernel": "k_tcw E + G (H(k+q) contraction + per-pair eigensolve; vertex contraction + "
                         "rotation and deltas of the reachable terms)",
               "work": f"{h + g} algorithmic contraction flops/pair ({h} in E, {g} in G) x {pairs} pairs per step",
               "kernel_ms": tot,
               "G": {"ms": g_ms, "launches": g_n, "tflops": g * pairs / (g_ms / 1e3) / 1e12,
                     "frac": g * pairs / (g_ms / 1e3) / 1e12 / peak},
               "E": {"ms": e_ms, "launches": e_n, "tflops": h * pairs / (e_ms / 1e3) / 1e12,
                     "frac": h * pairs / (e_ms / 1e3) / 1e12 / peak,
                     "note": "bound by the FP32 per-pair eigensolve, not the tensor pipe"}}
    out["executed_tflops"] = 3.0 * out["achieved"]
    out["executed_frac"] = 3.0 * out["frac"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "tf32x3", "bf16x3", "fp32", "fp64"])
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "fcc_nw4", "hex_nw5", "batch"])
    ap.add_argument("--other-steps", type=int, default=2, help="timed steps of the other split form (0: skip)")
    ap.add_argument("--fp64-k", type=int, default=8, help="k of the headline list timed in the plain FP64 form (0: skip)")
    ap.add_argument("--extras", type=int, default=1, help="also time the other configurations and the adjoint")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nk", type=int, default=0,
                    help="time only the first NK of the k list (a small case for ncu captures; not a bench line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)

    import torch
    import paper_1604_03525_gb300 as epw

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    precs = {"tf32x3": epw.TF32X3, "bf16x3": epw.BF16X3, "fp32": epw.FP32, "fp64": epw.FP64}
    name = AUTO_PRECISION[args.workload] if args.precision == "auto" else args.precision
    prec = precs[name]
    R = Runner(epw, torch, args.workload, rank, world, dev, args.nk)
    with ClockSampler(local) as clk:
        r = R.timed(args.steps, args.warmup, prec, barrier)
    t_local = float(np.sum(r["step_ms"]))
    if dist is not None:
        t = torch.tensor([t_local], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        # the shards' Im Sigma, gathered after the timed region (padded to the largest shard)
        from paper_1604_03525_gb300.shard import shard_bounds
        nmax = max(shard_bounds(len(R.wl.k), i, world)[1] - shard_bounds(len(R.wl.k), i, world)[0]
                   for i in range(world))
        pad = torch.zeros((nmax, R.wl.model.nw), dtype=torch.float64, device=dev)
        pad[:len(R.out)] = R.out
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        full = torch.cat([parts[i][:shard_bounds(len(R.wl.k), i, world)[1] - shard_bounds(len(R.wl.k), i, world)[0]]
                          for i in range(world)])
        assert full.shape[0] == len(R.wl.k) and bool(torch.all(full >= 0))
    else:
        t_max = t_local
    ms_per_step = t_max / args.steps
    value = R.pairs_total / (ms_per_step / 1e3)
    peaks, peak_src = measured_peaks()
    fused = args.workload == "fcc_nw4"
    roof = None
    if prec in (epw.BF16X3, epw.TF32X3):
        roof = roofline(R.wl.model, name, r, R.pairs, peaks, peak_src, fused)
        if fused:
            roof["traffic"], roof["traffic_source"] = profiled(TC_PROFILE, TC_SOURCE, "traffic", name)
        else:
            tpp, src = profiled(WIDE_PROFILE, WIDE_SOURCE, "traffic_per_pair", name)
            nlaunch = max(r["kern"][1], 1)
            roof["traffic"] = None if tpp is None else tpp * R.pairs / nlaunch
            roof["traffic_source"] = src + ("" if tpp is None else
                                            " (per-pair bytes of a smaller capture x the pairs of one G launch)")
    else:
        h, g, rot = flops_per_pair(R.wl.model)
        peak = 73.55 if prec == epw.FP32 else 1.257
        ach = (h + g + rot) * R.pairs / (r["kern"][0] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "peak_source": "measured FMA throughput (FP32 73.55 / FP64 1.257 TFLOP/s)",
                "work": f"{h + g + rot} algorithmic flops/pair x {R.pairs} pairs", "kernel_ms": r["kern"][0]}

    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": {"tf32x3": "tf32x3+f32+f64", "bf16x3": "bf16x3+f32+f64", "fp32": "f32+f64", "fp64": "f64"}[name],
        "data": "synthetic",
        "config": {"workload": DESCR[args.workload] + (f" (first {args.nk} k only)" if args.nk else ""),
                   "pairs_per_step": R.pairs_total,
                   "k_shard": "contiguous k slice per rank (strong scaling)", "precision": name,
                   "l2": "flushed between timed steps (256 MB write)"},
        "clocks": clk.summary(), "gpu_launches": int(r["launches"] // max(args.steps, 1) * args.steps),
        "roofline": roof,
    }
    if not args.no_e2e:
        e = R.e2e(prec, max(1, min(args.steps, 3)))
        if dist is not None:
            t = torch.tensor([R.pairs / e["value"]], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e["value"] = R.pairs_total / float(t.item())
        line["e2e"] = e
    if rank == 0 and world == 1:
        if args.other_steps > 0 and prec in (epw.BF16X3, epw.TF32X3):
            oname = "tf32x3" if name == "bf16x3" else "bf16x3"
            ro = R.timed(args.other_steps, 1, precs[oname])
            oms = float(np.mean(ro["step_ms"]))
            line["other_forms"] = {oname: {"value": R.pairs / (oms / 1e3), "unit": "pairs/s", "ms_per_step": oms,
                                           "roofline": roofline(R.wl.model, oname, ro, R.pairs, peaks, peak_src,
                                                                fused)}}
        if args.fp64_k > 0:
            # the plain FP64 GPU form (SIMT, FP64 contraction, eigensolve and sums) on the first
            # fp64_k k of the list x the full q list: seconds per k at this size
            nk64 = min(args.fp64_k, len(R.k))
            r64 = R.timed(1, 1, epw.FP64, k=R.k[:nk64])
            ms64 = float(np.mean(r64["step_ms"]))
            v64 = nk64 * len(R.wl.q) / (ms64 / 1e3)
            line["fp64_gpu_form"] = {"value": v64, "unit": "pairs/s", "ms_per_step": ms64,
                                     "sample": f"first {nk64} k x the full q list",
                                     "speedup_of_headline_form": value / v64}
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args.workload, *CPU_SAMPLE[args.workload])
        if args.extras and args.workload == WORKLOAD:
            line["c2"] = extra_fused(epw, torch, dev, peaks, peak_src)
            line["c5"] = extra_hex(epw, torch, dev, peaks, peak_src)
    if rank == 0:
        print(json.dumps(line))
    R.m.close()
    if dist is not None:
        dist.destroy_process_group()


def extra_fused(epw, torch, dev, peaks, peak_src):
    """The fcc nw=4 configuration on the fused single-kernel form (BF16x3), 10 steps."""
    R = Runner(epw, torch, "fcc_nw4", 0, 1, dev)
    r = R.timed(10, 3, epw.BF16X3)
    ms = float(np.mean(r["step_ms"]))
    roof = roofline(R.wl.model, "bf16x3", r, R.pairs, peaks, peak_src, True)
    roof["traffic"], roof["traffic_source"] = profiled(TC_PROFILE, TC_SOURCE, "traffic", "bf16x3")
    out = {"workload": DESCR["fcc_nw4"], "value": R.pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms,
           "precision": "bf16x3", "roofline": roof}
    R.m.close()
    return out


def extra_hex(epw, torch, dev, peaks, peak_src):
    """The hexagonal nw=5 configuration (BF16x3 forward) and its adjoint (TF32x3 and BF16x3)."""
    R = Runner(epw, torch, "hex_nw5", 0, 1, dev)
    r = R.timed(2, 1, epw.BF16X3)
    ms = float(np.mean(r["step_ms"]))
    out = {"workload": DESCR["hex_nw5"], "value": R.pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms,
           "precision": "bf16x3", "roofline": roofline(R.wl.model, "bf16x3", r, R.pairs, peaks, peak_src, False)}
    cot = torch.ones((len(R.k), R.wl.model.nw), dtype=torch.float64, device=dev)
    out["backward"] = {}
    for pname, p in (("tf32x3", epw.TF32X3), ("bf16x3", epw.BF16X3)):
        kw = dict(T=R.wl.T, EF=R.wl.EF, sigma=R.wl.sigma, precision=p)
        R.m.linewidth_backward(R.k, R.q, cot, R.wq, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R.m.linewidth_backward(R.k, R.q, cot, R.wq, **kw)
        e1.record()
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1)
        out["backward"][pname] = {
            "value": R.pairs / (bms / 1e3), "unit": "pairs/s", "ms_per_step": bms,
            "what": "dL/dg(Re,Rp), dL/dT, dL/dE_F of L = sum Im Sigma at the full size; g(k,q) recomputed "
                    "(forward contraction staged on the tensor cores, adjoint GEMMs in FP32)"}
    R.m.close()
    return out


if __name__ == "__main__":
    main()
