"""Benchmark: k.q pairs/s of the electron linewidth (Eq. linewidthel) on one GB300.

Workload: fcc lattice, nw=4 Wannier functions, 1 atom (3 modes), 135 Re and 135
Rp vectors (whole shells), 1000 k-points inside a 0.2 eV window of E_F, a
uniform 40^3 q grid (64,000 q), sigma = 20 meV, T = 300 K: 6.4e7 (k,q) pairs
per step.  A step is one epw_linewidth call: phases, phonons, k-side bands and
vertex, the per-pair interpolation/rotation/reduction and the final sum.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|fp32|fp64]
  python bench.py --impl reference     # the FP64 CPU oracle on a bounded sample
  python bench.py --workload diamond_nw8|hex_nw5|batch   # the other configurations (not the headline)

diamond_nw8: diamond two-atom basis, nw=8, 249 Re = Rp, 2000 k near the band edges x (60^3 grid +
1e5 random q), sigma = 10 meV.  hex_nw5: hexagonal three-atom cell, nw=5, ~300 R, 20^3 k x 40^3 q,
sigma = 15 meV, T = 50 K.  batch: uneven systems drawn as for the 64-system configuration, at
reduced sizes (stated in the line) so that the host can build the models, replayed as one CUDA graph.

Under torchrun each rank runs its own copy of the workload at one temperature
of the T sweep (300, 100, 50, 10 K): weak scaling, no data-path collective.
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

WORKLOAD = "fcc_nw4"
METRIC = "k·q pairs/s for ImΣ_nk on 1 GB300 (and % roofline) at stated error vs FP64 oracle"
T_SWEEP = [300.0, 100.0, 50.0, 10.0]
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def algorithmic_flops_per_pair(m):
    """Contractions S5+S7 per (k,q) pair (complex MAC = 8 flops).

    H(k+q): 8 nRe nw^2; g(k,q) U_k: 8 nRp 3nat nw^2; U_k+q^+ rotation: 8 3nat nw^3;
    mode projection: 8 (3nat)^2 nw^2.  Eigensolve sweeps and the delta/occupation
    terms are not counted (iterative / transcendental, not a fixed flop count).
    """
    nw, nm = m.nw, 3 * m.nat
    tensor = 8 * nw * nw * (len(m.Re) + nm * len(m.Rp))
    simt = 8 * nm * nw**3 + 8 * nm * nm * nw * nw
    return tensor, simt


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


TC_SOURCE = os.path.join(ROOT, "paper_1604_03525_gb300", "csrc", "epw_tc.cu")
TC_PROFILE = os.path.join(ROOT, "profiles", "k_tc_linewidth_fcc_nw4.md")


def profiled_traffic(form):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary.

    The summary records `traffic <form> <bytes> source-sha256 <hash>` lines; a
    value is used only while the kernel source still has that hash (otherwise
    the counters describe an older kernel and the traffic is reported as null).
    """
    import hashlib
    try:
        sha = hashlib.sha256(open(TC_SOURCE, "rb").read()).hexdigest()
        for line in open(TC_PROFILE):
            parts = line.strip().strip("`").split()
            if len(parts) == 5 and parts[0] == "traffic" and parts[1] == form and parts[3] == "source-sha256":
                if parts[4] == sha:
                    return float(parts[2]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, profiles/"
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


def cpu_baseline(wl_name, nk_s, nq_s):
    """The FP64 oracle (as it stands) on a bounded sample of the workload."""
    import oracle
    import workloads as W
    wl = W.make_workload(wl_name, nq_sub=nq_s)
    k = wl.k[::max(1, len(wl.k) // nk_s)][:nk_s]
    t0 = time.perf_counter()
    oracle.linewidth(wl.model, k, wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
    dt = time.perf_counter() - t0
    pairs = len(k) * len(wl.q)
    return {"value": pairs / dt, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(k)} k x {len(wl.q)} q (seeded subsample of the 40^3 grid), {pairs} pairs, {dt:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    import workloads as W
    oracle.build()
    nq_s = 512
    wl = W.make_workload(WORKLOAD, nq_sub=nq_s)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.linewidth(wl.model, wl.k, wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    pairs = len(wl.k) * len(wl.q)
    ms = 1e3 * float(np.mean(times))
    val = pairs / (ms / 1e3)
    sample = f"{len(wl.k)} k x {nq_s} q per step (seeded subsample of the 40^3 grid), {pairs} pairs"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fcc nw=4 nat=1, 135 Re/Rp, 1000 k (0.2 eV window) x 40^3 q, sigma=20 meV, T=300 K",
                   "sample_per_step": sample},
        "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args):
    """Uneven systems (the 64-system draw at reduced sizes) through one captured CUDA graph.

    The draw is the configuration's (nw, nat, lattice, R-shell target, k count, q grid per
    system) with nR <= 150, nk <= 1000, q grids 16^3..32^3 and nw <= 12 (the host builds every
    model in NumPy); systems outside the limits are dropped whole.  All jobs run
    split-BF16 (the fused kernel where the shape has one, else the staged tensor-core form).
    A step is one graph replay; the L2 is flushed between steps.
    """
    import torch
    import paper_1604_03525_gb300 as epw
    import workloads as W
    rank, world, local = dist_info()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = W.models.batch_specs(64, nR_range=(27, 150), nk_range=(50, 1000), nq_range=(16, 32), max_nw=12)
    jobs, pairs, tfl = [], 0, 0.0
    for sp in specs:
        wm, k, q = W.models.batch_system(sp)
        m = epw.Model(wm)
        jobs.append(dict(model=m, k=torch.tensor(k, device=dev), q=torch.tensor(q, device=dev), wq=None, T=300.0,
                         EF=0.0, sigma=0.05, precision=epw.BF16X3))
        pairs += len(k) * len(q)
        tfl += algorithmic_flops_per_pair(wm)[0] * len(k) * len(q)
    b = epw.Batch(jobs)  # autotunes, captures the graph and runs every job once
    for _ in range(args.warmup):
        b.run()
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
    print(json.dumps({
        "metric": METRIC, "value": pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32+f64", "data": "synthetic",
        "config": {"workload": f"uneven batch: {len(jobs)} systems of the 64-system draw (nw in "
                               f"{sorted({sp.nw for sp in specs})}, nat in {sorted({sp.nat for sp in specs})}, "
                               "nR 27..150, nk 50..1000, q 16^3..32^3), one CUDA graph replay per step",
                   "pairs_per_step": pairs, "precision": "bf16x3",
                   "l2": "flushed between timed steps (256 MB write)"},
        "clocks": clk.summary(), "gpu_launches": int(launches),
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "frac": ach / peaks["bf16_tflops_sustained"], "traffic": None,
                     "peak_source": f"{peak_src} bf16_tflops_sustained",
                     "work": f"{tfl:.3e} algorithmic contraction flops per replay (all systems)"},
        "e2e": None, "cpu_baseline": None,
    }))
    b.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "tf32x3", "bf16x3", "fp32", "fp64"])
    ap.add_argument("--other-steps", type=int, default=2, help="timed steps of the other tensor-core/FP32 forms")
    ap.add_argument("--backward-steps", type=int, default=3, help="timed adjoint calls (0: skip)")
    ap.add_argument("--se-steps", type=int, default=1,
                    help="timed complex self-energy + spectral function calls (100 k, 64 frequencies; 0: skip)")
    ap.add_argument("--phonon-steps", type=int, default=2,
                    help="timed phonon-side calls (Pi'', lambda, nesting over the same k x q; 0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 GPU form (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nk", type=int, default=0, help="profiling only: use the first NK k-points of the workload")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "diamond_nw8", "hex_nw5", "batch"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload != WORKLOAD:
        # the other single-system configurations: the split forms only (a plain FP64 or FP32
        # step of these sizes takes minutes), few steps (a step is seconds), no extra rows
        args.steps, args.warmup = min(args.steps, 2), min(args.warmup, 1)
        args.fp64_steps = args.backward_steps = args.phonon_steps = args.se_steps = 0
        args.no_e2e = True

    import torch
    import paper_1604_03525_gb300 as epw
    import workloads as W

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    headline = args.workload == WORKLOAD
    wl = W.make_workload(WORKLOAD, T=T_SWEEP[rank % len(T_SWEEP)]) if headline else W.make_workload(args.workload)
    if args.nk > 0:
        wl.k = wl.k[:args.nk]
    m = epw.Model(wl.model)
    dev = torch.device("cuda", local)
    k = torch.tensor(wl.k, device=dev)
    q = torch.tensor(wl.q, device=dev)
    wq = torch.tensor(wl.wq, device=dev)
    out = torch.empty((len(wl.k), wl.model.nw), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pairs = len(wl.k) * len(wl.q)

    precs = {"tf32x3": epw.TF32X3, "bf16x3": epw.BF16X3, "fp32": epw.FP32, "fp64": epw.FP64}
    if args.precision == "auto":
        # the fastest form that meets the 1e-4 target on this workload: split-BF16
        # (max relative error 3.4e-5 against the oracle at this size; TF32x3 1.2e-5)
        name = "bf16x3"
        try:
            m.linewidth(k[:8], q[:256], wq[:256], T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=epw.BF16X3)
        except epw.EPWError:
            name = "fp32"
    else:
        name = args.precision
    prec = precs[name]
    kw = dict(T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=prec, out=out)

    def timed_steps(nsteps, nwarm, precision):
        kw2 = dict(kw, precision=precision)
        for _ in range(nwarm):
            m.linewidth(k, q, wq, **kw2)
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        barrier()
        m.timing(True)
        l0 = epw.launch_count()
        for e0, e1 in evs:
            flush.zero_()  # evict L2 between timed steps (outside the timed events)
            e0.record(stream)
            m.linewidth(k, q, wq, **kw2)
            e1.record(stream)
        barrier()
        launches = epw.launch_count() - l0
        kms, kn = m.timing_read()
        m.timing(False)
        step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        return step_ms, kms / max(kn, 1), kn, launches

    with ClockSampler(local) as clk:
        step_ms, kern_ms, kern_n, launches = timed_steps(args.steps, args.warmup, prec)
    t_local = float(np.sum(step_ms))
    if dist is not None:
        t = torch.tensor([t_local], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    ms_per_step = t_max / args.steps
    value = world * pairs / (ms_per_step / 1e3)

    # end to end: host (pinned) buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        kh = torch.tensor(wl.k).pin_memory()
        qh = torch.tensor(wl.q).pin_memory()
        wh = torch.tensor(wl.wq).pin_memory()
        oh = torch.empty((len(wl.k), wl.model.nw), dtype=torch.float64).pin_memory()
        m.linewidth(kh, qh, wh, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=prec, out=oh)
        barrier()
        t0 = time.perf_counter()
        ne = max(1, min(args.steps, 5))
        for _ in range(ne):
            m.linewidth(kh, qh, wh, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=prec, out=oh)
        barrier()
        dt = (time.perf_counter() - t0) / ne
        e2e = {"value": world * pairs / dt, "unit": "pairs/s",
               "h2d_bytes_per_step": int(kh.nbytes + qh.nbytes + wh.nbytes), "d2h_bytes_per_step": int(oh.nbytes)}

    fp64 = None
    if args.fp64_steps > 0 and prec != epw.FP64:
        s64, k64, _, _ = timed_steps(args.fp64_steps, 1, epw.FP64)
        fp64 = {"value": pairs / (np.mean(s64) / 1e3), "unit": "pairs/s", "ms_per_step": float(np.mean(s64)),
                "kernel_ms": k64}
    backward = None
    if args.backward_steps > 0:
        # adjoint of sum_{k,n} Im Sigma_nk w.r.t. g(Re,Rp), T and E_F, device buffers, g(k,q)
        # recomputed: the tensor-core form (TF32x3) timed, the FP32 SIMT form once beside it
        cot = torch.ones((len(wl.k), wl.model.nw), dtype=torch.float64, device=dev)

        def time_backward(op, n):
            m.linewidth_backward(k, q, cot, wq, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=op)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(n):
                m.linewidth_backward(k, q, cot, wq, T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=op)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        bms = time_backward(epw.TF32X3, args.backward_steps)
        backward = {"value": pairs / (bms / 1e3), "unit": "pairs/s", "ms_per_step": bms, "precision": "tf32x3",
                    "what": "dL/dg(Re,Rp), dL/dT, dL/dE_F of L = sum Im Sigma; g(k,q) recomputed"}
        fms = time_backward(epw.FP32, 1)
        backward["fp32_simt"] = {"value": pairs / (fms / 1e3), "unit": "pairs/s", "ms_per_step": fms}
    phonon = None
    if args.phonon_steps > 0:
        # per-(q, nu) sums over the k list on the same workload: Pi''_qnu, lambda_qnu, nesting, N(E_F)
        pk = dict(T=wl.T, EF=wl.EF, sigma=wl.sigma, precision=prec)
        m.phonon_selfenergy(k, q, **pk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.phonon_steps):
            m.phonon_selfenergy(k, q, **pk)
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / args.phonon_steps
        phonon = {"value": pairs / (pms / 1e3), "unit": "pairs/s", "ms_per_step": pms, "precision": name,
                  "what": "Pi''_qnu (on shell), lambda_qnu, nesting zeta_q, N(E_F): per-q sums over the 1000 k"}
    selfen = None
    if args.se_steps > 0:
        # Sigma_nk(omega) and A_nk(omega) (Eqs. elselfenergy, spectral_funct) on 64 frequencies, first 100 k
        om = torch.linspace(-0.3, 0.3, 64, dtype=torch.float64, device=dev)
        sk = dict(T=wl.T, EF=wl.EF, delta=wl.sigma, precision=prec)
        m.selfenergy(k[:100], q, om, wq, **sk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.se_steps):
            m.selfenergy(k[:100], q, om, wq, **sk)
        e1.record()
        torch.cuda.synchronize()
        sms = e0.elapsed_time(e1) / args.se_steps
        sp = 100 * len(wl.q)
        selfen = {"value": sp / (sms / 1e3), "unit": "pairs/s", "ms_per_step": sms, "precision": name,
                  "what": "Sigma_nk(omega), A_nk(omega) on 64 frequencies: 100 k x the 40^3 q grid"}
    others = {}
    if args.other_steps > 0:
        forms = (("bf16x3", epw.BF16X3), ("tf32x3", epw.TF32X3), ("fp32", epw.FP32))
        for oname, op in (forms if headline else forms[:2]):
            if op == prec:
                continue
            try:
                so, ko, _, _ = timed_steps(args.other_steps, 1, op)
            except epw.EPWError:
                continue
            others[oname] = {"value": pairs / (np.mean(so) / 1e3), "unit": "pairs/s",
                             "ms_per_step": float(np.mean(so)), "kernel_ms": ko}

    peaks, peak_src = measured_peaks()
    tflops, sflops = algorithmic_flops_per_pair(wl.model)
    fused = wl.model.nw in (1, 2, 4) and 3 * wl.model.nat == 3
    if prec in (epw.BF16X3, epw.TF32X3) and not fused:
        # staged form: tcgen05 contraction per k chunk, then the per-pair eigensolve, rotation and
        # deltas on the CUDA cores (FP32), which dominate; the eigensolve's sweeps are not counted
        achieved = sflops * pairs / (kern_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": 73.55, "unit": "TFLOP/s", "frac": achieved / 73.55,
                "traffic": None, "peak_source": "measured FP32 FMA throughput",
                "work": f"{sflops} rotation + mode-projection flops/pair x {pairs} pairs (per-pair eigensolve "
                        f"not counted; the tensor-core contraction, {tflops} flops/pair, is a small share)"}
    elif prec in (epw.BF16X3, epw.TF32X3):
        achieved = tflops * pairs / (kern_ms / 1e3) / 1e12
        # a contraction takes the peak of its own dtype: tf32 = measured bf16 x nominal 1.1/2.25
        ratio = 1.0 if prec == epw.BF16X3 else 1.1 / 2.25
        peak = peaks["bf16_tflops_sustained"] * ratio
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None,
                "peak_source": f"{peak_src} bf16_tflops_sustained" + ("" if ratio == 1.0 else " x 1.1/2.25 (tf32)"),
                "work": f"{tflops} algorithmic contraction flops/pair x {pairs} pairs "
                        "(the 3-term split executes 3x this on the tensor pipe)"}
    else:
        # plain CUDA-core arithmetic: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz, FP64 1.25 TFLOP/s nominal
        # measured FMA rates of this machine's GB300 (8 independent chains per thread)
        peak = 73.55 if prec == epw.FP32 else 1.257
        achieved = (tflops + sflops) * pairs / (kern_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "measured FMA throughput (FP32 73.55 / FP64 1.257 TFLOP/s)", "work": f"{tflops + sflops} algorithmic flops/pair x {pairs} pairs"}
    if prec in (epw.BF16X3, epw.TF32X3) and fused:
        # the 3-term split (lo*hi + hi*lo + hi*hi) runs three MMAs per product on the tensor pipe
        roof["executed_tflops"] = 3.0 * achieved
        roof["executed_frac"] = 3.0 * achieved / peak
    roof["kernel_ms"] = kern_ms
    roof["kernel_launches"] = kern_n
    if prec in (epw.BF16X3, epw.TF32X3) and headline:
        roof["traffic"], roof["traffic_source"] = profiled_traffic("bf16x3" if prec == epw.BF16X3 else "tf32x3")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        nks, nqs = {WORKLOAD: (1000, 2560), "diamond_nw8": (64, 8192), "hex_nw5": (64, 16384)}[args.workload]
        cpu = cpu_baseline(args.workload, nks, nqs)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"tf32x3": "tf32x3+f32+f64", "bf16x3": "bf16x3+f32+f64", "fp32": "f32+f64",
                                                     "fp64": "f64"}[name],
            "data": "synthetic",
            "config": {"workload": ("fcc nw=4 nat=1, 135 Re/Rp, 1000 k (0.2 eV window) x 40^3 q, sigma=20 meV, "
                                    f"T={T_SWEEP[0]:.0f} K (rank r: T_sweep[r])") if headline else
                                   f"{wl.name}: nw={wl.model.nw} nat={wl.model.nat}, {len(wl.model.Re)} Re/Rp, "
                                   f"{len(wl.k)} k x {len(wl.q)} q, sigma={wl.sigma * 1e3:.0f} meV, T={wl.T:.0f} K",
                       "pairs_per_step_per_gpu": pairs,
                       "precision": name, "l2": "flushed between timed steps (256 MB write)"},
            "clocks": clk.summary(), "gpu_launches": int(launches), "roofline": roof,
            "e2e": e2e, "cpu_baseline": cpu, "fp64_gpu_form": fp64, "other_forms": others, "backward": backward, "phonon_side": phonon, "selfenergy": selfen,
        }
        print(json.dumps(line))
    m.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
