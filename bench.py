#!/usr/bin/env python
"""Benchmark: two-level MLC solve throughput (Mpoints/s) on synthetic bump charges.

One step = one full solve (all steps of Sec. 4: moments, local convolutions,
coarse charge, coarse solve, boundary values, Dirichlet solves) of the
128^3 workload (512 patches of 16^3, support 16, Q = 4, P = 4, FP64; 8 bumps
from seed 1) with the charge resident in HBM.  L2 is flushed (a 512 MB write)
between timed steps; the flush is outside the timed region.

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
Under torchrun each rank solves its own copy (independent problems, no
collective): weak scaling.
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

from paper_1702_08111_gb300 import inputs as I  # noqa: E402

METRIC = "MLC solve Mpoints/s at stated max error vs FP64 oracle"
WORKLOAD = "bumps8_128"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """SM clock, power and clock-event reasons sampled during the timed region:
    through NVML (ctypes, every 2 ms) when the device's PCI bus id is known,
    else nvidia-smi every 200 ms.  Only samples inside begin()/end() count."""

    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_index: int):
        self.cuda_index = cuda_index
        self.samples = []  # (time, sm_mhz, max_mhz, power_w, reason names)
        self.t0 = self.t1 = None
        self.source = None
        self._stop = threading.Event()
        self._th = None

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def _pci_bus_id(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.cuda_index)
            return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            return None

    def _nvml(self):
        import ctypes
        bus = self._pci_bus_id()
        if bus is None:
            return None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                return None
            try:
                reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
            except AttributeError:
                reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
            return lib, h, reasons
        except OSError:
            return None

    def _run_nvml(self, lib, h, reasons):
        import ctypes
        clk, mx, pw, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.perf_counter()
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    reasons(h, ctypes.byref(bits)) == 0):
                power = pw.value / 1e3 if lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0 else None
                names = [v for k, v in self.REASONS.items() if bits.value & k]
                self.samples.append((t, float(clk.value), float(mx.value), power, names))
            self._stop.wait(0.002)

    def _run_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        while not self._stop.is_set():
            try:
                t = time.perf_counter()
                out = subprocess.run(["nvidia-smi", "-i", str(self.cuda_index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                if len(f) >= 7 and f[0].replace(".", "").isdigit():
                    act = [names[k] for k in range(4) if f[3 + k].lower() == "active"]
                    power = float(f[2]) if f[2].replace(".", "").isdigit() else None
                    self.samples.append((t, float(f[0]), float(f[1]), power, act))
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        nv = self._nvml()
        if nv is not None:
            self.source = "nvml, 2 ms"
            self._th = threading.Thread(target=self._run_nvml, args=nv, daemon=True)
        else:
            self.source = "nvidia-smi, 200 ms"
            self._th = threading.Thread(target=self._run_smi, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        sel = [x for x in self.samples
               if self.t0 is None or (x[0] >= self.t0 and (self.t1 is None or x[0] <= self.t1))]
        if not sel:  # region shorter than the sampling period: nearest samples
            sel = self.samples[-2:]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        pw = [x[3] for x in sel if x[3] is not None]
        return {"sm_mhz": float(np.median([x[1] for x in sel])), "sm_max_mhz": max(x[2] for x in sel),
                "reasons": sorted({r for x in sel for r in x[4]}), "samples": len(sel),
                "power_w_median": float(np.median(pw)) if pw else None, "source": self.source}


def reduce_max_ms(ms: float, world: int, device: str = "cuda") -> float:
    """Slowest rank's time (the job's time): all-reduce MAX over the ranks."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(points_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput in Mpoints/s: every rank solves its own problem."""
    return world * points_per_rank / (ms_max * 1e-3) / 1e6


def time_plan(plan, f, phi, steps, warmup, flush, stream, world, clk=None):
    """Mean device time per solve (CUDA events on the launching stream, L2
    flushed between steps outside the timed region), then per-launch means
    from as many further solves run with per-launch timing on (the launches in
    sequence on one stream; not part of the timed region)."""
    import torch
    for _ in range(warmup):
        plan.solve(f, phi, stream)
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = 0.0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if clk is not None:
        clk.begin()
    for _ in range(steps):
        ev0.record(stream)
        plan.solve(f, phi, stream)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        flush.zero_()
    torch.cuda.synchronize()
    if clk is not None:
        clk.end()
    plan.set_timing(True)
    per_launch = {}
    for _ in range(steps):
        plan.solve(f, phi, stream)
        for k, v in plan.timing().items():
            per_launch[k] = per_launch.get(k, 0.0) + v
        flush.zero_()
    torch.cuda.synchronize()
    plan.set_timing(False)
    return total_ms / steps, {k: v / steps for k, v in per_launch.items()}


# FP32 pipe lane-instruction rate of one GB300 from its unit counts and
# maximum clock: 152 SMs x 128 FP32 lanes x 2.07 GHz (FADD, FMUL and FFMA
# issue at the same rate).  Both tiers run their FFTs on this pipe: the split
# tier in FP32, the FP64 tier in double-float (hi + lo FP32 pairs).
FP32_LANE_INST_PER_S = 152 * 128 * 2.07e9

# FP32 instructions of one (unnormalised) double-float operation: add =
# two-sum (6) + low parts (2); multiply = FMUL + 3 FFMA.
DF_ADD_INST, DF_MUL_INST = 8, 4


def fft64_schedule_inst(tier: str, sparse: bool, nin: int = 17) -> float:
    """FP32 instructions of one 64-point line transform in the slab kernel's
    schedule.  FP64 tier (double-float, radix 8 x 8 over an 8-thread group):
    16 radix-8 butterflies (52 real adds + 4 real multiplies each; 26 + 2 for
    a first-stage butterfly whose inputs 3..7 are zero, `sparse`) and 56
    twiddle products (7 per thread).  Split tier (FP32, radix 2 in one
    thread's registers): 6 stages of 32 butterflies (4 adds each; for inputs
    zero from nin <= 17 on, none in the first stage and 2 in the second) and 98
    nontrivial twiddle products (2 FMUL + 2 FFMA; twiddles 1 and -i cost
    nothing)."""
    if tier == "fp64":
        first = (26, 2) if sparse else (52, 4)
        adds = 8 * first[0] + 8 * 52
        muls = 8 * first[1] + 8 * 4
        # twiddle = 4 multiplies + 2 adds, all double-float
        return (adds + 56 * 2) * DF_ADD_INST + (muls + 56 * 4) * DF_MUL_INST
    if not sparse:
        return 6 * 32 * 4 + 98 * 4
    stage2 = 2 * max(0, min(nin, 32) - 16) if nin <= 17 else 32  # butterflies with two nonzero inputs
    return 4 * 32 * 4 + stage2 * 4 + 98 * 4


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one slab launch,
# from the ncu captures summarised in profiles/ (slab kernel unchanged since):
# the A1 spectra read and the A4 spectra written, no re-reads.
SLAB_DRAM_BYTES = {("bumps8_128", "fp64"): 508.528e6, ("bumps32_256_q6", "split"): 1.900593e9}


def slab_rows(w, ga):
    """z rows of the field box the inverse-x step reads (Omega_alpha rows and
    coarse rows), i.e. the inverse-y lines of a slab."""
    W = w.n + 2 * w.s + 1
    return sum(1 for zi in range(W) if (-ga <= zi - w.s <= w.n + ga) or (zi - w.s) % 4 == 0)


def roofline_for(w, plan, per_launch, tier):
    """Roofline of the dominant launch (the slab kernel).  Algorithmic work =
    nominal radix-2 FFT FLOPs (5 M log2 M per complex line) over the lines the
    pruned transform must produce (forward y on the n+1 nonzero z rows, forward
    and inverse z on all M columns, inverse y on the z rows read later), plus 2
    FLOPs per entry of the real-kernel product; FP64-equivalent FLOPs in the
    FP64 tier.  Peak = the FP32 pipe's instruction rate times the nominal FLOPs
    one FP32 instruction of the kernel's schedule carries: the rate the kernel
    would reach if the pipe issued nothing but its arithmetic."""
    info = plan.info
    N = w.N
    M, Mh, NP = info.M, info.M // 2 + 1, (N // w.n) ** 3
    nin = w.n + 1
    dom = max(per_launch, key=per_launch.get)
    if dom != "conv_slab" or M != 64:
        return None
    nz = slab_rows(w, info.g_alpha)
    line_flops = 5.0 * M * np.log2(M)
    nominal = (nin + 2 * M + nz) * line_flops + 2.0 * M * M
    prod_inst = M * M * (2 * DF_MUL_INST if tier == "fp64" else 2)
    inst = ((nin + M) * fft64_schedule_inst(tier, True, nin) + (M + nz) * fft64_schedule_inst(tier, False)
            + prod_inst)
    flops = NP * Mh * nominal
    achieved = flops / (per_launch[dom] * 1e-3) / 1e12
    peak = FP32_LANE_INST_PER_S * nominal / inst / 1e12
    basis = ("FP32 pipe 152 SMs x 128 lanes x 2.07 GHz = 40.27 T inst/s x %.4f nominal %s FLOP per FP32 "
             "instruction of the slab's %s schedule" % (nominal / inst, "FP64-equivalent" if tier == "fp64"
                                                        else "FP32", "double-float radix-8x8" if tier == "fp64"
                                                        else "FP32 radix-2 register"))
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": SLAB_DRAM_BYTES.get((w.name, tier)),
            "launch_ms": round(per_launch[dom], 4), "flops_per_launch": flops,
            "fp32_inst_per_launch": NP * Mh * inst, "peak_basis": basis}


def run_ours(args, rank, world):
    import torch
    from paper_1702_08111_gb300 import mlc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.device("cuda")
    w = I.workload(args.workload)
    N = w.N
    tier = "split" if w.charge_dtype == "f32" else "fp64"
    plan = mlc.Plan(N, w.n, w.s, w.P, w.Q, tier=mlc.MLC_TIER_SPLIT if tier == "split" else mlc.MLC_TIER_FP64)
    f_host = torch.from_numpy(w.charge())
    f = f_host.to(dev)
    phi = torch.empty((N, N, N), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        ms, per_launch = time_plan(plan, f, phi, args.steps, args.warmup, flush, stream, world, clk)
    ms = reduce_max_ms(ms, world)

    # end to end through the C ABI with host buffers (copies inside the call)
    f_pin = f_host.pin_memory()
    phi_pin = torch.empty((N, N, N), dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.solve_host(f_pin, phi_pin)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        plan.solve_host(f_pin, phi_pin)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms /= args.steps
    value = aggregate_value(float(N) ** 3, world, ms)
    res = {"value": value, "ms": ms, "e2e_ms": e2e_ms, "per_launch": per_launch,
           "roofline": roofline_for(w, plan, per_launch, tier), "clocks": clk.summary(),
           "phi": phi, "N": N, "tier": tier, "f_bytes": f_host.element_size() * N ** 3}
    del plan
    if args.extra and rank == 0:
        res["extra"] = run_extra(args, flush, stream)
    return res


def run_extra(args, flush, stream):
    """Secondary lines: the 256^3 Q=6 workload in the split and FP64 tiers."""
    import torch
    from paper_1702_08111_gb300 import mlc
    from oracle import closed_forms as CF
    w = I.workload("bumps32_256_q6")
    N = w.N
    f32 = torch.from_numpy(w.charge()).cuda()
    f64 = f32.double()
    out = {}
    phis = {}
    for tier, f in (("split", f32), ("fp64", f64)):
        plan = mlc.Plan(N, w.n, w.s, w.P, w.Q, tier=mlc.MLC_TIER_SPLIT if tier == "split" else mlc.MLC_TIER_FP64)
        phi = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
        steps = max(3, args.steps // 2)
        ms, pl = time_plan(plan, f, phi, steps, 3, flush, stream, 1)
        phis[tier] = phi.cpu().numpy()
        out[tier] = {"workload": "bumps32_256_q6", "tier": tier, "ms_per_step": round(ms, 3),
                     "value": round(float(N) ** 3 / (ms * 1e-3) / 1e6, 2), "unit": "Mpoints/s",
                     "roofline": roofline_for(w, plan, pl, tier),
                     "per_launch_ms": {k: round(v, 4) for k, v in pl.items()}}
        del plan
    ex = CF.bumps_potential(N, w.bumps)
    d = np.abs(phis["split"] - phis["fp64"]).max() / np.abs(phis["fp64"]).max()
    out["split"]["max_rel_err_vs_fp64_gpu"] = float(d)
    out["fp64"]["max_rel_err_vs_closed_form"] = float(np.abs(phis["fp64"] - ex).max() / np.abs(ex).max())
    out["split"]["max_rel_err_vs_closed_form"] = float(np.abs(phis["split"] - ex).max() / np.abs(ex).max())
    out["split_over_fp64_speedup"] = round(out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"], 3)
    del phis
    out["split_batched"] = run_batched_256(args, flush, stream, w)
    out["split_batched_over_fp64_speedup"] = round(
        out["split_batched"]["value"] / out["fp64"]["value"], 3)
    out["batch"] = run_batch(args, flush, stream)
    out["serving"] = run_serving(args)
    return out


def run_batched_256(args, flush, stream, w, nprob=4):
    """The split tier at 256^3 in its batched form: nprob problems of the
    256^3 Q = 6 geometry (32 bumps each; seeds 3, 13, 23, 33) in one
    mlc_batch_solve (shared per-patch launches, per-problem coarse steps on
    parallel graph branches).  Mpoints/s over all problems."""
    import torch
    from paper_1702_08111_gb300 import mlc
    ws = [I.Workload(w.name, w.N, w.n, w.s, w.Q, bumps=I.draw_bumps(32, 3 + 10 * k), charge_dtype="f32")
          for k in range(nprob)]
    plans = [mlc.Plan(x.N, x.n, x.s, x.P, x.Q, tier=mlc.MLC_TIER_SPLIT) for x in ws]
    fs = [torch.from_numpy(x.charge()).cuda() for x in ws]
    phis = [torch.empty((x.N,) * 3, dtype=torch.float64, device="cuda") for x in ws]
    for _ in range(3):
        mlc.batch_solve(plans, fs, phis, stream)
        flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(3, args.steps // 2)
    tot = 0.0
    for _ in range(steps):
        e0.record(stream)
        mlc.batch_solve(plans, fs, phis, stream)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        flush.zero_()
    ms = tot / steps
    res = {"workload": f"{nprob} x bumps32_256_q6 (seeds 3, 13, 23, 33)", "problems": nprob,
           "ms_per_batch": round(ms, 3), "ms_per_problem": round(ms / nprob, 3),
           "value": round(nprob * float(w.N) ** 3 / (ms * 1e-3) / 1e6, 2), "unit": "Mpoints/s",
           "batch_choice": mlc.batch_choice(plans, fs, phis)}
    del plans, fs, phis
    return res


def run_batch(args, flush, stream):
    """48 uneven problems (sides 32..160), split tier, through mlc_batch_solve
    (one graph per patch geometry) versus the same problems one by one."""
    import torch
    from paper_1702_08111_gb300 import mlc
    probs = I.batch_problems(48, 4)
    groups = {}
    for w in probs:
        groups.setdefault((w.n, w.s), []).append(w)
    plans, fs, phis = {}, {}, {}
    for key, ws in groups.items():
        plans[key] = [mlc.Plan(w.N, w.n, w.s, w.P, w.Q, tier=mlc.MLC_TIER_SPLIT) for w in ws]
        fs[key] = [torch.from_numpy(w.charge().astype(np.float32)).cuda() for w in ws]
        phis[key] = [torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda") for w in ws]
    pts = float(sum(w.N ** 3 for w in probs))

    def step_batch():
        for key in groups:
            mlc.batch_solve(plans[key], fs[key], phis[key], stream)

    def step_single():
        for key in groups:
            for p, f, ph in zip(plans[key], fs[key], phis[key]):
                p.solve(f, ph, stream)

    res = {}
    for name, fn in (("batched_graph", step_batch), ("one_by_one", step_single)):
        for _ in range(3):
            fn()
            flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        steps = max(3, args.steps // 2)
        for _ in range(steps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            flush.zero_()
        ms = tot / steps
        res[name] = {"ms_per_step": round(ms, 3), "value": round(pts / (ms * 1e-3) / 1e6, 2), "unit": "Mpoints/s"}
    res["problems"] = len(probs)
    res["groups"] = {f"n{k[0]}_s{k[1]}": len(v) for k, v in groups.items()}
    res["speedup_over_one_by_one"] = round(res["one_by_one"]["ms_per_step"] / res["batched_graph"]["ms_per_step"], 3)
    return res


def run_serving(args, nreq=200):
    """Continuous-batching server on the first `nreq` requests of the serving
    mix: saturated throughput first, then Poisson arrivals at 0.7 x that rate;
    p50/p99 latency (enqueue -> completion)."""
    import torch
    from paper_1702_08111_gb300 import mlc
    reqs = I.serving_requests(2000, 5)[:nreq]
    data = []
    for w, tier in reqs:
        f = w.charge()
        t = torch.from_numpy(f.astype(np.float32) if tier == "split" else f).cuda()
        data.append((w, tier, t, torch.empty((w.N,) * 3, dtype=torch.float64, device="cuda")))
    srv = mlc.Server(120 << 30, max_batch=8)

    def submit(k):
        w, tier, f, phi = data[k]
        return srv.enqueue(f, phi, w.N, w.n, w.s, w.P, w.Q,
                           tier=mlc.MLC_TIER_SPLIT if tier == "split" else mlc.MLC_TIER_FP64)

    # warm-up: every distinct plan once (plan creation is not serving latency)
    seen = {}
    for k, (w, tier, _, _) in enumerate(data):
        seen.setdefault((w.N, w.Q, tier), k)
    for t in [submit(k) for k in seen.values()]:
        srv.wait(t)
    # saturated: all at once
    t0 = time.perf_counter()
    for t in [submit(k) for k in range(len(data))]:
        srv.wait(t)
    sat_s = time.perf_counter() - t0
    rate = 0.7 * len(data) / sat_s
    rng = np.random.default_rng(55)
    gaps = rng.exponential(1.0 / rate, size=len(data))
    tickets = []
    t0 = time.perf_counter()
    next_t = t0
    for k in range(len(data)):
        next_t += gaps[k]
        while time.perf_counter() < next_t:
            time.sleep(min(0.0005, max(0.0, next_t - time.perf_counter())))
        tickets.append(submit(k))
    lats = []
    for t in tickets:
        st, lat, q = srv.wait(t)
        lats.append(lat)
    total_s = time.perf_counter() - t0
    srv.close()
    pts = float(sum(w.N ** 3 for w, _, _, _ in data))
    return {"requests": len(data), "rate_req_per_s": round(rate, 2),
            "saturated_req_per_s": round(len(data) / sat_s, 2),
            "p50_ms": round(float(np.percentile(lats, 50)), 3), "p99_ms": round(float(np.percentile(lats, 99)), 3),
            "Mpoints_per_s_at_rate": round(pts / total_s / 1e6, 2),
            "Mpoints_per_s_saturated": round(pts / sat_s / 1e6, 2),
            "distinct_plans": len(seen), "hbm_budget_gb": 120, "max_batch": 8}


def cpu_oracle_solve(w, nodes_sample=None):
    from oracle import mlc_oracle as O
    G1 = O.dgf_octant(w.Q, 128, 2)
    prm = O.Params(N=w.N, n=w.n, s=w.s, Q=w.Q, P=w.P)
    f = w.charge()
    t0 = time.perf_counter()
    phi = O.solve_open(prm, f, G1=G1)
    return phi, time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", dest="extra", action="store_false")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w = I.workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args, w)

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    line = None
    if rank == 0:
        cpu = None
        err = None
        if not args.no_cpu_baseline and world == 1:
            phi_o, t = cpu_oracle_solve(w)
            got = r["phi"].cpu().numpy()
            err = float(np.abs(got - phi_o).max() / np.abs(phi_o).max())
            cpu = {"value": round(float(w.N) ** 3 / t / 1e6, 4), "unit": "Mpoints/s",
                   "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"one full oracle solve of {args.workload} ({t:.1f} s; DGF table prebuilt)"}
        N = r["N"]
        e2e_val = float(N) ** 3 / (r["e2e_ms"] * 1e-3) / 1e6
        launches = 13
        line = {
            "metric": METRIC, "value": round(r["value"], 3), "unit": "Mpoints/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32x2",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": w.N, "patch": w.n, "support": w.s, "Q": w.Q,
                       "P": w.P, "tier": "fp64",
                       "arithmetic": "double-float (pairs of f32, ~48-bit significand) on the FP32 pipe; "
                                     "f64 in the moments, the plan tables and the f/phi conversions",
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"independent problem per GPU x{world}"},
            "max_rel_err_vs_oracle": err,
            "e2e": {"value": round(e2e_val, 3), "unit": "Mpoints/s",
                    "h2d_bytes_per_step": int(r["f_bytes"]), "d2h_bytes_per_step": int(N ** 3 * 8)},
            "gpu_launches": launches * args.steps,
            "roofline": r["roofline"], "cpu_baseline": cpu, "clocks": r["clocks"],
            "per_launch_ms": {k: round(v, 4) for k, v in r["per_launch"].items()},
        }
        if "extra" in r:
            line["extra"] = r["extra"]
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def run_reference(args, w):
    """Time the CPU oracle as it stands on a bounded sample of the workload."""
    from oracle import mlc_oracle as O
    # bounded sample: the 64^3 sub-problem with the workload's patch geometry and
    # charge recipe (8 patches instead of 512), one full oracle solve per step
    sub = I.Workload(w.name + "_sample64", 64, w.n, w.s, w.Q, w.P, bumps=I.draw_bumps(8, 1))
    G1 = O.dgf_octant(w.Q, 128, 2)
    prm = O.Params(N=64, n=w.n, s=w.s, Q=w.Q, P=w.P)
    f = sub.charge()
    for _ in range(args.warmup):
        O.solve_open(prm, f, G1=G1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.solve_open(prm, f, G1=G1)
    dt = (time.perf_counter() - t0) / args.steps
    val = 64.0 ** 3 / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 5), "unit": "Mpoints/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": w.N, "patch": w.n, "support": w.s, "Q": w.Q, "P": w.P,
                   "tier": "fp64"},
        "cpu_baseline": {"value": round(val, 5), "unit": "Mpoints/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "64^3 sub-problem (8 patches of 16^3, support 16, 8 bumps, seed 1) per step"},
        "e2e": {"value": round(val, 5), "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
