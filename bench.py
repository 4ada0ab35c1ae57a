#!/usr/bin/env python3
"""Benchmark: performance index PID (Sec. 4.1, Def. PID: time of one RHS evaluation / #DOF, in ns) of the
flux-differencing LGL-DGSEM RHS on GB300, FP64 (headline) and FP32-flux mode.

Workload: 3D compressible Euler, inviscid Taylor-Green vortex at Mach 0.1 on the periodic curvilinear mesh
[-pi, pi]^3 with x_i = xi_i + 0.1 sin(xi_1) sin(xi_2) sin(xi_3), 16^3 elements, polydeg 3 (262,144 DOF),
Ranocha volume flux, Ranocha + local Lax-Friedrichs surface flux. One step = one dg_step of the four-stage
low-storage RK4 (4 RHS evaluations + 4 fused stage updates); PID = step time / (4 * #DOF).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch with torchrun: the mesh grows with N along its last direction (N x 16 element layers, periodic)
and is cut into N slabs of 16^3 elements, one per rank (weak scaling); every Runge-Kutta stage packs the slab's two
boundary face planes, exchanges them with the neighbouring ranks over NCCL and unpacks them into the ghost layer
before the stage's kernels. The step time is the max over ranks.
--impl reference times the CPU oracle (plain C, FP64, one core) on a bounded element sample of the same
workload, one oracle RHS evaluation per step.
"""
from __future__ import annotations

import argparse
import ctypes
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

NELEM = [16, 16, 16]
POLYDEG = 3
MACH = 0.1
AMP = 0.1
STAGES = 4  # classical RK4, low-storage form (per stage: interface kernel + volume kernel with fused update)
METRIC = "PID (ns per DOF per RHS eval), FP64 vs FP32, 1xGB300, with roofline fraction"
WORKLOAD = "3D Euler inviscid Taylor-Green vortex M=0.1, curvilinear periodic [-pi,pi]^3 16^3 hex, p=3 (262,144 DOF)"
WORKLOAD_SHORT = "TGV M=0.1, curved periodic 16^3 hex, p=3 (262,144 DOF), RK4 step, Ranocha+LLF"
L2_FLUSH_BYTES = 512 << 20

# Algorithmic FLOPs of the volume kernel per DOF (3D, p = 3, series branch of both logarithmic means, a
# division or reciprocal counted as one flop, an FMA as two): 4.5 node pairs per DOF x 98 flops per pair
# (directional Ranocha flux 72 + averaged normal 6 + two-sided accumulation 20), 13 flops of primitive variables
# and 30 flops of direction sums, surface lift and Jacobian scaling per node, and 20 flops of the fused RK4
# stage update (5 values x 4).
VOLUME_FLOPS_PER_DOF = 4.5 * 98 + 13 + 30 + 20
# Algorithmic HBM bytes of the volume kernel per DOF in dg_step: the stage state 40 (FP64) + Ja 72 (FP64; 36 as
# the FP32 copy) + 1/J 8 + interface fluxes 2d/(p+1) = 1.5 face nodes per DOF x 5 values (8 B FP64, 4 B FP32)
# + the fused RK4 update, averaged over the 4 stages: (80 + 160 + 160 + 120)/4 = 130 (u, y, acc streams).
VOLUME_BYTES_PER_DOF_F64 = 40 + 72 + 8 + 1.5 * 5 * 8 + 130
VOLUME_BYTES_PER_DOF_F32 = 40 + 36 + 8 + 1.5 * 5 * 4 + 130
NELEM_LARGE = [32, 32, 32]  # the precision workload: 2,097,152 DOF, inputs larger than L2


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (debug runs)")
    ap.add_argument("--only", default="", help="comma-separated subset of fp64_16,fp32_16,fp64_32,fp32_32, "
                    "variants, ablation, gauss, staging, launch, rhs, batch, diff (profiling runs; prints one line per "
                    "configuration instead of the contract line)")
    ap.add_argument("--extras", default="", help="comma-separated sub-benchmarks to run before the contract line "
                    "(%s, or all); each prints its own line" % ",".join(EXTRAS))
    ap.add_argument("--details", default="", help="also write every result of the run to this JSON file")
    ap.add_argument("--slabs", action="store_true", help="run the partitioned path (slabs with halo exchanges) also "
                    "at N = 1, as one slab that is its own neighbour")
    return ap.parse_args(argv)


# ------------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)  # nvidia-smi's first sample

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi -lms 200 around the timed region"}


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml, ctypes) every 5 ms from a thread while the
    timed region runs (a region of tens of milliseconds sees no nvidia-smi sample at its 200 ms period). Reads only.
    The device is found by the UUID CUDA reports for it."""
    NVML_CLOCK_SM = 1
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, lib, handle):
        self.lib, self.handle = lib, handle
        self.samples = []
        self.thread = None
        self.stop_event = threading.Event()
        self.reasons_fn = None
        for name in ("nvmlDeviceGetCurrentClocksEventReasons", "nvmlDeviceGetCurrentClocksThrottleReasons"):
            fn = getattr(lib, name, None)
            if fn is not None:
                fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]
                fn.restype = ctypes.c_int
                self.reasons_fn = fn
                break
        lib.nvmlDeviceGetClockInfo.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint)]
        lib.nvmlDeviceGetClockInfo.restype = ctypes.c_int
        lib.nvmlDeviceGetMaxClockInfo.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint)]
        lib.nvmlDeviceGetMaxClockInfo.restype = ctypes.c_int
        mx = ctypes.c_uint(0)
        self.max_mhz = mx.value if lib.nvmlDeviceGetMaxClockInfo(handle, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0 \
            else None

    @classmethod
    def open(cls, device):
        """A sampler for the torch device, or None when NVML or the device cannot be had."""
        try:
            import torch
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            lib.nvmlInit_v2.restype = ctypes.c_int
            if lib.nvmlInit_v2() != 0:
                return None
            handle = ctypes.c_void_p()
            uuid = str(torch.cuda.get_device_properties(device).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            lib.nvmlDeviceGetHandleByUUID.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
            lib.nvmlDeviceGetHandleByUUID.restype = ctypes.c_int
            if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(handle)) != 0 or not handle.value:
                return None
            return cls(lib, handle)
        except (OSError, AttributeError, RuntimeError, ValueError):
            return None

    def _poll(self):
        clk, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self.stop_event.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.handle, self.NVML_CLOCK_SM, ctypes.byref(clk)) == 0:
                bits = rs.value if self.reasons_fn is not None and self.reasons_fn(self.handle, ctypes.byref(rs)) == 0 \
                    else 0
                self.samples.append((clk.value, bits))
            time.sleep(0.005)

    def start(self):
        self.thread = threading.Thread(target=self._poll, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_event.set()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [c for c, _ in self.samples]
        reasons = sorted({name for _, bits in self.samples for bit, name in self.REASONS.items() if bits & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "NVML, every 5 ms during the timed region"}


def clock_sampler(local_rank: int, device):
    """NVML sampling during the timed region where NVML is available, else nvidia-smi at its 200 ms period."""
    s = NvmlClockSampler.open(device)
    return s if s is not None else ClockSampler(local_rank)


# ------------------------------------------------------------------------------------------------------
# the volume kernel's sources (the launcher and the tile schedule included)
DIGEST_SOURCES = ("dgmath.cuh", "kernels.cuh", "volume.cu", "volume_impl.cuh", "volume_inst.cu", "volume_pipe.cuh",
                  "tile_plan.h")


def source_digest(root: str = ROOT) -> str:
    """sha256 (first 16 hex digits) of the volume kernel's sources with comments and blank lines removed: it changes
    with the compiled code, not with its comments."""
    h = hashlib.sha256()
    for f in DIGEST_SOURCES:
        with open(os.path.join(root, "paper_2112_10517_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update((code + "\n").encode())
    return h.hexdigest()[:16]


PROFILE_JSON = os.path.join("profiles", "volume_kernel_tgv32_p3.json")


def committed_capture(root: str = ROOT):
    """The keyed figures of the committed ncu capture of the volume kernel (32^3, p = 3; inputs larger than L2), or
    None unless the capture was taken on the current kernel source (its source digest matches)."""
    path = os.path.join(root, PROFILE_JSON)
    if not os.path.exists(path):
        return None
    try:
        cap = json.load(open(path))
    except ValueError:
        return None
    return cap if cap.get("source_digest") == source_digest(root) else None


def committed_traffic(precision: str, ndofs: int, root: str = ROOT):
    """DRAM bytes per volume-kernel launch: bytes per DOF from the committed capture times the DOF of this launch;
    None unless the capture was taken on the current kernel source."""
    cap = committed_capture(root)
    if cap is None or precision not in cap:
        return None
    return float(cap[precision]["traffic_bytes_per_dof"]) * ndofs


def committed_utilization(precision: str, root: str = ROOT):
    """The ncu view of the same kernel: FP64-pipe activity and DRAM throughput as fractions of their peaks; None
    unless the capture was taken on the current kernel source."""
    cap = committed_capture(root)
    if cap is None or precision not in cap:
        return None
    return {"fp64_pipe_active": cap[precision]["fp64_pipe_active"],
            "dram_throughput": cap[precision]["dram_throughput"], "capture": PROFILE_JSON}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except ValueError:
            pass
    return {}


# HBM bandwidth when MEASURED_PEAKS.json is absent: an earlier STREAM-style copy on a GB300 of this pool
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else the fallback figure."""
    v = measured_peaks().get("hbm_gbs")
    if isinstance(v, (int, float)) and v > 0:
        return float(v), "measured hbm_gbs"
    return HBM_FALLBACK_GBS, "fallback 6.8 TB/s"


def alu_peaks():
    """FP64 and FP32 FMA rates measured live with libdgpeaks (flop/s, FMA = 2 flop)."""
    import ctypes
    from paper_2112_10517_gb300 import build as _b
    lib = ctypes.CDLL(_b.lib_path("libdgpeaks.so"))
    out = {}
    for kind, name in ((0, "fp64"), (1, "fp32")):
        ops = ctypes.c_double()
        rc = lib.dgpk_measure(kind, ctypes.c_double(0.05), ctypes.byref(ops), None)
        out[name] = 2.0 * ops.value if rc == 0 else None
    return out


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (the step time of a multi-GPU run is that of its slowest rank)."""
    import torch
    if not torch.distributed.is_initialized() or torch.distributed.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_pid(ms_per_step: float, ndofs_per_rank: int, world: int, rhs_per_step: int = STAGES) -> float:
    """PID of the whole job: step time over all DOF processed by all ranks (weak scaling: each rank its own copy)."""
    return ms_per_step * 1e6 / (rhs_per_step * ndofs_per_rank * world)


def make_state(ctx):
    from paper_2112_10517_gb300 import inputs
    return inputs.taylor_green(ctx.node_coords(), mach=MACH)


def make_case(nelem, precision, rank, world, slabs=False, **kw):
    """The context of one rank and a function doing one RK4 step on it: the whole mesh at N = 1; at N > 1 the
    rank's slab of a mesh of nelem[2] x N layers on [-pi, (2N - 1) pi] along the last direction, stepped stage by
    stage with a halo exchange before each stage (partition.Slab)."""
    from paper_2112_10517_gb300 import dg, partition
    if world == 1 and not slabs:
        ctx = dg.DG(3, nelem, POLYDEG, lo=[-math.pi] * 3, hi=[math.pi] * 3, mapping="sine", amp=AMP, surface="llf",
                    precision=precision, **kw)
        return ctx, (lambda u, dt, scratch, stream: ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch,
                                                             stream=stream))
    glob = [nelem[0], nelem[1], nelem[2] * world]
    b, e = partition.slab_plan(glob[2], world)[rank]
    ctx = dg.DG(3, glob, POLYDEG, lo=[-math.pi] * 3, hi=[math.pi, math.pi, (2 * world - 1) * math.pi],
                mapping="sine", amp=AMP, surface="llf", precision=precision, part=(b, e), **kw)
    slab = partition.Slab(ctx, rank, world)
    return ctx, (lambda u, dt, scratch, stream: slab.step(u, scratch, dt, dg.DG_RK4_CLASSIC))


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2112_10517_gb300 import build as _b
    if rank == 0 or world == 1:
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2112_10517_gb300 import dg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    only = [x for x in args.only.split(",") if x]
    peaks_alu = alu_peaks() if rank == 0 and not only else {}
    results = {}
    runs = [("fp64_16", NELEM, "fp64", True), ("fp32_16", NELEM, "fp32", False),
            ("fp64_32", NELEM_LARGE, "fp64", False), ("fp32_32", NELEM_LARGE, "fp32", False)]
    if only:
        runs = [(lab, ne, pr, main) for lab, ne, pr, main in runs if lab in only]
    for label, nelem, precision, main in runs:
        ctx, step = make_case(nelem, precision, rank, world, slabs=args.slabs)
        slab_path = world > 1 or args.slabs
        u0 = make_state(ctx)
        u = torch.from_numpy(u0).to(dev)
        scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device=dev)
        # time step: CFL 0.5 on the smallest node spacing (TGV speed |v| + c <= 1 + 1/M)
        dt = 0.5 * (2 * math.pi / nelem[0]) / (POLYDEG + 1) ** 2 / (1.0 + 1.0 / MACH)
        for _ in range(args.warmup):
            step(u, dt, scratch, stream)
        torch.cuda.synchronize()
        if ctx.check_status() != dg.DG_OK:
            raise RuntimeError("non-physical state during warm-up")
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = clock_sampler(local_rank, dev) if main else None
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        # CUDA events around every 13th launch of the dominant (volume) kernel only: the roofline's kernel time
        # (13 is coprime to the 4 stages per step, so every stage is sampled; an event pair between two dependent
        # kernels undoes their programmatic overlap, so fewer pairs perturb the timed steps less); the interface
        # kernel is timed in a second pass below, so that the timed region carries no more events than needed
        ctx.profile(True, kernels=[dg.KERNEL_VOLUME], every=13)
        launches0 = ctx.launch_count()
        for k in range(args.steps):
            flush.zero_()  # evict L2 (larger than the 126 MB L2) between timed steps
            starts[k].record(stream)
            step(u, dt, scratch, stream)
            ends[k].record(stream)
        torch.cuda.synchronize()
        launches = ctx.launch_count() - launches0
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop() if clocks else None
        vol_ms, vol_n = ctx.profile_read(dg.KERNEL_VOLUME)
        ctx.profile(False)
        per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms = max_over_ranks(sum(per_step) / args.steps, dev)
        ms_std = statistics.pstdev(per_step) if len(per_step) > 1 else 0.0
        # the interface kernel's time per launch, from a second pass of the same steps with events around it only
        ctx.profile(True, kernels=[dg.KERNEL_INTERFACE])
        for k in range(args.steps):
            flush.zero_()
            step(u, dt, scratch, stream)
        torch.cuda.synchronize()
        ifc_ms, ifc_n = ctx.profile_read(dg.KERNEL_INTERFACE)
        ctx.profile(False)
        # the same eager steps without any per-launch profiling events (the cost of that instrumentation)
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step(u, dt, scratch, stream)
            ends[k].record(stream)
        torch.cuda.synchronize()
        nms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps, dev)
        # the same step captured once in a CUDA graph (8 kernels) and replayed per step: the launch gaps go away
        # (the library neither allocates nor synchronizes in dg_step); timed separately, same L2 flushes. (One GPU:
        # a slab's step has halo exchanges between its stages.)
        gms = None
        if not slab_path:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(stream)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                step(u, dt, scratch, side)
            for _ in range(2):
                graph.replay()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                graph.replay()
                ends[k].record(stream)
            torch.cuda.synchronize()
            gms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
        status = ctx.check_status()
        if status != dg.DG_OK:
            raise RuntimeError("non-physical state during the timed steps")
        ndofs = ctx.ndofs
        pid = whole_job_pid(ms, ndofs, world)
        vol_avg_s = vol_ms / max(vol_n, 1) * 1e-3
        res = {"ms_per_step": ms, "pid_ns": pid, "pid_std_ns": whole_job_pid(ms_std, ndofs, world) if ms_std else 0.0,
               "launches": launches, "clocks": clk,
               "volume_ms_avg": vol_avg_s * 1e3, "interface_ms_avg": ifc_ms / max(ifc_n, 1),
               "volume_share_of_step": vol_avg_s * 1e3 * STAGES / ms if ms > 0 else None,
               "graph_ms_per_step": gms, "graph_pid_ns": whole_job_pid(gms, ndofs, world) if gms else None,
               "noprof_pid_ns": whole_job_pid(nms, ndofs, world)}
        # e2e: the same step through the C ABI with the state in pinned host memory (dg_step_host: host->device copy,
        # the step, device->host copy of the new state, all inside the timed region)
        # (a slab at N > 1: the same copies around the slab's step, through the partition module's Slab)
        if main:
            u_host = torch.from_numpy(u0).pin_memory()
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

            def host_step():
                if not slab_path:
                    ctx.step_host(u_host, dt, dg.DG_RK4_CLASSIC, stream=stream)
                else:
                    u.copy_(u_host, non_blocking=True)
                    step(u, dt, scratch, stream)
                    u_host.copy_(u, non_blocking=True)
            for k in range(args.warmup):
                host_step()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()
                e0[k].record(stream)
                host_step()
                e1[k].record(stream)
            torch.cuda.synchronize()
            ems = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / args.steps, dev)
            res["e2e_pid_ns"] = whole_job_pid(ems, ndofs, world)
            res["e2e_bytes"] = int(u_host.numel() * 8)
        # roofline of the dominant kernel (volume): FP64 is bound by the FP64 pipe, FP32 by HBM
        vflops = VOLUME_FLOPS_PER_DOF * ndofs
        if precision == "fp64":
            peak = peaks_alu.get("fp64")
            achieved = vflops / vol_avg_s / 1e12
            res["roofline"] = {"bound": "alu", "achieved": achieved,
                               "peak": peak / 1e12 if peak else None, "unit": "TFLOP/s",
                               "frac": achieved / (peak / 1e12) if peak else None,
                               "traffic": committed_traffic("fp64", ndofs),
                               "peak_src": "measured FP64 FMA x2 (libdgpeaks)",
                               "algorithmic_flops_per_launch": vflops,
                               "ncu_utilization": committed_utilization("fp64")}
        else:
            hbm, hbm_src = hbm_peak()
            vbytes = VOLUME_BYTES_PER_DOF_F32 * ndofs
            achieved = vbytes / vol_avg_s / 1e9
            peak32 = peaks_alu.get("fp32")
            res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                               "frac": achieved / hbm, "traffic": committed_traffic("fp32", ndofs),
                               "peak_src": hbm_src,
                               "algorithmic_bytes_per_launch": vbytes,
                               "ncu_utilization": committed_utilization("fp32"),
                               "alu_frac_of_fp32_peak": (vflops / vol_avg_s) / peak32 if peak32 else None}
        res["ndofs"] = ndofs
        results[label] = res
        del ctx, u, scratch
    return results, peaks_alu


BATCH_N = 64


def batch_specs(seed: int = 0):
    """The batching workload: 64 instances, n^3 elements with n uniform in {4..16}, degree uniform in {2..5}."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(int(rng.integers(4, 17)), int(rng.integers(2, 6))) for _ in range(BATCH_N)]


def run_batch(args, dev):
    """PID of one batched RHS over all instances (dg_batch_rhs), FP64 and FP32, after autotuning."""
    import torch
    from paper_2112_10517_gb300 import dg, inputs
    out = {}
    specs = batch_specs()
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    for precision, logs in (("fp64", False), ("fp32", False), ("fp64", True), ("fp32", True)):
        ctxs, us, dus = [], [], []
        for k, (n, p) in enumerate(specs):
            ctx = dg.DG(3, [n, n, n], p, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision=precision,
                        precompute_logs=logs)
            u = inputs.smooth_random(ctx.node_coords(), seed=1000 + k)
            ctxs.append(ctx)
            us.append(torch.from_numpy(u).to(dev))
            dus.append(torch.empty_like(us[-1]))
        batch = dg.DGBatch(ctxs, us, dus)
        tuning = batch.autotune()
        for _ in range(args.warmup):
            batch.rhs()
        torch.cuda.synchronize()
        # the batch RHS (memset, interface launch, one persistent launch per degree) captured once in a CUDA graph
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            batch.rhs(stream=side)
        graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        bad = [i for i, c in enumerate(ctxs) if c.check_status() != dg.DG_OK]
        if bad:
            raise RuntimeError("non-physical state in batch instances %s" % bad)
        out[precision + ("_precomputed_logs" if logs else "")] = {
            "pid_ns": ms * 1e6 / batch.ndofs, "ms_per_batch_rhs": ms,
            "tuning": {"threads_per_cta": tuning[0], "ctas_per_sm": tuning[1]}}
        out["ndofs"] = batch.ndofs
        batch.close()
        del ctxs, us, dus
    out["workload"] = ("64 independent 3D Euler instances, n^3 elements (n uniform in 4..16), polydeg uniform "
                       "in 2..5, seeded smooth random states, curvilinear periodic [-pi,pi]^3, Ranocha + LLF, "
                       "one dg_batch_rhs (interface launch + one persistent volume launch per degree) per step, "
                       "captured once in a CUDA graph and replayed; inputs larger than L2")
    out["speedup_fp32_vs_fp64"] = out["fp64"]["pid_ns"] / out["fp32"]["pid_ns"]
    return out


def run_variants(args, dev):
    """dg_rhs throughput of the flux and geometry variants on the 32^3, p = 3 Taylor-Green vortex: Ranocha and
    Shima et al. volume fluxes, curvilinear (sine-perturbed) and Cartesian (affine, constant metrics) meshes,
    FP64 and FP32 flux arithmetic. L2 is flushed before every timed call."""
    import torch
    from paper_2112_10517_gb300 import dg, inputs
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for flux in ("ranocha", "shima"):
        for geo in ("curved", "cartesian"):
            for precision in ("fp64", "fp32"):
                kw = dict(mapping="sine", amp=AMP) if geo == "curved" else dict(mapping="affine")
                ctx = dg.DG(3, NELEM_LARGE, POLYDEG, lo=lo, hi=hi, surface="llf", precision=precision, flux=flux,
                            **kw)
                u = torch.from_numpy(inputs.taylor_green(ctx.node_coords(), mach=MACH)).to(dev)
                du = torch.empty_like(u)
                for _ in range(args.warmup):
                    ctx.rhs(u, du)
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                ctx.profile(True)
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    ctx.rhs(u, du)
                    b.record(stream)
                torch.cuda.synchronize()
                vol_ms, vol_n = ctx.profile_read(dg.KERNEL_VOLUME)
                ctx.profile(False)
                if ctx.check_status() != dg.DG_OK:
                    raise RuntimeError("non-physical state in the variant runs")
                ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
                out["%s_%s_%s" % (flux, geo, precision)] = {"ms": ms, "pid_ns": ms * 1e6 / ctx.ndofs,
                                                            "volume_ms": vol_ms / max(vol_n, 1)}
                del ctx, u, du
    out["workload"] = ("dg_rhs (one RHS: interface + volume kernel) on the 32^3, p = 3 Taylor-Green vortex, Mach 0.1, "
                       "2,097,152 DOF; curved = sine-perturbed mesh, cartesian = affine mesh; L2 flushed per call")
    return out


def run_staging(args, dev):
    """The RK4 step (dg_step, fused stage update) with the two ways the volume kernel stages a tile: bulk
    asynchronous copies that overlap the computation of a persistent CTA's tiles (pipelined) and direct loads by
    one CTA per tile (direct), FP32 and FP64 flux arithmetic. Taylor-Green vortex, p = 3 at 16^3 and 32^3, and
    p = 1, 2, 4, 5, 6, 7 at about 2M DOF; L2 flushed before every timed step."""
    import torch
    from paper_2112_10517_gb300 import dg
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    # (precision, p, elements per direction): p = 3 on the bench meshes, and p = 1, 2, 4, 5, 6, 7 at about 2M DOF
    cases = [("fp32", 3, NELEM[0]), ("fp32", 3, NELEM_LARGE[0]), ("fp64", 3, NELEM[0]), ("fp64", 3, NELEM_LARGE[0]),
             ("fp32", 1, 64), ("fp32", 5, 18), ("fp32", 7, 16), ("fp64", 1, 64), ("fp64", 5, 18), ("fp64", 7, 16),
             ("fp32", 2, 43), ("fp32", 4, 26), ("fp32", 6, 18), ("fp64", 2, 43), ("fp64", 4, 26), ("fp64", 6, 18)]
    for precision, p, ne in cases:
        nelem = [ne] * 3
        for staging in ("pipelined", "direct"):
            ctx = dg.DG(3, nelem, p, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision=precision,
                        staging=staging)
            u = torch.from_numpy(make_state(ctx)).to(dev)
            scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device=dev)
            dt = 0.5 * (2 * math.pi / ne) / (p + 1) ** 2 / (1.0 + 1.0 / MACH)
            for _ in range(args.warmup):
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            ctx.profile(True)
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
                b.record(stream)
            torch.cuda.synchronize()
            vol_ms, vol_n = ctx.profile_read(dg.KERNEL_VOLUME)
            ctx.profile(False)
            if ctx.check_status() != dg.DG_OK:
                raise RuntimeError("non-physical state or wait timeout in the staging runs")
            ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            key = "%s_%d_%s" % (precision, ne, staging) if p == POLYDEG else "%s_p%d_%d_%s" % (precision, p, ne, staging)
            out[key] = {"pid_ns": whole_job_pid(ms, ctx.ndofs, 1), "volume_ms": vol_ms / max(vol_n, 1)}
            del ctx, u, scratch
    out["workload"] = ("dg_step (RK4) on the Taylor-Green vortex, sine-perturbed mesh: p = 3 at 16^3 and 32^3 elements "
                       "(keys fp32_16 ...), p = 1 at 64^3, 2 at 43^3, 4 at 26^3, 5 at 18^3, 6 at 18^3, 7 at 16^3 (keys "
                       "fp32_p7_16 ...); FP32 and "
                       "FP64 flux arithmetic; volume_ms = the volume kernel's event time per launch")
    return out


def run_rhs_pid(args, dev, runs: int = 5, calls: int = 20):
    """The PID of one dg_rhs evaluation (Sec. 4.1, Def. PID: time of one RHS / #DOF), mean and standard deviation
    over `runs` runs, each the mean of `calls` calls with L2 flushed before every call and CUDA events around the
    call alone; with the volume and interface kernels' own event times per DOF. Taylor-Green vortex, p = 3,
    sine-perturbed mesh at 16^3 and 32^3 elements, FP64 and FP32."""
    import statistics
    import torch
    from paper_2112_10517_gb300 import dg
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for precision, ne in (("fp64", NELEM[0]), ("fp32", NELEM[0]), ("fp64", NELEM_LARGE[0]), ("fp32", NELEM_LARGE[0])):
        ctx = dg.DG(3, [ne] * 3, POLYDEG, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision=precision)
        u = torch.from_numpy(make_state(ctx)).to(dev)
        du = torch.empty_like(u)
        for _ in range(max(args.warmup, 3)):
            ctx.rhs(u, du)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
        means = []
        for _ in range(runs):
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.rhs(u, du)
                b.record(stream)
            torch.cuda.synchronize()
            means.append(sum(a.elapsed_time(b) for a, b in ev) / calls)
        # the kernels' own times: a separate pass with events around each kernel
        ctx.profile(True)
        for _ in range(calls):
            flush.zero_()
            ctx.rhs(u, du)
        torch.cuda.synchronize()
        vol_ms, vol_n = ctx.profile_read(dg.KERNEL_VOLUME)
        ifc_ms, ifc_n = ctx.profile_read(dg.KERNEL_INTERFACE)
        ctx.profile(False)
        if ctx.check_status() != dg.DG_OK:
            raise RuntimeError("non-physical state in the RHS runs")
        nd = ctx.ndofs
        out["%s_%d" % (precision, ne)] = {
            "pid_ns": statistics.mean(means) * 1e6 / nd, "pid_std_ns": statistics.pstdev(means) * 1e6 / nd,
            "volume_pid_ns": vol_ms / max(vol_n, 1) * 1e6 / nd, "interface_pid_ns": ifc_ms / max(ifc_n, 1) * 1e6 / nd}
        del ctx, u, du
    out["workload"] = ("dg_rhs (interface kernel + volume kernel storing du) on the Taylor-Green vortex, sine-perturbed "
                       "mesh, p = 3 at 16^3 and 32^3 elements; %d runs of %d calls, L2 flushed before every call; "
                       "pid_std_ns over the runs' means; volume/interface_pid_ns from the kernels' own events"
                       % (runs, calls))
    return out


def run_launch_modes(args, dev):
    """The RK4 step (dg_step) with the interface and pipelined volume kernels launched as programmatic dependents
    of the kernel before them (overlap, the default) and as ordinary launches (serial): eager steps without
    profiling events, and the same step captured in a CUDA graph and replayed. Taylor-Green vortex, p = 3 at 16^3
    and 32^3 elements, FP64 and FP32; L2 flushed before every timed step."""
    import torch
    from paper_2112_10517_gb300 import dg
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for precision, ne in (("fp64", NELEM[0]), ("fp32", NELEM[0]), ("fp64", NELEM_LARGE[0]), ("fp32", NELEM_LARGE[0])):
        for launch in ("overlap", "serial"):
            ctx = dg.DG(3, [ne] * 3, POLYDEG, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf",
                        precision=precision, launch=launch)
            u = torch.from_numpy(make_state(ctx)).to(dev)
            scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device=dev)
            dt = 0.5 * (2 * math.pi / ne) / (POLYDEG + 1) ** 2 / (1.0 + 1.0 / MACH)
            for _ in range(args.warmup):
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
                b.record(stream)
            torch.cuda.synchronize()
            eager = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(stream)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch, stream=side)
            for _ in range(2):
                graph.replay()
            torch.cuda.synchronize()
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                graph.replay()
                b.record(stream)
            torch.cuda.synchronize()
            gms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            if ctx.check_status() != dg.DG_OK:
                raise RuntimeError("non-physical state or wait timeout in the launch-mode runs")
            out["%s_%d_%s" % (precision, ne, launch)] = {"pid_ns": whole_job_pid(eager, ctx.ndofs, 1),
                                                        "graph_pid_ns": whole_job_pid(gms, ctx.ndofs, 1)}
            del ctx, u, scratch, graph
    out["workload"] = ("dg_step (RK4) on the Taylor-Green vortex, sine-perturbed mesh, p = 3 at 16^3 and 32^3 "
                       "elements; pid_ns eager without profiling events, graph_pid_ns as graph replays")
    return out


def run_reference_pressure(args, dev):
    """The FP32 flux mode's RK4 step (dg_step) without and with the reference pressure p_ref = 1/(gamma M^2)
    (dg_opts.p_ref: the momentum equations' pressure terms on p - p_ref), Taylor-Green vortex p = 3 at 16^3 and
    32^3 elements; eager steps without profiling events, L2 flushed before every timed step."""
    import torch
    from paper_2112_10517_gb300 import dg
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    p0 = 1.0 / (1.4 * MACH ** 2)
    out = {}
    for ne in (NELEM[0], NELEM_LARGE[0]):
        for name, pref in (("plain", 0.0), ("p_ref", p0)):
            ctx = dg.DG(3, [ne] * 3, POLYDEG, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision="fp32",
                        p_ref=pref)
            u = torch.from_numpy(make_state(ctx)).to(dev)
            scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device=dev)
            dt = 0.5 * (2 * math.pi / ne) / (POLYDEG + 1) ** 2 / (1.0 + 1.0 / MACH)
            for _ in range(args.warmup):
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            torch.cuda.synchronize()
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.step(u, dt, dg.DG_RK4_CLASSIC, scratch=scratch)
                b.record(stream)
            torch.cuda.synchronize()
            if ctx.check_status() != dg.DG_OK:
                raise RuntimeError("non-physical state in the reference-pressure runs")
            ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            out["fp32_%d_%s" % (ne, name)] = {"pid_ns": whole_job_pid(ms, ctx.ndofs, 1), "ms_per_step": ms}
            del ctx, u, scratch
    out["workload"] = ("dg_step (RK4), FP32 flux mode, Taylor-Green vortex Mach 0.1, sine-perturbed mesh, p = 3 at "
                       "16^3 and 32^3 elements, without and with p_ref = 1/(gamma M^2)")
    return out


def run_logmean_ablation(args, dev):
    """Volume-term time of the log-mean variants (Sec. 3.1: Algorithms 2/3 with divisions, with the polynomial 1/log
    form; Sec. 7.2: logarithms precomputed per node) against the default (no division, one shared reciprocal),
    on the three initial conditions of the paper's ablation, 2D and 3D, p = 3 and 7, on the sine-perturbed mesh of
    [-5, 5]^d. FP64; FP32 for 3D p = 3. Each entry is the mean of `steps` dg_rhs calls, L2 flushed before each.
    Every variant runs the per-tile volume kernel, so that the log mean is the only difference."""
    import torch
    from paper_2112_10517_gb300 import dg, inputs
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    geos = [(3, [32, 32, 32], 3, "fp64"), (3, [16, 16, 16], 7, "fp64"), (2, [256, 256], 3, "fp64"),
            (2, [128, 128], 7, "fp64"), (3, [32, 32, 32], 3, "fp32")]
    variants = [("default", {}), ("precomputed_logs", dict(precompute_logs=True)), ("alg23", dict(logmean="alg")),
                ("alg23_poly", dict(logmean="alg_poly"))]
    out = {}
    for nd, nelem, p, precision in geos:
        lo, hi = [-5.0] * nd, [5.0] * nd
        states = None
        geo = {}
        for vname, vkw in variants:
            # all variants on the per-tile kernel (the pipelined one serves the default log mean only)
            ctx = dg.DG(nd, nelem, p, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision=precision,
                        staging="direct", **vkw)
            if states is None:
                xyz = ctx.node_coords()
                states = {"vortex": inputs.isentropic_vortex(xyz, eps=20.0), "sine": inputs.sine_paper(xyz),
                          "random": inputs.random_state(xyz, seed=0)}
            for ic, u0 in states.items():
                u = torch.from_numpy(u0).to(dev)
                du = torch.empty_like(u)
                for _ in range(args.warmup):
                    ctx.rhs(u, du)
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                ctx.profile(True)
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    ctx.rhs(u, du)
                    b.record(stream)
                torch.cuda.synchronize()
                vol_ms, vol_n = ctx.profile_read(dg.KERNEL_VOLUME)
                ctx.profile(False)
                if ctx.check_status() != dg.DG_OK:
                    raise RuntimeError("non-physical state in the log-mean ablation")
                geo.setdefault(ic, {})[vname] = {
                    "volume_ms": vol_ms / max(vol_n, 1),
                    "rhs_ms": sum(a.elapsed_time(b) for a, b in ev) / args.steps}
                del u, du
            del ctx
        for ic, row in geo.items():
            base = row["default"]["volume_ms"]
            for vname in row:
                row[vname]["volume_rel_to_default"] = row[vname]["volume_ms"] / base
            row["precomputed_rel_to_per_pair"] = row["precomputed_logs"]["volume_ms"] / base
        out["%dd_p%d_%s" % (nd, p, precision)] = geo
    out["workload"] = ("dg_rhs on the sine-perturbed mesh of [-5,5]^d: 3D 32^3 p=3 and 16^3 p=7 (2,097,152 DOF), "
                       "2D 256^2 p=3 and 128^2 p=7 (1,048,576 DOF); initial conditions: isentropic vortex eps=20, "
                       "rho = 2 + prod sin(pi x/5) with p = rho^gamma, seeded random; Ranocha + LLF")
    return out


def run_gauss(args, dev):
    """Legendre-Gauss collocation with entropy projection (Sec. 6) against LGL-DGSEM on the same affine mesh:
    dg_rhs time per DOF and the per-kernel breakdown (entropy projection, interface flux, volume term), Taylor-Green
    vortex on [-pi, pi]^3, FP64, EC surface fluxes as in the paper's Gauss runs. L2 flushed before every call."""
    import torch
    from paper_2112_10517_gb300 import dg, inputs
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    out = {}
    for nelem, p in (([32, 32, 32], 3), ([16, 16, 16], 7)):
        row = {}
        for nodes in ("lgl", "gauss"):
            ctx = dg.DG(3, nelem, p, lo=lo, hi=hi, mapping="affine", surface="ec", nodes=nodes)
            u = torch.from_numpy(inputs.taylor_green(ctx.node_coords(), mach=MACH)).to(dev)
            du = torch.empty_like(u)
            for _ in range(args.warmup):
                ctx.rhs(u, du)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            ctx.profile(True)
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.rhs(u, du)
                b.record(stream)
            torch.cuda.synchronize()
            parts = {name: ctx.profile_read(kid)[0] / args.steps for name, kid in
                     (("volume_ms", dg.KERNEL_VOLUME), ("interface_ms", dg.KERNEL_INTERFACE),
                      ("projection_ms", dg.KERNEL_PROJECT))}
            ctx.profile(False)
            if ctx.check_status() != dg.DG_OK:
                raise RuntimeError("non-physical state in the Gauss comparison")
            ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
            row[nodes] = dict(ms=ms, pid_ns=ms * 1e6 / ctx.ndofs, **parts)
            del ctx, u, du
        row["gauss_over_lgl"] = row["gauss"]["pid_ns"] / row["lgl"]["pid_ns"]
        out["3d_%d_p%d" % (nelem[0], p)] = row
    out["workload"] = ("dg_rhs, Taylor-Green vortex Mach 0.1 on the affine [-pi,pi]^3 mesh, 32^3 p=3 and 16^3 p=7 "
                       "(2,097,152 DOF), Ranocha's flux, EC surface flux, FP64; LGL-DGSEM vs Legendre-Gauss "
                       "collocation with entropy projection")
    return out


def run_diff_and_scale(args, dev):
    """The differentiation workload (dg_vjp on 8^3, p = 4, FP64) and forward RHS throughput at 64^3, p = 3."""
    import torch
    from paper_2112_10517_gb300 import dg, inputs
    lo, hi = [-math.pi] * 3, [math.pi] * 3

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    out = {}
    ctx = dg.DG(3, [8, 8, 8], 4, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf")
    u = torch.from_numpy(inputs.smooth_random(ctx.node_coords(), seed=40)).to(dev)
    g = torch.from_numpy(inputs.perturbation(tuple(u.shape), 41)).to(dev)
    du, ub = torch.empty_like(u), torch.empty_like(u)
    ms_f = timed(lambda: ctx.rhs(u, du))
    ms_b = timed(lambda: ctx.vjp(u, g, ub))
    out["vjp_8cubed_p4_fp64"] = {"rhs_ms": ms_f, "vjp_ms": ms_b, "vjp_over_rhs": ms_b / ms_f,
                                 "pid_rhs_ns": ms_f * 1e6 / ctx.ndofs, "pid_vjp_ns": ms_b * 1e6 / ctx.ndofs}
    del ctx, u, g, du, ub
    for precision in ("fp64", "fp32"):
        ctx = dg.DG(3, [64, 64, 64], 3, lo=lo, hi=hi, mapping="sine", amp=AMP, surface="llf", precision=precision)
        u = torch.from_numpy(inputs.taylor_green(ctx.node_coords(), mach=MACH)).to(dev)
        du = torch.empty_like(u)
        ms = timed(lambda: ctx.rhs(u, du))
        out["rhs_64cubed_p3_" + precision] = {"ms": ms, "pid_ns": ms * 1e6 / ctx.ndofs, "ndofs": ctx.ndofs}
        del ctx, u, du
    out["workload"] = ("dg_vjp vs dg_rhs on 3D curvilinear 8^3, p = 4, FP64 (smooth random state); dg_rhs at 64^3, "
                       "p = 3 (16.8M DOF) Taylor-Green, FP64 and FP32; back-to-back calls, inputs larger than L2 "
                       "at 64^3")
    return out


def oracle_pid(seconds_target: float, elements=None):
    """Time the CPU oracle RHS on the same workload; returns (pid_ns, sample description, reps)."""
    import numpy as np
    import oracle as orc
    from paper_2112_10517_gb300 import inputs
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    xyz = orc.coords(3, NELEM, lo, hi, POLYDEG, mapping=1, amp=AMP)
    Ja, J = orc.metrics(3, POLYDEG, xyz)
    u = inputs.taylor_green(xyz, mach=MACH)
    E = u.shape[0]
    b, e = (0, E) if elements is None else elements
    nd = (e - b) * u.shape[2]
    reps, t0 = 0, time.perf_counter()
    while True:
        orc.rhs(3, POLYDEG, NELEM, Ja, J, u, llf=True, elem_range=(b, e))
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target and reps >= 2:
            break
    return el / (reps * nd) * 1e9, reps, nd


def _oracle_slice(job):
    """Worker of oracle_pid_all_cores (a spawned process): `reps` oracle RHS evaluations of elements [b, e)."""
    import oracle as orc
    Ja, J, u, b, e, reps = job
    t0 = time.perf_counter()
    for _ in range(reps):
        orc.rhs(3, POLYDEG, NELEM, Ja, J, u, llf=True, elem_range=(b, e))
    return time.perf_counter() - t0


def oracle_pid_all_cores(reps: int = 8):
    """The same oracle RHS split over all host cores by element ranges (spawned processes, one per core): the
    parallel wall time of `reps` full evaluations, as ns per DOF per RHS; returns (pid_ns, cores)."""
    import multiprocessing as mp
    import oracle as orc
    from paper_2112_10517_gb300 import inputs
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    xyz = orc.coords(3, NELEM, lo, hi, POLYDEG, mapping=1, amp=AMP)
    Ja, J = orc.metrics(3, POLYDEG, xyz)
    u = inputs.taylor_green(xyz, mach=MACH)
    E = u.shape[0]
    cores = max(1, min(os.cpu_count() or 1, E))
    bounds = [(E * k // cores, E * (k + 1) // cores) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_slice, [(Ja, J, u, b, e, 1) for b, e in bounds])  # warm-up: imports and the library
        times = pool.map(_oracle_slice, [(Ja, J, u, b, e, reps) for b, e in bounds])
    return max(times) / (reps * u.shape[0] * u.shape[2]) * 1e9, cores


def arm_config(args, world):
    """The contract line's config, the same on both arms (the reference arm's sample is in its cpu_baseline)."""
    return {"workload": WORKLOAD_SHORT, "l2": "flushed each step",
            "parallelism": "slabs+halo" if world > 1 or args.slabs else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    # each step: one oracle RHS evaluation on a fixed sample of 512 elements (1/8 of the mesh, 32,768 DOF)
    import numpy as np
    from paper_2112_10517_gb300 import inputs
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    xyz = orc.coords(3, NELEM, lo, hi, POLYDEG, mapping=1, amp=AMP)
    Ja, J = orc.metrics(3, POLYDEG, xyz)
    u = inputs.taylor_green(xyz, mach=MACH)
    sample = (1536, 2048)
    nd = (sample[1] - sample[0]) * u.shape[2]
    for _ in range(args.warmup):
        orc.rhs(3, POLYDEG, NELEM, Ja, J, u, llf=True, elem_range=sample)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.rhs(3, POLYDEG, NELEM, Ja, J, u, llf=True, elem_range=sample)
        times.append(time.perf_counter() - t0)
    ms = sum(times) / len(times) * 1e3
    pid = ms * 1e6 / nd
    line = {"metric": METRIC, "value": pid, "unit": "ns/DOF/RHS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": arm_config(args, world),
            "cpu_baseline": {"value": pid, "unit": "ns/DOF/RHS", "cores": 1, "kind": "oracle",
                             "sample": "one oracle RHS evaluation per step on elements 1536-2047 (512 of the "
                                       "4096) of the 16^3 Taylor-Green mesh (%s)" % WORKLOAD},
            "e2e": {"value": pid, "unit": "ns/DOF/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The sub-benchmarks beyond the headline (--extras): each prints its own line before the contract line.
EXTRAS = ("batch", "diff", "variants", "ablation", "gauss", "staging", "launch", "rhs", "pref")
CONTRACT_LINE_MAX_BYTES = 1200


def sig(x, digits: int = 4):
    """x rounded to `digits` significant digits (None stays None): keeps the contract line short."""
    if x is None or not isinstance(x, float) or x == 0.0 or not math.isfinite(x):
        return x
    return round(x, digits - 1 - int(math.floor(math.log10(abs(x)))))


def contract_line(args, world: int, results: dict, cpu) -> dict:
    """The one JSON line the benchmark contract asks for, printed last: the FP64 headline (16^3, p = 3 RK4 step),
    its roofline, the CPU oracle, the end-to-end figure through the host-state entry point, clocks, and the FP32
    mode and the 32^3 precision workload as single numbers. Everything else goes to earlier lines."""
    r64, r32 = results["fp64_16"], results.get("fp32_16")
    b64, b32 = results.get("fp64_32"), results.get("fp32_32")
    rf = r64["roofline"]
    clk = r64.get("clocks") or {}
    line = {
        "metric": METRIC, "value": sig(r64["pid_ns"]), "value_std": sig(r64["pid_std_ns"], 2), "unit": "ns/DOF/RHS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sig(r64["ms_per_step"]),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args, world),
        "roofline": {"bound": rf["bound"], "achieved": sig(rf["achieved"]), "peak": sig(rf["peak"]),
                     "unit": rf["unit"], "frac": sig(rf["frac"], 3), "traffic": sig(rf["traffic"]),
                     "peak_src": rf["peak_src"]},
        "cpu_baseline": cpu,
        "e2e": {"value": sig(r64.get("e2e_pid_ns")), "unit": "ns/DOF/RHS",
                "h2d_bytes_per_step": r64.get("e2e_bytes"), "d2h_bytes_per_step": r64.get("e2e_bytes")},
        "gpu_launches": r64["launches"],
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons")},
    }
    if r32:
        line["fp32"] = {"value": sig(r32["pid_ns"]), "ms_per_step": sig(r32["ms_per_step"]),
                        "hbm_frac": sig(r32["roofline"]["frac"], 3)}
    if b64 and b32:
        line["p3_32cubed"] = {"fp64": sig(b64["pid_ns"]), "fp32": sig(b32["pid_ns"]),
                              "fp64_frac": sig(b64["roofline"]["frac"], 3), "fp32_frac": sig(b32["roofline"]["frac"], 3)}
    return line


def compact_cpu_baseline(cpu):
    """The cpu_baseline object of the contract line (the full record goes to a detail line)."""
    if cpu is None:
        return None
    out = {"value": sig(cpu["value"]), "unit": cpu["unit"], "cores": cpu["cores"], "kind": cpu["kind"],
           "sample": "full 16^3 mesh RHS x%d, 1 core" % cpu["reps"]}
    if cpu.get("all_cores"):
        out["all_cores_value"] = sig(cpu["all_cores"]["value"])
        out["all_cores"] = cpu["all_cores"]["cores"]
    return out


def emit(name: str, payload, sink: dict):
    """One detail line (printed before the contract line) and its entry in the details file."""
    sink[name] = payload
    print(json.dumps({"bench_detail": name, "result": payload}), flush=True)


def main(argv=None):
    args = parse_args(argv)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    results, peaks_alu = run_ours(args, rank, world, local_rank)
    dev = torch.device("cuda", local_rank)
    runners = {"batch": run_batch, "diff": run_diff_and_scale, "variants": run_variants,
               "ablation": run_logmean_ablation, "gauss": run_gauss, "staging": run_staging,
               "launch": run_launch_modes, "rhs": run_rhs_pid, "pref": run_reference_pressure}
    if rank == 0 and args.only:
        for label, res in results.items():
            print(json.dumps({"configuration": label, "pid_ns": res["pid_ns"], "noprof_pid_ns": res["noprof_pid_ns"],
                              "graph_pid_ns": res["graph_pid_ns"], "ms_per_step": res["ms_per_step"],
                              "volume_ms": res["volume_ms_avg"], "interface_ms": res["interface_ms_avg"],
                              "e2e_pid_ns": res.get("e2e_pid_ns")}),
                  flush=True)
        for name in args.only.split(","):
            if name in runners:
                print(json.dumps({"configuration": name, "result": runners[name](args, dev)}), flush=True)
    elif rank == 0:
        details = {}
        for label, res in results.items():
            emit(label, res, details)
        emit("alu_peaks_measured_tflops", {k: (v / 1e12 if v else None) for k, v in peaks_alu.items()}, details)
        wanted = EXTRAS if args.extras == "all" else [x for x in args.extras.split(",") if x]
        for name in wanted:
            if name not in runners:
                raise SystemExit("unknown --extras entry %r (choose from %s)" % (name, ", ".join(EXTRAS)))
            emit(name, runners[name](args, dev), details)
        cpu = None
        if not args.no_cpu_baseline and world == 1:  # the oracle baseline: rank 0 at N = 1 only
            pid_cpu, reps, nd = oracle_pid(10.0)
            cpu = {"value": pid_cpu, "unit": "ns/DOF/RHS", "cores": 1, "kind": "oracle", "reps": reps,
                   "sample": "%d oracle RHS evaluations of the full 16^3 p=3 mesh (%d DOF each), 1 core" % (reps, nd)}
            pid_all, cores = oracle_pid_all_cores()
            cpu["all_cores"] = {"value": pid_all, "unit": "ns/DOF/RHS", "cores": cores,
                                "sample": "8 oracle RHS evaluations of the full 16^3 p=3 mesh split by element "
                                          "ranges over %d spawned processes (parallel wall time)" % cores}
            emit("cpu_baseline", cpu, details)
        line = contract_line(args, world, results, compact_cpu_baseline(cpu))
        if args.details:
            with open(args.details, "w") as fh:
                json.dump({"contract": line, "details": details}, fh, indent=1)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
