#!/usr/bin/env python3
"""Throughput of one RPMD time step (B300, sm_103a) on synthetic flexible water.

Default workload: 4,096 q-SPC/Fw-style waters (12,288 atoms, 49.7 A box, rc 9 A),
P = 32 beads, 300 K, dt 0.5 fs, PILE thermostat, mixed precision (FP32 pair
math, int64 fixed-point forces, FP64 modes and integrator).

A "step" is one full BAOAB step of the hot path: B-A-O-A in normal modes with
the bead transform, the centroid-list check (and rebuild when due), the
nonbonded and bonded bead forces, the force projection and the closing B.
For adQTB the once-per-segment work (spectra, gamma update, next colored-noise
segment) is included, amortised over the segment's steps.
Each timed step is bracketed by CUDA events on the library's stream; the L2 is
flushed (a 256 MB write) between steps, outside the events.

``--impl reference`` times the FP64 CPU oracle on the same workload instead.
Under torchrun every rank runs an independent replica (the path is replicas
only on one-GPU machines); rank 0 prints the line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# load every kernel of the library at start-up: the first replay of a rarely taken
# conditional branch (a list rebuild) must not pay for lazy module loading in a timed step
os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")

METRIC = "atom·bead·steps/s (ns/day) RPMD & adQTB water vs FP64 GPU path at stated error"
UNIT = "atom·bead·steps/s"
# Algorithmic FP32 flops per in-cutoff bead pair (FMA = 2) of the DSF Coulomb force on both
# atoms, and the extra flops of the LJ term on O-O pairs.
FLOPS_PAIR = 45
FLOPS_LJ = 8


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks of the initialised process group (the job's time is
    its slowest rank's), followed by a barrier."""
    import torch
    import torch.distributed as td
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    td.barrier()
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class _NvmlCtypes:
    """The few NVML calls the clock sampler makes, through ctypes on the driver's
    libnvidia-ml.so.1, for hosts without the pynvml module.  Names, signatures and the
    clock-event reason bits follow the public nvml.h."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} returned {rc}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2(), "nvmlInit_v2")

    def nvmlShutdown(self):
        self.lib.nvmlShutdown()

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.c.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.c.c_uint(i), self.c.byref(h)), "GetHandleByIndex")
        return h

    def nvmlDeviceGetHandleByUUID(self, uuid):
        h = self.c.c_void_p()
        u = uuid if isinstance(uuid, bytes) else uuid.encode()
        self._ok(self.lib.nvmlDeviceGetHandleByUUID(self.c.c_char_p(u), self.c.byref(h)), "GetHandleByUUID")
        return h

    def _clock(self, fn, h, kind):
        v = self.c.c_uint()
        self._ok(fn(h, self.c.c_int(kind), self.c.byref(v)), "clock query")
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h, kind)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h, kind)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.c.byref(v)), "clock event reasons")
        return v.value


class ClockSampler:
    """SM clock and throttle-reason samples during the timed region: NVML polled every 2 ms
    from a thread (a timed region of a few milliseconds still gets samples), else nvidia-smi
    at its 50 ms floor."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        # nvidia-smi numbers every GPU of the node: map the CUDA device ordinal through
        # CUDA_VISIBLE_DEVICES (an index or a UUID) so that the samples are this rank's GPU's
        vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
        self.index = vis[index] if index < len(vis) else str(index)
        self.rows = []
        self.proc = None
        self.thread = None

    def _nvml_loop(self, nv, handle):
        reasons = [("hw_slowdown", nv.nvmlClocksEventReasonHwSlowdown),
                   ("hw_thermal_slowdown", nv.nvmlClocksEventReasonHwThermalSlowdown),
                   ("sw_thermal_slowdown", nv.nvmlClocksEventReasonSwThermalSlowdown),
                   ("sw_power_cap", nv.nvmlClocksEventReasonSwPowerCap)]
        mx = nv.nvmlDeviceGetMaxClockInfo(handle, nv.NVML_CLOCK_SM)
        while not self.stop.is_set():
            sm = nv.nvmlDeviceGetClockInfo(handle, nv.NVML_CLOCK_SM)
            bits = nv.nvmlDeviceGetCurrentClocksEventReasons(handle)
            self.rows.append([str(sm), str(mx)] + ["Active" if bits & b else "Not Active" for _, b in reasons])
            time.sleep(0.002)

    def __enter__(self):
        self.stop = threading.Event()
        try:
            try:
                import pynvml as nv
            except ImportError:
                nv = _NvmlCtypes()
            nv.nvmlInit()
            idx = self.index
            if idx.isdigit():
                handle = nv.nvmlDeviceGetHandleByIndex(int(idx))
            else:
                try:
                    handle = nv.nvmlDeviceGetHandleByUUID(idx)
                except Exception:
                    handle = nv.nvmlDeviceGetHandleByUUID(idx.encode())
            self.nvml = nv
            self.thread = threading.Thread(target=self._nvml_loop, args=(nv, handle), daemon=True)
            self.thread.start()
            return self
        except Exception as e:   # no NVML here: fall back to nvidia-smi, and say why
            self.nvml = None
            self.nvml_error = f"{type(e).__name__}: {e}"[:120]
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def __exit__(self, *a):
        self.stop.set()
        if getattr(self, "nvml", None) is not None:
            self.thread.join(timeout=2)
            try:
                self.nvml.nvmlShutdown()
            except Exception:
                pass
            return
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    **({"nvml_error": self.nvml_error} if getattr(self, "nvml_error", None) else {})}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[2 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows),
                "source": ("nvml, 2 ms" if getattr(self, "nvml", None) is not None else "nvidia-smi, 50 ms")
                + (" (ctypes)" if isinstance(getattr(self, "nvml", None), _NvmlCtypes) else ""),
                **({"nvml_error": self.nvml_error} if getattr(self, "nvml_error", None) else {})}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


SKIN = None   # --skin: the neighbour-list skin (A) in place of the workload's own


def _config(name):
    import dataclasses
    from paper_2212_03137_b300.workloads import CONFIGS
    cfg = CONFIGS[name]
    return dataclasses.replace(cfg, skin=SKIN) if SKIN is not None else cfg


def _workload_conf(name, cfg, ws):
    """The workload a line measures (the same dict on both arms)."""
    conf = {"workload": name, "n_molecules": cfg.n_mol, "n_atoms": 3 * cfg.n_mol, "beads": cfg.P, "box_A": cfg.box,
            "rc_A": cfg.rc, "skin_A": cfg.skin, "dt_fs": cfg.dt_fs, "temperature_K": cfg.temperature,
            "thermostat": cfg.thermostat, "precision": cfg.precision,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"}
    if "respa" in cfg.extra:
        conf.update({"respa_inner_steps": int(cfg.extra["respa"]),
                     "contracted_beads": int(cfg.extra.get("contracted_beads", 0)),
                     "step": "one RESPA outer step; the metric counts its inner time steps"})
    return conf


def _batch_conf(cfgs, ws):
    return {"workload": "batch_256", "n_systems": len(cfgs),
            "n_molecules_range": [min(c.n_mol for c in cfgs), max(c.n_mol for c in cfgs)],
            "beads": sorted({c.P for c in cfgs}), "density_g_cm3": 1.0, "dt_fs": 0.5, "temperature_K": 300.0,
            "thermostat": "pile", "precision": "mixed", "l2": "flushed between timed steps (256 MB write)",
            "parallelism": f"replicas x{ws}"}


def _host():
    """The host the CPU baseline ran on: CPU model and the cores the OS reports."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def _sampled_force_error(h, cfg, n_mol=40, seed=5):
    """RMS relative error of the GPU forces of bead 0 on the atoms of n_mol sampled molecules
    against the oracle's brute-force sum for those atoms (any box size; FP64)."""
    from oracle import water as ow
    from paper_2212_03137_b300 import qhp
    from paper_2212_03137_b300.workloads import WATER_FF as W
    ff = ow.ForceField(eps=W["eps"], sigma=W["sigma"], q_O=W["q_O"], k_b=W["k_b"], r0=W["r0"],
                       k_theta=W["k_theta"], theta0=math.radians(W["theta0_deg"]), alpha=W["alpha"], rc=cfg.rc,
                       m_O=W["m_O"], m_H=W["m_H"])
    box = cfg.system()
    qhp.qhp_compute_forces(h)
    F = qhp.qhp_get_forces(h)[0]
    x = qhp.qhp_get_beads(h)[0]
    mols = np.sort(np.random.default_rng(seed).choice(box.n_mol, min(n_mol, box.n_mol), replace=False))
    atoms = np.concatenate([np.arange(3 * m, 3 * m + 3) for m in mols])
    Fo = ow.nonbonded_on_atoms(x, atoms, box.types, box.molecule, box.box, ff) + ow.bonded(x[atoms], box.box, ff)[1]
    return float(np.sqrt(np.sum((F[atoms] - Fo) ** 2) / np.sum(Fo ** 2)))


def run_ours(args, ws, rank, local):
    import torch
    from paper_2212_03137_b300 import build, qhp

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = _config(args.workload)
    sysobj = qhp.System.from_config(cfg, seed=cfg.seed + 1000 * rank)
    h = sysobj.h
    # one explicit stream for the library's kernels, the L2 flush and the timing events
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    qhp.qhp_set_stream(h, stream.cuda_stream)
    qhp.qhp_set_graph_mode(h, not args.direct_launch)
    inner = int(cfg.extra.get("respa", 1))        # time steps per call (RESPA outer step)
    if "respa" in cfg.extra:
        qhp.qhp_set_respa(h, inner, int(cfg.extra.get("contracted_beads", 0)))
    N, P = sysobj.n_atoms, sysobj.P
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step = qhp.qhp_step_adqtb if cfg.thermostat == "adqtb" else qhp.qhp_step_rpmd

    # warm-up (compiles the step graph, fills the list)
    for _ in range(args.warmup):
        step(h, 1)
    qhp.qhp_sync(h)
    pairs, oo_pairs = qhp.qhp_count_pairs(h)
    if "respa" in cfg.extra:
        # the pair kernel runs on the contracted beads: the in-cutoff pair count of the full
        # ring polymer scaled by Pc/P (an estimate: the bead-pair density is the same)
        pc = int(cfg.extra.get("contracted_beads", 0)) or P
        pairs, oo_pairs = pairs * pc // P, oo_pairs * pc // P
    qhp.qhp_set_profiling(h, True)
    step(h, 1)
    qhp.qhp_sync(h)

    dist = ws > 1
    if dist:
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize(dev)
    info0 = qhp.qhp_get_info(h)
    launches0, rebuilds0 = info0.kernel_launches, info0.rebuilds
    step_ms, pair_ms, stages = [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                       # evict L2 between timed steps (outside the events)
            e0.record(stream)
            step(h, 1)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            pr = qhp.qhp_get_profile(h)
            pair_ms.append(pr.pair_ms)
            stages.append([pr.integrate_ms, pr.list_ms, pr.pair_ms, pr.bonded_ms, pr.project_ms])
    info1 = qhp.qhp_get_info(h)
    launches = info1.kernel_launches - launches0
    rebuilds = info1.rebuilds - rebuilds0
    total_ms = float(np.sum(step_ms))
    seg = None
    if cfg.thermostat == "adqtb":
        # Once per segment the step also runs the spectra, the gamma update and the next
        # noise segment.  Whole-job throughput carries that work amortised over the segment:
        # the timed steps that ended a segment are replaced by regular steps plus their
        # share, and when none fell in the window one segment-end step is timed on its own.
        step0 = info1.step - args.steps
        ends = [k for k in range(args.steps) if (step0 + k + 1) % cfg.n_seg == 0]
        regular = [t for k, t in enumerate(step_ms) if k not in ends]
        mean_reg = float(np.mean(regular))
        if ends:
            end_ms = float(np.mean([step_ms[k] for k in ends]))
        else:
            left = cfg.n_seg - 1 - (info1.step % cfg.n_seg)
            if left:
                step(h, left)
            flush.zero_()
            e0.record(stream)
            step(h, 1)
            e1.record(stream)
            e1.synchronize()
            end_ms = e0.elapsed_time(e1)
        extra = max(0.0, end_ms - mean_reg)
        total_ms = args.steps * (mean_reg + extra / cfg.n_seg)
        seg = {"segment_end_step_ms": end_ms, "segment_work_ms": extra, "n_seg": cfg.n_seg,
               "amortised_ms_per_step": extra / cfg.n_seg, "timed_segment_ends": len(ends)}
    if dist:
        total_ms = max_over_ranks(total_ms, dev)
    qhp.qhp_set_profiling(h, False)

    units = N * P * args.steps * inner * ws
    value = units / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    steps_per_s = 1e3 / ms_per_step
    ns_day = steps_per_s * inner * cfg.dt_fs * 86400.0 / 1e6

    out = None
    if rank == 0:
        peaks, src = _peaks()
        clocks = clk.summary()
        smax = float(peaks.get("sm_max_mhz", 2032.0))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        fp64 = cfg.precision == "fp64"
        # FP32: 128 FMA lanes per SM; FP64 runs at 1/64 of that rate on this part
        lanes = 2 if fp64 else 128
        peak_tflops = n_sm * lanes * 2 * smax * 1e6 / 1e12
        flops_launch = FLOPS_PAIR * pairs + FLOPS_LJ * oo_pairs
        mean_pair_ms = float(np.mean(pair_ms))
        achieved = flops_launch / (mean_pair_ms * 1e-3) / 1e12
        traffic = _profile_traffic("pair", args.workload)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if fp64 else "f32/i64/f64 (mixed)", "data": "synthetic",
            "ns_per_day": ns_day,
            "config": _workload_conf(args.workload, cfg, ws),
            "launch": "direct kernel launches" if args.direct_launch else "one CUDA graph per step",
            "roofline": {"kernel": "nonbonded pair kernel", "bound": "alu", "achieved": achieved,
                         "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": traffic, "pairs_per_launch": pairs, "oo_pairs_per_launch": oo_pairs,
                         "flops_per_launch": flops_launch, "mean_launch_ms": mean_pair_ms,
                         "share_of_step": mean_pair_ms / ms_per_step,
                         "peak_source": f"{'FP64' if fp64 else 'FP32'} FMA: {n_sm} SMs x {lanes} lanes x 2 x "
                                        f"{smax:.0f} MHz ({src} clock)"},
            "clocks": clocks,
            "gpu_launches": int(launches),
            "stage_ms": dict(zip(["integrate_transform", "list_check_rebuild", "pair", "bonded", "project_kick"],
                                 [round(float(x), 5) for x in np.mean(np.array(stages), axis=0)])),
            "list_rebuilds": int(rebuilds), "list_entries": int(info1.list_entries),
        }
        if seg is not None:
            out["adqtb_segment"] = seg
    if args.e2e:
        e2e = _e2e(args, h, N, P, step, dev, ws, inner)
        if rank == 0:
            out["e2e"] = e2e
    if args.fp64 and rank == 0:
        out["fp64_gpu_path"] = _fp64_path(args, cfg, dev, flops_launch, n_sm, smax)
        out["speedup_vs_fp64_gpu_path"] = value / ws / out["fp64_gpu_path"]["value"]
    if rank == 0 and args.workload == "grad_216w":
        out["gradient"] = _time_gradient(qhp, h, cfg, N, P)
    if rank == 0 and getattr(args, "sampled_error", False):
        out["force_error_rms_rel_vs_oracle"] = _sampled_force_error(h, cfg)
        out["force_error_sample"] = "bead 0 of 40 sampled molecules, oracle brute-force sum for those atoms"
    sysobj.close()
    if rank == 0 and args.cpu_baseline:
        cb, err = _cpu_baseline(cfg, args)
        out["cpu_baseline"] = cb
        if err is not None:
            out["force_error_rms_rel_vs_oracle"] = err
    return out


def run_batch(args, ws, rank, local):
    """256 independent boxes (64-2,048 waters, P from {4..64}) stepped by the batched launches."""
    import torch
    from paper_2212_03137_b300 import build, qhp
    from paper_2212_03137_b300.workloads import batch_configs

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfgs = batch_configs(seed=1234 + 1000 * rank)
    systems = [qhp.System.from_config(c) for c in cfgs]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    b = qhp.Batch(systems)
    qhp.qhp_batch_set_stream(b.h, stream.cuda_stream)
    tuned = qhp.qhp_batch_autotune(b.h, 3)
    units_step = sum(s.n_atoms * s.P for s in systems)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        b.step(1)
    b.sync()
    pairs = oo = 0
    for s in systems:
        p_, o_ = qhp.qhp_count_pairs(s.h)
        pairs += p_
        oo += o_
    dist = ws > 1
    if dist:
        import torch.distributed as td
        td.barrier()
    torch.cuda.synchronize(dev)
    i0 = qhp.qhp_batch_get_info(b.h)
    step_ms, stages = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            b.step(1)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            pr = qhp.qhp_batch_get_profile(b.h)
            stages.append([pr.integrate_ms, pr.list_ms, pr.pair_ms, pr.bonded_ms, pr.project_ms])
    b.sync()
    i1 = qhp.qhp_batch_get_info(b.h)
    total_ms = float(np.sum(step_ms))
    if dist:
        total_ms = max_over_ranks(total_ms, dev)
    value = units_step * args.steps * ws / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    out = None
    if rank == 0:
        peaks, src = _peaks()
        smax = float(peaks.get("sm_max_mhz", 2032.0))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_tflops = n_sm * 128 * 2 * smax * 1e6 / 1e12
        st = np.mean(np.array(stages), axis=0)
        flops = FLOPS_PAIR * pairs + FLOPS_LJ * oo
        achieved = flops / (st[2] * 1e-3) / 1e12
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/i64/f64 (mixed)", "data": "synthetic",
            "ns_per_day": 1e3 / ms_per_step * 0.5 * 86400.0 / 1e6,
            "config": _batch_conf(cfgs, ws),
            "atom_beads_per_step": units_step,
            "tuned_warps_per_atom": {str(k): v for k, v in tuned.items()},
            "launch": "one CUDA graph per batched step",
            "roofline": {"kernel": "batched force kernel (pair and bonded items; FLOPs count the pairs)",
                         "bound": "alu", "achieved": achieved,
                         "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": _profile_traffic("pair", "batch_256"), "pairs_per_launch": pairs,
                         "oo_pairs_per_launch": oo, "flops_per_launch": flops, "mean_launch_ms": float(st[2]),
                         "share_of_step": float(st[2]) / ms_per_step,
                         "peak_source": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 x {smax:.0f} MHz ({src} clock)"},
            "clocks": clk.summary(),
            "gpu_launches": int(i1.kernel_launches - i0.kernel_launches),
            "stage_ms": dict(zip(["integrate_transform_check", "rebuild_bodies", "forces", "bonded (in forces)",
                                  "project_kick"], [round(float(x), 5) for x in st])),
            "list_rebuilds": int(i1.rebuilds - i0.rebuilds),
        }
    if args.e2e:
        # public API with host buffers: every box's momenta live on the host between steps
        # (uploaded from pinned memory, one batched step, read back) and every box's
        # centroids are read back as the result
        import torch as _t
        pins = [_t.from_numpy(qhp.qhp_get_modes(s.h)[1]).pin_memory() for s in systems]
        ptrs = [qhp.C.cast(p.data_ptr(), qhp._DP) for p in pins]
        cents = [np.empty((s.n_atoms, 3)) for s in systems]
        n = max(1, min(args.steps, 20))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(n):
            for s, ptr in zip(systems, ptrs):
                qhp.lib().qhp_set_modes(s.h, None, ptr)
            b.step(1)
            for s, ptr, c in zip(systems, ptrs, cents):
                qhp.lib().qhp_get_modes(s.h, None, ptr)
                qhp.lib().qhp_get_centroid(s.h, c.ctypes.data_as(qhp._DP))
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        if rank == 0:
            out["e2e"] = {"value": units_step * n * ws / dt, "unit": UNIT,
                          "h2d_bytes_per_step": int(sum(p.numel() * 8 for p in pins)),
                          "d2h_bytes_per_step": int(sum(p.numel() * 8 for p in pins) + sum(c.nbytes for c in cents))}
    if rank == 0 and getattr(args, "sampled_error", False):
        # three boxes of different bead counts, bead 0 of 40 sampled molecules each
        picks = [min(range(len(cfgs)), key=lambda k: (cfgs[k].P != P, cfgs[k].n_mol)) for P in (4, 16, 64)]
        errs = [_sampled_force_error(systems[k].h, cfgs[k]) for k in picks]
        out["force_error_rms_rel_vs_oracle"] = max(errs)
        out["force_error_sample"] = f"boxes {picks} (P = 4, 16, 64), bead 0 of 40 sampled molecules each; worst"
    if rank == 0 and args.fp64:
        out["fp64_gpu_path"] = _batch_fp64_sample(cfgs, dev)
        out["speedup_vs_fp64_gpu_path"] = value / ws / out["fp64_gpu_path"]["value"]
    b.close()
    for s in systems:
        s.close()
    if rank == 0 and args.cpu_baseline:
        rng = np.random.default_rng(7)
        picks = sorted(rng.choice(len(cfgs), 8, replace=False))
        t_tot = u_tot = 0.0
        for k in picks:
            t, u, *_ = _oracle_sample(cfgs[k], min(2, cfgs[k].P))
            t_tot += t
            u_tot += u
        out["cpu_baseline"] = {"value": u_tot / t_tot, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"FP64 oracle on 8 of the 256 boxes (indices {list(map(int, picks))}): "
                                         "forces of 2 beads each + one BAOAB update, numpy, 1 thread"}
    return out


def _batch_fp64_sample(cfgs, dev, n=12, steps=3):
    """The batch's boxes on the plain FP64 GPU path, one system at a time: n boxes spread over
    the size and bead-count range, each timed over a few steps; the rate is their atom-bead
    steps over their summed time (the FP64 path has no batched launch)."""
    import torch
    from paper_2212_03137_b300 import qhp
    order = sorted(range(len(cfgs)), key=lambda k: cfgs[k].n_mol * cfgs[k].P)
    picks = [order[int(round(i * (len(order) - 1) / (n - 1)))] for i in range(n)]
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    units = ms = 0.0
    for k in picks:
        s = qhp.System.from_config(cfgs[k], precision="fp64")
        qhp.qhp_set_stream(s.h, stream.cuda_stream)
        qhp.qhp_step_rpmd(s.h, 1)
        qhp.qhp_sync(s.h)
        e0.record(stream)
        qhp.qhp_step_rpmd(s.h, steps)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        units += s.n_atoms * s.P * steps
        s.close()
    return {"value": units / (ms * 1e-3), "unit": UNIT, "ms_sampled": ms,
            "sample": f"{n} of the {len(cfgs)} boxes (indices {picks}), {steps} steps each, one system at a time"}


def _time_gradient(qhp, h, cfg, N, P, block=15, reps=3):
    """Wall time of the differentiable segment: J = (1/K) sum_k V(Q_0,k) over K = cfg.steps
    BAOAB steps with the noise held fixed, and dJ/dtheta by the checkpointed adjoint (forward
    segment, replays from checkpoints every `block` steps, backward sweep).  The call is
    synchronous, so host wall time brackets the device work."""
    import time
    K = int(cfg.steps)
    qhp.qhp_segment_grad(h, K, block, 0)   # warm-up
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        J, g = qhp.qhp_segment_grad(h, K, block, 0)
        ts.append(time.perf_counter() - t0)
    t = float(np.median(ts))
    return {"K": K, "checkpoint_block": block, "observable": "centroid potential energy V(Q_0)",
            "parameters": ["eps", "sigma", "q_O", "k_b", "k_theta"], "s_per_gradient": t,
            "atom_bead_steps_per_s": N * P * K / t, "J": J, "dJ_dtheta": [float(x) for x in g]}


def _e2e(args, h, N, P, step, dev, ws, inner=1):
    """Public API with host buffers: the state's momenta live on the host between steps.  Per
    step: upload them (pinned), step, read the new momenta back and the centroids (the
    result).  The round trip keeps the dynamics exact (positions stay on the device)."""
    import torch
    from paper_2212_03137_b300 import qhp
    Q, Pm = qhp.qhp_get_modes(h)
    pin = torch.from_numpy(Pm).pin_memory()
    cent = np.empty((N, 3))
    ptr = qhp.C.cast(pin.data_ptr(), qhp._DP)
    n = max(1, args.steps)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(n):
        qhp.lib().qhp_set_modes(h, None, ptr)
        step(h, 1)
        qhp.lib().qhp_get_modes(h, None, ptr)
        qhp.lib().qhp_get_centroid(h, cent.ctypes.data_as(qhp._DP))
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    return {"value": N * P * n * inner * ws / dt, "unit": UNIT, "h2d_bytes_per_step": int(Pm.nbytes),
            "d2h_bytes_per_step": int(Pm.nbytes + cent.nbytes)}


def _fp64_path(args, cfg, dev, flops=None, n_sm=None, smax=None):
    """The same workload on the plain FP64 GPU path (FP64 pair math, FP64 forces), with the FP64
    pair kernel's own fraction of the FP64 peak (the same algorithmic flops per launch)."""
    import torch
    from paper_2212_03137_b300 import qhp
    s = qhp.System.from_config(cfg, precision="fp64")
    stream = torch.cuda.current_stream(dev)
    assert stream.cuda_stream != 0, "timing needs an explicit stream"
    qhp.qhp_set_stream(s.h, stream.cuda_stream)
    qhp.qhp_set_profiling(s.h, True)
    step = qhp.qhp_step_adqtb if cfg.thermostat == "adqtb" else qhp.qhp_step_rpmd
    step(s.h, 1)
    qhp.qhp_sync(s.h)
    k = max(2, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot, pair = 0.0, []
    for _ in range(k):
        e0.record(stream)
        step(s.h, 1)
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        pair.append(qhp.qhp_get_profile(s.h).pair_ms)
    s.close()
    out = {"value": s.n_atoms * s.P * k / (tot * 1e-3), "unit": UNIT, "ms_per_step": tot / k, "steps": k}
    if flops and n_sm and smax and min(pair) > 0:
        peak = n_sm * 2 * 2 * smax * 1e6 / 1e12   # FP64: 2 FMA lanes per SM on this part
        achieved = flops / (float(np.mean(pair)) * 1e-3) / 1e12
        out["pair_roofline"] = {"kernel": "FP64 pair kernel", "bound": "alu", "achieved": achieved, "peak": peak,
                                "unit": "TFLOP/s", "frac": achieved / peak, "mean_launch_ms": float(np.mean(pair)),
                                "peak_source": f"FP64 FMA: {n_sm} SMs x 2 lanes x 2 x {smax:.0f} MHz"}
    return out


def _oracle_sample(cfg, n_beads):
    """Time the FP64 oracle (as it stands) on a bounded sample of one step: the forces of
    n_beads of the P beads (oracle cell-list pair sum) plus one full BAOAB update of every mode.
    Returns (seconds, atom-bead units covered, sampled bead positions, their oracle forces)."""
    import math as _m
    from oracle import rpmd as orp
    from oracle import water as ow
    from paper_2212_03137_b300.workloads import WATER_FF as W
    box = cfg.system()
    ff = ow.ForceField(eps=W["eps"], sigma=W["sigma"], q_O=W["q_O"], k_b=W["k_b"], r0=W["r0"],
                       k_theta=W["k_theta"], theta0=_m.radians(W["theta0_deg"]), alpha=W["alpha"], rc=cfg.rc,
                       m_O=W["m_O"], m_H=W["m_H"])
    prm = orp.Params(P=cfg.P, temperature=cfg.temperature, dt=cfg.dt_fs * 1e-3, gamma0=cfg.gamma0, seed=cfg.seed)
    m = ff.masses(box.types)
    st = orp.init_state(box.pos, m, prm)
    fn = ow.make_force_fn(box.types, box.molecule, box.box, ff, cells=True)
    xb = orp.beads(st, cfg.P)[:n_beads]
    t0 = time.perf_counter()
    _, F = fn(xb)
    t_force = time.perf_counter() - t0
    st.f = np.zeros_like(st.Q)
    t0 = time.perf_counter()
    orp.kick(st, 0.5 * prm.dt)
    orp.free_flow(st, prm, m, 0.5 * prm.dt)
    orp.ou(st, prm, m, prm.dt)
    orp.free_flow(st, prm, m, 0.5 * prm.dt)
    orp.kick(st, 0.5 * prm.dt)
    t_int = time.perf_counter() - t0
    return t_force + t_int * n_beads / cfg.P, box.n_atoms * n_beads, xb, F, t_force, t_int


def _cpu_baseline(cfg, args, n_beads=2):
    """cpu_baseline leg: the oracle timed on the host cores, and the GPU force error on the
    same sampled beads at the same initial state."""
    from paper_2212_03137_b300 import qhp
    n_beads = min(n_beads, cfg.P)
    t, units, xb, F, t_force, t_int = _oracle_sample(cfg, n_beads)
    err = None
    s = qhp.System.from_config(cfg)
    try:
        qhp.qhp_compute_forces(s.h)
        Fg = qhp.qhp_get_forces(s.h)[:n_beads]
        xg = qhp.qhp_get_beads(s.h)[:n_beads]
        if np.abs(xg - xb).max() < 1e-9:
            err = float(np.sqrt(np.sum((Fg - F) ** 2) / np.sum(F ** 2)))
    finally:
        s.close()
    return ({"value": units / t, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host(),
             "sample": f"FP64 oracle as it stands (numpy, 1 thread): forces of {n_beads} of {cfg.P} beads "
                       f"({t_force:.1f} s) + one BAOAB update of all modes ({t_int:.2f} s); the rate is "
                       f"extrapolated to a full step by counting {n_beads}/{cfg.P} of its atom-beads"}, err)


def run_reference(args, ws, rank, local):
    """Reference arm: the FP64 CPU oracle; each timed step is a one-bead sample of the workload."""
    if rank != 0:
        return None
    k = max(1, args.steps)
    t_tot, units = 0.0, 0
    if args.workload == "batch_256":
        from paper_2212_03137_b300.workloads import batch_configs
        cfgs = batch_configs()
        picks = [int(x) for x in np.random.default_rng(7).choice(len(cfgs), 8, replace=False)]
        for it in range(k):
            t, u, *_ = _oracle_sample(cfgs[picks[it % 8]], 1)
            t_tot += t
            units += u
        cfg = cfgs[picks[0]]
        sample = f"FP64 oracle: one box per step from 8 of the 256 boxes {picks}, forces of 1 bead + one BAOAB update"
        conf = _batch_conf(cfgs, ws)
    else:
        cfg = _config(args.workload)
        for _ in range(k):
            t, u, *_ = _oracle_sample(cfg, 1)
            t_tot += t
            units += u
        sample = f"FP64 oracle: forces of 1 of {cfg.P} beads + one BAOAB update of all modes scaled by 1/{cfg.P}"
        conf = _workload_conf(args.workload, cfg, ws)
    value = units / t_tot
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": k, "warmup": args.warmup,
            "ms_per_step": t_tot / k * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": conf,
            "method": "the FP64 CPU oracle on the host (one process, numpy on one thread); the GPU arm's L2 "
                      "flush and launch mode do not apply",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host(),
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _profile_traffic(kind, workload):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None when there is
    no capture for this workload or the kernel source has changed since it was taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "pair_traffic.txt")
    src = os.path.join(ROOT, "paper_2212_03137_b300", "csrc", "forces.cu")
    if not os.path.exists(p):
        return None
    with open(src, "rb") as fh:
        sha = hashlib.sha256(fh.read()).hexdigest()
    with open(p) as fh:
        for line in fh:
            f = line.split()
            if len(f) == 4 and not f[0].startswith("#") and f[0] == workload and f[1] == kind and f[3] == sha:
                return float(f[2])
    return None


DEFAULT_WORKLOAD = "rpmd_mixed_4096w"
OTHER_WORKLOADS = ("adqtb_mixed_72000w", "batch_256", "grad_216w")


def _other_workloads(args, ws, rank, local):
    """The 72,000-water adQTB box, the 256-box batch and the 216-water gradient workload, each
    timed like the default one (its own K steps after W warm-up steps, L2 flushed between
    steps) with its dominant kernel's roofline, the plain FP64 GPU path where it is a
    different path, and a force error against the oracle on sampled atoms."""
    import copy
    keep = ("value", "unit", "ms_per_step", "ns_per_day", "dtype", "config", "launch", "roofline", "clocks",
            "gpu_launches", "stage_ms", "list_rebuilds", "adqtb_segment", "gradient", "fp64_gpu_path",
            "speedup_vs_fp64_gpu_path", "force_error_rms_rel_vs_oracle", "force_error_sample",
            "atom_beads_per_step", "tuned_warps_per_atom")
    res = {}
    for name in OTHER_WORKLOADS:
        sub = copy.copy(args)
        sub.workload = name
        sub.e2e = False
        sub.cpu_baseline = False
        sub.fp64 = name != "grad_216w"        # that workload is itself the FP64 path
        sub.sampled_error = True
        r = run_batch(sub, ws, rank, local) if name == "batch_256" else run_ours(sub, ws, rank, local)
        if rank == 0:
            res[name] = {k: v for k, v in r.items() if k in keep}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    # the default run also times the other configurations (at N = 1) under "workloads"
    ap.add_argument("--only-default", dest="all_workloads", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    # kernel-by-kernel launches instead of step graphs, for profiler launch lists
    ap.add_argument("--direct-launch", action="store_true")
    ap.add_argument("--skin", type=float, default=None, help="neighbour-list skin in A (default: the workload's)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    global SKIN
    SKIN = args.skin
    ws, rank, local = _dist()
    if ws > 1:
        import torch
        import torch.distributed as td
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        td.init_process_group(backend=backend)
    if args.impl == "reference":
        out = run_reference(args, ws, rank, local)
    elif args.workload == "batch_256":
        out = run_batch(args, ws, rank, local)
    else:
        out = run_ours(args, ws, rank, local)
        if args.workload == DEFAULT_WORKLOAD and args.all_workloads and ws == 1:
            out["workloads"] = _other_workloads(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
