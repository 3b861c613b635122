"""Throughput benchmark of the CSPH-TVD + Exner step on GB300.

Workload: half-wet fractal terrain, 16384 x 16384 cells (268M), dx = 5 m,
20 m relief with a carved channel, 50 % wet with a 2 m dam-break step so
fronts move, Manning n per 64 x 64 block, FP32 state with FP64 dt / mass
bookkeeping; K timed steps.  Metric: Gcell-updates/s, counting every cell of
the grid each step (HGS-skipped dry blocks included).

One JSON line on rank 0:
  value       device-timed (CUDA events on the solver's stream), inputs resident
  e2e         the same through the C ABI with host buffers: H2D of the state,
              K steps, D2H of the state, all inside the timed region
  roofline    the fused step kernel against the measured HBM copy bandwidth;
              algorithmic bytes = 32 B x cells of the computed and copied blocks
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload
With --impl reference, the oracle arm alone.  With --gpus N under torchrun,
N independent replicas (the method is single-GPU): value = all cells / max time.
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

METRIC = "Gcell-updates/s per CSPH-TVD+Exner step"
UNIT = "Gcell/s"
BYTES_PER_CELL = 32  # FP32 AoS {H, Hu, Hv, b}: 16 B read + 16 B write


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _max_over_ranks(x, world):
    """The largest value of x over all ranks (x itself on one rank); NCCL
    reduces device tensors, gloo host tensors."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _aggregate_rate(cells_per_step, steps, seconds, world):
    """Whole-job Gcell/s: the cell updates of all ranks over the slowest
    rank's time (each rank runs the same workload: weak scaling)."""
    return float(cells_per_step) * steps * world / seconds / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("swe_kernels.cuh", "swe_launch.cuh", "swe_internal.h"):
        with open(os.path.join(ROOT, "paper_2103_15196_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_kv():
    """Key: value lines of the committed ncu summary of the step kernel, or {}
    if absent or taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", "step_kernel_fp32_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        return kv if kv.get("kernel_source_hash") == _kernel_hash() else {}
    except Exception:
        return {}


def _profile_traffic(n):
    """DRAM bytes per launch of the step kernel (ncu), scaled to this grid."""
    kv = _profile_kv()
    return float(kv["dram_bytes_per_cell"]) * n * n if "dram_bytes_per_cell" in kv else None


# GB300 instruction issue: 152 SMs x 4 schedulers x 1 warp-instruction per clock
ISSUE_WARPS_PER_CLOCK = 152 * 4


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes): SM
    clock, its maximum, power draw and the active clock-event reasons."""
    SM = 1                                   # NVML_CLOCK_SM
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, pci_bus_id):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle for " + pci_bus_id)
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        ct = self.ct
        sm, mx, mw, r = ct.c_uint(0), ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, ct.byref(sm))
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ct.byref(mx))
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
        self.reasons_fn(self.h, ct.byref(r))
        names = [v for k, v in self.BITS.items() if r.value & k]
        return float(sm.value), float(mx.value), mw.value / 1000.0, names


class Clocks:
    """Samples the SM clock, power and clock-event reasons every 100 ms on a
    host thread (NVML, read only; nvidia-smi as a fallback), started before
    the warm-up.  summary() keeps the samples taken between start() and
    stop(), i.e. during the timed region."""

    def __init__(self, index):
        self.index = str(index)
        self.pci = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(index)
            self.pci = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            self.index = self.pci
        except Exception:
            pass
        self.samples = []           # (host time, sm_mhz, max_mhz, watts, [reasons])
        self.proc = None
        self.nvml = None
        self.source = None
        self.t0 = None
        self.t1 = None
        self._halt = threading.Event()

    def wait_first(self, timeout=20.0):
        """Blocks until the sampler has delivered a sample (or timeout s)."""
        t = time.time()
        while (self.proc or self.nvml) and not self.samples and time.time() - t < timeout:
            time.sleep(0.05)

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __enter__(self):
        try:
            self.nvml = _Nvml(self.pci) if self.pci else None
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.source = "nvml"
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _poll(self):
        while not self._halt.is_set():
            try:
                self.samples.append((time.time(),) + self.nvml.sample())
            except Exception:
                return
            self._halt.wait(0.1)

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            s = [p.strip() for p in line.split(",")]
            if len(s) >= 7 and s[0].replace(".", "").isdigit():
                try:
                    self.samples.append((time.time(), float(s[0]), float(s[1]), float(s[2]),
                                         [names[i] for i in range(4) if s[3 + i].lower() == "active"]))
                except ValueError:
                    pass

    def __exit__(self, *a):
        self._halt.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        t0 = self.t0 if self.t0 is not None else -float("inf")
        t1 = self.t1 if self.t1 is not None else float("inf")
        samples = [x for x in self.samples if t0 <= x[0] <= t1]
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        sm = [x[1] for x in samples]
        reasons = sorted({r for x in samples for r in x[4]})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(x[2] for x in samples),
                "power_w_max": max(x[3] for x in samples), "reasons": reasons, "samples": len(samples),
                "source": self.source}


def _issue_object(gcell_s, clocks):
    """What bounds the step kernel: warp-instructions per cell (ncu, same
    kernel source, the benchmark's block shape) times the measured cell rate,
    against the issue peak at the sampled SM clock (one warp-instruction per
    scheduler per clock); the thread-instructions beside it."""
    kv = _profile_kv()
    if "warp_inst_per_cell" not in kv:
        return None
    wpc = float(kv["warp_inst_per_cell"])
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = ISSUE_WARPS_PER_CLOCK * mhz * 1e6 / 1e12
    ach = gcell_s * 1e9 * wpc / 1e12
    return {"bound": "instruction issue", "warp_inst_per_cell": wpc,
            "thread_inst_per_cell": float(kv.get("thread_inst_per_cell", "nan")), "achieved": ach, "peak": peak,
            "unit": "T warp-instructions/s", "frac": ach / peak}


def _step_launches(n, K):
    """Kernel launches of run_steps(K): graphs of m steps (m by grid size, as
    the library chooses it), each a compaction then, per step, the step kernel
    and the commit-and-list kernel; the remaining steps one by one (three
    launches each)."""
    m = 8 if n * n >= (1 << 24) else (32 if n * n >= (1 << 20) else 128)
    return (K // m) * (1 + 2 * m) + (K % m) * 3


def make_workload(n, seed=3, wet_fraction=0.5):
    from paper_2103_15196_gb300 import inputs as I
    return I.half_wet(n, dx=5.0, seed=seed, wet_fraction=wet_fraction)


def cpu_baseline(sc, budget_s=12.0, win=1024):
    """The FP64 oracle as it stands, on windows of the workload's first state,
    all host cores: cell-updates/s (dt from the window's own Eq. 7 terms)."""
    from oracle import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    n = sc.nx
    w = min(win, n)
    y0 = x0 = (n - w) // 2
    sl = (slice(y0, y0 + w), slice(x0, x0 + w))
    H = np.ascontiguousarray(sc.H[sl], dtype=np.float64)
    b = np.ascontiguousarray(sc.b[sl], dtype=np.float64)
    Z = np.zeros_like(H)
    ncell = np.ascontiguousarray(sc.manning_per_cell()[sl], dtype=np.float64)
    p = O.Params(nx=w, ny=w, dx=sc.dx, tile_x=64, tile_y=64)
    st = O.State(H, Z, Z.copy(), b)
    cells, t0 = 0, time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        st, info = O.step(p, st, ncell)
        cells += w * w
        steps += 1
    el = time.perf_counter() - t0
    # the same oracle on one core (a 256^2 window, a few seconds), beside it
    O.set_threads(1)
    w1 = min(256, n)
    s1 = (slice((n - w1) // 2, (n - w1) // 2 + w1),) * 2
    st1 = O.State(np.ascontiguousarray(sc.H[s1], dtype=np.float64), np.zeros((w1, w1)), np.zeros((w1, w1)),
                  np.ascontiguousarray(sc.b[s1], dtype=np.float64))
    p1 = O.Params(nx=w1, ny=w1, dx=sc.dx, tile_x=64, tile_y=64)
    n1 = np.ascontiguousarray(sc.manning_per_cell()[s1], dtype=np.float64)
    c1, t1, k1 = 0, time.perf_counter(), 0
    while time.perf_counter() - t1 < budget_s / 4 or k1 == 0:
        st1, _ = O.step(p1, st1, n1)
        c1 += w1 * w1
        k1 += 1
    e1 = time.perf_counter() - t1
    O.set_threads(cores)
    return {"value": cells / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps (K1-K8, HGS on) of the central {w}x{w} window "
                      f"of the {n}^2 workload, {el:.1f} s",
            "single_core": {"value": c1 / e1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"{k1} steps of the central {w1}x{w1} window, {e1:.1f} s"}}


def run_reference(args):
    """The FP64 CPU oracle on the host cores: K steps of a central window of
    the workload, the window sized so the K + W steps take ~ref_seconds."""
    from oracle import oracle as O
    rank, world, _ = _dist()
    if rank != 0:
        return
    n = args.size
    sc = make_workload(n)
    cores = O.set_threads(os.cpu_count() or 1)

    def window(w):
        y0 = (n - w) // 2
        sl = (slice(y0, y0 + w), slice(y0, y0 + w))
        H = np.ascontiguousarray(sc.H[sl], dtype=np.float64)
        Z = np.zeros_like(H)
        st = O.State(H, Z, Z.copy(), np.ascontiguousarray(sc.b[sl], dtype=np.float64))
        ncell = np.ascontiguousarray(sc.manning_per_cell()[sl], dtype=np.float64)
        return O.Params(nx=w, ny=w, dx=sc.dx, tile_x=64, tile_y=64), st, ncell

    p, st, ncell = window(256)
    t0 = time.perf_counter()
    O.step(p, st, ncell)
    per_cell = (time.perf_counter() - t0) / (256 * 256)
    per_step = args.ref_seconds / max(1, args.steps + args.warmup)
    w = int(min(min(n, 2048), max(64, (per_step / per_cell) ** 0.5)))
    p, st, ncell = window(w)
    for _ in range(args.warmup):
        st, _ = O.step(p, st, ncell)
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        st, _ = O.step(p, st, ncell)
    el = time.perf_counter() - t0
    v = float(w) * w * max(1, args.steps) / el / 1e9
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"{args.steps} FP64 oracle steps (K1-K8, HGS on) of the central {w}x{w} window of the "
                    f"{n}^2 workload, {el:.1f} s"}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"half-wet fractal terrain {n}x{n}, dx=5 m, Manning per 64^2 block; "
                                   f"oracle on its central {w}x{w} window", "grid": n},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(args, torch, swe):
    """The batched ensemble: 64 flood scenarios, sides 32*U{8..64} (256..2048), per-scenario
    terrain seed, Manning n ~ U[0.02, 0.06], inflow peak ~ U[50, 1000] m^3/s,
    d50 scale ~ U[0.5, 2]; one persistent launch per run, autotuned blocks.
    Returns aggregate Gcell/s and the same scenarios run one after another."""
    from paper_2103_15196_gb300 import inputs as I
    specs = I.ensemble_specs(args.ens_n, seed=4)
    scs = [I.ensemble_scenario(sp["side"], sp["seed"], sp["manning"], sp["peak"], sp["d50_scale"]) for sp in specs]
    cells_per_step = float(sum(sc.nx * sc.ny for sc in scs))
    stream = torch.cuda.Stream()
    E = swe.Ensemble([dict(nx=sc.nx, ny=sc.ny, dx=sc.dx, d50=sc.d50) for sc in scs], stream=stream.cuda_stream)

    def load(m, sc):
        m.set_manning(sc.manning, block=sc.manning_block)
        m.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
        m.set_state(sc.H.astype(np.float32), sc.Hu.astype(np.float32), sc.Hv.astype(np.float32),
                    sc.b.astype(np.float32))

    for m, sc in zip(E.members, scs):
        load(m, sc)
    bw, th = E.autotune(5)
    K = args.ens_steps
    E.run(3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    E.run(K)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    E.close()
    # the same scenarios, one solver after another (each its own graphs)
    seq_ms = 0.0
    for sc in scs:
        S = swe.Solver(sc.nx, sc.ny, sc.dx, precision="fp32", stream=stream.cuda_stream, d50=sc.d50)
        load(S, sc)
        S.run_steps(3)
        S.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.run_steps(K)
        b.record(stream)
        b.synchronize()
        seq_ms += a.elapsed_time(b)
        S.close()
    return {"metric": "aggregate Gcell-updates/s, 64-scenario ensemble", "value": cells_per_step * K / (ms * 1e-3) / 1e9,
            "unit": UNIT, "scenarios": len(scs), "cells_per_step": int(cells_per_step), "steps": K,
            "ms_per_step": ms / K, "launches_per_run": 1, "block": [bw - 8, th],
            "sequential_value": cells_per_step * K / (seq_ms * 1e-3) / 1e9,
            "speedup_vs_sequential": seq_ms / ms,
            "config": "sides 32*U{8..64}, half-wet fractal terrain + channel + inflow hydrograph, "
                      "n~U[0.02,0.06], peak~U[50,1000], d50 scale~U[0.5,2], FP32, seed 4"}


def run_hgs_flood(args, torch, swe):
    """The dry-block skip (K1, Sec. 3) on the kind of scene it is for: the
    flood-channel terrain at the benchmark's size, initially dry, water
    entering through the channel head (inflow hydrograph peaking at
    500 m^3/s).  The same steps with the skip on and off (off: on the same
    blocks, on the library's default blocks for the grid and on 248-column
    blocks of the default height, the speed-up taken against the fastest);
    rates count every cell of the grid per step."""
    from paper_2103_15196_gb300 import inputs as I
    n, K, W = args.size, args.hgs_steps, 5
    sc = I.flood_channel(n, dx=5.0, seed=2, peak=500.0)
    stream = torch.cuda.Stream()
    out = {}
    bc = args.hgs_block_cols
    for name, skip, rows, cols in (("on", 1, args.hgs_tile_rows, bc), ("off", 0, args.hgs_tile_rows, bc),
                                   ("off_default_blocks", 0, 0, 0), ("off_256_columns", 0, 0, 256)):
        S = swe.Solver(n, n, 5.0, precision="fp32", stream=stream.cuda_stream, hgs_skip=skip,
                       tile_rows=rows, block_cols=cols)
        S.set_manning(sc.manning, block=sc.manning_block)
        S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
        S.set_state(*(np.asarray(a, dtype=np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b)))
        S.run_steps(W)
        S.sync()
        d0 = S.diag()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.run_steps(K)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        d1 = S.diag()
        out[name] = {"value": _aggregate_rate(float(n) * n, K, ms * 1e-3, 1), "ms_per_step": ms / K,
                     "active_cell_fraction": (d1["cells_computed"] - d0["cells_computed"]) / (float(n) * n * K),
                     "wet_cells_end": d1["wet_cells"], "t_end": d1["t"]}
        S.close()
    off = max(out["off"]["value"], out["off_default_blocks"]["value"], out["off_256_columns"]["value"])
    return {"workload": f"flood channel {n}x{n}, initially dry, inflow on the channel head, steps {W}..{W + K}",
            "tile_rows": args.hgs_tile_rows, "block_cols": bc,
            "unit": UNIT, "skip_on": out["on"], "skip_off": out["off"],
            "skip_off_default_blocks": out["off_default_blocks"], "skip_off_256_columns": out["off_256_columns"],
            "speedup": out["on"]["value"] / off}


def run_surrogate(args, torch, swe):
    """The learned bed surrogate.  2000 samples (500 snapshots x 4
    tiles of 1024^2) of (state, bed change over K = 50 steps) from solver runs
    on the 2048^2 flood-channel terrain class (fractal DEM + carved channel,
    half wet with a dam-break step, inflow hydrograph), training on the GPU,
    then an unseen scenario run with surrogate windows (water advanced K/f
    steps, bed by the network; every judge_every-th window run by the plain
    solver and judged) against the plain coupled method."""
    from paper_2103_15196_gb300 import inputs as I
    K, T, n, f, J = 50, 1024, 2048, args.sur_f, args.sur_judge
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    def scenario(seed):
        return I.ensemble_scenario(n, seed=seed, manning=0.035, peak=500.0, d50_scale=1.0)

    def solver(sc):
        S = swe.Solver(n, n, 5.0, precision="fp32", stream=sp)
        S.set_manning(sc.manning, block=sc.manning_block)
        S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
        S.set_state(*(a.astype(np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b)))
        return S

    t_all = time.perf_counter()
    sv = solver(scenario(7000))
    sv.run_steps(args.sur_spin)
    H, Hu, Hv, b0 = sv.get_state(np.float32)
    sv.run_steps(K)
    b1 = sv.get_state(np.float32)[3]
    db = (b1 - b0).astype(np.float64)
    wet = H > 1e-4
    sp_ = np.sqrt((np.where(wet, Hu / np.maximum(H, 1e-4), 0) ** 2 + np.where(wet, Hv / np.maximum(H, 1e-4), 0) ** 2))
    vs = float(np.sqrt(np.mean(sp_[wet] ** 2))) + 1e-6 if wet.any() else 1.0
    norm = [float(H.mean()), float(H.std()) + 1e-6, float(b0.mean()), float(b0.std()) + 1e-6,
            vs, vs ** 3, float(db.std()) + 1e-9, (float(db.std()) + 1e-9) / K]
    sv.close()
    net = swe.Surrogate(tile=T, max_batch=4, seed=0, stream=sp)
    net.set_norm(norm)
    net.set_loss(args.sur_loss)
    nsnap = args.sur_samples // 4
    X = torch.empty((nsnap * 4, T, T, 8), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((nsnap * 4, T, T), dtype=torch.float32, device="cuda")
    nscen = max(1, nsnap // args.sur_snaps_per_run)

    def sample_run(seed, Xs, Ys, count, k0):
        """count windows of one scenario, a skipped window between samples:
        its start bed, two coupled steps (the bed saved between them; the
        network's input state), then the rest of the K coupled steps (the
        target)."""
        sv = solver(scenario(seed))
        sv.run_steps(args.sur_spin)
        for j in range(count):
            net.save_bed(sv)
            sv.run_steps(1)
            net.save_mid(sv)
            sv.run_steps(1)
            net.pack_state(sv, Xs[4 * (k0 + j):4 * (k0 + j) + 4])
            sv.run_steps(K - 2)
            net.pack_target(sv, Ys[4 * (k0 + j):4 * (k0 + j) + 4])
            sv.run_steps(K * args.sur_gap)
        sv.close()

    k = 0
    for r in range(nscen):
        cnt = nsnap // nscen if r < nscen - 1 else nsnap - k
        sample_run(7100 + r, X, Y, cnt, k)
        k += cnt
    nval = args.sur_val // 4
    Xv = torch.empty((nval * 4, T, T, 8), dtype=torch.bfloat16, device="cuda")
    Yv = torch.empty((nval * 4, T, T), dtype=torch.float32, device="cuda")
    sample_run(7500, Xv, Yv, nval, 0)
    ov = torch.empty((4, T, T), dtype=torch.float32, device="cuda")

    def validate():
        """Relative L1 on held-out windows (output units) of the network, of
        the linear extrapolation of the two coupled steps (channel 6, the
        network's base) and of the first step alone (channel 6 - channel 5),
        both masked as the network's output is."""
        e_net = e_lin = e_lin1 = ref = outside = 0.0
        for j in range(nval):
            net.forward(Xv[4 * j:4 * j + 4], ov, 4)
            torch.cuda.synchronize()
            o = ov.cpu().numpy().astype(np.float64)
            y = Yv[4 * j:4 * j + 4].cpu().numpy().astype(np.float64)
            xs = Xv[4 * j:4 * j + 4, :, :, 5:8].float().cpu().numpy().astype(np.float64)
            e_net += np.abs(o - y).sum()
            e_lin += np.abs(xs[..., 1] * xs[..., 2] - y).sum()
            e_lin1 += np.abs((xs[..., 1] - xs[..., 0]) * xs[..., 2] - y).sum()
            outside += np.abs(y * (xs[..., 2] == 0)).sum()
            ref += np.abs(y).sum()
        validate.outside = outside / ref
        return e_net / ref, e_lin / ref, e_lin1 / ref

    t_data = time.perf_counter() - t_all
    # training
    t0 = time.perf_counter()
    g = torch.Generator().manual_seed(0)
    steps, losses = 0, []
    lr0 = args.sur_lr
    val_curve = []
    v_net, v_lin, v_lin1 = validate()
    best = (v_net, [net.params(i) for i in range(6)])
    val_curve.append((0, v_net))
    # a fixed number of steps with a step-based schedule (a linear decay to a
    # tenth): the training kernels are deterministic, so is the trained network
    total = args.sur_train_steps
    every = max(1, total // args.sur_val_points)
    while steps < total:
        for i in torch.randperm(nsnap, generator=g).tolist():
            loss = net.train_step(X[4 * i:4 * i + 4], Y[4 * i:4 * i + 4], 4, lr0 * (0.1 + 0.9 * (1 - steps / total)))
            losses.append(loss)
            steps += 1
            if steps % every == 0 and steps < total:
                vn, _, _ = validate()
                val_curve.append((steps, vn))
                if vn < best[0]:
                    best = (vn, [net.params(j) for j in range(6)])
            if steps == total:
                break
    vn, _, _ = validate()
    val_curve.append((steps, vn))
    if vn < best[0]:
        best = (vn, [net.params(j) for j in range(6)])
    for j, (Wm, b_) in enumerate(best[1]):
        net.set_params(j, Wm, b_)
    t_train = time.perf_counter() - t0
    # forward time of one 2048^2 domain (4 tiles)
    outb = torch.empty((4, T, T), dtype=torch.float32, device="cuda")
    net.forward(X[0:4], outb, 4)
    fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fa.record(stream)
    for _ in range(5):
        net.forward(X[0:4], outb, 4)
    fb.record(stream)
    fb.synchronize()
    fwd_ms = fa.elapsed_time(fb) / 5
    del X, Y, outb, Xv, Yv, ov
    torch.cuda.empty_cache()
    # evaluation on an unseen scenario: plain coupled method vs surrogate windows
    sc = scenario(7999)
    R = args.sur_windows
    A = solver(sc)
    A.run_steps(args.sur_spin)
    A.sync()
    ta = A.t
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    A.run_steps(K * R)
    e1.record(stream)
    e1.synchronize()
    wall_p = e0.elapsed_time(e1) * 1e-3
    bed_p = A.t - ta
    A.close()
    rate_p = bed_p / wall_p

    def surrogate_run(f_, J_):
        Bs = solver(sc)
        Bs.run_steps(args.sur_spin)
        Bs.sync()
        w0 = time.perf_counter()
        st_ = net.run(Bs, R, K=K, f=f_, judge_every=J_, bound=args.sur_bound)
        wall = time.perf_counter() - w0
        Bs.close()
        return st_, wall

    st, wall_s = surrogate_run(f, J)
    rate_s = st.bed_time / wall_s
    variants = []
    for v in filter(None, args.sur_variants.split(",")):
        fv, jv = (int(x) for x in v.split(":"))
        sv_, wv = surrogate_run(fv, jv)
        variants.append({"f": fv, "judge_every": jv, "speedup": sv_.bed_time / wv / rate_p,
                         "err_mean": sv_.err_mean, "err_max": sv_.err_max, "err_linear_mean": sv_.err_linear_mean,
                         "elev_err_max": sv_.elev_err_max, "mode": sv_.mode})
    net.close()
    out = {"metric": "surrogate bed simulated-time rate / plain method's, at judged error",
           "speedup": rate_s / rate_p, "rate_plain_s_per_s": rate_p, "rate_surrogate_s_per_s": rate_s,
           "K": K, "f": f, "judge_every": J, "loss": args.sur_loss, "lr": args.sur_lr, "bound": args.sur_bound, "windows": R,
           "stats": st.as_dict(), "variants": variants,
           "validation": {"samples": nval * 4, "err_linear": v_lin, "err_linear_first_step": v_lin1,
                          "err_network_best": best[0], "gain_vs_linear": best[0] / v_lin,
                          "change_outside_mask": validate.outside, "curve": val_curve},
           "train_steps": steps,
           # mean training loss over the first and the last twentieth of the steps
           "train_loss_first": float(np.mean(losses[:max(1, len(losses) // 20)])),
           "train_loss_last": float(np.mean(losses[-max(1, len(losses) // 20):])),
           "samples": nsnap * 4, "tile": T, "forward_ms_2048sq": fwd_ms,
           "plain_window_ms": wall_p * 1e3 / R,
           "seconds": {"data": t_data, "train": t_train, "eval": wall_p + wall_s},
           "error_metric": "err_*: relative L1 of the predicted bed change against the plain solver's over the "
                           "judged window; elev_err_max: relative L1 of the bed elevation"}
    return out


def run_ours(args):
    import torch
    from paper_2103_15196_gb300 import swe

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    n, K, W = args.size, args.steps, args.warmup
    sc = make_workload(n, wet_fraction=args.wet_fraction)
    stream = torch.cuda.Stream()
    S = swe.Solver(n, n, 5.0, precision="fp32", stream=stream.cuda_stream, hgs_skip=0 if args.hgs_off else 1,
                   tile_rows=args.tile_rows, block_cols=args.block_cols)
    S.set_manning(sc.manning, block=64)
    H32 = [np.ascontiguousarray(a, dtype=np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b)]
    S.set_state(*H32)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # --- device-timed region, inputs resident
    clk = Clocks(local).__enter__()
    clk.wait_first()
    S.run_steps(W)
    S.sync()
    d0 = S.diag()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    ev0.record(stream)
    S.run_steps(K)
    ev1.record(stream)
    ev1.synchronize()
    clk.stop()
    clk.__exit__(None, None, None)
    torch.cuda.synchronize()
    barrier()
    ms = _max_over_ranks(ev0.elapsed_time(ev1), world)
    S.sync()
    d1 = S.diag()
    value = _aggregate_rate(float(n) * n, K, ms * 1e-3, world)
    comp = d1["cells_computed"] - d0["cells_computed"]
    copied = d1["cells_copied"] - d0["cells_copied"]
    alg_bytes_launch = BYTES_PER_CELL * (comp + copied) / K
    peak, peak_kind = _peaks()
    achieved = alg_bytes_launch / (ms * 1e-3 / K) / 1e9
    traffic = _profile_traffic(n)

    # --- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Ke = max(1, min(K, args.e2e_steps))
        host_in = [torch.from_numpy(a).pin_memory().numpy() for a in H32]
        host_out = [torch.empty((n, n), dtype=torch.float32).pin_memory().numpy() for _ in range(4)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.set_state(*host_in)
        S.run_steps(Ke)
        S.get_state(out=host_out)
        t1 = time.perf_counter()
        barrier()
        el = _max_over_ranks(t1 - t0, world)
        e2e = {"value": _aggregate_rate(float(n) * n, Ke, el, world), "unit": UNIT,
               "h2d_bytes_per_step": int(4 * n * n * 4 / Ke), "d2h_bytes_per_step": int(4 * n * n * 4 / Ke),
               "steps": Ke, "seconds": el}
    dd = S.diag()
    S.close()
    ens = None
    if world == 1 and not args.no_ensemble:
        ens = run_ensemble(args, torch, swe)
    hgs_flood = None
    if world == 1 and not args.no_hgs_flood:
        hgs_flood = run_hgs_flood(args, torch, swe)
    sur = None
    if world == 1 and not args.no_surrogate:
        sur = run_surrogate(args, torch, swe)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(sc, budget_s=args.cpu_seconds)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.wet_fraction:.0%}-wet fractal terrain {n}x{n} ({n * n} cells), dx=5 m, 20 m relief, "
                               f"carved channel, 2 m dam-break step, Manning per 64^2 block, FP32 state, "
                               f"FP64 dt/accumulators, HGS {'off' if args.hgs_off else 'on'}",
                   "grid": n, "l2_flush": "inputs larger than L2 (2 x 4.3 GB ping-pong state)",
                   "parallelism": f"{world} independent replica(s)",
                   "block": [dd["tile_x"], dd["tile_y"]]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": f"step_kernel<float,{dd['tile_x'] + 8}> (variant without source terms)",
                     "algorithmic_bytes_per_launch": alg_bytes_launch,
                     "note": "launch duration = timed region / K (includes the commit-and-list kernel "
                             "of each step and a compaction per graph replay)"},
        "issue": _issue_object(value, clk.summary()),
        "hgs": {"active_cell_fraction": comp / (float(n) * n * K), "copied_cell_fraction": copied / (float(n) * n * K),
                "all_cell_equiv_GBps": BYTES_PER_CELL * n * n / (ms * 1e-3 / K) / 1e9,
                "wet_cells_end": dd["wet_cells"], "t_end": dd["t"]},
        "e2e": e2e,
        "gpu_launches": _step_launches(n, K),
        "clocks": clocks,
        "cpu_baseline": cb,
        "ensemble": ens,
        "hgs_flood": hgs_flood,
        "surrogate": sur,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--hgs-off", action="store_true")
    ap.add_argument("--wet-fraction", type=float, default=0.5, help="initially wet fraction of the terrain")
    ap.add_argument("--tile-rows", type=int, default=0, help="rows per block strip (0: library default)")
    ap.add_argument("--block-cols", type=int, default=0, help="threads per block, 128 or 256 (0: default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-hgs-flood", action="store_true")
    ap.add_argument("--hgs-steps", type=int, default=200)
    ap.add_argument("--hgs-tile-rows", type=int, default=8, help="block strip height of the dry-start flood leg")
    ap.add_argument("--hgs-block-cols", type=int, default=256, help="threads per block of the dry-start flood leg")
    ap.add_argument("--ens-n", type=int, default=64)
    ap.add_argument("--ens-steps", type=int, default=100)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-only", action="store_true", help="run only the learned bed surrogate experiment")
    ap.add_argument("--sur-samples", type=int, default=2000)
    ap.add_argument("--sur-snaps-per-run", type=int, default=25)
    ap.add_argument("--sur-spin", type=int, default=300)
    ap.add_argument("--sur-train-steps", type=int, default=9000, help="Adam steps (batches of 4 tiles)")
    ap.add_argument("--sur-lr", type=float, default=1e-3)
    ap.add_argument("--sur-windows", type=int, default=200)
    ap.add_argument("--sur-f", type=int, default=25)
    ap.add_argument("--sur-judge", type=int, default=20)
    ap.add_argument("--sur-bound", type=float, default=0.35,
                    help="judged relative L1 of the window's bed change above which the plain solver takes over")
    ap.add_argument("--sur-loss", default="l1", choices=["mse", "l1"])
    ap.add_argument("--sur-gap", type=int, default=1, help="windows skipped between training samples")
    ap.add_argument("--sur-val", type=int, default=80, help="held-out validation samples (tiles)")
    ap.add_argument("--sur-val-points", type=int, default=6)
    ap.add_argument("--sur-variants", default="10:10,10:20,25:10",
                    help="extra f:judge_every evaluations of the trained network")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.surrogate_only:
        import torch
        from paper_2103_15196_gb300 import swe
        print(json.dumps({"surrogate": run_surrogate(args, torch, swe)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
