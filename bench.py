"""Benchmark: chunked 3D Gaussian + erode/dilate on a 1024^3 uint16 volume.

One step = the whole filtering path on one synthetic porous-media tomogram
(1024^3 uint16, 2 GiB): Gaussian sigma = 1, 2, 4 (FP32 accumulation, FP32
outputs) and grayscale erosion and dilation with a ball of radius 3 (exact,
uint16 outputs). `value` is volume voxels per second through the whole step
with inputs and outputs resident in HBM; `e2e` is the same step through the
C ABI with pinned host buffers (one hp_multi3d call per step: the
out-of-core executor streams each slab once for all five filters,
host<->device copies inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hp|reference]

`--impl reference` times the CPU oracle (the test oracle, single-threaded
FP64 C) on bounded sub-boxes of the same workload.

The default line also carries, besides the step: the FP32 FMA roofline of
the dominant kernel against the derived peak (this device's SM count x 128
lanes x 2 x max clock) and libhp's measured FMA probe; `bank` (the 512^3
float16 12-filter bank over 37 bricks, one graph launch); `spheres128` and
`autograd256` (the 128^3 pipeline and the 256^3 forward + backward); `ooc` (2048^3
uint16 out of core under an 8e9-byte budget, with a host-link probe at each
op's brick size and byte mix and the fraction of the link bound reached;
`--no-ooc` skips it); and the oracle timed single-threaded (`cpu_baseline`)
and as its OpenMP build on every host core (`cpu_baseline_mt`).

Other measured configurations, one JSON line each (not the benchmark step):
`--workload ooc2048` (2048^3 uint16 out-of-core under an 8e9-byte budget,
host-link efficiency), `spheres128` (128^3 float32 Gaussian -> threshold ->
cube morphology), `open1024` (1024^3 uint16 opening, closing, top-hat,
unsharp mask and Gaussian local threshold), `features1024` (1024^3 uint16
Hessian components and eigenvalues, box-window mean / Niblack / Sauvola
thresholds), `morph512` (512^3 uint16 erosion with cubes and balls of
radius 7 to 16),
`sweep` (out-of-core Gaussian on 1 to 16 GiB slabs under an 8e9-byte budget),
`bank512` (512^3 float16 12-filter bank over 37 bricks,
FMA roofline), `autograd256` (256^3 float32 forward + backward).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxels/s for chunked 3D Gaussian + erode/dilate at 1024³ uint16; % of HBM peak"
N = 1024
SIGMAS = (1.0, 2.0, 4.0)
BALL_R = 3
SEED = 2511118900 + 1


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2032.0)), "measured"
    except Exception:
        return 6400.0, 2032.0, "fallback"


class ClockSampler:
    """SM clock, its maximum and the clock-event (throttle) reasons, sampled
    during the timed region: NVML polled from a thread every 5 ms, or
    nvidia-smi every 20 ms where NVML cannot be opened (its first sample
    taken before the timed region starts). Reads only."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.nv = None
        self.samples: list[tuple[float, int]] = []
        self.mx = None
        self.stop = threading.Event()
        self.nvml_error = None
        self.first = threading.Event()

    @staticmethod
    def _nvml_lib():
        """(max SM clock, SM clock, reasons) readers for one device handle:
        the pynvml binding where installed, else NVML's C API through ctypes
        (nvmlInit_v2, nvmlDeviceGetHandleByUUID / ByIndex_v2,
        nvmlDeviceGetClockInfo, nvmlDeviceGetMaxClockInfo,
        nvmlDeviceGetCurrentClocksEventReasons; NVML_CLOCK_SM = 1; reason
        bits sw_power_cap 0x4, hw_slowdown 0x8, sw_thermal 0x20, hw_thermal
        0x40)."""
        try:
            import pynvml as nv
            nv.nvmlInit()
            reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            return (nv.nvmlDeviceGetHandleByUUID, nv.nvmlDeviceGetHandleByIndex,
                    lambda h: nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM),
                    lambda h: nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM), reasons, "pynvml")
        except ImportError:
            pass
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")

        def ok(rc):
            if rc != 0:
                raise RuntimeError(f"NVML error {rc}")
        ok(lib.nvmlInit_v2())

        def by_uuid(u):
            h = ctypes.c_void_p()
            ok(lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)))
            return h

        def by_index(i):
            h = ctypes.c_void_p()
            ok(lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(i), ctypes.byref(h)))
            return h

        def clock(fn):
            def get(h):
                v = ctypes.c_uint()
                ok(fn(h, ctypes.c_int(1), ctypes.byref(v)))
                return v.value
            return get
        rfn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def reasons(h):
            v = ctypes.c_ulonglong()
            ok(rfn(h, ctypes.byref(v)))
            return v.value
        return (by_uuid, by_index, clock(lib.nvmlDeviceGetMaxClockInfo),
                clock(lib.nvmlDeviceGetClockInfo), reasons, "ctypes")

    def _nvml(self):
        import torch
        by_uuid, by_index, max_clock, clock, reasons, how = self._nvml_lib()
        try:  # the CUDA device's own GPU, whatever NVML's enumeration order
            u = str(torch.cuda.get_device_properties(self.index).uuid)
            h = by_uuid(u if u.startswith("GPU-") else "GPU-" + u)
        except Exception:
            h = by_index(self.index)
        self.bits = (0x8, 0x40, 0x20, 0x4)  # NAMES order
        self.mx = float(max_clock(h))

        def poll():
            while not self.stop.is_set():
                try:
                    self.samples.append((float(clock(h)), int(reasons(h))))
                except Exception:
                    pass
                self.stop.wait(0.005)
        self.nv = how
        self.t = threading.Thread(target=poll, daemon=True)
        self.t.start()

    def __enter__(self):
        try:
            self._nvml()
            return self
        except Exception as e:
            self.nv = None
            self.nvml_error = f"{type(e).__name__}: {e}"[:160]
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=3.0)
            self.lines.clear()  # keep only samples taken from here on
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def __exit__(self, *exc):
        if self.nv is not None:
            self.stop.set()
            self.t.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], self.mx, set()
        if self.nv is not None:
            for mhz, r in self.samples:
                sm.append(mhz)
                for nm, b in zip(self.NAMES, self.bits):
                    if r & b:
                        reasons.add(nm)
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                    "reasons": sorted(reasons), "samples": len(sm), "source": f"nvml ({self.nv}), 5 ms"}
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(self.NAMES, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
               "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 20 ms"}
        if self.nvml_error:
            out["nvml_error"] = self.nvml_error
        return out


def _traffic(kernel: str, nvox: int):
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    capture (one-pass DRAM counters at the captured volume, scaled by the
    voxel count where the bench runs another size: an estimate there, since
    halo re-reads grow with the volume); None when that kernel is not the
    captured one or its sources changed since the capture."""
    if kernel != "gauss_s4":
        return None
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic_gauss_zr_r12_porous.json")) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return (rec["dram_read_bytes"] + rec["dram_write_bytes"]) * nvox / rec["captured_voxels"]
    except Exception:
        return None


def fma_peaks(hp, torch, sm_max_mhz: float):
    """FP32 FMA ceilings in TFLOP/s: derived (SM count of this device x 128
    FP32 lanes x 2 flop x max SM clock) and measured (libhp's FMA probe:
    packed FMA chains on every SM, CUDA events)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    derived = sms * 128 * 2 * sm_max_mhz * 1e6 / 1e12
    measured = hp.probe_fp32_fma(5) / 1e12
    return derived, measured, sms


def bank_measure(hp, torch, synth, steps: int, warmup: int, peak_derived: float,
                 peak_measured: float, hbm_gbs: float):
    """The 512^3 float16 12-filter bank (G, GM, LoG at sigma 0.7, 1, 2, 4)
    over 37 seeded k-d bricks, one graph launch per bank: ms per bank and
    its FMA and HBM rooflines."""
    n = 512
    f = synth.porous_f16(n, synth.SEED_BASE + 3)
    x = torch.from_numpy(f).cuda()
    bank = [(k, s) for s in BANK_SIGMAS for k in (hp.G, hp.GM, hp.LOG)]
    bricks = synth.kd_bricks(n, 37, synth.SEED_BASE + 3)
    outs = [torch.empty((n, n, n), dtype=torch.float16, device="cuda") for _ in bank]
    stream = torch.cuda.current_stream()
    ms, clk = _timed(lambda: hp.filterbank3d(x, bank, outs=outs, bricks=bricks), steps,
                     max(3, warmup), stream)
    hp.stream_status(stream)
    kernels = int(hp.stats()["bank_kernels"])
    nvox = n ** 3
    # per sigma, each pass 2r+1 taps: x pass 3 orders; y pass y0(X0), y0(X1),
    # y1(X0), and y2(X0) + y0(X2) summed (5 passes); z pass G, D_z, D_zz,
    # D_x, D_y and D_xx + D_yy (6): 14 passes
    fma = sum(14 * (2 * int(np.floor(3 * s + 0.5)) + 1) for s in BANK_SIGMAS)
    tflops = nvox * fma * 2 / (ms / 1e3) / 1e12
    gbs = nvox * (2 + 2 * len(bank)) / (ms / 1e3) / 1e9
    del outs, x
    return {"ms": ms, "voxels_per_s": nvox / (ms / 1e3), "kernels_per_launch": kernels,
            "fma_per_voxel": fma, "TFLOP/s": tflops, "alu_frac": tflops / peak_derived,
            "alu_frac_of_measured": tflops / peak_measured, "GB/s": gbs,
            "hbm_frac": gbs / hbm_gbs, "clocks": clk,
            "workload": "porous 512^3 f16 -> 12 x f16 (G, GM, LoG at sigma 0.7/1/2/4), 37 k-d bricks"}


def reduce_over_ranks(local_ms: float, ws: int, units_per_rank: float, device=None):
    """Whole-job timing of N replicas: the slowest rank's time (max over
    ranks) and the units all ranks processed per second. Uses the default
    process group when ws > 1."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return total_ms, ws * units_per_rank / (total_ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(budget_s: float, seed_volume=None):
    """Time the oracle on sub-boxes of the workload for about budget_s
    seconds; returns (voxels/s, sample description)."""
    import oracle
    import synth
    f = seed_volume
    if f is None:
        f, _ = synth.porous((96, 96, 96), SEED)    # same recipe, a smaller drawing
    n = f.shape[0]
    b = 16
    rng = np.random.default_rng(7)
    voxels, t0, boxes = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s:
        lo = [int(v) for v in rng.integers(0, n - b, 3)]
        for s in SIGMAS:
            r = oracle.radius(s)
            ilo = [max(0, c - r) for c in lo]
            ihi = [min(n, c + b + r) for c in lo]
            oracle.gaussian3d(f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]], s, gdims=f.shape,
                              in_lo=ilo, out_lo=lo, out_shape=(b, b, b))
        ilo = [max(0, c - BALL_R) for c in lo]
        ihi = [min(n, c + b + BALL_R) for c in lo]
        part = f[ilo[0]:ihi[0], ilo[1]:ihi[1], ilo[2]:ihi[2]]
        for dil in (False, True):
            oracle.morph3d(part, oracle.SE_BALL, BALL_R, dil, gdims=f.shape, in_lo=ilo, out_lo=lo,
                           out_shape=(b, b, b))
        voxels += b ** 3
        boxes += 1
    dt = time.perf_counter() - t0
    return voxels / dt, f"{boxes} random {b}^3 output boxes (with halos) of the step, {dt:.1f} s"


def cpu_ops_sample(ops, seconds_per_op: float = 3.0, n: int = 48):
    """Time the oracle (single-threaded FP64 C) on each named op of a
    workload, on an n^3 drawing of the same porous generator, for about
    seconds_per_op each: {name: voxels/s} and the sample description."""
    import oracle
    import synth
    f, _ = synth.porous((n, n, n), SEED)
    res = {}
    for name, fn in ops:
        calls, t0 = 0, time.perf_counter()
        while True:
            fn(f)
            calls += 1
            dt = time.perf_counter() - t0
            if dt >= seconds_per_op:
                break
        res[name] = calls * n ** 3 / dt
    return res, f"the oracle on a {n}^3 drawing of the same porous generator, ~{seconds_per_op:.0f} s per op"


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(min(per_step, 2.0))
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, sample = cpu_oracle_sample(per_step)
        vals.append(v)
    dt = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {
        "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic porous tomogram (seeded), bounded sub-box sample",
        "config": {"workload": "porous 1024^3 u16: gaussian s=1,2,4 -> f32; erode+dilate ball r=3",
                   "sample": sample},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_hp(args):
    import torch
    import torch.distributed as dist

    import paper_2511_11890_b300 as hp
    import synth

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_gbs, sm_max_mhz, peak_kind = _peaks()

    N = args.size
    f, porosity = synth.porous(N, SEED)
    x = torch.from_numpy(f).to(dev)
    outs_g = [torch.empty((N, N, N), dtype=torch.float32, device=dev) for _ in SIGMAS]
    out_e = torch.empty((N, N, N), dtype=torch.uint16, device=dev)
    out_d = torch.empty((N, N, N), dtype=torch.uint16, device=dev)
    stream = torch.cuda.current_stream(dev)
    names = [f"gauss_s{s:g}" for s in SIGMAS] + ["erode_ball3", "dilate_ball3"]

    def step(evs=None):
        k = 0
        for s, o in zip(SIGMAS, outs_g):
            hp.gaussian3d(x, s, out=o)
            if evs is not None:
                evs[k].record(stream)
            k += 1
        hp.erode3d(x, "ball", BALL_R, out=out_e)
        if evs is not None:
            evs[k].record(stream)
        hp.dilate3d(x, "ball", BALL_R, out=out_d)
        if evs is not None:
            evs[k + 1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    # timed region: K steps, events between the five kernels of every step
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in names] for _ in range(args.steps)]
    first = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        start.record(stream)
        for i in range(args.steps):
            first[i].record(stream)
            step(ev[i])
        end.record(stream)
        torch.cuda.synchronize()
    hp.stream_status(stream)
    total_ms = start.elapsed_time(end)
    per = {nm: 0.0 for nm in names}
    for i in range(args.steps):
        prev = first[i]
        for nm, e in zip(names, ev[i]):
            per[nm] += prev.elapsed_time(e) / args.steps
            prev = e
    total_ms, value = reduce_over_ranks(total_ms, ws, args.steps * N ** 3, dev)

    # per-kernel rooflines: algorithmic bytes (u16 in + out) and FP32 FMAs
    nvox = N ** 3
    kern = {}
    fma_peak_tflops, fma_measured_tflops, sms = fma_peaks(hp, torch, sm_max_mhz)
    for s, nm in zip(SIGMAS, names):
        r = int(np.floor(3 * s + 0.5))
        byts = nvox * (2 + 4)
        flops = nvox * 3 * (2 * r + 1) * 2
        ms = per[nm]
        kern[nm] = {"ms": ms, "GB/s": byts / ms / 1e6, "hbm_frac": byts / ms / 1e6 / hbm_gbs,
                    "TFLOP/s": flops / ms / 1e9, "alu_frac": flops / ms / 1e9 / fma_peak_tflops,
                    "alu_frac_of_measured": flops / ms / 1e9 / fma_measured_tflops}
    for nm in names[3:]:
        byts = nvox * 4
        ms = per[nm]
        kern[nm] = {"ms": ms, "GB/s": byts / ms / 1e6, "hbm_frac": byts / ms / 1e6 / hbm_gbs}
    dom = max(names, key=lambda k: per[k])
    dk = kern[dom]
    if "alu_frac" in dk and dk["alu_frac"] > dk["hbm_frac"]:
        roof = {"bound": "alu", "achieved": dk["TFLOP/s"], "peak": fma_peak_tflops,
                "unit": "TFLOP/s", "frac": dk["alu_frac"], "traffic": None,
                "kernel": dom,
                "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock",
                "measured_peak": fma_measured_tflops,
                "frac_of_measured": dk["alu_frac_of_measured"],
                "measured_peak_kind": "libhp FMA probe (packed fma.rn.f32x2 chains, CUDA events)"}
    else:
        roof = {"bound": "hbm", "achieved": dk["GB/s"], "peak": hbm_gbs, "unit": "GB/s",
                "frac": dk["hbm_frac"], "traffic": None, "kernel": dom, "peak_kind": peak_kind}
    roof["traffic"] = _traffic(dom, nvox)
    step_bytes = nvox * (3 * 6 + 2 * 4)
    hbm_step_frac = step_bytes / (total_ms / args.steps) / 1e6 / hbm_gbs

    del outs_g, out_e, out_d
    torch.cuda.empty_cache()
    # configuration 4: the filter bank (one graph launch per bank); configs 1
    # and 5: the 128^3 pipeline and the 256^3 forward + backward
    bank = cfg1 = cfg5 = None
    if rank == 0 and not args.no_bank:
        bank = bank_measure(hp, torch, synth, args.steps, args.warmup, fma_peak_tflops,
                            fma_measured_tflops, hbm_gbs)
        torch.cuda.empty_cache()
        cfg1 = spheres128_measure(hp, torch, synth, args.steps, args.warmup)
        cfg5 = autograd256_measure(hp, torch, synth, args.steps, args.warmup)
        torch.cuda.empty_cache()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(f).pin_memory()
        oh = [torch.empty((N, N, N), dtype=torch.float32).pin_memory() for _ in SIGMAS]
        eh = torch.empty((N, N, N), dtype=torch.uint16).pin_memory()
        dh = torch.empty((N, N, N), dtype=torch.uint16).pin_memory()

        ops = [("gauss", s) for s in SIGMAS] + [("erode", "ball", BALL_R), ("dilate", "ball", BALL_R)]

        def hstep():
            # the whole step in one call: each halo-padded slab of the input
            # crosses the host link once, all five filters run on it
            hp.multi3d(xh, ops, outs=oh + [eh, dh])
            st = hp.stats()
            return st["h2d_bytes"], st["d2h_bytes"]

        hstep()
        ke = max(1, min(args.steps, 3))
        if ws > 1:
            dist.barrier()  # the ranks start together; the slowest one sets the time
        t0 = time.perf_counter()
        for _ in range(ke):
            h2d, d2h = hstep()
        dt = time.perf_counter() - t0
        e2e_ms, e2e_value = reduce_over_ranks(dt * 1e3, ws, ke * nvox, dev)
        e2e = {"value": e2e_value, "unit": "voxels/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke,
               "link_GB/s": (h2d + d2h) / (e2e_ms / 1e3 / ke) / 1e9,
               "call": "hp_multi3d on pinned host buffers (one out-of-core pass, 5 outputs)"}
        del xh, oh, eh, dh

    # configuration 3: out of core at 2048^3 under an 8e9-byte budget
    ooc = None
    if rank == 0 and not args.no_ooc:
        del x
        torch.cuda.empty_cache()
        ooc = ooc_measure(hp, torch, steps=2)

    cpu = cpu_mt = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        nproc = os.cpu_count() or 1
        v, sample = cpu_oracle_sample(args.cpu_seconds)
        cpu = {"value": v, "unit": "voxels/s", "cores": 1, "kind": "oracle", "sample": sample,
               "nproc": nproc}
        import oracle
        oracle.use_threads(True)
        try:
            v, sample = cpu_oracle_sample(max(4.0, args.cpu_seconds / 2))
        finally:
            oracle.use_threads(False)
        cpu_mt = {"value": v, "unit": "voxels/s", "cores": nproc,
                  "kind": "oracle, the same source built with OpenMP over z", "sample": sample,
                  "nproc": nproc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": f"synthetic porous tomogram (seeded, porosity {porosity:.3f})",
            "config": {"workload": f"porous {N}^3 u16: gaussian s=1,2,4 -> f32; erode+dilate ball r=3",
                       "volume": [N, N, N], "parallelism": "replicas" if ws > 1 else "single",
                       "l2": f"input ({2 * N ** 3 / 2 ** 30:.3g} GiB) and outputs "
                             f"({16 * N ** 3 / 2 ** 30:.3g} GiB) larger than L2",
                       "hbm_frac_of_step": hbm_step_frac},
            "roofline": roof, "kernels": kern, "cpu_baseline": cpu, "cpu_baseline_mt": cpu_mt,
            "e2e": e2e, "gpu_launches": 5 * args.steps, "clocks": clk.summary(),
            "bank": bank, "ooc": ooc, "spheres128": cfg1, "autograd256": cfg5,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def link_probe(chunk: int, d2h_per_h2d: float, seconds: float = 1.0):
    """Pinned host <-> device copy rates (GB/s) with chunks of the brick
    size, each leg for at least `seconds`: H2D alone, D2H alone, and both
    directions at once with D2H bytes = d2h_per_h2d x H2D bytes (the mix of
    the operation being measured), two streams per direction. The link
    bound of an operation moving (h, d) bytes is then
    max(h / h2d, d / d2h, (h + d) / both) seconds."""
    import torch
    dchunk = max(1 << 20, int(chunk * d2h_per_h2d) // 4096 * 4096)
    hs = [torch.empty(chunk, dtype=torch.uint8).pin_memory() for _ in range(2)]
    ds = [torch.empty(chunk, dtype=torch.uint8, device="cuda") for _ in range(2)]
    hd = [torch.empty(dchunk, dtype=torch.uint8).pin_memory() for _ in range(2)]
    dd = [torch.empty(dchunk, dtype=torch.uint8, device="cuda") for _ in range(2)]
    st = [torch.cuda.Stream() for _ in range(4)]

    def run(h2d: bool, d2h: bool):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb_h = nb_d = 0
        i = 0
        while True:
            if h2d:
                with torch.cuda.stream(st[i % 2]):
                    ds[i % 2].copy_(hs[i % 2], non_blocking=True)
                nb_h += chunk
            if d2h:
                with torch.cuda.stream(st[2 + i % 2]):
                    hd[i % 2].copy_(dd[i % 2], non_blocking=True)
                nb_d += dchunk
            i += 1
            if i % 4 == 0:
                torch.cuda.synchronize()
                if time.perf_counter() - t0 >= seconds:
                    break
        dt = time.perf_counter() - t0
        return nb_h / dt / 1e9, nb_d / dt / 1e9

    run(True, True)  # warm-up
    h2d, _ = run(True, False)
    _, d2h = run(False, True)
    bh, bd = run(True, True)
    return {"chunk_bytes": chunk, "h2d": h2d, "d2h": d2h, "both_h2d": bh, "both_d2h": bd,
            "both_total": bh + bd, "d2h_per_h2d": dchunk / chunk}


def link_bound_s(h2d_bytes: int, d2h_bytes: int, probe: dict) -> float:
    """Seconds the host link needs for these bytes at the probe's rates."""
    return max(h2d_bytes / 1e9 / probe["h2d"], d2h_bytes / 1e9 / probe["d2h"],
               (h2d_bytes + d2h_bytes) / 1e9 / probe["both_total"])


def ooc_measure(hp, torch, f=None, steps: int = 2):
    """Out-of-core 2048^3 uint16 (pinned host buffers, budget 8e9 B):
    Gaussian sigma 3 (f32) and ball-5 dilation (u16); per op the best of
    `steps` timed calls after one warm-up, the bytes moved, the link probe
    at the op's brick size and byte mix, and the fraction of the link bound
    reached."""
    import synth
    n, budget = 2048, 8_000_000_000
    if f is None:
        f, _ = synth.porous(n, 2511118900 + 2)
    xh = torch.from_numpy(f).pin_memory()
    del f
    og = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    od = torch.empty((n, n, n), dtype=torch.uint16).pin_memory()
    old = hp.get_memory_budget()
    hp.set_memory_budget(budget)
    res = {}
    try:
        for name, fn in (("gauss_s3", lambda: hp.gaussian3d(xh, 3.0, out=og)),
                         ("dilate_ball5", lambda: hp.dilate3d(xh, "ball", 5, out=od))):
            fn()
            times = []
            for _ in range(max(1, steps)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                times.append(time.perf_counter() - t0)
            st = hp.stats()
            dt = min(times)
            chunk = int(min(1 << 30, max(1 << 26, st["h2d_bytes"] // max(1, st["bricks"]))))
            probe = link_probe(chunk // 4096 * 4096, st["d2h_bytes"] / max(1, st["h2d_bytes"]))
            bound = link_bound_s(st["h2d_bytes"], st["d2h_bytes"], probe)
            res[name] = {"s": dt, "voxels_per_s": n ** 3 / dt, "bricks": st["bricks"],
                         "h2d_bytes": st["h2d_bytes"], "d2h_bytes": st["d2h_bytes"],
                         "peak_device_bytes": st["peak_device_bytes"], "budget_bytes": budget,
                         "link_GBps": (st["h2d_bytes"] + st["d2h_bytes"]) / dt / 1e9,
                         "probe_GBps": probe, "link_bound_s": bound, "link_frac": bound / dt}
    finally:
        hp.set_memory_budget(old)
        del xh, og, od
    return res


def run_outofcore(args):
    """2048^3 uint16 porous volume in pinned host memory under an 8e9-byte
    budget: Gaussian sigma 3 (f32 out) and ball-5 dilation (u16 out), each
    streamed through the device in halo-padded bricks."""
    import torch

    import paper_2511_11890_b300 as hp
    n = 2048
    res = ooc_measure(hp, torch, steps=args.steps)
    total = sum(v["s"] for v in res.values())
    line = {"metric": "voxels/s, out-of-core 2048^3 uint16 under an 8e9-byte budget "
                      "(gaussian s=3 + ball-5 dilation); % of host link",
            "value": 2 * n ** 3 / total, "unit": "voxels/s", "n_gpus": 1, "steps": args.steps,
            "higher_is_better": True, "data": "synthetic porous tomogram (seeded)",
            "config": {"workload": "porous 2048^3 u16, pinned host buffers, budget 8e9 B"},
            "ops": res}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args):
    """Size sweep of the out-of-core Gaussian (sigma 3, f32 out) under an
    8e9-byte budget: uint16 slabs of 2048 x 2048 x nz for nz = 128 .. 2048
    (1 to 16 GiB of input), as in the paper's time-versus-size and
    memory-versus-budget figures. Per size: time, bricks, peak library
    device bytes during the call and library device bytes left after it."""
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    n, budget = 2048, 8_000_000_000
    f, _ = synth.porous(n, 2511118900 + 2)
    xh = torch.from_numpy(f).pin_memory()
    del f
    og = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    hp.set_memory_budget(budget)
    rows = []
    for nz in (128, 256, 512, 1024, 2048):
        x, o = xh[:nz], og[:nz]
        hp.gaussian3d(x, 3.0, out=o)  # warm-up
        times = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hp.gaussian3d(x, 3.0, out=o)
            times.append(time.perf_counter() - t0)
        st = hp.stats()
        dt = min(times)
        rows.append({"nz": nz, "input_GiB": nz * n * n * 2 / 2 ** 30, "s": dt,
                     "voxels_per_s": nz * n * n / dt, "bricks": st["bricks"],
                     "link_GBps": (st["h2d_bytes"] + st["d2h_bytes"]) / dt / 1e9,
                     "peak_device_bytes": st["peak_device_bytes"],
                     "live_device_bytes_after": st["live_device_bytes"]})
    line = {"metric": "seconds per out-of-core Gaussian (sigma 3) vs input size, 8e9-byte budget",
            "value": rows[-1]["s"], "unit": "s", "n_gpus": 1, "steps": args.steps,
            "higher_is_better": False, "data": "synthetic porous tomogram (seeded)",
            "config": {"workload": "porous u16 slabs 2048 x 2048 x nz, pinned host buffers, budget 8e9 B"},
            "sizes": rows}
    print(json.dumps(line), flush=True)
    return 0


def _timed(fn, steps, warmup, stream):
    """CUDA-event time (ms per call) of fn() over `steps` calls after
    `warmup` untimed ones, with clocks sampled during the timed region."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clk.summary()


def run_open1024(args):
    """1024^3 uint16 porous volume: opening, closing and white top-hat with
    the r = 3 ball (compositions of the erosion and dilation kernels through
    a scratch volume), the unsharp mask (sigma 2, amount 1) and the Gaussian
    local threshold (sigma 2)."""
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    n = N
    f, _ = synth.porous(n, SEED)
    x = torch.from_numpy(f).cuda()
    o = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    hbm_gbs, _, peak_kind = _peaks()
    nvox = n ** 3
    res, clks = {}, {}
    # algorithmic bytes per voxel: two passes of 2 B in + 2 B out; the
    # top-hat adds its difference (2 B in, 2 B opening in, 2 B out)
    for name, fn, bpv in (("open", hp.open3d, 8), ("close", hp.close3d, 8), ("tophat", hp.tophat3d, 14)):
        ms, clk = _timed(lambda fn=fn: fn(x, "ball", BALL_R, out=o), args.steps, max(3, args.warmup), stream)
        gbs = nvox * bpv / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "GB/s": gbs, "hbm_frac": gbs / hbm_gbs}
        clks[name] = clk
    # unsharp mask sigma 2, amount 1 (float32 out): the Gaussian (2 B in, 4 B
    # out) and the epilogue (2 B in, 4 B in, 4 B out)
    g = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    ms, _ = _timed(lambda: hp.unsharp3d(x, 2.0, 1.0, out=g), args.steps, max(3, args.warmup), stream)
    res["unsharp_s2"] = {"ms": ms, "GB/s": nvox * 16 / (ms / 1e3) / 1e9,
                         "hbm_frac": nvox * 16 / (ms / 1e3) / 1e9 / hbm_gbs}
    # Gaussian local threshold sigma 2 (uint8 out): the Gaussian into scratch
    # (2 B in, 4 B out) and the comparison (2 B + 4 B in, 1 B out)
    u = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    ms, _ = _timed(lambda: hp.threshold_local3d(x, 2.0, 0.0, out=u), args.steps, max(3, args.warmup), stream)
    res["threshold_local_s2"] = {"ms": ms, "GB/s": nvox * 13 / (ms / 1e3) / 1e9,
                                 "hbm_frac": nvox * 13 / (ms / 1e3) / 1e9 / hbm_gbs}
    hp.stream_status(stream)
    import oracle
    cpu, sample = cpu_ops_sample([
        ("open", lambda v: oracle.open3d(v, oracle.SE_BALL, BALL_R)),
        ("close", lambda v: oracle.close3d(v, oracle.SE_BALL, BALL_R)),
        ("tophat", lambda v: oracle.tophat3d(v, oracle.SE_BALL, BALL_R)),
        ("unsharp_s2", lambda v: oracle.unsharp3d(v, 2.0, 1.0)),
        ("threshold_local_s2", lambda v: oracle.threshold_local(v, 2.0, 0.0))])
    line = {"metric": "voxels/s, 1024^3 uint16 opening (ball r = 3)", "value": nvox / (res["open"]["ms"] / 1e3),
            "unit": "voxels/s", "n_gpus": 1, "steps": args.steps, "ms_per_step": res["open"]["ms"],
            "higher_is_better": True, "dtype": "u16", "data": "synthetic porous tomogram (seeded)",
            "config": {"workload": "porous 1024^3 u16: opening, closing, white top-hat, ball r = 3"},
            "ops": res, "hbm_peak_kind": peak_kind, "gpu_launches": 2 * args.steps,
            "clocks": clks["open"],
            "cpu_baseline": {"value": cpu["open"], "unit": "voxels/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "ops": cpu}}
    print(json.dumps(line), flush=True)
    return 0


def run_morph512(args):
    """512^3 uint16 porous volume: erosion with large structuring elements,
    cubes of radius 7 and 16 (van Herk / Gil-Werman line passes through key
    scratch, 20 B/voxel) and balls of radius 7, 10, 13 and 16 (tiled z-march,
    2 B in and 2 B out per voxel)."""
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    n = 512
    f, _ = synth.porous(n, 5)
    x = torch.from_numpy(f).cuda()
    o = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    hbm_gbs, _, peak_kind = _peaks()
    nvox = n ** 3
    res, clks = {}, {}
    for se, r, bpv in (("cube", 7, 20), ("cube", 16, 20), ("ball", 7, 4), ("ball", 10, 4),
                       ("ball", 13, 4), ("ball", 16, 4)):
        ms, clks[f"{se}{r}"] = _timed(lambda: hp.erode3d(x, se, r, out=o), args.steps,
                                      max(3, args.warmup), stream)
        gbs = nvox * bpv / (ms / 1e3) / 1e9
        res[f"erode_{se}{r}"] = {"ms": ms, "voxels_per_s": nvox / (ms / 1e3), "GB/s": gbs,
                                 "hbm_frac": gbs / hbm_gbs}
    hp.stream_status(stream)
    import oracle
    cpu, sample = cpu_ops_sample([("erode_cube7", lambda v: oracle.erode3d(v, oracle.SE_CUBE, 7)),
                                  ("erode_ball7", lambda v: oracle.erode3d(v, oracle.SE_BALL, 7))],
                                 3.0, 32)
    line = {"metric": "voxels/s, 512^3 uint16 erosion with the radius-7 cube", "unit": "voxels/s",
            "value": res["erode_cube7"]["voxels_per_s"], "n_gpus": 1, "steps": args.steps,
            "ms_per_step": res["erode_cube7"]["ms"], "higher_is_better": True, "dtype": "u16",
            "data": "synthetic porous tomogram (seeded)",
            "config": {"workload": "porous 512^3 u16: erosion, cube r = 7, 16; ball r = 7, 10, 13, 16"},
            "ops": res, "hbm_peak_kind": peak_kind, "gpu_launches": 3 * args.steps,
            "clocks": clks["cube7"],
            "cpu_baseline": {"value": cpu["erode_cube7"], "unit": "voxels/s", "cores": 1,
                             "kind": "oracle", "sample": sample, "ops": cpu}}
    print(json.dumps(line), flush=True)
    return 0


def run_features1024(args):
    """1024^3 uint16 porous volume: the Hessian feature set at sigma 2 (the
    six second-derivative components to float32, and the three ascending
    eigenvalues per voxel) and the box-window local thresholds (mean,
    Niblack, Sauvola; radius 7, a 15^3 window) to uint8."""
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    n = N
    f, _ = synth.porous(n, SEED)
    x = torch.from_numpy(f).cuda()
    stream = torch.cuda.current_stream()
    hbm_gbs, sm_max_mhz, peak_kind = _peaks()
    fma_derived, fma_measured, _ = fma_peaks(hp, torch, sm_max_mhz)
    nvox = n ** 3
    res, clks = {}, {}
    # Hessian components: six separable passes of r = 6 (13 taps per axis,
    # 3 x 13 FMAs per voxel each), 2 B in and 4 B out per component
    outs = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(6)]
    ms, clks["hessian"] = _timed(lambda: hp.hessian3d(x, 2.0, outs=outs), args.steps, max(3, args.warmup), stream)
    fma = 6 * 3 * 13
    tflops = 2 * fma * nvox / (ms / 1e3) / 1e12
    res["hessian_components_s2"] = {"ms": ms, "fma_per_voxel": fma, "TFLOP/s": tflops,
                                    "alu_frac": tflops / fma_derived,
                                    "alu_frac_of_measured": tflops / fma_measured,
                                    "GB/s": nvox * 36 / (ms / 1e3) / 1e9}
    del outs
    # eigenvalues: the six components into library scratch, then the
    # closed-form 3 x 3 symmetric eigenvalues (24 B in, 12 B out per voxel)
    eig = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(3)]
    ms, _ = _timed(lambda: hp.hessian3d(x, 2.0, eigenvalues=True, outs=eig), args.steps,
                   max(3, args.warmup), stream)
    res["hessian_eigenvalues_s2"] = {"ms": ms, "voxels_per_s": nvox / (ms / 1e3),
                                     "note": "components (6 x 39 FMA/voxel) + eigenvalue epilogue"}
    del eig
    # box-window thresholds, three passes through scratch: x (2 B in, 12 B
    # out: the window sum as u32 and the sum of squares as u64), y (12 in,
    # 12 out), z fused with the decision (12 + 2 in, 1 out): 53 B/voxel
    u = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    for method, k, c in (("mean", 0.0, 0.0), ("niblack", -0.2, 0.0), ("sauvola", 0.34, 32768.0)):
        ms, clks[method] = _timed(lambda: hp.threshold_box3d(x, method, 7, k, c, out=u), args.steps,
                                  max(3, args.warmup), stream)
        gbs = nvox * 53 / (ms / 1e3) / 1e9
        res[f"threshold_box_{method}_r7"] = {"ms": ms, "voxels_per_s": nvox / (ms / 1e3),
                                             "GB/s": gbs, "hbm_frac": gbs / hbm_gbs}
    hp.stream_status(stream)
    import oracle
    cpu, sample = cpu_ops_sample([
        ("hessian_components_s2", lambda v: oracle.hessian3d(v, 2.0)),
        ("hessian_eigenvalues_s2", lambda v: oracle.hessian_eigenvalues(v, 2.0)),
        ("threshold_box_mean_r7", lambda v: oracle.threshold_box(v, oracle.LOCAL_MEAN, 7, 0.0, 0.0)),
        ("threshold_box_niblack_r7", lambda v: oracle.threshold_box(v, oracle.LOCAL_NIBLACK, 7, -0.2, 0.0)),
        ("threshold_box_sauvola_r7", lambda v: oracle.threshold_box(v, oracle.LOCAL_SAUVOLA, 7, 0.34, 32768.0))])
    h = res["hessian_components_s2"]
    line = {"metric": "voxels/s, 1024^3 uint16 Hessian components (sigma 2)", "value": nvox / (h["ms"] / 1e3),
            "unit": "voxels/s", "n_gpus": 1, "steps": args.steps, "ms_per_step": h["ms"],
            "higher_is_better": True, "dtype": "f32", "data": "synthetic porous tomogram (seeded)",
            "config": {"workload": "porous 1024^3 u16: Hessian components and eigenvalues (sigma 2); "
                                   "box-window mean / Niblack / Sauvola thresholds (radius 7)"},
            "ops": res, "hbm_peak_kind": peak_kind,
            "fma_peak_tflops": {"derived": fma_derived, "measured": fma_measured},
            "gpu_launches": 6 * args.steps, "clocks": clks["hessian"],
            "cpu_baseline": {"value": cpu["hessian_components_s2"], "unit": "voxels/s", "cores": 1,
                             "kind": "oracle", "sample": sample, "ops": cpu}}
    print(json.dumps(line), flush=True)
    return 0


def spheres128_measure(hp, torch, synth, steps: int, warmup: int):
    """128^3 float32 spheres: Gaussian sigma 2 -> threshold 0.5 to uint8 ->
    erosion and dilation with the 3^3 cube (the unchunked pipeline): ms per
    pipeline (four launches through the C ABI)."""
    n = 128
    f = synth.spheres(n, 40, synth.SEED_BASE + 0)
    x = torch.from_numpy(f).cuda()
    g = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    t = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    e = torch.empty_like(t)
    d = torch.empty_like(t)
    stream = torch.cuda.current_stream()

    def step():
        hp.gaussian3d(x, 2.0, out=g)
        hp.threshold3d(g, 0.5, out=t)
        hp.erode3d(t, "cube", 1, out=e)
        hp.dilate3d(t, "cube", 1, out=d)

    ms, clk = _timed(step, steps, max(3, warmup), stream)
    hp.stream_status(stream)
    return {"ms": ms, "voxels_per_s": n ** 3 / (ms / 1e3), "launches": 4, "clocks": clk,
            "workload": "spheres 128^3 f32: gaussian s=2, threshold 0.5, cube-3 erode + dilate",
            "note": "8 MiB volume, L2-resident: bound by host launch latency"}


def run_spheres128(args):
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    m = spheres128_measure(hp, torch, synth, args.steps, args.warmup)
    line = {"metric": "voxels/s, 128^3 float32 pipeline: gaussian s=2, threshold 0.5, cube-3 erode+dilate",
            "value": m["voxels_per_s"], "unit": "voxels/s", "n_gpus": 1, "steps": args.steps,
            "ms_per_step": m["ms"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic spheres (seeded)",
            "config": {"workload": "spheres 128^3 f32, 40 balls r 4-16, sigma 0.05 noise",
                       "l2": "8 MiB volume: L2-resident, latency-bound (voxels/s only)"},
            "gpu_launches": 4 * args.steps, "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


BANK_SIGMAS = (0.7, 1.0, 2.0, 4.0)


def run_bank512(args):
    """512^3 float16 porous volume: Gaussian, gradient magnitude and LoG at
    sigma 0.7, 1, 2, 4 (12 float16 outputs) over 37 uneven bricks, in one
    persistent graph-captured launch per bank."""
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    hbm_gbs, sm_max_mhz, peak_kind = _peaks()
    derived, measured, sms = fma_peaks(hp, torch, sm_max_mhz)
    b = bank_measure(hp, torch, synth, args.steps, args.warmup, derived, measured, hbm_gbs)
    line = {"metric": "voxels/s, 512^3 float16 12-filter bank (G, GM, LoG at sigma 0.7/1/2/4), 37 bricks",
            "value": b["voxels_per_s"], "unit": "voxels/s", "n_gpus": 1, "steps": args.steps,
            "ms_per_step": b["ms"], "higher_is_better": True, "dtype": "f32 (f16 storage)",
            "data": "synthetic porous tomogram (seeded), 37 seeded k-d bricks",
            "config": {"workload": b["workload"] + f", {b['kernels_per_launch']} persistent kernel(s) per launch"},
            "roofline": {"bound": "alu", "achieved": b["TFLOP/s"], "peak": derived, "unit": "TFLOP/s",
                         "frac": b["alu_frac"], "fma_per_voxel": b["fma_per_voxel"],
                         "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock",
                         "measured_peak": measured, "frac_of_measured": b["alu_frac_of_measured"],
                         "hbm": {"GB/s": b["GB/s"], "frac": b["hbm_frac"], "peak_kind": peak_kind}},
            "gpu_launches": b["kernels_per_launch"] * args.steps, "clocks": b["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def autograd256_measure(hp, torch, synth, steps: int, warmup: int):
    """256^3 float32 spheres: forward 12-filter bank + erosion (5^3 cube),
    loss = sum of w * features with seeded N(0,1) fields, hand-written
    backward through torch.autograd: ms per forward + backward."""
    from paper_2511_11890_b300 import autograd as hpa
    n = 256
    f = synth.spheres(n, 320, synth.SEED_BASE + 4)
    x = torch.from_numpy(f).cuda().requires_grad_(True)
    bank = [(k, s) for s in BANK_SIGMAS for k in (hp.G, hp.GM, hp.LOG)]
    ws = [torch.from_numpy(synth.normal_field((n, n, n), synth.SEED_BASE + 40 + i)).cuda()
          for i in range(len(bank) + 1)]
    stream = torch.cuda.current_stream()

    def step():
        x.grad = None
        feats = hpa.bank_and_erosion(x, bank, "cube", 2)
        loss = sum((F * w).sum() for F, w in zip(feats, ws))
        loss.backward()

    ms, clk = _timed(step, steps, max(3, warmup), stream)
    hp.stream_status(stream)
    del x, ws
    return {"ms": ms, "voxels_per_s": n ** 3 / (ms / 1e3), "clocks": clk,
            "workload": "spheres 256^3 f32: 12-filter bank + cube-5 erosion, forward + backward",
            "note": "the weighted sums of the loss run as torch reductions"}


def run_autograd256(args):
    import torch

    import paper_2511_11890_b300 as hp
    import synth
    m = autograd256_measure(hp, torch, synth, args.steps, args.warmup)
    line = {"metric": "voxels/s, 256^3 float32 forward + backward (12-filter bank + cube-5 erosion)",
            "value": m["voxels_per_s"], "unit": "voxels/s", "n_gpus": 1, "steps": args.steps,
            "ms_per_step": m["ms"], "higher_is_better": True, "dtype": "f32",
            "data": "synthetic spheres (seeded), seeded N(0,1) loss weights",
            "config": {"workload": "spheres 256^3 f32, 320 balls; loss = sum w_k * feature_k",
                       "note": m["note"]},
            "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hp", choices=["hp", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-bank", action="store_true", help="skip the 512^3 filter-bank leg")
    ap.add_argument("--no-ooc", action="store_true", help="skip the 2048^3 out-of-core leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="porous1024",
                    choices=["porous1024", "ooc2048", "spheres128", "bank512", "autograd256",
                             "open1024", "features1024", "morph512", "sweep"])
    ap.add_argument("--size", type=int, default=N,
                    help="edge of the in-HBM volume (1024 is the benchmark; smaller sizes "
                         "are for profiling captures)")
    args = ap.parse_args()
    if args.workload == "ooc2048":
        return run_outofcore(args)
    if args.workload == "spheres128":
        return run_spheres128(args)
    if args.workload == "bank512":
        return run_bank512(args)
    if args.workload == "autograd256":
        return run_autograd256(args)
    if args.workload == "open1024":
        return run_open1024(args)
    if args.workload == "features1024":
        return run_features1024(args)
    if args.workload == "morph512":
        return run_morph512(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_hp(args)


if __name__ == "__main__":
    sys.exit(main())
