#!/usr/bin/env python3
"""Benchmark of the GB300 hydro path: one FP64 MUSCL-Hancock/HLLC step of a 512^3 periodic grid.

Workload (the single-uniform-grid configuration): 512^3 periodic box, Gaussian random k^-4
velocities at rms Mach 5, lognormal density (sigma 1), cold gas P/rho = 1e-4 plus a Sedov cell
(E = 1 in one cell); MinMod PLM + HLLC, CFL 0.8, gamma 5/3; each step's dt is the CFL dt of its
input, fused into the previous step's epilogue (device-resident, no host sync per step).  The
state (5.4 GB in FP64) is far larger than L2, so no flush is needed between steps.

Prints one JSON line: value = interior cells x steps / time (Mcell-updates/s, whole job), the
roofline of the step kernel (the method's algorithmic bytes and flops per launch / CUDA-event
duration, against the measured HBM and the arithmetic peak of the pipe that runs them), the
clocks seen during the timed region, an end-to-end number through the C ABI with host buffers,
the CPU oracle as a reported baseline, the other forms (native FP64, FP32, mixed, mixed-precision
batched AMR patches and oct groups, PPM, MHD, the two-level AMR cycle, adjoint/forward ratios,
1024^3 graph-captured run) beside it, and for the headline and every form the error of one more
step against the FP64 oracle on sampled cells, patches or oct groups (err_vs_oracle; the oracle
runs in the CPU oracle leg, rank 0, after every timed region).

The headline step runs in double-float arithmetic (--precision df64): the double state with every
operation of the scheme on pairs of floats, which meets the FP64 parity bar and runs on the FP32
pipes; the native-FP64 step is reported beside it (forms.fp64_512).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--precision df64|fp64|fp32|mixed]
Under torchrun (N > 1) every rank runs the same workload on its own GPU (replicas: the path
does not shard); value sums all ranks' cells over the slowest rank's time.
"""
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

import torch  # noqa: E402

# Algorithmic arithmetic per interior cell of one step (binary +, -, *, / and sqrt, each 1),
# counted stage by stage on a 64^3 sample of each workload (tests/test_bench_constants.py
# recomputes them): recovery 12 + slopes + predictor 56 + 3 x face (states + HLLC) + update 35.
ALG_FLOPS_PER_CELL = {"turb_minmod": 375.0, "turb_mc": 402.0, "mach10_mc": 387.0}
# The same step in double-float arithmetic (the df64 precision): each operation of the scheme
# becomes FP32 operations of the double-word algorithms -- add/sub 11 (TwoSum of the high words,
# the low words' sum, Fast2Sum), mul 8 (TwoProd by FMA, a cross product and FMA, Fast2Sum), div 23,
# sqrt 12 -- applied to the oracle's count by kind on the same sample (+- 178.3, * 167.5, / 22.9,
# sqrt 6.0 per cell).  Reported beside the roofline as the emulation's work, not the method's.
DF_COST = {"addsub": 11, "mul": 8, "div": 23, "sqrt": 12}
ALG_DF_FLOPS_PER_CELL = {"turb_minmod": 3900.0}
BYTES_PER_CELL = {"fp64": 80.0, "fp32": 40.0, "mixed": 80.0, "df64": 80.0}  # 5 fields read + 5 written

PRECISION_TEXT = {
    "df64": "FP64 step in double-float arithmetic (double state; every operation on pairs of floats)",
    "fp64": "FP64 step in native double arithmetic",
    "fp32": "FP32 step with the pressure recovery in error-free float transformations",
    "mixed": "double state, FP32 bulk, double recovery and update accumulation"}
PARITY_TEXT = {
    "df64": "<= 1e-12 relative per step against the FP64 oracle (tests/test_gpu_forward.py, fp64 bar)",
    "fp64": "<= 1e-12 relative per step against the FP64 oracle (tests/test_gpu_forward.py)",
    "fp32": "<= 1e-5 relative after one step against the FP64 oracle; conservation 1e-6 over 100 steps "
            "(tests/test_gpu_forward.py)",
    "mixed": "<= 1e-5 relative after one step against the FP64 oracle (tests/test_gpu_forward.py)"}

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# Arithmetic peaks from unit counts and the maximum SM clock (2070 MHz), 152 SMs:
# FP32 128 FMA lanes/SM/clk -> 80.5 TFLOP/s; FP64 2 DFMA/SM/clk -> 1.26 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--precision", default="df64", choices=["fp64", "fp32", "mixed", "df64"])
    p.add_argument("--forms", default="all", help="comma list of extra forms, 'all' or 'none'")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--tuning", default="auto", help="'auto' (autotune) or '<tile id>:<zchunk>'")
    p.add_argument("--npatch", type=int, default=4096, help="patches of the batched form")
    p.add_argument("--ngroups", type=int, default=262144, help="oct groups of the batched form")
    p.add_argument("--adj-n", type=int, default=64, help="grid edge of the adjoint form")
    p.add_argument("--adj-precisions", default="df64,fp64,fp32", help="precisions of the adjoint form")
    p.add_argument("--mhd-precisions", default="fp64,df64,fp32,mixed", help="precisions of the MHD form")
    p.add_argument("--forms-only", action="store_true",
                   help="run only the extra forms and print their JSON (for profiling them alone)")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources the uniform-grid step kernel's code is compiled from (its launcher and the other
# kernels live elsewhere): a committed ncu summary carries their hash, and its DRAM traffic is
# used only while they are unchanged.
STEP_SOURCES = ("df.cuh", "hydro_device.cuh", "step_tile.cuh")


def kernel_source_hash(files=STEP_SOURCES):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1412_0934_gb300", "csrc")
    for fn in sorted(files):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_hash") != kernel_source_hash():
            return None, "stale"
        return float(kv["dram_bytes_per_launch_full"]), os.path.relpath(path, ROOT)
    except Exception:
        return None, "absent"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.lines = []
        self.proc = None
        sel = []
        try:
            uuid = str(torch.cuda.get_device_properties(device).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi"] + sel + ["--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def job_time_ms(ms, world, device):
    """The job's timed-region duration: the maximum over ranks of each rank's own (replicas)."""
    if world == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def e2e_summary(ms, cells):
    """End-to-end throughput from the wall-clock times (ms) of individual steps over `cells` cells: the
    median step sets the value, the mean step mean_value; the slowest step is kept beside them."""
    s = sorted(ms)
    k = len(s)
    med = s[k // 2] if k % 2 else 0.5 * (s[k // 2 - 1] + s[k // 2])
    mean = sum(s) / k
    return {"value": cells / med / 1e3, "unit": "Mcell-updates/s", "steps": k, "ms_per_step_median": round(med, 3),
            "mean_value": cells / mean / 1e3, "ms_per_step_max": round(s[-1], 3)}


def job_value(cells, steps, world, t_max_ms):
    """Whole-job throughput in Mcell-updates/s: every rank's cells over the slowest rank's time."""
    return world * cells * steps / (t_max_ms / 1e3) / 1e6


# ----------------------------------------------------------------------------- workloads
def turbulent(n, precision, device, seed=2, mach=5.0, sigma=1.0, p_over_rho=1e-4, sedov=True):
    import workloads
    U = workloads.turbulent_state(n, seed=seed, mach=mach, sigma_rho=sigma, p_over_rho=p_over_rho, sedov=sedov,
                                  device=device)
    if precision == "fp32":
        U = U.float()
    return U.contiguous()


TUNING = "auto"


TILE_NAMES = {0: "16x16", 1: "32x8", 2: "8x8", 3: "32x16", 4: "16x16/1 block per SM"}


def tune(hy, ctx, a, b, dx, dts):
    """Autotune tile shape and z-chunk on this machine (writes b), or apply a fixed --tuning."""
    pa, pb = hy.patch(a, 0, dx), hy.patch(b, 0, dx)
    hy.hydro_cfl_dt(ctx, pa, dts[0:1])
    if TUNING == "auto":
        hy.hydro_autotune(ctx, pa, pb, dts[0:1])
    else:
        t, z = (int(x) for x in TUNING.split(":"))
        hy.hydro_set_tuning(ctx, t, z)
    t, z = hy.hydro_get_tuning(ctx)
    return {"tile": TILE_NAMES[t], "zchunk": z}


def time_steps(hy, ctx, a, b, dx, dts, steps, warmup, stream, per_launch=True):
    """warmup + steps ping-pong steps with device-resident dt; returns (ms total, per-launch ms list,
    final state tensor, launches in the timed region)."""
    pa, pb = hy.patch(a, 0, dx), hy.patch(b, 0, dx)
    hy.hydro_cfl_dt(ctx, pa, dts[0:1])
    cur = 0
    for i in range(warmup):
        src, dst = (pa, pb) if cur == 0 else (pb, pa)
        hy.hydro_step(ctx, src, dst, dts[i:i + 1], dts[i + 1:i + 2])
        cur ^= 1
    torch.cuda.synchronize()
    launches0 = hy.hydro_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(steps):
        k = warmup + i
        src, dst = (pa, pb) if cur == 0 else (pb, pa)
        if per_launch:
            ev[i][0].record(stream)
        hy.hydro_step(ctx, src, dst, dts[k:k + 1], dts[k + 1:k + 2])
        if per_launch:
            ev[i][1].record(stream)
        cur ^= 1
    t1.record(stream)
    torch.cuda.synchronize()
    launches = hy.hydro_launch_count(ctx) - launches0
    per = [s.elapsed_time(e) for s, e in ev] if per_launch else []
    return t0.elapsed_time(t1), per, (a if cur == 0 else b), launches


def roofline(precision, cells, per_ms, flops_per_cell, hbm_gbs, peak_src, traffic):
    """Roofline object of the step kernel from the method's own work: algorithmic bytes per launch
    (BYTES_PER_CELL) against the measured HBM peak, and algorithmic flops per launch (the oracle's
    count of the scheme's +, -, *, / and sqrt) against the arithmetic peak of the pipe that runs them
    (FP64 for the native-double step, FP32 for the others); the binding roof is the one with the
    larger fraction.  For the double-float step the FP32 operations that emulate those flops are
    reported beside it (emulated_fp32_*), not as the method's work."""
    avg_s = statistics.mean(per_ms) / 1e3
    bytes_launch = cells * BYTES_PER_CELL[precision]
    flops_launch = cells * flops_per_cell
    gbs = bytes_launch / avg_s / 1e9
    tfl = flops_launch / avg_s / 1e12
    fpeak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    hbm_frac = gbs / hbm_gbs
    alu_frac = tfl / fpeak
    common = {"hbm_frac": round(hbm_frac, 4), "alu_frac": round(alu_frac, 4),
              "alu_peak_tflops": round(fpeak, 2), "alu_peak_source": "unit counts x 2070 MHz",
              "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": peak_src, "avg_launch_ms": round(avg_s * 1e3, 4),
              "algorithmic_bytes_per_launch": bytes_launch, "algorithmic_flops_per_launch": flops_launch,
              "algorithmic_flops_per_cell": flops_per_cell}
    if precision == "df64":
        em = ALG_DF_FLOPS_PER_CELL["turb_minmod"]
        etfl = cells * em / avg_s / 1e12
        common.update({"emulated_fp32_ops_per_cell": em, "emulated_fp32_tflops": round(etfl, 3),
                       "emulated_fp32_frac": round(etfl / FP32_PEAK_TFLOPS, 4)})
    if alu_frac >= hbm_frac:
        r = {"bound": "alu", "achieved": round(tfl, 3), "peak": round(fpeak, 2), "unit": "TFLOP/s",
             "frac": round(alu_frac, 4)}
    else:
        r = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s", "frac": round(hbm_frac, 4)}
    r["traffic"] = traffic
    r.update(common)
    return r


# ----------------------------------------------------------------------------- parity samples
# Every form, after its timed region, takes one more step (or adjoint step) and copies to the host
# the inputs and GPU outputs of sampled cells, whole patches or oct groups.  No oracle code runs
# here: the CPU oracle leg (cpu_oracle_leg, rank 0 only, after every timed region) computes the same
# outputs in FP64 and attaches the normwise error per field to the form (err_vs_oracle).
CHECKS = []


def sample_cells(shape, count, seed):
    """Random cells plus the box corners, both sides of 16- and 32-cell tile seams and of 32-, 64- and
    128-plane z-chunk seams, and the 7^3 block around the box centre (the Sedov cell of the
    turbulence boxes: where the step changes the state most, its time step set by the blast) (z, y, x)."""
    import numpy as np
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    cells = [tuple(int(rng.integers(0, m)) for m in shape) for _ in range(count)]
    for dz in range(-3, 4):
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                cells.append(((nz // 2 + dz) % nz, (ny // 2 + dy) % ny, (nx // 2 + dx) % nx))
    for z in (0, 31, 32, 63, 64, 127, 128, nz - 1):
        for y in (0, 15, 16, ny - 1):
            for x in (0, 31, 32, nx - 1):
                cells.append((z % nz, y % ny, x % nx))
    return np.array(sorted(set(cells)))


def neighbourhoods(U, cells, r):
    """(S, F, 2r+1, 2r+1, 2r+1) periodic neighbourhoods of the cells (z, y, x), gathered on U's device."""
    F, NZ, NY, NX = U.shape
    c = torch.as_tensor(cells, device=U.device, dtype=torch.long)
    o = torch.arange(-r, r + 1, device=U.device)
    iz = (c[:, 0, None] + o) % NZ
    iy = (c[:, 1, None] + o) % NY
    ix = (c[:, 2, None] + o) % NX
    flat = (iz[:, :, None, None] * NY + iy[:, None, :, None]) * NX + ix[:, None, None, :]
    return U.reshape(F, -1)[:, flat].permute(1, 0, 2, 3, 4).double().cpu().numpy()


def record_cells(path, scheme, U_in, U_out, dx, dt, limiter, count=600, seed=0, note=None):
    """Sampled cells of one periodic step U_in -> U_out (scheme plm, ppm or mhd)."""
    r = 3 if scheme == "ppm" else 2
    cells = sample_cells(tuple(U_in.shape[1:]), count, seed)
    ci = torch.as_tensor(cells, device=U_out.device)
    got = U_out[:, ci[:, 0], ci[:, 1], ci[:, 2]].double().cpu().numpy().T
    CHECKS.append({"path": path, "scheme": scheme, "inputs": neighbourhoods(U_in, cells, r), "got": got, "dx": dx,
                   "dt": [dt] * len(cells), "limiter": limiter, "what": "%d sampled cells" % len(cells), "note": note})


def record_boxes(path, scheme, boxes, limiter, what):
    """Whole ghosted boxes (patches, oct stencils): [(ghosted input, GPU interior output, dx, dt)]."""
    CHECKS.append({"path": path, "scheme": scheme, "boxes": boxes, "limiter": limiter, "what": what})


def oracle_errors(checks):
    """The CPU oracle's outputs for every recorded sample and the normwise error per field of the
    GPU's (max over samples of |gpu - oracle| / max over samples of |oracle|), by form."""
    import numpy as np
    import oracle
    from oracle import mhd as omhd
    from oracle import ppm as oppm
    acc = {}
    for c in checks:
        cfg = oracle.config(limiter=c["limiter"] if c["limiter"] != "ppm" else "minmod")
        step = {"plm": lambda g, dx, dt: oracle.step_patch(g, dx, dt, cfg),
                "ppm": lambda g, dx, dt: oppm.step_patch(g, dx, dt, cfg),
                "mhd": lambda g, dx, dt: omhd.step_patch(g, dx, dt, cfg, limiter=c["limiter"])}.get(c["scheme"])
        if c["scheme"] == "adjoint":
            w = oracle.step_periodic_adjoint(c["U"], c["lam_out"], c["dx"], c["dt"], cfg)
            F = w.shape[0]
            want, got = w.reshape(F, -1).T, c["got"].reshape(F, -1).T
        elif "inputs" in c:
            want = np.stack([step(g, c["dx"], dt).reshape(g.shape[0]) for g, dt in zip(c["inputs"], c["dt"])])
            got = np.asarray(c["got"], dtype=np.float64)
        else:
            ws, gs = [], []
            for Ug, out, dx, dt in c["boxes"]:
                w = step(Ug, dx, dt)
                ws.append(w.reshape(w.shape[0], -1).T)
                gs.append(np.asarray(out, dtype=np.float64).reshape(w.shape[0], -1).T)
            want, got = np.concatenate(ws), np.concatenate(gs)
        a = acc.setdefault(tuple(c["path"]), {"want": [], "got": [], "what": c["what"], "note": c.get("note")})
        a["want"].append(want)
        a["got"].append(got)
    res = {}
    for path, a in acc.items():
        want, got = np.concatenate(a["want"]), np.concatenate(a["got"])
        scale = np.maximum(np.abs(want).max(axis=0), 1e-300)
        per_field = (np.abs(got - want).max(axis=0) / scale).tolist()
        e = {"max": float("%.3g" % max(per_field)), "per_field": [float("%.3g" % v) for v in per_field],
             "samples": a["what"], "metric": "per field max|gpu - oracle| / max|oracle| over the samples (FP64 oracle)"}
        if a["note"]:
            e["note"] = a["note"]
        res[path] = e
    return res


# ----------------------------------------------------------------------------- forms
def record_step(hy, ctx, src, dst, dx, d, path, scheme, limiter, count=600):
    """One more step src -> dst at the form's tuning (dt d: the fused CFL dt of src), sampled."""
    hy.hydro_step(ctx, hy.patch(src, 0, dx), hy.patch(dst, 0, dx), d)
    torch.cuda.synchronize()
    record_cells(path, scheme, src, dst, dx, d.item(), limiter, count=count, seed=len(CHECKS) + 17)


def form_uniform(hy, n, precision, limiter, steps, warmup, flops_key, mach=5.0, sigma=1.0, p_over_rho=1e-4,
                 sedov=True, seed=2, graph=False, path=None):
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision=precision, limiter=limiter)
    a = turbulent(n, precision, "cuda", seed=seed, mach=mach, sigma=sigma, p_over_rho=p_over_rho, sedov=sedov)
    b = torch.empty_like(a)
    dx = 1.0 / n
    cells = n ** 3
    if graph:
        hist = torch.empty(steps + 1, dtype=torch.float64, device="cuda")
        pa, pb = hy.patch(a, 0, dx), hy.patch(b, 0, dx)
        tuning = tune(hy, ctx, a, b, dx, hist)
        hy.hydro_run(ctx, pa, pb, steps, hist, use_graph=True)  # capture + first replay (warm-up)
        torch.cuda.synchronize()
        a.copy_(turbulent(n, precision, "cuda", seed=seed, mach=mach, sigma=sigma, p_over_rho=p_over_rho,
                          sedov=sedov))
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        hy.hydro_run(ctx, pa, pb, steps, hist, use_graph=True)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        rc, bits = hy.hydro_get_error(ctx)
        out = {"cells": cells, "steps": steps, "ms_per_step": ms / steps,
               "mcell_updates_per_s": cells * steps / (ms / 1e3) / 1e6, "graph": True, "error_bits": bits,
               "tuning": tuning}
        if path:
            # one more step from the GPU's own state after the timed steps, and the cells of that
            # state whose internal energy is negative (their pressure is floored, HYDRO_EBIT_P_FLOOR)
            neg = 0
            for z in range(0, n, 64):
                W = a[:, z:z + 64].double()
                neg += int(((W[4] - 0.5 * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / W[0]) < 0).sum().item())
            del W
            d = torch.empty(1, dtype=torch.float64, device="cuda")
            hy.hydro_cfl_dt(ctx, pa, d)
            hy.hydro_step(ctx, pa, pb, d)
            torch.cuda.synchronize()
            out["negative_internal_energy_cells_after_last_step"] = neg
            record_cells(path, "plm", a, b, dx, d.item(), limiter, count=400, seed=31,
                         note="one further step from the GPU's state after the %d timed steps; that state has "
                              "%d cells (%.2g of all) with negative internal energy, floored by the scheme"
                              % (steps, neg, neg / cells))
    else:
        dts = torch.empty(warmup + steps + 1, dtype=torch.float64, device="cuda")
        tuning = tune(hy, ctx, a, b, dx, dts)
        if limiter == "ppm":
            tuning["tile"] = "16x16"  # the PPM kernel's one tile shape; only the z chunk is tuned
        ms, per, final, launches = time_steps(hy, ctx, a, b, dx, dts, steps, warmup, stream)
        rc, bits = hy.hydro_get_error(ctx)
        if path:
            record_step(hy, ctx, final, b if final is a else a, dx, dts[warmup + steps:warmup + steps + 1], path,
                        "ppm" if limiter == "ppm" else "plm", limiter)
        hbm, src = peaks()
        out = {"cells": cells, "steps": steps, "ms_per_step": ms / steps,
               "mcell_updates_per_s": cells * steps / (ms / 1e3) / 1e6, "error_bits": bits, "tuning": tuning}
        if flops_key is None:  # operations not counted for this form: the HBM fraction only
            out["hbm_frac"] = cells * BYTES_PER_CELL[precision] / (statistics.mean(per) / 1e3) / 1e9 / hbm
        else:
            out["roofline"] = roofline(precision, cells, per, ALG_FLOPS_PER_CELL[flops_key], hbm, src, None)
    del a, b
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_batched(hy, steps, warmup, npatch=4096, ngroups=262144):
    """4096 AMR patches (edges {8..48}, cubes and 2:1 boxes, levels 0-5, own dx and CFL dt) in one
    persistent launch per step, plus 262144 oct groups; mixed precision."""
    import numpy as np
    import workloads
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision="mixed")
    parent = turbulent(256, "mixed", "cuda", seed=3, sedov=False)
    descs = workloads.patch_set(npatch, seed=3)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=3)
    ins, outs, keep = [], [], []
    interior = 0
    ghosted = 0
    for d, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (d["nx"], d["ny"], d["nz"])).contiguous()
        Vg = torch.empty_like(Ug)
        keep += [Ug, Vg]
        ins.append(hy.patch(Ug, 2, d["dx"], d["level"]))
        outs.append(hy.patch(Vg, 2, d["dx"], d["level"]))
        interior += d["nx"] * d["ny"] * d["nz"]
        ghosted += Ug[0].numel()
    n = len(ins)
    dt = torch.empty(n, dtype=torch.float64, device="cuda")
    dn = torch.empty(n, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(ctx, ins, dt)
    if TUNING == "auto":
        hy.hydro_autotune(ctx, ins, outs, dt)  # tile shape and z chunk for this patch set
    tt, tz = hy.hydro_get_tuning(ctx)
    per_class = [hy.hydro_get_class_tuning(ctx, k) for k in range(hy.NUM_PATCH_CLASSES)]
    for _ in range(warmup):
        hy.hydro_step(ctx, ins, outs, dt, dn)
    torch.cuda.synchronize()
    l0 = hy.hydro_launch_count(ctx)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_step(ctx, ins, outs, dt, dn)  # same input each step: the per-patch dt stays valid
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    launches = (hy.hydro_launch_count(ctx) - l0) / steps
    rng_s = np.random.default_rng(41)
    big = sorted(range(n), key=lambda i: -descs[i]["nx"] * descs[i]["ny"] * descs[i]["nz"])[:2]
    picks = sorted(set(big) | set(int(i) for i in rng_s.choice(n, 22, replace=False)))
    dth = dt.cpu().numpy()
    record_boxes(("mixed_batched",), "plm",
                 [(keep[2 * i].cpu().numpy(), keep[2 * i + 1][:, 2:-2, 2:-2, 2:-2].cpu().numpy(), descs[i]["dx"],
                   float(dth[i])) for i in picks], "minmod", "%d whole patches (the 2 largest among them)" % len(picks))
    # oct groups
    og = workloads.oct_origins(ngroups, parent.shape[1:], seed=3)
    g = workloads.gather_octs(parent, og).contiguous()
    go = torch.empty((5, ngroups, 2, 2, 2), dtype=torch.float64, device="cuda")
    dto = torch.tensor([0.5 * dt.min().item()], dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        hy.hydro_step_octs(ctx, g, go, 1.0 / 256, dto)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_step_octs(ctx, g, go, 1.0 / 256, dto)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_o = t0.elapsed_time(t1) / steps
    sel = torch.as_tensor(np.sort(rng_s.choice(ngroups, 400, replace=False)), device="cuda")

    def record_octs(key, stencils, outs, what):
        record_boxes(("mixed_batched", key), "plm",
                     [(st, o, 1.0 / 256, dto.item()) for st, o in zip(stencils, outs)], "minmod", what)

    record_octs("octs", g[:, sel].permute(1, 0, 2, 3, 4).cpu().numpy(),
                go[:, sel].permute(1, 0, 2, 3, 4).cpu().numpy(), "400 whole oct groups")
    # the same groups read in place from the level grid (no gathered copy), in Morton order of
    # their origins (the space-filling-curve order a tree code keeps its octs in)
    oa = np.asarray(og)
    key = np.zeros(len(oa), dtype=np.int64)
    for b in range(21):
        for d in range(3):
            key |= ((oa[:, d] >> b) & 1).astype(np.int64) << (3 * b + d)
    od = torch.as_tensor(oa[np.argsort(key, kind="stable")], dtype=torch.int32, device="cuda").contiguous()
    lv = hy.patch(parent, 0, 1.0 / 256)
    for _ in range(warmup):
        hy.hydro_step_octs_level(ctx, lv, od, go, dto)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_step_octs_level(ctx, lv, od, go, dto)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_l = t0.elapsed_time(t1) / steps
    st_l = workloads.gather_octs(parent, od[sel].cpu().numpy()).permute(1, 0, 2, 3, 4).cpu().numpy()
    record_octs("octs_level", st_l, go[:, sel].permute(1, 0, 2, 3, 4).cpu().numpy(), "400 whole oct groups")
    # the level stored oct-major (128^3 octs) with its device-built Morton order and neighbour
    # table (the device chunk builder); the same groups, then every oct of the level in Morton
    # order, stepped through the table
    no = 128 ** 3
    V = parent.reshape(5, 128, 2, 128, 2, 128, 2).permute(0, 1, 3, 5, 2, 4, 6).reshape(5, no, 8).contiguous()
    Vo = torch.empty_like(V)
    idx = torch.arange(no, device="cuda", dtype=torch.int32)
    pos = torch.stack([idx % 128, (idx // 128) % 128, idx // (128 * 128)], dim=1).contiguous()
    order = torch.empty(no, dtype=torch.int32, device="cuda")
    nbr = torch.empty((no, 27), dtype=torch.int32, device="cuda")
    for _ in range(warmup):
        hy.hydro_octs_build(ctx, pos, (128, 128, 128), order, nbr)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_octs_build(ctx, pos, (128, 128, 128), order, nbr)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_b = t0.elapsed_time(t1) / steps
    ol = (od[:, 0] // 2 + 128 * (od[:, 1] // 2 + 128 * (od[:, 2] // 2))).to(torch.int32).contiguous()
    timed = {}
    for name, lst in (("groups", ol), ("level", order)):
        for _ in range(warmup):
            hy.hydro_step_octs_table(ctx, V, Vo, nbr, lst, 1.0 / 256, dto)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            hy.hydro_step_octs_table(ctx, V, Vo, nbr, lst, 1.0 / 256, dto)
        t1.record(stream)
        torch.cuda.synchronize()
        timed[name] = t0.elapsed_time(t1) / steps
        # the octs stepped (oct-major: cell (i, j, k) of oct o at o * 8 + (k * 2 + j) * 2 + i)
        pick = sel if name == "groups" else torch.as_tensor(np.sort(rng_s.choice(no, 400, replace=False)),
                                                             device="cuda")
        octs_sel = lst[pick].long()
        pos_s = pos[octs_sel]
        st_t = workloads.gather_octs(parent, (2 * pos_s).cpu().numpy()).permute(1, 0, 2, 3, 4).cpu().numpy()
        got_t = Vo[:, octs_sel].reshape(5, -1, 2, 2, 2).permute(1, 0, 2, 3, 4).cpu().numpy()
        record_octs("octs_table" if name == "groups" else "octs_table_level", st_t, got_t, "400 whole octs")
    ms_t, ms_tl = timed["groups"], timed["level"]
    # coarse-to-fine ghost fill of the same patch set from a 128^3 coarse level (fine dx = 1/256)
    coarse = turbulent(128, "mixed", "cuda", seed=3, sedov=False)
    rng = np.random.default_rng(14)
    gorig = [(int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(rng.integers(0, 256))) for _ in descs]
    gfine = [hy.patch(keep[2 * i], 2, 1.0 / 256) for i in range(n)]
    gcoarse = hy.patch(coarse, 0, 1.0 / 128)
    # arguments marshalled once: the 4096-patch ctypes array would cost the host more than the fill
    gf_a, gn = hy._parray(gfine)
    go_i, gc = hy._ints(gorig), ctypes.byref(gcoarse.c)

    def fill():
        if hy.lib().hydro_fill_ghosts(ctx.handle, gc, gf_a, go_i, gn) != hy.HYDRO_OK:
            raise RuntimeError("hydro_fill_ghosts failed")

    for _ in range(warmup):
        fill()
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        fill()
    t1.record(stream)
    torch.cuda.synchronize()
    ms_g = t0.elapsed_time(t1) / steps
    nghost = ghosted - interior
    rc, bits = hy.hydro_get_error(ctx)
    hbm, src = peaks()
    bytes_p = (ghosted * 5 * 8 + interior * 5 * 8)
    bytes_o = ngroups * (216 + 8) * 5 * 8
    out = {"patches": n, "interior_cells": interior, "ghosted_cells": ghosted, "ms_per_step": ms,
           "mcell_updates_per_s": interior / (ms / 1e3) / 1e6, "launches_per_step": launches,
           "tuning": {"tile": TILE_NAMES[tt], "zchunk": tz,
                      "per_patch_class": [{"tile": TILE_NAMES[t], "zchunk": z} for t, z in per_class]},
           "hbm_frac": bytes_p / (ms / 1e3) / 1e9 / hbm,
           "octs": {"groups": ngroups, "ms_per_step": ms_o, "mcell_updates_per_s": ngroups * 8 / (ms_o / 1e3) / 1e6,
                    "hbm_frac": bytes_o / (ms_o / 1e3) / 1e9 / hbm},
           "octs_level": {"groups": ngroups, "ms_per_step": ms_l,
                          "mcell_updates_per_s": ngroups * 8 / (ms_l / 1e3) / 1e6,
                          "hbm_frac": ngroups * (80 + 8) * 5 * 8 / (ms_l / 1e3) / 1e9 / hbm,
                          "note": "stencils read in place from the 256^3 level (80 needed cells per group, "
                                  "8 written), groups in Morton order; no gathered copy"},
           "octs_table": {"groups": ngroups, "ms_per_step": ms_t,
                          "mcell_updates_per_s": ngroups * 8 / (ms_t / 1e3) / 1e6,
                          "hbm_frac": ngroups * ((80 + 8) * 5 * 8 + 27 * 4) / (ms_t / 1e3) / 1e9 / hbm,
                          "note": "the same groups read from the oct-major level through the device-built "
                                  "neighbour table (80 needed cells + 27 table entries per group, 8 written)"},
           "octs_table_level": {"octs": no, "ms_per_step": ms_tl,
                                "mcell_updates_per_s": no * 8 / (ms_tl / 1e3) / 1e6,
                                "hbm_frac": no * (8 * 5 * 8 * 2 + 27 * 4) / (ms_tl / 1e3) / 1e9 / hbm,
                                "note": "every oct of the 256^3 level in Morton order through the table "
                                        "(each cell read once from HBM and written once, plus the table)"},
           "octs_build": {"octs": no, "ms": ms_b, "mocts_per_s": no / (ms_b / 1e3) / 1e6,
                          "note": "Morton order and 27-entry neighbour table of the level's 128^3 octs "
                                  "(bitmap over the key space, prefix sums, O(1) rank lookups)"},
           "ghost_fill": {"ghost_cells": nghost, "ms": ms_g, "mcells_per_s": nghost / (ms_g / 1e3) / 1e6,
                          "hbm_frac": (nghost + 128 ** 3) * 5 * 8 / (ms_g / 1e3) / 1e9 / hbm,
                          "note": "2 ghost layers of the 4096 patches prolonged from a 128^3 coarse level "
                                  "(writes + one read of the coarse level)"},
           "error_bits": bits}
    del keep, parent, g, go, od, coarse, V, Vo, pos, order, nbr, ol
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_ppm_batched(hy, steps, warmup, npatch=4096, precision="mixed"):
    """The PPM step of the 4096-patch AMR set (three ghost layers per patch) in one persistent
    launch per step, per-patch dt and fused dt_next."""
    import workloads
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision=precision, limiter="ppm")
    parent = turbulent(256, precision, "cuda", seed=3, sedov=False)
    descs = workloads.patch_set(npatch, seed=3)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=3)
    ins, outs, keep = [], [], []
    interior = ghosted = 0
    for d, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (d["nx"], d["ny"], d["nz"]), ghost=3).contiguous()
        Vg = torch.empty_like(Ug)
        keep += [Ug, Vg]
        ins.append(hy.patch(Ug, 3, d["dx"], d["level"]))
        outs.append(hy.patch(Vg, 3, d["dx"], d["level"]))
        interior += d["nx"] * d["ny"] * d["nz"]
        ghosted += Ug[0].numel()
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    dn = torch.empty_like(dt)
    hy.hydro_cfl_dt(ctx, ins, dt)
    if TUNING == "auto":
        hy.hydro_autotune(ctx, ins, outs, dt)
    tt, tz = hy.hydro_get_tuning(ctx)
    for _ in range(warmup):
        hy.hydro_step(ctx, ins, outs, dt, dn)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_step(ctx, ins, outs, dt, dn)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    rc, bits = hy.hydro_get_error(ctx)
    import numpy as np
    rng_s = np.random.default_rng(43)
    dth = dt.cpu().numpy()
    picks = sorted(int(i) for i in rng_s.choice(len(ins), 8, replace=False))
    record_boxes(("ppm_batched_mixed",), "ppm",
                 [(keep[2 * i].double().cpu().numpy(), keep[2 * i + 1][:, 3:-3, 3:-3, 3:-3].double().cpu().numpy(),
                   descs[i]["dx"], float(dth[i])) for i in picks], "ppm", "%d whole patches" % len(picks))
    hbm, src = peaks()
    es = 4 if precision == "fp32" else 8
    out = {"patches": len(ins), "interior_cells": interior, "ghosted_cells": ghosted, "ms_per_step": ms,
           "mcell_updates_per_s": interior / (ms / 1e3) / 1e6, "tuning": {"tile": "16x16", "zchunk": tz},
           "hbm_frac": (ghosted + interior) * 5 * es / (ms / 1e3) / 1e9 / hbm, "error_bits": bits,
           "note": "PPM on the patch set of mixed_batched with three ghost layers per patch"}
    del keep, parent
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_mhd(hy, precision, steps, warmup, n=256):
    """Ideal MHD with GLM cleaning on an n^3 periodic box (smooth magnetised gas, plasma beta 0.5,
    rms Mach 2): steps chained through the fused dt."""
    import workloads
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision=precision, limiter="minmod")
    dtype = torch.float32 if precision == "fp32" else torch.float64
    a = workloads.mhd_state(n, seed=7, beta=0.5, mach=2.0, device="cuda").to(dtype).contiguous()
    b = torch.empty_like(a)
    dx = 1.0 / n
    dts = torch.empty(warmup + steps + 1, dtype=torch.float64, device="cuda")
    hy.hydro_mhd_cfl_dt(ctx, a, dx, dts[0:1])
    for i in range(warmup):
        hy.hydro_mhd_step(ctx, a, b, dx, dts[i:i + 1], dts[i + 1:i + 2])
        a, b = b, a
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        k = warmup + i
        hy.hydro_mhd_step(ctx, a, b, dx, dts[k:k + 1], dts[k + 1:k + 2])
        a, b = b, a
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    rc, bits = hy.hydro_get_error(ctx)
    k = warmup + steps
    hy.hydro_mhd_step(ctx, a, b, dx, dts[k:k + 1])
    torch.cuda.synchronize()
    record_cells(("mhd_256_" + precision,), "mhd", a, b, dx, dts[k].item(), "minmod", count=300, seed=51)
    hbm, src = peaks()
    es = 4 if precision == "fp32" else 8
    fused = precision in ("fp32", "mixed")
    out = {"cells": n ** 3, "steps": steps, "ms_per_step": ms, "mcell_updates_per_s": n ** 3 / (ms / 1e3) / 1e6,
           "hbm_frac": n ** 3 * 2 * 9 * es / (ms / 1e3) / 1e9 / hbm, "launches_per_step": 2 if fused else 4,
           "error_bits": bits,
           "note": ("the step's constants, then one fused tile kernel (32x8 columns marching in z through "
                    "shared memory, fused dt), no per-cell scratch" if fused else
                    "the step's constants, then three kernels (predict, face fluxes, update + fused dt) with "
                    "81 scratch elements per cell")}
    del a, b
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_mhd_patches(hy, precision, steps, warmup, npatch=512):
    """MHD on AMR patches (two ghost layers, the patch-size mix of the batched hydro form, cut from
    a 256^3 magnetised-gas parent), one batched call per step, per-patch dt and fused dt_next."""
    import workloads
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision=precision, limiter="minmod")
    dtype = torch.float32 if precision == "fp32" else torch.float64
    parent = workloads.mhd_state(256, seed=7, beta=0.5, mach=2.0, device="cuda").to(dtype)
    descs = workloads.patch_set(npatch, seed=3)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=3)
    ins, outs, keep = [], [], []
    interior = 0
    _, NZ, NY, NX = parent.shape
    for d, o in zip(descs, origins):
        ix = (torch.arange(o[0] - 2, o[0] + d["nx"] + 2, device="cuda") % NX)
        iy = (torch.arange(o[1] - 2, o[1] + d["ny"] + 2, device="cuda") % NY)
        iz = (torch.arange(o[2] - 2, o[2] + d["nz"] + 2, device="cuda") % NZ)
        Ug = parent[:, iz][:, :, iy][:, :, :, ix].contiguous()
        Vg = torch.empty_like(Ug)
        keep += [Ug, Vg]
        ins.append(hy.MhdPatch(Ug, 2, d["dx"], d["level"]))
        outs.append(hy.MhdPatch(Vg, 2, d["dx"], d["level"]))
        interior += d["nx"] * d["ny"] * d["nz"]
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    dn = torch.empty_like(dt)
    hy.hydro_mhd_cfl_patches(ctx, ins, dt)
    for _ in range(warmup):
        hy.hydro_mhd_step_patches(ctx, ins, outs, dt, dn)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        hy.hydro_mhd_step_patches(ctx, ins, outs, dt, dn)  # same input each step: the per-patch dt stays valid
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    rc, bits = hy.hydro_get_error(ctx)
    # sampled cells of sampled patches: each cell's 5^3 neighbourhood inside its ghosted input
    import numpy as np
    rng_s = np.random.default_rng(53)
    dth = dt.cpu().numpy()
    nbs, got, dxs, dtl = [], [], [], []
    for i in sorted(int(i) for i in rng_s.choice(len(ins), 12, replace=False)):
        Ug, Vg = keep[2 * i], keep[2 * i + 1]
        d = descs[i]
        for _ in range(25):
            x, y, z = (int(rng_s.integers(0, m)) for m in (d["nx"], d["ny"], d["nz"]))
            nbs.append(Ug[:, z:z + 5, y:y + 5, x:x + 5].double().cpu().numpy())
            got.append(Vg[:, z + 2, y + 2, x + 2].double().cpu().numpy())
            dxs.append(d["dx"])
            dtl.append(float(dth[i]))
    for dxv in sorted(set(dxs)):  # one record per cell size (the oracle takes one dx per record)
        idx = [j for j, v in enumerate(dxs) if v == dxv]
        CHECKS.append({"path": ("mhd_patches_fp32",), "scheme": "mhd", "inputs": np.stack([nbs[j] for j in idx]),
                       "got": np.stack([got[j] for j in idx]), "dx": dxv, "dt": [dtl[j] for j in idx],
                       "limiter": "minmod", "what": "%d sampled cells of 12 patches" % len(nbs)})
    out = {"patches": len(ins), "interior_cells": interior, "ms_per_step": ms,
           "mcell_updates_per_s": interior / (ms / 1e3) / 1e6,
           "launches_per_step": 2 if precision in ("fp32", "mixed") else 4, "error_bits": bits,
           "note": "MHD on the first 512 patches of the batched hydro form's patch set, two ghost layers"
                   + ("; the step's constants, then one fused tile kernel over 32x8x32 tiles of every patch"
                      if precision in ("fp32", "mixed") else "")}
    del keep, parent
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_amr_level(hy, steps, warmup, n=256, pieces=16, seed=15):
    """One two-level AMR cycle, mixed precision: a 256^3 fine level tiled by 16^3 patches of random
    even edges (cuts at random even positions per axis) over a 128^3 coarse level.  Per cycle: the
    coarse step with the flux registers of the coarse boxes under the patches; fine ghosts
    prolonged from the coarse level and exchanged between siblings; the fine patches' registers
    and their batched step; refluxing and average-down onto the coarse level (one fine substep per
    coarse step here: the kernels' costs, not a time-refinement schedule)."""
    import numpy as np
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision="mixed")
    coarse = turbulent(n // 2, "mixed", "cuda", seed=seed, sedov=False)
    fine = turbulent(n, "mixed", "cuda", seed=seed + 1, sedov=False)
    rng = np.random.default_rng(seed)
    axes = []
    for _ in range(3):
        c = 2 * np.sort(rng.choice(np.arange(1, n // 2), pieces - 1, replace=False))
        e = np.concatenate([[0], c, [n]])
        axes.append(list(zip(e[:-1].tolist(), np.diff(e).tolist())))
    ins, outs, keep, origins = [], [], [], []
    interior = 0
    for z0, nz in axes[2]:
        for y0, ny in axes[1]:
            for x0, nx in axes[0]:
                Ug = torch.zeros((5, nz + 4, ny + 4, nx + 4), dtype=torch.float64, device="cuda")
                Ug[:, 2:-2, 2:-2, 2:-2] = fine[:, z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
                Vg = torch.empty_like(Ug)
                keep += [Ug, Vg]
                ins.append(hy.patch(Ug, 2, 1.0 / n))
                outs.append(hy.patch(Vg, 2, 1.0 / n))
                origins.append((x0, y0, z0))
                interior += nx * ny * nz
    del fine
    cp = hy.patch(coarse, 0, 2.0 / n)
    coarse2 = torch.empty_like(coarse)
    cp2 = hy.patch(coarse2, 0, 2.0 / n)
    per = (n, n, n)
    boxes_o = [(o[0] // 2, o[1] // 2, o[2] // 2) for o in origins]
    boxes_n = [(p.c.nx // 2, p.c.ny // 2, p.c.nz // 2) for p in ins]
    rc_regs = [torch.zeros(5 * hy.register_size(*b), dtype=torch.float64, device="cuda") for b in boxes_n]
    rf_regs = [torch.zeros(5 * hy.register_size(p.c.nx, p.c.ny, p.c.nz), dtype=torch.float64, device="cuda")
               for p in ins]
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    dtc = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_fill_ghosts(ctx, cp, ins, origins)
    hy.hydro_exchange_ghosts(ctx, ins, origins, per)
    hy.hydro_cfl_dt(ctx, ins, dt)
    hy.hydro_cfl_dt(ctx, cp, dtc)
    if TUNING == "auto":
        hy.hydro_autotune(ctx, ins, outs, dt)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    names = ["coarse_registers", "coarse_step", "fill_from_coarse", "exchange", "fine_registers", "fine_step",
             "reflux_and_average_down"]
    # the C calls with their arguments marshalled once (the 4096-patch ctypes arrays would
    # otherwise cost the host milliseconds per call, and the GPU would wait for them)
    L, H = hy.lib(), ctx.handle
    cpc, cp2c = ctypes.byref(cp.c), ctypes.byref(cp2.c)
    ins_a, npat = hy._parray(ins)
    outs_a, _ = hy._parray(outs)
    org_i, bo_i, bn_i = hy._ints(origins), hy._ints(boxes_o), hy._ints(boxes_n)
    rc_p, rf_p = hy._ptrs(rc_regs), hy._ptrs(rf_regs)
    per_i = (ctypes.c_int * 3)(*per)
    dt_p, dtc_p = dt.data_ptr(), dtc.data_ptr()

    def chk(rc):
        if rc != hy.HYDRO_OK:
            raise RuntimeError("AMR cycle call failed: %d" % rc)

    def one():
        ev[0].record(stream)
        chk(L.hydro_level_fluxes(H, cpc, bo_i, bn_i, npat, dtc_p, rc_p, 0))
        ev[1].record(stream)
        chk(L.hydro_step(H, cpc, cp2c, 1, dtc_p, None))
        ev[2].record(stream)
        chk(L.hydro_fill_ghosts(H, cpc, ins_a, org_i, npat))
        ev[3].record(stream)
        chk(L.hydro_exchange_ghosts(H, ins_a, org_i, npat, per_i))
        ev[4].record(stream)
        chk(L.hydro_patch_fluxes(H, ins_a, npat, dt_p, rf_p, 0))
        ev[5].record(stream)
        chk(L.hydro_step(H, ins_a, outs_a, npat, dt_p, None))
        ev[6].record(stream)
        chk(L.hydro_reflux(H, cp2c, bo_i, bn_i, npat, rc_p, rf_p))
        chk(L.hydro_average_down(H, cp2c, outs_a, org_i, npat))
        ev[7].record(stream)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    parts = np.zeros(7)
    for _ in range(steps):
        one()
        torch.cuda.synchronize()
        parts += [ev[i].elapsed_time(ev[i + 1]) for i in range(7)]
    parts /= steps
    rng_s = np.random.default_rng(47)
    dth = dt.cpu().numpy()
    picks = sorted(int(i) for i in rng_s.choice(len(ins), 10, replace=False))
    record_boxes(("amr_level_mixed",), "plm",
                 [(keep[2 * i].cpu().numpy(), keep[2 * i + 1][:, 2:-2, 2:-2, 2:-2].cpu().numpy(), 1.0 / n,
                   float(dth[i])) for i in picks], "minmod",
                 "the fine step of %d whole patches (ghosts prolonged and exchanged on the GPU)" % len(picks))
    ghosts = sum(t[0].numel() for t in keep[0::2]) - interior
    rc, bits = hy.hydro_get_error(ctx)
    t, z = hy.hydro_get_tuning(ctx)
    out = {"patches": len(ins), "fine_interior_cells": interior, "coarse_cells": (n // 2) ** 3,
           "ghost_cells": ghosts, "ms": {k: round(v, 4) for k, v in zip(names, parts)},
           "mcell_updates_per_s": (interior + (n // 2) ** 3) / (parts.sum() / 1e3) / 1e6,
           "fine_step_only_mcell_updates_per_s": interior / (parts[5] / 1e3) / 1e6,
           "tuning": {"tile": TILE_NAMES[t], "zchunk": z}, "error_bits": bits}
    del keep, coarse, coarse2
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()
    return out


def form_adjoint(hy, precision, n=64, nsteps=40):
    """Adjoint/forward time ratio on the 64^3 periodic grid (one step each, and the 40-step
    checkpointed gradient against the 40-step forward)."""
    from paper_1412_0934_gb300 import autograd as hag
    import workloads
    stream = torch.cuda.current_stream()
    dtype = torch.float32 if precision == "fp32" else torch.float64
    ctx = hy.hydro_init(precision=precision)
    U = workloads.turbulent_state(n, seed=4, mach=2.0, sedov=False, device="cuda").to(dtype).contiguous()
    V = torch.empty_like(U)
    L = torch.randn(U.shape, dtype=dtype, device="cuda")
    M = torch.empty_like(U)
    dx = 1.0 / n
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(ctx, hy.patch(U, 0, dx), dt)
    pU, pV, pL, pM = (hy.patch(t, 0, dx) for t in (U, V, L, M))
    hy.hydro_autotune(ctx, pU, pV, dt)  # the forward at its best tile shape for this grid
    reps = 50
    for _ in range(5):
        hy.hydro_step(ctx, pU, pV, dt)
        hy.hydro_adjoint_step(ctx, pU, dt, pL, pM)
    torch.cuda.synchronize()
    t0, t1, t2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t0.record(stream)
    for _ in range(reps):
        hy.hydro_step(ctx, pU, pV, dt)
    t1.record(stream)
    for _ in range(reps):
        hy.hydro_adjoint_step(ctx, pU, dt, pL, pM)
    t2.record(stream)
    torch.cuda.synchronize()
    f_ms, a_ms = t0.elapsed_time(t1) / reps, t1.elapsed_time(t2) / reps
    CHECKS.append({"path": ("adjoint_" + precision,), "scheme": "adjoint", "U": U.double().cpu().numpy(),
                   "lam_out": L.double().cpu().numpy(), "got": M.double().cpu().numpy(), "dx": dx, "dt": dt.item(),
                   "limiter": "minmod",
                   "what": "one adjoint step of the whole %d^3 grid (the 40-step checkpointed gradient is "
                           "compared with the oracle's chained adjoint in tests/test_gpu_adjoint.py)" % n})
    # 40-step run: forward only vs forward + checkpointed gradient
    W = workloads.turbulent_state(n, seed=4, mach=2.0, sedov=False, device="cuda")
    rho0 = (W[0]).to(dtype).requires_grad_(True)
    vel0 = (W[1:4] / W[0]).to(dtype).requires_grad_(True)
    p0 = ((2.0 / 3.0) * (W[4] - 0.5 * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / W[0])).to(dtype)
    target = torch.ones_like(rho0)
    sim = hag.Simulation(ctx, (n, n, n), dx, nsteps=nsteps, checkpoint_every=8)

    def grad_run():
        rho0.grad, vel0.grad = None, None
        loss = ((sim(rho0, vel0, p0) - target) ** 2).sum()
        loss.backward()

    with torch.no_grad():
        sim.forward_only(rho0, vel0, p0)
    grad_run()  # warm-up: the autograd graph and the allocator's blocks
    torch.cuda.synchronize()
    runs = 3
    t0.record(stream)
    with torch.no_grad():
        for _ in range(runs):
            sim.forward_only(rho0, vel0, p0)
    t1.record(stream)
    for _ in range(runs):
        grad_run()
    t2.record(stream)
    torch.cuda.synchronize()
    fwd40, grad40 = t0.elapsed_time(t1) / runs, t1.elapsed_time(t2) / runs
    rc, bits = hy.hydro_get_error(ctx)
    t, z = hy.hydro_get_tuning(ctx)
    hy.hydro_finalize(ctx)
    return {"n": n, "forward_tuning": [t, z], "forward_ms": f_ms, "adjoint_ms": a_ms, "adjoint_over_forward": a_ms / f_ms,
            "steps40_forward_ms": fwd40, "steps40_forward_plus_gradient_ms": grad40,
            "gradient_over_forward_40": grad40 / fwd40, "error_bits": bits}


def cpu_baseline(n, seconds, steps_cap=1000):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same workload (an n^3 box of
    the same distributions), timed on this host's cores."""
    import numpy as np
    import oracle
    import workloads
    U = workloads.turbulent_state(n, seed=2, mach=5.0, sedov=True).numpy()
    dx = 1.0 / n
    cfg = oracle.config()
    t0 = time.perf_counter()
    steps = 0
    while steps < steps_cap and (time.perf_counter() - t0) < seconds:
        dt = oracle.cfl_periodic(U, dx, cfg)
        U = oracle.step_periodic(U, dx, dt, cfg)
        steps += 1
    el = time.perf_counter() - t0
    threads = oracle.threads()
    return {"value": n ** 3 * steps / el / 1e6, "unit": "Mcell-updates/s", "cores": threads, "kind": "oracle",
            "sample": "%d^3 box of the same workload (lognormal rho, k^-4 Mach-5 velocities, P/rho=1e-4, Sedov "
                      "cell), %d FP64 steps incl. CFL dt, %.1f s" % (n, steps, el)}


def cpu_oracle_leg(line, seconds):
    """The leg of the run that executes the CPU oracle, after every timed region: its timed baseline
    (cpu_baseline) and its outputs for the samples each form recorded, whose errors it attaches
    (err_vs_oracle of the headline and of each form)."""
    line["cpu_baseline"] = cpu_baseline(128, seconds)
    try:
        errs = oracle_errors(CHECKS)
    except Exception as e:  # reported, not fatal
        line["err_vs_oracle"] = {"error": repr(e)[:300]}
        return
    forms = line.get("forms", {})
    for path, e in errs.items():
        if path == ("headline",):
            line["err_vs_oracle"] = e
            continue
        node = forms.get(path[0])
        for k in path[1:]:
            node = node.get(k) if isinstance(node, dict) else None
        if isinstance(node, dict):
            node["err_vs_oracle"] = e


# ----------------------------------------------------------------------------- arms
def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle  # the reference arm is the CPU oracle
    import workloads
    n = 96
    # the sample is generated outside the timed region; each step is the oracle's CFL dt and step
    U = workloads.turbulent_state(n, seed=2, mach=5.0, sedov=True).numpy()
    dx = 1.0 / n
    cfg = oracle.config()

    def step(U):
        return oracle.step_periodic(U, dx, oracle.cfl_periodic(U, dx, cfg), cfg)

    for _ in range(args.warmup):
        U = step(U)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = step(U)
    el = time.perf_counter() - t0
    threads = oracle.threads()
    value = n ** 3 * args.steps / el / 1e6
    line = {"impl": "reference", "metric": "Mcell-updates/s per hydro step (1 GB300)", "value": value,
            "unit": "Mcell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle; each step one %d^3 sample of the 512^3 periodic Mach-5 k^-4 "
                                   "turbulence box (lognormal rho sigma 1, P/rho 1e-4, Sedov cell), MinMod, CFL 0.8"
                                   % n},
            "cpu_baseline": {"value": value, "unit": "Mcell-updates/s", "cores": threads, "kind": "oracle",
                             "sample": "%d^3 box of the headline workload, stepped on (CFL dt included); the "
                                       "state generated before the timed steps" % n},
            "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_forms(hy, args, n, precision):
    """The extra forms beside the headline (each failure reported, not fatal)."""
    forms = [] if args.forms == "none" else (
        ["fp64", "fp32", "mixed", "ppm", "mhd", "batched", "amr", "adjoint", "graph1024"] if args.forms == "all"
        else args.forms.split(","))
    forms = [f for f in forms if f != precision]
    extra = {}
    for f in forms:
        try:
            if f in ("fp32", "mixed"):
                extra[f + "_512"] = form_uniform(hy, n, f, "minmod", args.steps, args.warmup, "turb_minmod",
                                                 path=(f + "_512",))
            elif f == "fp64_256":
                extra["fp64_256"] = form_uniform(hy, 256, "fp64", "minmod", args.steps, args.warmup,
                                                 "turb_minmod", path=("fp64_256",))
            elif f in ("fp64", "df64"):
                extra[f + "_512"] = form_uniform(hy, n, f, "minmod", args.steps, args.warmup, "turb_minmod",
                                                 path=(f + "_512",))
            elif f == "batched":
                extra["mixed_batched"] = form_batched(hy, max(3, args.steps // 2), 2, npatch=args.npatch,
                                                      ngroups=args.ngroups)
            elif f == "adjoint":
                for prec in args.adj_precisions.split(","):
                    extra["adjoint_" + prec] = form_adjoint(hy, prec, n=args.adj_n)
            elif f == "amr":
                extra["amr_level_mixed"] = form_amr_level(hy, max(3, args.steps // 2), 2)
            elif f == "ppm":
                for prec in ("df64", "fp32"):
                    key = "ppm_%d_%s" % (n, prec)
                    extra[key] = form_uniform(hy, n, prec, "ppm", args.steps, args.warmup, None, path=(key,))
                extra["ppm_batched_mixed"] = form_ppm_batched(hy, max(3, args.steps // 2), 2, npatch=args.npatch)
            elif f == "mhd":
                for prec in args.mhd_precisions.split(","):
                    extra["mhd_256_" + prec] = form_mhd(hy, prec, args.steps, args.warmup)
                if "fp32" in args.mhd_precisions.split(","):
                    extra["mhd_patches_fp32"] = form_mhd_patches(hy, "fp32", max(3, args.steps // 2), 2)
            elif f == "graph1024":
                extra["graph_1024_fp32_mc"] = form_uniform(hy, 1024, "fp32", "mc", 20, 0, "mach10_mc", mach=10.0,
                                                           sigma=1.5, p_over_rho=1e-5, sedov=False, seed=5,
                                                           graph=True, path=("graph_1024_fp32_mc",))
        except Exception as e:  # a failing extra form is reported, not fatal
            extra[f] = {"error": repr(e)[:300]}
    return extra


def main():
    global TUNING
    args = parse()
    TUNING = args.tuning
    if args.impl == "reference":
        return reference_arm(args)
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1412_0934_gb300 as hy

    precision = args.precision
    n = args.n
    if args.forms_only:
        print(json.dumps(run_forms(hy, args, n, precision)), flush=True)
        return 0
    dx = 1.0 / n
    cells = n ** 3
    stream = torch.cuda.current_stream()
    ctx = hy.hydro_init(precision=precision, limiter="minmod")
    a = turbulent(n, precision, "cuda")
    b = torch.empty_like(a)
    dts = torch.empty(args.warmup + args.steps + 1, dtype=torch.float64, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    tuning = tune(hy, ctx, a, b, dx, dts)
    barrier()
    with ClockSampler(local) as clk:
        ms, per, final, launches = time_steps(hy, ctx, a, b, dx, dts, args.steps, args.warmup, stream)
    barrier()
    rc, bits = hy.hydro_get_error(ctx)
    if rc != hy.HYDRO_OK:
        print("device error bits %#x" % bits, file=sys.stderr)
    if rank == 0:  # one more step at the timed tuning, sampled for the CPU oracle leg
        record_step(hy, ctx, final, b if final is a else a, dx, dts[args.warmup + args.steps:], ("headline",), "plm",
                    "minmod", count=1000)
    t_max = job_time_ms(ms, world, "cuda")
    value = job_value(cells, args.steps, world, t_max)
    hbm, src = peaks()
    traffic, tsrc = profile_traffic("step_uniform_512_%s.txt" % precision)
    roof = roofline(precision, cells, per, ALG_FLOPS_PER_CELL["turb_minmod"], hbm, src, traffic)
    roof["traffic_source"] = tsrc

    # end to end through the C ABI with the state in (page-locked) host memory: hydro_step_host
    # copies the state in, steps it and copies the result out every step, pipelined over z slabs;
    # host buffers ping-pong, each step's dt is the fused CFL dt of the previous step's result.
    e2e_steps = 12
    esz = a.element_size()
    hbuf = [torch.empty(a.shape, dtype=a.dtype, pin_memory=True) for _ in range(2)]  # page-locked, no staging copy
    hbuf[0].copy_(a)
    hd = torch.empty(e2e_steps + 2, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(ctx, hy.patch(a, 0, dx), hd[0:1])
    hy.hydro_step_host(ctx, hy.host_patch(hbuf[0], dx), hy.host_patch(hbuf[1], dx), hd[0:1], hd[1:2])  # warm-up
    hbuf.reverse()
    barrier()
    e2e_ms = []
    for k in range(1, e2e_steps + 1):
        t0 = time.perf_counter()
        hy.hydro_step_host(ctx, hy.host_patch(hbuf[0], dx), hy.host_patch(hbuf[1], dx), hd[k:k + 1], hd[k + 1:k + 2])
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        hbuf.reverse()
    barrier()
    e2e = e2e_summary(e2e_ms, world * cells)
    e2e.update({"h2d_bytes_per_step": 5 * (n + 2) * n * n * esz, "d2h_bytes_per_step": 5 * cells * esz,
                "note": "hydro_step_host: state in page-locked host memory, copied in (plus 2 wrap planes) and out "
                        "every step, overlapped with the step kernel over z slabs; wall clock of each step "
                        "(host call to synchronize); value from the median step, mean_value from the mean (the "
                        "host link of this shared machine stalls now and then for a few hundred ms)"})
    del hbuf, a, b, final
    hy.hydro_finalize(ctx)
    torch.cuda.empty_cache()

    line = {"metric": "Mcell-updates/s per hydro step (1 GB300)", "value": round(value, 2),
            "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "f64-state/f32",
                      "df64": "f64 state, double-float (f32 pair) arithmetic"}[precision],
            "data": "synthetic",
            "config": {"workload": "%d^3 periodic uniform grid, Gaussian k^-4 velocities at rms Mach 5, lognormal rho "
                                   "(sigma 1), P/rho = 1e-4, Sedov cell E=1; MinMod PLM + HLLC, CFL 0.8, gamma 5/3; "
                                   "%s; dt from the fused CFL of each step" % (n, PRECISION_TEXT[precision]),
                       "parity": PARITY_TEXT[precision],
                       "cells": cells, "state_bytes": 5 * cells * esz,
                       "l2": "inputs larger than L2 (state %.1f GB vs 129 MB L2); no flush" % (5 * cells * esz / 1e9),
                       "parallelism": "replicas x%d" % world, "tuning": tuning},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "device_error_bits": bits}

    if rank == 0:
        extra = run_forms(hy, args, n, precision)
        line["forms"] = extra
        if args.cpu_seconds > 0:
            cpu_oracle_leg(line, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
