"""Benchmark of the fused rrBGK stream+collide update on GB300.

Default workload: the D3Q19 round jet, 384 x 256 x 256 cells, FP32 population
storage (top-hat velocity inflow of diameter 24 at Ma 0.3 with 1% seeded
noise, ambient at rest, 32-cell sponges and zero-gradient outflow on the five
open faces, tau for Re_D = 1e4).  One "step" is one time step of the whole
lattice: one launch of the fused kernel.

Prints one JSON line (rank 0).  `value` is whole-job MLUPS (cells x steps /
s) with the populations resident in HBM; `e2e` is the same metric through
the public C ABI with host buffers (initial rho, u uploaded and final rho, u
read back inside the timed region).  `roofline` reports the fused kernel's
algorithmic HBM bandwidth (2 Q s bytes per cell update) against the measured
copy bandwidth.  `cpu_baseline` times the FP64 CPU oracle on a bounded sample.

--impl reference times the FP64 CPU oracle itself on that sample.
--gpus N under torchrun runs N independent replicas (one solve per GPU; a
single solve is not sharded), weak scaling, max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline, D3Q19 regularized LBM; FP16-store speedup; p99 latency"
CS = 1.0 / math.sqrt(3.0)


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def jet_spec(nx=384, ny=256, nz=256, diameter=24.0, sponge=32, Ma=0.3, Re=1e4, chi=0.5, seed=3,
             noise=0.01):
    """The round jet: top-hat inflow (tanh shear layer of momentum thickness
    R/20), Ma 0.3, Re_D, 1% seeded inlet noise, sponges chi_max 0.5."""
    U = Ma * CS
    tau = 3 * U * diameter / Re + 0.5
    return dict(n=(nx, ny, nz), diameter=diameter, sponge=sponge, U=U, tau=tau, chi=chi, seed=seed,
                noise=noise, theta=diameter / 40.0, lattice=1)


def jet_workload_name(nx, ny, nz, lattice="D3Q19"):
    """The workload both benchmark arms name in their config."""
    return (f"{lattice} round jet {nx}x{ny}x{nz}, Re_D 1e4, Ma 0.3, two-lattice pull, fused inflow/outflow/sponge "
            "(storage precision in config.storage)")


def configure_gpu(lbm, spec, precision, stream):
    from paper_1710_02065_gb300 import inputs
    nx, ny, nz = spec["n"]
    s = lbm.Solver(spec.get("lattice", lbm.LBM_D3Q19), spec["n"], spec["tau"], precision, Ma_ref=0.3, stream=stream)
    prof = inputs.top_hat_profile(ny, nz, ny / 2, nz / 2, spec["diameter"] / 2, spec["U"], spec["theta"])
    lbm.lbm_set_boundary(s.h, lbm.LBM_FACE_XM, lbm.LBM_BC_VELOCITY, None, prof)
    for f in range(1, 6):
        lbm.lbm_set_boundary(s.h, f, lbm.LBM_BC_OUTFLOW)
        lbm.lbm_set_sponge(s.h, f, spec["sponge"], spec["chi"], 1.0, (0.0, 0.0, 0.0))
    lbm.lbm_set_inlet_noise(s.h, spec["seed"], spec["noise"])
    return s


def configure_oracle(spec):
    import oracle
    from paper_1710_02065_gb300 import inputs
    nx, ny, nz = spec["n"]
    P = oracle.Problem(oracle.D3Q19, spec["n"], spec["tau"])
    prof = inputs.top_hat_profile(ny, nz, ny / 2, nz / 2, spec["diameter"] / 2, spec["U"], spec["theta"])
    P.set_boundary(0, oracle.VELOCITY, (0, 0, 0), prof)
    for f in range(1, 6):
        P.set_boundary(f, oracle.OUTFLOW)
        P.set_sponge(f, spec["sponge"], spec["chi"], 1.0, (0, 0, 0))
    P.noise_seed, P.noise_amp = spec["seed"], spec["noise"]
    n = P.ncell
    f = P.equilibrium(np.ones(n), np.zeros((n, 3)))
    return P, f


SAMPLE_SPEC = dict(nx=96, ny=64, nz=64, diameter=6.0, sponge=8)  # the jet scaled by 1/4
REF_SAMPLE_SPEC = dict(nx=64, ny=48, nz=48, diameter=4.5, sponge=6)  # about 0.3 s per oracle step


def time_oracle(max_seconds=15.0, max_steps=40, min_steps=2):
    """MLUPS of the FP64 CPU oracle (one thread) on the jet scaled to 96 x 64 x 64."""
    spec = jet_spec(**SAMPLE_SPEC)
    P, f = configure_oracle(spec)
    f = P.run(f, 1)  # warm-up (builds the oracle)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps and (steps < min_steps or time.perf_counter() - t0 < max_seconds):
        f = P.run(f, 1, step0=1 + steps)
        steps += 1
    dt = time.perf_counter() - t0
    mlups = P.ncell * steps / dt / 1e6
    return mlups, steps, dt, P.ncell


def _oracle_replica(steps):
    """One independent oracle solve of the 96 x 64 x 64 sample (a pool worker)."""
    spec = jet_spec(**SAMPLE_SPEC)
    P, f = configure_oracle(spec)
    f = P.run(f, 1)
    t0 = time.perf_counter()
    f = P.run(f, steps, step0=1)
    return P.ncell, steps, t0, time.perf_counter()


def time_oracle_all_cores(cores=None, steps=6):
    """Aggregate MLUPS of `cores` independent single-threaded oracle solves
    running at once (one per host core; spawned processes, so it is safe after
    CUDA initialisation).  The oracle itself is unchanged: this is replica
    throughput, the way the host would run many independent problems."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_replica, [steps] * cores)
    t0 = min(r[2] for r in res)
    t1 = max(r[3] for r in res)
    cells = sum(r[0] * r[1] for r in res)
    return cells / (t1 - t0) / 1e6, cores, steps, t1 - t0


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # nvidia-smi needs a moment before its first sample
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("rr.cuh", "step.cuh", "step_vec.cuh", "step_rows.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1710_02065_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == src:
            return float(parts[2])
    return None


def recorded_fp64_inst(kernel_key: str):
    """(FP64 thread instructions, FP64 flops) per cell from the committed ncu
    counts, if they were taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_fp64_inst.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel_key and parts[1] == src:
            return float(parts[2]), float(parts[3])
    return None


# GB300 FP64: 1.25 TFLOP/s nominal = 625 G FMA instructions/s (no measured FP64 peak is available)
FP64_INST_PEAK_G = 625.0


def issue_peak_g(sm_mhz=None):
    """Warp instructions per second the SMs can issue (G/s): 152 SMs x 4
    schedulers x one warp instruction per cycle at the SM clock sampled during
    the timed region (the 2070 MHz maximum when no sample exists)."""
    return 152 * 4 * (sm_mhz or 2070.0) / 1e3


def recorded_issue(kernel_key: str, grid: str):
    """Warp instructions per cell from the committed ncu counts, if taken on
    the current kernel source and on the same grid (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_issue.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel_key and parts[1] == src and parts[2] == grid:
            return float(parts[3])
    return None


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(v: float, pg, world: int) -> float:
    if pg is None or world == 1:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ---------------------------------------------------------------------------
# timing of one precision
# ---------------------------------------------------------------------------
def time_precision(lbm, torch, spec, precision, steps, warmup, pg, stream, tune=True, launch=None):
    """launch: a fixed (kind, knob) candidate instead of tuning, e.g. ("cell", 64)."""
    from paper_1710_02065_gb300 import autotune
    s = configure_gpu(lbm, spec, precision, stream.cuda_stream)
    n = s.ncell
    s.set_state(np.ones(n), np.zeros((n, 3)))
    tuned = {}
    if launch is not None:
        if not autotune.apply(s.h, launch):
            raise SystemExit(f"--launch {launch[0]}:{launch[1]} does not apply to this lattice / size")
    elif tune:
        tuned = autotune.autotune(s.h, precision, stream, steps=5, torch=torch)[1]
    launch = autotune.describe(s.h)
    lbm.lbm_step(s.h, warmup)
    s.sync()
    info0 = s.info()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    barrier(pg)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            lbm.lbm_step(s.h, 1)
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total_ms = ev[0].elapsed_time(ev[steps])
    info1 = s.info()
    m, j, rc = s.reduce()
    s.close()
    return dict(total_ms=total_ms, per_ms=per, launches=info1["launches"] - info0["launches"],
                bytes_per_cell=info1["bytes_per_cell"], ncell=n, stable=(rc == 0),
                launch=launch, tuning={k: round(ms, 4) for k, ms in tuned.items()})


def e2e_run(lbm, torch, spec, precision, steps, stream):
    """Through the public API with host buffers: upload rho, u from pinned
    memory, advance `steps`, read rho, u back.  FP32 and 16-bit storage move
    FP32 host arrays (lbm_set_state_f32 / lbm_moments_f32: their populations
    carry FP32 precision at most), FP64 storage FP64 arrays."""
    s = configure_gpu(lbm, spec, precision, stream.cuda_stream)
    n = s.ncell
    f32 = precision != lbm.LBM_FP64
    dt = torch.float32 if f32 else torch.float64
    rho_t = torch.ones(n, dtype=dt).pin_memory()
    u_t = torch.zeros((n, 3), dtype=dt).pin_memory()
    rho_o = torch.empty(n, dtype=dt).pin_memory()
    u_o = torch.empty((n, 3), dtype=dt).pin_memory()
    rho, u, ro, uo = rho_t.numpy(), u_t.numpy(), rho_o.numpy(), u_o.numpy()
    up = (lambda: lbm.lbm_set_state_f32(s.h, rho, u)) if f32 else (lambda: s.set_state(rho, u))
    down = (lambda: lbm.lbm_moments_f32(s.h, ro, uo, None)) if f32 else (lambda: lbm.lbm_moments(s.h, ro, uo, None))
    # one untimed pass to page everything in
    up()
    lbm.lbm_step(s.h, 2)
    down()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    up()  # returns once the field is written (it checks the values)
    t1 = time.perf_counter()
    lbm.lbm_step(s.h, steps)
    down()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s.close()
    return dict(seconds=t2 - t0, upload_s=t1 - t0, h2d=(rho.nbytes + u.nbytes) / steps,
                d2h=(ro.nbytes + uo.nbytes) / steps, host_dtype="fp32" if f32 else "fp64")


def _pprime_compare(runs, checkpoints, ref_name):
    out = {}
    for name in runs:
        if name == ref_name:
            continue
        out[name] = {}
        for c in checkpoints:
            ref = runs[ref_name][c]
            d = runs[name][c] - ref
            scale = np.abs(ref).max()
            out[name][str(c)] = {"max_rel": float(np.abs(d).max() / scale),
                                 "rms_rel": float(np.sqrt(np.mean(d * d)) / scale)}
    out["max_abs_p_ref"] = {str(c): float(np.abs(runs[ref_name][c]).max()) for c in checkpoints}
    return out


def _gpu_pprime(lbm, make, checkpoints):
    s = make()
    t, fields = 0, {}
    for c in checkpoints:
        lbm.lbm_step(s.h, c - t)
        t = c
        rho = np.zeros(s.ncell)
        lbm.lbm_moments(s.h, rho, None, None)
        fields[c] = (rho - 1.0) / 3.0
    s.close()
    return fields


def _oracle_pprime(P, f, checkpoints, threads):
    t, fields = 0, {}
    for c in checkpoints:
        f = P.run(f, c - t, step0=t, threads=threads)
        t = c
        rho, _, _ = P.moments(f)
        fields[c] = (rho - 1.0) / 3.0
    return fields


def pprime_errors(lbm, torch, stream, threads=None):
    """Error of p' = c_s^2 (rho - 1) for each storage precision against the FP64
    oracle (the reference, run on `threads` host threads -- bitwise the
    single-threaded oracle), with the GPU FP64 path as a second column:
      * the round jet scaled to 96x64x64 (D = 6, sponges 8, Ma 0.3) at Re_D
        1250 with a D/20 shear layer, at steps 100, 500, 1000 (at Re_D 2500,
        the full-size lattice viscosity, this copy leaves the stable range
        before step 1000); the ambient is at rest, so the default storage
        shift is the rest state already
      * the D2Q9 128^2 acoustic pulse (amplitude 1e-3, laminar, tau 0.6) on a
        mean flow u0 = (0.05, 0), steps 50 and 200; 16-bit storage with the
        default shift (f - w) and shifted by the mean-flow equilibrium
        (f - feqH(1, u0), lbm_set_storage_shift)"""
    threads = threads or os.cpu_count() or 1
    res = {"oracle_threads": threads}
    spec = jet_spec(Re=1250.0, **SAMPLE_SPEC)
    spec["theta"] = spec["diameter"] / 20.0
    cps = (100, 500, 1000)
    runs = {}
    for name in ("fp64", "fp32", "fp16", "bf16"):
        def make(name=name):
            s = configure_gpu(lbm, spec, lbm.PRECISIONS[name], stream.cuda_stream)
            s.set_state(np.ones(s.ncell), np.zeros((s.ncell, 3)))
            return s
        runs[name] = _gpu_pprime(lbm, make, cps)
    t0 = time.perf_counter()
    P, f = configure_oracle(spec)
    runs["oracle"] = _oracle_pprime(P, f, cps, threads)
    jet_s = time.perf_counter() - t0
    res["jet_96x64x64_Re1250"] = {
        "vs_oracle": _pprime_compare(runs, cps, "oracle"),
        "vs_gpu_fp64": _pprime_compare({k: v for k, v in runs.items() if k != "oracle"}, cps, "fp64"),
        "oracle_seconds": round(jet_s, 1)}
    from paper_1710_02065_gb300 import inputs
    import oracle
    u0 = (0.05, 0.0, 0.0)
    rho0, uu0 = inputs.gaussian_pulse_2d(128, 1e-3, 6.0, u0[:2])
    cps2 = (50, 200)
    runs = {}
    for name, shift in (("fp64", None), ("fp32", None), ("fp16", None), ("bf16", None),
                        ("fp16_shift_u0", u0), ("bf16_shift_u0", u0)):
        def make(name=name, shift=shift):
            s = lbm.Solver(lbm.LBM_D2Q9, (128, 128, 1), 0.6, lbm.PRECISIONS[name[:4]], stream=stream.cuda_stream)
            if shift is not None:
                lbm.lbm_set_storage_shift(s.h, shift)
            s.set_state(rho0, uu0)
            return s
        runs[name] = _gpu_pprime(lbm, make, cps2)
    P = oracle.Problem(oracle.D2Q9, (128, 128), 0.6)
    runs["oracle"] = _oracle_pprime(P, P.equilibrium(rho0, uu0), cps2, threads)
    res["acoustic_pulse_d2q9_128_u0.05"] = {
        "vs_oracle": _pprime_compare(runs, cps2, "oracle"),
        "vs_gpu_fp64": _pprime_compare({k: v for k, v in runs.items() if k != "oracle"}, cps2, "fp64")}
    res["reference"] = ("FP64 oracle (vs_oracle) and the GPU FP64 path (vs_gpu_fp64); errors relative to "
                        "max |p'| of the reference at that step; *_shift_u0: stored as f - feqH(1, u0)")
    return res


def stability_ab(lbm, stream, n=128, U=0.1, taus=(0.5001, 0.5002, 0.5005, 0.501, 0.502, 0.505)):
    """A/B of the collision models on the periodic double shear layer (D2Q9
    n^2, U = 0.1, kappa = 80, delta = 0.05, FP64 storage): for each tau the
    step at which the populations stop being finite (checked every n/U/8
    steps up to 2 n / U, two convective times), or None when the run stays
    finite.  Sec. I of the paper motivates rrBGK by the instability of the
    plain BGK at low viscosity."""
    from paper_1710_02065_gb300 import inputs as _inp
    rho0, u0 = _inp.double_shear_layer(n, U)
    horizon = int(round(2 * n / U))
    chunk = max(1, horizon // 16)
    out = {"workload": f"D2Q9 double shear layer {n}^2, U {U}, kappa 80, delta 0.05, FP64, {horizon} steps",
           "rrBGK": {}, "BGK": {}}
    for name, model in (("rrBGK", lbm.LBM_COLLISION_RR), ("BGK", lbm.LBM_COLLISION_BGK)):
        for tau in taus:
            s = lbm.Solver(lbm.LBM_D2Q9, (n, n, 1), tau, lbm.LBM_FP64, stream=stream.cuda_stream)
            lbm.lbm_set_collision(s.h, model)
            s.set_state(rho0, u0)
            t, failed = 0, None
            while t < horizon:
                lbm.lbm_step(s.h, chunk)
                t += chunk
                _, _, rc = s.reduce()
                if rc != 0:
                    failed = t
                    break
            out[name][str(tau)] = failed
            s.close()
    return out


# ---------------------------------------------------------------------------
# cylinder workloads (single level and 2:1 two-level) and serving
# ---------------------------------------------------------------------------
def strouhal(signal, dt_steps, D, U):
    """Dominant frequency of a lift signal (FFT peak with parabolic refinement),
    as St = f D / U with f in 1/steps."""
    x = np.asarray(signal) - np.mean(signal)
    n = len(x)
    win = np.hanning(n)
    spec = np.abs(np.fft.rfft(x * win, 8 * n))
    k = int(np.argmax(spec[1:])) + 1
    a, b, c = np.log(spec[k - 1] + 1e-300), np.log(spec[k] + 1e-300), np.log(spec[k + 1] + 1e-300)
    kk = k + 0.5 * (a - c) / (a - 2 * b + c)
    f = kk / (8 * n * dt_steps)
    return f * D / U


def record_series(lbm, torch, s, total, every, level, probes=None):
    """Advance `total` steps and record lift/drag of `level` (and p' at the
    probe cells) every `every` steps into device memory, read back once at the
    end: the samples are taken in stream order without host round trips.
    Returns (wall seconds, forces [n, 3], p' [n, len(probes)] or None)."""
    n = (total + every - 1) // every
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    P = torch.zeros((n, len(probes)), dtype=torch.float64, device="cuda") if probes else None
    cells = torch.tensor(probes, dtype=torch.int64, device="cuda") if probes else None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n):
        lbm.lbm_step(s.h, min(every, total - k * every))
        lbm.lbm_force_async(s.h, level, F[k].data_ptr())
        if probes:
            lbm.lbm_probe_async(s.h, len(probes), cells.data_ptr(), P[k].data_ptr())
    s.sync()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return wall, F.cpu().numpy(), (P.cpu().numpy() if probes else None)


def run_cylinder(lbm, torch, args):
    """Single-level D2Q9 cylinder: 1600x800, D = 40 at (400, 400), Ma 0.2,
    Re 150, inflow on -x, 100-cell sponge + zero-gradient outflow on +x, y
    periodic, +-1% seeded u_y at t = 0.  Lift and drag every 10 steps."""
    from paper_1710_02065_gb300 import inputs
    nx, ny, D = 1600, 800, 40.0
    U = 0.2 * CS
    tau = 3 * U * D / 150.0 + 0.5
    stream = torch.cuda.Stream()
    s = lbm.Solver(lbm.LBM_D2Q9, (nx, ny, 1), tau, lbm.PRECISIONS[args.precision], Ma_ref=0.2,
                   stream=stream.cuda_stream)
    solid = inputs.cylinder_mask(nx, ny, 400, 400, D)
    rho, u = inputs.uniform_flow_perturbed(nx, ny, U, 2)
    u[solid == 1] = 0.0
    lbm.lbm_set_boundary(s.h, 0, 1, (U, 0, 0))
    lbm.lbm_set_boundary(s.h, 1, 2)
    lbm.lbm_set_sponge(s.h, 1, 100, 0.5, 1.0, (U, 0, 0))
    lbm.lbm_set_geometry(s.h, solid)
    s.set_state(rho, u)
    total = args.cyl_steps
    every = 10
    probes = [400 + nx * 700, 1200 + nx * 400]
    wall, Fs, pp = record_series(lbm, torch, s, total, every, 0, probes)
    drag, lift = list(Fs[:, 0]), list(Fs[:, 1])
    _, _, rc = s.reduce()
    s.close()
    half = len(lift) // 2
    q = 0.5 * U * U * D
    return {"workload": "D2Q9 cylinder 1600x800, D=40, Ma 0.2, Re 150, single level", "steps": total,
            "St": strouhal(lift[half:], every, D, U), "Cd_mean": float(np.mean(drag[half:]) / q),
            "Cl_amplitude": float((np.max(lift[half:]) - np.min(lift[half:])) / 2 / q),
            "probe_pprime_rms": [float(np.std(np.array(pp)[half:, k])) for k in range(2)],
            "mlups_incl_sampling": nx * ny * total / wall / 1e6, "stable": rc == 0, "tau": tau}


def run_cylinder_two_level(lbm, torch, args):
    """2:1 two-level D2Q9 cylinder: coarse 800x400 (D_c = 20), fine patch over
    coarse [160, 480] x [120, 280] (641 x 321 fine nodes) holding the cylinder
    at coarse (200, 200) (D_f = 40), same Ma, Re, inflow, sponge (50 coarse
    cells) and seeds as the single-level run.  Lift/drag on the fine level."""
    from paper_1710_02065_gb300 import inputs
    nxc, nyc, Dc = 800, 400, 20.0
    Df = 2 * Dc
    U = 0.2 * CS
    tau_f = 3 * U * Df / 150.0 + 0.5
    tau_c = (tau_f + 0.5) / 2
    stream = torch.cuda.Stream()
    s = lbm.Solver(lbm.LBM_D2Q9, (nxc, nyc, 1), tau_c, lbm.PRECISIONS[args.precision], Ma_ref=0.2,
                   stream=stream.cuda_stream)
    lbm.lbm_set_boundary(s.h, 0, 1, (U, 0, 0))
    lbm.lbm_set_boundary(s.h, 1, 2)
    lbm.lbm_set_sponge(s.h, 1, 50, 0.5, 1.0, (U, 0, 0))
    rho, u = inputs.uniform_flow_perturbed(nxc, nyc, U, 2)
    s.set_state(rho, u)
    X0, Y0, Wc, Hc = 160, 120, 320, 160
    lbm.lbm_set_level_streams(s.h, args.level_streams)
    lbm.lbm_add_refinement_patch(s.h, (X0, Y0, 0), (Wc, Hc, 1))
    nfx, nfy = 2 * Wc + 1, 2 * Hc + 1
    solid_f = inputs.cylinder_mask(nfx, nfy, 2 * (200 - X0), 2 * (200 - Y0), Df)
    rho_f, u_f = inputs.uniform_flow_perturbed(nfx, nfy, U, 3)
    u_f[solid_f == 1] = 0.0
    lbm.lbm_set_geometry_level(s.h, 1, solid_f)
    lbm.lbm_set_state_level(s.h, 1, rho_f, u_f)
    lbm.lbm_set_state(s.h, rho, u)
    total = args.cyl_steps // 2  # coarse steps covering the same physical time
    every = 5
    wall, Fs, _ = record_series(lbm, torch, s, total, every, 1)
    drag, lift = list(Fs[:, 0]), list(Fs[:, 1])
    _, _, rc = s.reduce()
    s.close()
    half = len(lift) // 2
    q = 0.5 * U * U * Df
    cells = nxc * nyc + 2 * nfx * nfy
    return {"workload": "D2Q9 cylinder, 2:1 two-level: coarse 800x400 + fine 641x321", "coarse_steps": total,
            "St": strouhal(lift[half:], 2 * every, Df, U), "Cd_mean": float(np.mean(drag[half:]) / q),
            "Cl_amplitude": float((np.max(lift[half:]) - np.min(lift[half:])) / 2 / q),
            "mlups_incl_sampling": cells * total / wall / 1e6, "stable": rc == 0, "tau_c": tau_c, "tau_f": tau_f}


def run_cylinder_three_level(lbm, torch, args):
    """Three nested levels (the paper's cylinder uses four): coarse 400x200
    (D = 10), level 1 over coarse [40, 240] x [50, 150] (401 x 201, D = 20),
    level 2 over level-1 [60, 260] x [40, 160] (401 x 241, D = 40 around the
    cylinder and 7 D of its wake); the cylinder at coarse (100, 100), same
    Ma, Re, inflow, sponge (25 coarse cells) and seeds as the single-level
    run.  Lift/drag on the finest level; cell updates per coarse step:
    coarse + 2 x level 1 + 4 x level 2."""
    from paper_1710_02065_gb300 import inputs
    U = 0.2 * CS
    D2 = 40.0
    tau = [0.0, 0.0, 3 * U * D2 / 150.0 + 0.5]
    tau[1] = (tau[2] + 0.5) / 2
    tau[0] = (tau[1] + 0.5) / 2
    nxc, nyc = 400, 200
    stream = torch.cuda.Stream()
    s = lbm.Solver(lbm.LBM_D2Q9, (nxc, nyc, 1), tau[0], lbm.PRECISIONS[args.precision], Ma_ref=0.2,
                   stream=stream.cuda_stream)
    lbm.lbm_set_boundary(s.h, 0, 1, (U, 0, 0))
    lbm.lbm_set_boundary(s.h, 1, 2)
    lbm.lbm_set_sponge(s.h, 1, 25, 0.5, 1.0, (U, 0, 0))
    rho, u = inputs.uniform_flow_perturbed(nxc, nyc, U, 2)
    s.set_state(rho, u)
    patches = [((40, 50, 0), (200, 100, 1)), ((60, 40, 0), (200, 120, 1))]
    lbm.lbm_set_level_streams(s.h, args.level_streams)
    for o, e in patches:
        lbm.lbm_add_refinement_patch(s.h, o, e)
    ext1, _ = lbm.lbm_level_info(s.h, 1)
    ext2, _ = lbm.lbm_level_info(s.h, 2)
    # cylinder centre in level-2 nodes: coarse (100, 100) -> level 1 (120, 100) -> level 2 (120, 120)
    solid = inputs.cylinder_mask(ext2[0], ext2[1], 120.0, 120.0, D2)
    lbm.lbm_set_geometry_level(s.h, 2, solid)
    r1, u1 = inputs.uniform_flow_perturbed(ext1[0], ext1[1], U, 3)
    r2, u2 = inputs.uniform_flow_perturbed(ext2[0], ext2[1], U, 4)
    u2[solid == 1] = 0.0
    lbm.lbm_set_state_level(s.h, 2, r2, u2)
    lbm.lbm_set_state_level(s.h, 1, r1, u1)
    lbm.lbm_set_state(s.h, rho, u)
    total = args.cyl_steps // 4  # coarse steps covering the same physical time as the single-level run
    every = 5
    wall, Fs, _ = record_series(lbm, torch, s, total, every, 2)
    drag, lift = list(Fs[:, 0]), list(Fs[:, 1])
    _, _, rc = s.reduce()
    s.close()
    half = len(lift) // 2
    q = 0.5 * U * U * D2
    cells = nxc * nyc + 2 * ext1[0] * ext1[1] + 4 * ext2[0] * ext2[1]
    return {"workload": f"D2Q9 cylinder, three nested levels: coarse 400x200 + {ext1[0]}x{ext1[1]} + "
                        f"{ext2[0]}x{ext2[1]}", "coarse_steps": total,
            "St": strouhal(lift[half:], 4 * every, D2, U), "Cd_mean": float(np.mean(drag[half:]) / q),
            "Cl_amplitude": float((np.max(lift[half:]) - np.min(lift[half:])) / 2 / q),
            "mlups_incl_sampling": cells * total / wall / 1e6, "stable": rc == 0, "tau": tau}


def run_jet_two_level(lbm, torch, args):
    """2:1 two-level round jet (D3Q19, or D3Q27 with --lattice): the 384x256x256 jet lattice (FP32,
    Re_D 1e4, sponges, inlet noise) with a fine patch over the near-nozzle
    region, coarse [2, 66] x [96, 160] x [96, 160] (129^3 fine nodes, the
    inlet disc of diameter 24 in the middle of its cross-section).  Cell
    updates per coarse step: coarse cells + 2 x fine cells; time by CUDA
    events over args.steps coarse steps after args.warmup."""
    spec = jet_spec()
    spec["lattice"] = {"d3q19": lbm.LBM_D3Q19, "d3q27": lbm.LBM_D3Q27}[args.lattice]
    stream = torch.cuda.Stream()
    s = configure_gpu(lbm, spec, lbm.PRECISIONS[args.precision], stream.cuda_stream)
    lbm.lbm_set_level_streams(s.h, args.level_streams)
    n = s.ncell
    X0, Y0, Z0, W = 2, 96, 96, 64
    lbm.lbm_add_refinement_patch(s.h, (X0, Y0, Z0), (W, W, W))
    ext, tau_f = lbm.lbm_level_info(s.h, 1)
    nf = int(np.prod(ext))
    lbm.lbm_set_state_level(s.h, 1, np.ones(nf), np.zeros((nf, 3)))
    s.set_state(np.ones(n), np.zeros((n, 3)))
    lbm.lbm_step(s.h, args.warmup)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    info0 = s.info()
    with torch.cuda.stream(stream):
        e0.record(stream)
        lbm.lbm_step(s.h, args.steps)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = s.info()["launches"] - info0["launches"]
    _, _, rc = s.reduce()
    rf = np.zeros(nf)
    lbm.lbm_moments_level(s.h, 1, rf, None, None)
    s.close()
    cells = n + 2 * nf
    return {"workload": f"{args.lattice.upper()} round jet 384x256x256 + 2:1 patch {ext[0]}x{ext[1]}x{ext[2]} over the nozzle, "
                        f"{args.precision}", "metric": "cell updates per second (coarse + 2 x fine per coarse step)",
            "mlups": cells * args.steps / (ms / 1e3) / 1e6, "ms_per_coarse_step": ms / args.steps,
            "coarse_steps": args.steps, "launches_per_coarse_step": launches / args.steps,
            "level_streams": "concurrent" if args.level_streams else "in order",
            "tau_c": spec["tau"], "tau_f": tau_f, "stable": rc == 0 and bool(np.isfinite(rf).all())}


def run_serving(lbm, torch, args):
    from paper_1710_02065_gb300 import inputs, serving
    reqs = inputs.serving_requests(args.requests, seed=5, rate_per_s=args.rate, steps_scale=args.steps_scale)
    out = serving.serve(reqs, hbm_budget_bytes=int(args.budget_gb * (1 << 30)), max_slots=256,
                        steps_per_round=args.round_steps, aa=args.streaming == "aa", tune=not args.no_tune)
    out["workload"] = (f"{args.requests} requests, Poisson arrivals {args.rate}/s, D2Q9 pulses 64^2-1024^2 and "
                       f"D3Q19 Taylor-Green 32^3-192^3, steps x{args.steps_scale}, FP32/FP16, "
                       f"{args.streaming} streaming")
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    if out.get("gpu_gbs"):
        out["roofline"] = {"bound": "hbm", "achieved": out["gpu_gbs"], "peak": peak, "unit": "GB/s",
                           "frac": out["gpu_gbs"] / peak, "traffic": None,
                           "kernel": "k_batched (rounds' graphs incl. the per-domain advance)",
                           "bytes": "2 Q s per cell update of every request, over the device time of the rounds"}
    out["arrival_rate_note"] = ("default rate 9.7/s: 0.8 x the 12.1 requests/s this stream was served at when "
                                "saturated by the first engine (35.0 G cell updates/s), kept for comparison; the "
                                "current engine serves it at 13.8 requests/s saturated (1.48e12 cell updates at "
                                "39.9 G/s with arrivals at 40/s), so 9.7/s is 0.70 x saturation")
    return out


def run_batched(lbm, torch, args):
    """The serving engine's batched update (k_batched) on a fixed batch: `--batch
    KxN` periodic requests of N^3 (D3Q19 / D3Q27) or N^2 (D2Q9) cells at rest,
    one (lattice, precision) group, `--round-steps` steps per round; after
    `--warmup` warm rounds, `--steps` rounds are timed by the device time of
    their graphs (k_batched per step plus the per-domain advance).  The
    roofline is 2 Q s bytes per cell update over that time."""
    k, n = (int(v) for v in args.batch.lower().split("x"))
    lat = {"d2q9": lbm.LBM_D2Q9, "d3q19": lbm.LBM_D3Q19, "d3q27": lbm.LBM_D3Q27}[args.lattice]
    prec = lbm.PRECISIONS[args.precision]
    q = {lbm.LBM_D2Q9: 9, lbm.LBM_D3Q19: 19, lbm.LBM_D3Q27: 27}[lat]
    s_bytes = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[args.precision]
    ext = (n, n, 1) if lat == lbm.LBM_D2Q9 else (n, n, n)
    cells = k * ext[0] * ext[1] * ext[2]
    srv = lbm.lbm_server_create(16 << 30, 256, None)
    try:
        if args.streaming == "aa":
            lbm.lbm_server_set_streaming(srv, lbm.LBM_STREAM_AA)
        if args.launch:
            v, w = (int(t) for t in args.launch.split("x"))
            lbm.lbm_server_set_launch(srv, lat, prec, v, w)
        for _ in range(k):
            lbm.lbm_server_submit(srv, lat, prec, ext, 0.6, 1 << 40)
        for _ in range(args.warmup):
            lbm.lbm_server_run(srv, args.round_steps)
        torch.cuda.synchronize()
        t0 = lbm.lbm_server_gpu_time(srv)
        w0 = time.perf_counter()
        for _ in range(args.steps):
            lbm.lbm_server_run(srv, args.round_steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        ms = lbm.lbm_server_gpu_time(srv) - t0
        v, w = lbm.lbm_server_get_launch(srv, lat, prec)
    finally:
        lbm.lbm_server_destroy(srv)
    updates = cells * args.round_steps * args.steps
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    gbs = 2 * q * s_bytes * updates / (ms / 1e3) / 1e9
    return {"workload": f"batched update, {k} periodic {args.lattice.upper()} requests of "
                        f"{'x'.join(str(e) for e in ext)} cells at rest, {args.precision} storage, "
                        f"{args.streaming} streaming",
            "metric": "MLUPS", "value": updates / (ms / 1e3) / 1e6, "unit": "MLUPS",
            "rounds": args.steps, "steps_per_round": args.round_steps, "warmup_rounds": args.warmup,
            "device_ms": ms, "wall_ms": 1e3 * wall, "cells": cells,
            "launch": {"cells_per_lane": v, "warps_per_block": w},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "kernel": "k_batched (+ k_batch_advance per step)",
                         "bytes_per_cell": 2 * q * s_bytes}}


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    """The FP64 CPU oracle, timed on the host cores on the jet scaled to 96x64x64."""
    if rank != 0:
        return
    spec = jet_spec(**REF_SAMPLE_SPEC)
    P, f = configure_oracle(spec)
    for k in range(args.warmup):
        f = P.run(f, 1, step0=k)
    t0 = time.perf_counter()
    f = P.run(f, args.steps, step0=args.warmup)
    dt = time.perf_counter() - t0
    mlups = P.ncell * args.steps / dt / 1e6
    sample = f"D3Q19 round jet scaled to 64x48x48 (D=4.5, sponge 6), FP64 oracle, {args.steps} timed steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": jet_workload_name(384, 256, 256), "cells": 384 * 256 * 256,
                   "storage": "fp64 (the oracle)", "sample": "64x48x48 copy of the jet per step",
                   "inlet": "top hat, tanh shear layer theta = D/40, Ma 0.3, 1% seeded noise",
                   "parallelism": "none (host, 1 thread)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--no-extra", action="store_true", help="skip the other storage precisions")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--no-tune", action="store_true", help="use the default launch shape (no autotuning)")
    ap.add_argument("--launch", default=None,
                    help="fixed kernel and launch shape for the main precision instead of tuning: "
                         "cell:BLOCK, vec2:BLOCK, vec4:BLOCK or rows:STAGES; batched workload: VxW, cells per "
                         "lane x warps per block")
    ap.add_argument("--workload", default="jet", choices=["jet", "cylinder", "cylinder2level", "cylinder3level",
                                                          "jet2level", "serving", "batched"],
                    help="jet: the headline benchmark line; the others print their own JSON line")
    ap.add_argument("--cyl-steps", type=int, default=40000, help="fine-resolution steps of the cylinder runs")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--rate", type=float, default=9.7,
                    help="serving arrival rate (requests/s); the default 9.7/s is 0.70 x the 13.8 requests/s "
                         "this stream is served at when saturated (1.48e12 cell updates at 39.9 G/s)")
    ap.add_argument("--steps-scale", type=float, default=1.0, help="serving: scale of per-request steps")
    ap.add_argument("--budget-gb", type=float, default=8.0, help="serving: HBM budget for populations")
    ap.add_argument("--round-steps", type=int, default=100, help="serving: steps per batched round")
    ap.add_argument("--streaming", default="pull", choices=["pull", "aa"],
                    help="serving: streaming pattern of the requests (aa: one lattice each)")
    ap.add_argument("--level-streams", type=int, default=1, choices=[0, 1],
                    help="refined workloads: 1 runs the refined levels concurrently with the level-0 update "
                         "(lbm_set_level_streams), 0 in order on one stream")
    ap.add_argument("--lattice", default="d3q19", choices=["d2q9", "d3q19", "d3q27"],
                    help="lattice of the jet (d3q19, the benchmark line, or d3q27), two-level jet and batched "
                         "workloads")
    ap.add_argument("--batch", default="8x128",
                    help="batched workload: KxN, K periodic requests of N^3 (N^2 for D2Q9) cells")
    ap.add_argument("--grid", default="384x256x256",
                    help="jet extents NXxNYxNZ; inlet diameter and sponges scale with NX/384")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        if pg is not None:
            pg.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    from paper_1710_02065_gb300 import build
    if rank == 0:
        build.build()
    barrier(pg)
    from paper_1710_02065_gb300 import lbm

    if args.workload != "jet":
        fn = {"cylinder": run_cylinder, "cylinder2level": run_cylinder_two_level,
              "cylinder3level": run_cylinder_three_level, "jet2level": run_jet_two_level, "serving": run_serving,
              "batched": run_batched}
        out = fn[args.workload](lbm, torch, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if pg is not None:
            pg.destroy_process_group()
        return

    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    scale = nx / 384.0
    spec = jet_spec(nx, ny, nz, diameter=24.0 * scale, sponge=max(2, int(round(32 * scale))))
    if args.lattice == "d2q9":
        raise SystemExit("the jet workload is 3D: --lattice d3q19 or d3q27")
    lat = args.lattice
    spec["lattice"] = {"d3q19": lbm.LBM_D3Q19, "d3q27": lbm.LBM_D3Q27}[lat]
    prec = lbm.PRECISIONS[args.precision]
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    fixed = None
    if args.launch:
        kind, knob = args.launch.split(":")
        fixed = (kind, int(knob))
    main_run = time_precision(lbm, torch, spec, prec, args.steps, args.warmup, pg, stream, tune=not args.no_tune,
                              launch=fixed)
    clk = clocks.stop()
    total_s = max_over_ranks(main_run["total_ms"] / 1e3, pg, world)
    ncell = main_run["ncell"]
    value = world * ncell * args.steps / total_s / 1e6
    per = np.array(main_run["per_ms"])
    kernel_ms = float(per.mean())
    bpc = main_run["bytes_per_cell"]
    achieved = bpc * ncell / (kernel_ms / 1e3) / 1e9
    peaks = measured_peaks()
    if peaks and "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    kind = main_run["launch"]["kernel"]
    kname = {"rows": "k_stream_collide_rows", "cell": "k_stream_collide"}.get(kind, "k_stream_collide_vec")
    key = f"{kname}_{lat}_{args.precision}_jet{nx}x{ny}x{nz}"
    traffic = recorded_traffic(key)

    extra = {}
    # the other precisions, lattices and studies are properties of one GPU: the
    # single-GPU run reports them, replica runs (N > 1) time the main line only
    run_extra = not args.no_extra and world == 1
    if not args.no_extra and world > 1:
        extra["note"] = "per-GPU extras (other precisions, D3Q27, p' errors, A/B, serving) are in the N = 1 run"
    if run_extra:
        for name in ("fp16", "bf16", "fp64"):
            if name == args.precision:
                continue
            r = time_precision(lbm, torch, spec, lbm.PRECISIONS[name], max(20, args.steps // 4),
                               args.warmup, pg, stream, tune=not args.no_tune)
            k_ms = float(np.mean(r["per_ms"]))
            extra[name] = {"launch": r["launch"], "mlups": r["ncell"] / (k_ms / 1e3) / 1e6,
                           "gbs": r["bytes_per_cell"] * r["ncell"] / (k_ms / 1e3) / 1e9,
                           "frac_of_measured_hbm": r["bytes_per_cell"] * r["ncell"] / (k_ms / 1e3) / 1e9 / peak}
            if name in ("fp16", "bf16") and r["launch"]["kernel"] == "vec2" and r["launch"]["streaming"] == "pull":
                ins = recorded_issue(f"k_stream_collide_vec_{lat}_{name}_jet", args.grid.lower())
                if ins is not None:
                    rate = extra[name]["mlups"] / 1e3  # G cells/s
                    mhz = (clk or {}).get("sm_mhz")
                    ipk = issue_peak_g(mhz)
                    extra[name]["roofline"] = {
                        "bound": "alu", "achieved": rate * ins, "peak": ipk, "unit": "G warp instr/s",
                        "frac": rate * ins / ipk, "warp_inst_per_cell": ins, "sm_mhz": mhz or 2070.0,
                        "peak_source": "152 SMs x 4 schedulers x the median SM clock sampled during the main "
                                       "timed region (one warp instruction per scheduler per cycle); counts "
                                       "from profiles/ncu_issue.txt, taken on this grid"}
            if name == "fp64":
                kk = "k_stream_collide_vec" if r["launch"]["kernel"].startswith("vec") else "k_stream_collide"
                ins = recorded_fp64_inst(f"{kk}_{lat}_fp64_jet")
                if ins is not None and r["launch"]["kernel"] in ("cell", "vec2"):
                    rate = extra[name]["mlups"] / 1e3  # G cells/s
                    extra[name]["roofline"] = {
                        "bound": "alu", "achieved": rate * ins[0], "peak": FP64_INST_PEAK_G,
                        "unit": "G FP64 instr/s", "frac": rate * ins[0] / FP64_INST_PEAK_G,
                        "fp64_inst_per_cell": ins[0], "fp64_tflops": rate * ins[1] / 1e3,
                        "peak_source": "nominal 1.25 TFLOP/s FP64 (625 G FMA/s); counts from profiles/ncu_fp64_inst.txt"}
        # the same jet on D3Q27 (complete third order; 27 populations, 216 B per cell in FP32)
        if lat == "d3q19":
            spec27 = dict(spec, lattice=lbm.LBM_D3Q27)
            r = time_precision(lbm, torch, spec27, lbm.PRECISIONS[args.precision], max(20, args.steps // 4),
                               args.warmup, pg, stream, tune=not args.no_tune)
            k_ms = float(np.mean(r["per_ms"]))
            extra["d3q27_" + args.precision] = {
                "launch": r["launch"], "mlups": r["ncell"] / (k_ms / 1e3) / 1e6,
                "gbs": r["bytes_per_cell"] * r["ncell"] / (k_ms / 1e3) / 1e9,
                "frac_of_measured_hbm": r["bytes_per_cell"] * r["ncell"] / (k_ms / 1e3) / 1e9 / peak}
        if "fp16" in extra:
            extra["fp16_store_speedup"] = extra["fp16"]["mlups"] / (ncell / (kernel_ms / 1e3) / 1e6)
        if "bf16" in extra:
            extra["bf16_store_speedup"] = extra["bf16"]["mlups"] / (ncell / (kernel_ms / 1e3) / 1e6)

    if run_extra:
        extra["pprime_error"] = pprime_errors(lbm, torch, stream)
        extra["stability_ab"] = stability_ab(lbm, stream)
        from paper_1710_02065_gb300 import inputs as _inp, serving as _srv
        reqs = _inp.serving_requests(96, seed=5, rate_per_s=40.0, steps_scale=0.1)
        sv = _srv.serve(reqs, hbm_budget_bytes=8 << 30, max_slots=256, steps_per_round=50, tune=not args.no_tune)
        sv["workload"] = ("serving sample: 96 requests, Poisson 40/s, steps x0.1 (the full stream is "
                          "--workload serving)")
        extra["serving"] = sv

    e2e = None if args.no_e2e else e2e_run(lbm, torch, spec, prec, args.steps, stream)
    e2e_s = max_over_ranks(e2e["seconds"], pg, world) if e2e else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        mlups_cpu, st, dt, nc = time_oracle()
        cpu = {"value": mlups_cpu, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"D3Q19 round jet scaled to 96x64x64 ({nc} cells), {st} FP64 steps in {dt:.1f} s, 1 thread"}
        try:
            agg, nproc, rst, rdt = time_oracle_all_cores()
            cpu["all_cores"] = {"value": agg, "unit": "MLUPS", "cores": nproc,
                                "sample": f"{nproc} independent 96x64x64 oracle solves at once, "
                                          f"{rst} FP64 steps each, {rdt:.1f} s wall"}
        except Exception as e:  # a host without process spawning still reports the 1-thread figure
            cpu["all_cores"] = {"unavailable": repr(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": jet_workload_name(nx, ny, nz, lat.upper()),
                       "cells": ncell, "tau": spec["tau"], "storage": args.precision,
                       "inlet": "top hat, tanh shear layer theta = D/40, Ma 0.3, 1% seeded noise",
                       "launch": main_run["launch"], "autotune_ms_per_step": main_run["tuning"],
                       "l2": "inputs larger than L2 (populations %.2f GB per lattice)" % (bpc / 2 * ncell / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "kernel": f"{kname}<{lat.upper()}>", "bytes_per_cell": bpc,
                         "kernel_ms": kernel_ms},
            "cpu_baseline": cpu,
            "e2e": ({"value": world * ncell * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                     "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                     "steps": args.steps, "host_dtype": e2e["host_dtype"],
                     "upload_ms": 1e3 * e2e["upload_s"]} if e2e else None),
            "gpu_launches": main_run["launches"],
            "clocks": clk,
            "stable": main_run["stable"],
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
