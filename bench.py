"""Benchmark of the split-step Crank-Nicolson hot path (arXiv:2009.13507) on GB300.

Workload (one benchmark step): the 2D spin-1 imaginary-time run on a 256 x 256
grid, dx = dy = 0.05 on [-6.4, 6.4)^2, isotropic trap, c0 = 50, c2 = 1, Rashba
SO gamma = 0.8, Rabi Omega = 0.5, random-phase Gaussian initial state (seeded),
dt = 2e-4, 2000 time steps with renormalisation every step, then the
observables (energy, norms, rms sizes). Complex128 state (plain FP64 form).
Metric: grid point-steps per second (one point = all three spin components
advanced by one full time step).

Also reported on the same line: the complex64 precision form on the same
workload (FP64 reductions) with its energy error against the FP64 path, the
FP64-accurate double-float form (FP32 pairs) with its state and energy error
against the FP64 path, the dominant kernel's roofline, the oracle on the host
cores (cpu_baseline) and the end-to-end throughput through the C ABI with host
buffers.

--impl reference times the FP64 CPU oracle on every host core instead (OpenMP
over points and lines; the whole workload per step when it fits the time
budget, else a stated shorter sample of it).

Multi-GPU: the single-grid step does not shard (replicas only): with N ranks
every rank runs its own replica, value = all ranks' point-steps / max time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 256
DX = 0.05
NSTEPS = 2000
PHYS = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
WORKLOAD = "2D spin-1 imaginary time, 256x256, dx=0.05, c0=50, c2=1, Rashba gamma=0.8, Omega=0.5, dt=2e-4, 2000 steps"
METRIC = "point-steps/s"
# Algorithmic FP64 flops per grid point of the pointwise kernel (SO + CALCNU +
# HERM, imaginary time, 2D Rashba), counted from the formulas it evaluates
# (FMA = 2 flops; exp by its degree-9 Taylor polynomial).
POINTWISE_FLOPS = 263
# Algorithmic FP64 flops per grid point of one Crank-Nicolson sweep (three
# component lines; real tables in imaginary time): forward 6, backward 8,
# carry fix-up 4, 2w - x 4 per component.
CN_FLOPS = 66
# Nominal FP64 rate: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 1.259
# The oracle's sample: the whole 2000-step workload on every host core (~3 s on 16 Arm cores)
# and 600 steps on one thread (~8 s).
CPU_SAMPLE_STEPS = NSTEPS
CPU_SINGLE_STEPS = 600
# DRAM bytes (read + write) of one launch of the dominant kernel on this workload in an ncu capture
# (cold L2): None whenever the kernel changed after the capture.
HEAD_TRAFFIC_BYTES = 3251968


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_hbm_gbs():
    """The HBM copy bandwidth measured on this GPU pool (MEASURED_PEAKS.json beside this
    file, GB/s), or None when the file is absent."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def hbm_view(effective_gbps: float) -> dict:
    """Effective bandwidth of the step's two streaming passes (192 algorithmic bytes per
    point-step) against the measured HBM copy peak; the state is L2-resident, so this is
    context, not the binding roof (the FP64 ALU is)."""
    peak = measured_hbm_gbs()
    return {"algorithmic_bytes_per_point_step": 192, "effective_GBps": effective_gbps,
            "peak_GBps": peak, "peak_source": "measured copy bandwidth" if peak else None,
            "frac": effective_gbps / peak if peak else None}


def max_over_ranks(t: float, device=None) -> float:
    """Max of t over the ranks of the default process group (t itself when
    there is no group or a single rank): the replicas' benchmark time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_value(points_per_rank: int, world_size: int, t_ms: float) -> float:
    """Whole-job point-steps/s of world_size independent replicas that each
    advance points_per_rank point-steps, timed by the slowest rank (t_ms)."""
    return world_size * points_per_rank / (t_ms * 1e-3)


def bench_config(ws: int) -> dict:
    """The workload description shared by both arms (the oracle arm reports the same dict)."""
    return {"workload": WORKLOAD, "precision": "complex128 (plain FP64 form)", "grid": [NX, NY],
            "l2": "GPU arm: 256 MiB L2 flush between benchmark steps (the 3 MiB state is L2-resident within a "
                  "run); oracle arm: host caches as they are",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def cpu_oracle_rate(steps: int = CPU_SAMPLE_STEPS, threads: int = 1):
    """The FP64 CPU oracle (as it stands) on the same workload: `steps` time steps of
    256x256 plus the observables, on `threads` OpenMP threads (<= 0: every core this
    process may use). Returns (point-steps/s, seconds, threads used)."""
    from oracle import oracle as O
    from paper_2009_13507_gb300 import inputs as I
    O.build()
    n = O.set_threads(threads)
    try:
        prob = O.Problem(dim=2, nx=NX, ny=NY, dx=DX, dy=DX, **PHYS)
        psi = I.gaussian_phase_2d(NX, NY, DX, DX, seed=0)
        t0 = time.perf_counter()
        out = O.step(prob, psi, steps, True)
        O.observables(prob, out)
        t = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    return NX * NY * steps / t, t, n


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on every host core, each benchmark step
    the 256x256 workload from its initial state plus the observables. A benchmark
    step runs all 2000 time steps when the K timed steps fit in about two and a
    half minutes at the rate measured on a short probe, otherwise a shorter
    sample of the same workload (stated in the line)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_rate(5, 0)
    r_probe, _t, cores = cpu_oracle_rate(40, 0)
    budget_s = 150.0
    steps_per = NSTEPS
    if args.steps * NX * NY * NSTEPS / r_probe > budget_s:
        steps_per = max(50, int(budget_s * r_probe / (args.steps * NX * NY)))
    wall = []
    for _ in range(args.steps):
        _r, t, cores = cpu_oracle_rate(steps_per, 0)
        wall.append(t)
    ms = statistics.mean(wall) * 1e3
    value = NX * NY * steps_per / (ms * 1e-3)
    r1, t1, _ = cpu_oracle_rate(100, 1)
    sample = ("%d of the workload's %d time steps per benchmark step (plus the observables), %d OpenMP threads"
              % (steps_per, NSTEPS, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "time_steps_per_bench_step": steps_per,
        "config": bench_config(ws),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": r1, "cores": 1,
                                           "sample": "100 time steps of the workload (%.1f s)" % t1}},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def extra_workloads(dev, reps=2):
    """The other workloads of the method, each measured with CUDA events on its
    solver's stream after one warm-up run (rank 0 only):
      1d_imag       1D, Nx = 256, dx = 0.05, c0 = 10, c2 = -0.5, gamma p_x Sigma_x (0.5),
                    Omega = 0.2, dt = 1e-4, 10,000 imaginary-time steps, complex128 (and the
                    double-float and complex64 forms with their energy error)
      quench        2D 512 x 512, dx = 0.04, the 2D physics above; ground state prepared
                    in FP64 (3000 imaginary-time steps, untimed), then Omega 0.5 -> 0 and
                    10,000 real-time steps at dt = 1e-4 in complex64 and complex128
                    (energy / norm of complex64 against complex128 after 10,000 steps, and
                    of both against the FP64 oracle on every host core after 1,000)
      batched       64 instances (32 1D nx ~ U{128..1024}, 32 2D n ~ U{128..384}), per-instance
                    (gamma, Omega, c0, c2) drawn, 1,000 imaginary-time steps, autotuned tiles
      adjoint       2D 256 x 256 real time, 500 steps at dt = 2e-4, gradient of the
                    final-density loss w.r.t. Omega(t) and (wx, wy), checkpoint every 50
                    (the loss also against the FP64 oracle)
      step_options  the headline workload with Strang splitting, with the SO substep by
                    Crank-Nicolson, and with both (complex128)
      large         the 2D physics above at 2048 x 2048 and 4096 x 4096 (dx = 0.05), 10
                    imaginary-time steps in complex64, double-float and complex128: the state
                    (100 MB to 805 MB) does not fit in L2, so the two streaming passes go to HBM;
                    effective GB/s (96 / 192 algorithmic bytes per point-step) against the
                    measured HBM copy peak
    """
    import numpy as np
    import torch

    from paper_2009_13507_gb300 import inputs as I
    from paper_2009_13507_gb300 import sgpe

    def ev_time(stream, fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    out = {}
    # 1D imaginary time in the three precisions
    d1 = {}
    for prec in ("c128", "cdf", "c64"):
        s1 = sgpe.Solver(1, 256, dx=0.05, precision=prec, device=dev)
        s1.set_params(sgpe.Physics(c0=10.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2, dt=1e-4, renorm=1))
        p1 = torch.from_numpy(I.gaussian_jitter_1d(256, 0.05, seed=0)).to(dev).to(s1.cdtype)
        ms = []
        for r in range(reps + 1):
            s1.load_state(p1)
            t = ev_time(s1.stream, lambda: s1.step_imag(10000))
            if r:
                ms.append(t)
        d1[prec] = {"value": 256 * 10000 / (statistics.mean(ms) * 1e-3), "ms": statistics.mean(ms),
                    "E": s1.energy()["E"]}
    out["1d_imag"] = {"value": d1["c128"]["value"], "unit": METRIC, "ms": d1["c128"]["ms"], "E": d1["c128"]["E"],
                      "precision": "complex128",
                      "cdf_value": d1["cdf"]["value"],
                      "cdf_energy_rel_err_vs_fp64": abs(d1["cdf"]["E"] - d1["c128"]["E"]) / abs(d1["c128"]["E"]),
                      "c64_value": d1["c64"]["value"],
                      "c64_energy_rel_err_vs_fp64": abs(d1["c64"]["E"] - d1["c128"]["E"]) / abs(d1["c128"]["E"])}
    # 512 x 512 real-time quench
    n3, dx3 = 512, 0.04
    phys = dict(PHYS)
    prep = sgpe.Solver(2, n3, n3, dx=dx3, device=dev)
    prep.set_params(sgpe.Physics(**phys))
    prep.set_state(I.gaussian_phase_2d(n3, n3, dx3, dx3, seed=0))
    prep.step_imag(3000)
    prep.energy()
    ground = prep.psi.clone()
    prep.stream.synchronize()
    q = {}
    for prec in ("c128", "c64"):
        s3 = sgpe.Solver(2, n3, n3, dx=dx3, precision=prec, device=dev)
        s3.set_params(sgpe.Physics(**dict(phys, omega=0.0, dt=1e-4, renorm=0)))
        g = ground.to(s3.cdtype)
        s3.load_state(g)
        s3.step_real(100)  # warm-up (graph capture)
        s3.load_state(g)
        e0 = s3.energy()
        t = ev_time(s3.stream, lambda: s3.step_real(10000))
        e = s3.energy()
        q[prec] = {"value": n3 * n3 * 10000 / (t * 1e-3), "ms": t, "E0": e0["E"], "E": e["E"], "N": e["N"]}
    # against the FP64 oracle (every host core): the first 1000 quench steps from the same ground state
    from oracle import oracle as O
    O.build()
    n_orc = 1000
    ground_h = ground.cpu().numpy()
    prob3 = O.Problem(dim=2, nx=n3, ny=n3, dx=dx3, dy=dx3, **dict(phys, omega=0.0, dt=1e-4, renorm=0))
    cores = O.set_threads(0)
    t0 = time.perf_counter()
    ref3 = O.observables(prob3, O.step(prob3, ground_h, n_orc, False))
    t_orc = time.perf_counter() - t0
    O.set_threads(1)
    vs_oracle = {}
    for prec in ("c128", "c64"):
        s3 = sgpe.Solver(2, n3, n3, dx=dx3, precision=prec, device=dev)
        s3.set_params(sgpe.Physics(**dict(phys, omega=0.0, dt=1e-4, renorm=0)))
        s3.load_state(ground.to(s3.cdtype))
        s3.step_real(n_orc)
        e = s3.energy()
        vs_oracle[prec] = {"energy_rel_err": abs(e["E"] - ref3["E"]) / abs(ref3["E"]),
                           "norm_err": abs(e["N"] - ref3["N"])}
    out["quench"] = {"value": q["c64"]["value"], "unit": METRIC, "precision": "complex64 (FP64 reductions)",
                     "fp64_value": q["c128"]["value"],
                     "vs_oracle_after_1000_steps": vs_oracle,
                     "oracle": {"steps": n_orc, "seconds": t_orc, "cores": cores},
                     "energy_rel_err_vs_fp64_gpu_10000_steps": abs(q["c64"]["E"] - q["c128"]["E"]) / abs(q["c128"]["E"]),
                     "norm_err_vs_fp64_gpu_10000_steps": abs(q["c64"]["N"] - q["c128"]["N"]),
                     "energy_drift_fp64": q["c128"]["E"] - q["c128"]["E0"], "detail": q}
    # batched
    inst = []
    for t in I.batch_table(0):
        d = dict(t)
        d.update(dx=0.05, dy=0.05, so_type=1, dt=(1e-4 if t["dim"] == 1 else 2e-4), renorm=1)
        inst.append(d)
    bres = {}
    for prec in ("c128", "c64"):
        bs = sgpe.BatchSolver(inst, precision=prec, device=dev)
        tiles = bs.autotune(2)
        states = [I.gaussian_phase_2d(s["nx"], s["ny"], s["dx"], s["dy"], seed=100 + i) if s["dim"] == 2
                  else I.gaussian_jitter_1d(s["nx"], s["dx"], seed=100 + i, amp=1e-2) for i, s in enumerate(bs.specs)]
        packed = bs.pack(states)
        torch.cuda.synchronize(dev)
        ms = []
        for r in range(reps + 1):
            bs.load_state(packed)
            t = ev_time(bs.stream, lambda: bs.step_imag(1000))
            if r:
                ms.append(t)
        obs = bs.energy()
        pts = sum(s["nx"] * s["ny"] for s in bs.specs)
        bres[prec] = {"value": pts * 1000 / (statistics.mean(ms) * 1e-3), "ms": statistics.mean(ms),
                      "tiles": tiles, "E": obs[:, 5].copy(), "launches_per_step": bs.launches_per_step()}
    err = float(np.max(np.abs(bres["c64"]["E"] - bres["c128"]["E"]) / np.abs(bres["c128"]["E"])))
    out["batched"] = {"value": bres["c128"]["value"], "unit": METRIC, "precision": "complex128",
                      "c64_value": bres["c64"]["value"], "c64_energy_max_rel_err_vs_fp64": err,
                      "ms": bres["c128"]["ms"], "c64_ms": bres["c64"]["ms"], "tiles_c128": bres["c128"]["tiles"],
                      "tiles_c64": bres["c64"]["tiles"], "instances": len(inst),
                      "launches_per_step": bres["c128"]["launches_per_step"]}
    # large grids: HBM-resident state
    peak = measured_hbm_gbs()
    big = {}
    for n4 in (2048, 4096):
        for prec in ("c64", "cdf", "c128"):
            sl = sgpe.Solver(2, n4, n4, dx=DX, precision=prec, device=dev)
            sl.set_params(sgpe.Physics(**PHYS))
            pl = torch.from_numpy(I.gaussian_phase_2d(n4, n4, DX, DX, seed=0)).to(sl.cdtype).to(dev)
            # (the double-float state is 16 bytes a complex number, like complex128)
            ms = []
            for r in range(reps + 1):
                sl.load_state(pl)
                t = ev_time(sl.stream, lambda: sl.step_imag(10))
                if r:
                    ms.append(t)
            t_step = statistics.mean(ms) / 10
            rate = n4 * n4 / (t_step * 1e-3)
            gbs = rate * (96 if prec == "c64" else 192) / 1e9
            big["%s_%d" % (prec, n4)] = {"value": rate, "us_per_step": t_step * 1e3, "effective_GBps": gbs,
                                         "frac_of_measured_hbm": gbs / peak if peak else None}
            del sl, pl
            torch.cuda.empty_cache()
    out["large"] = {"unit": METRIC, "hbm_peak_GBps": peak, "detail": big}
    # adjoint
    ares = {}
    tgt = I.gaussian_target(NX, NY, DX, DX, seed=7)
    psi0 = I.gaussian_phase_2d(NX, NY, DX, DX, seed=0)
    for prec in ("c64", "c128"):
        sa = sgpe.Solver(2, NX, NY, dx=DX, precision=prec, device=dev)
        sa.set_params(sgpe.Physics(**dict(PHYS, renorm=0)))
        p0 = torch.from_numpy(psi0).to(sa.cdtype).to(dev)
        om = np.full(500, 0.5)
        times = []
        for r in range(reps + 1):
            sa.load_state(p0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            L, dom, dw = sa.loss_grad(om, tgt, checkpoint_every=50)
            if r:
                times.append((time.perf_counter() - t0) * 1e3)
        ares[prec] = {"ms_per_gradient": statistics.mean(times), "loss": L, "dL_dwx": dw[0], "dL_dwy": dw[1]}
    # the loss of the same 500 real-time steps by the FP64 oracle (every host core)
    proba = O.Problem(dim=2, nx=NX, ny=NY, dx=DX, dy=DX, **dict(PHYS, renorm=0))
    O.set_threads(0)
    psiN = O.step(proba, psi0, 500, False, omega_t=np.full(500, 0.5))
    O.set_threads(1)
    L_orc = DX * DX * float(np.sum((np.sum(np.abs(psiN) ** 2, axis=0) - tgt) ** 2))
    # the step options on the headline workload (complex128, 2000 imaginary-time steps)
    var = {}
    for name, kw in (("strang", dict(split=1)), ("so_crank_nicolson", dict(so_mode=1)),
                     ("strang_so_crank_nicolson", dict(split=1, so_mode=1))):
        sv = sgpe.Solver(2, NX, NY, dx=DX, precision="c128", device=dev)
        sv.set_params(sgpe.Physics(**dict(PHYS, **kw)))
        pv = torch.from_numpy(psi0.astype(np.complex128)).to(dev)
        ms = []
        for r in range(reps + 1):
            sv.load_state(pv)
            t = ev_time(sv.stream, lambda: sv.step_imag(NSTEPS))
            if r:
                ms.append(t)
        var[name] = {"value": NX * NY * NSTEPS / (statistics.mean(ms) * 1e-3), "ms": statistics.mean(ms),
                     "E": sv.energy()["E"], "launches_per_step": sv.launches_per_step()}
    out["step_options"] = var
    out["adjoint"] = {"value": ares["c64"]["ms_per_gradient"], "unit": "ms per gradient", "precision": "complex64",
                      "fp64_ms_per_gradient": ares["c128"]["ms_per_gradient"],
                      "loss_rel_err_vs_oracle": {p_: abs(ares[p_]["loss"] - L_orc) / L_orc for p_ in ("c64", "c128")},
                      "loss_rel_err_vs_fp64": abs(ares["c64"]["loss"] - ares["c128"]["loss"]) / ares["c128"]["loss"],
                      "dL_dwx_rel_err_vs_fp64": abs(ares["c64"]["dL_dwx"] - ares["c128"]["dL_dwx"])
                      / abs(ares["c128"]["dL_dwx"])}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (forms)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_2009_13507_gb300 import inputs as I
    from paper_2009_13507_gb300 import sgpe

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    psi0 = I.gaussian_phase_2d(NX, NY, DX, DX, seed=0)
    solver = sgpe.Solver(2, NX, NY, dx=DX, precision="c128", device=dev)
    solver.set_params(sgpe.Physics(**PHYS))
    psi0_dev = torch.from_numpy(psi0.astype(np.complex128)).to(dev)
    stream = solver.stream
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # reset to the resident initial state (device copy inside libsgpe; resets the pending scale)
    def reset(s, p0):
        s.load_state(p0)

    def timed_run(s, p0, steps, warmup):
        for _ in range(warmup):
            reset(s, p0)
            s.step_imag(NSTEPS)
            s.energy_array()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        energies = []
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(steps):
            reset(s, p0)
            flush_buf.zero_()  # L2 flush (256 MiB) between benchmark steps, outside the events
            torch.cuda.synchronize(dev)
            evs[k][0].record(s.stream)
            s.step_imag(NSTEPS)
            energies.append(s.energy_array())  # observables (synchronises)
            evs[k][1].record(s.stream)
        torch.cuda.synchronize(dev)
        barrier()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, energies, wall

    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else local)
    clocks.start()
    ms64, en64, _ = timed_run(solver, psi0_dev, args.steps, args.warmup)
    clk = clocks.stop()
    t_step = max_over_ranks(statistics.mean(ms64), dev)  # ms per benchmark step, slowest rank
    point_steps = NX * NY * NSTEPS
    value = replica_value(point_steps, ws, t_step)

    # per-kernel device times (CUDA events on the solver's stream, eager launches, same workload)
    reset(solver, psi0_dev)
    kms, kcnt = solver.profile_steps(NSTEPS, True)
    e_prof = solver.energy_array()
    fused = int(kcnt[1]) == 0  # pointwise + CN-x in one kernel
    names = ["pointwise+cn_x" if fused else "pointwise", "cn_x", "cn_y", "finalize"]
    kavg = {names[i]: kms[i] / max(int(kcnt[i]), 1) for i in range(4) if int(kcnt[i]) > 0}
    dom = max(kavg, key=lambda n: kavg[n])
    share = {n: kms[i] / kms.sum() for i, n in enumerate(names) if int(kcnt[i]) > 0}
    dom_ms = kavg[names[0]]
    dom_flops = POINTWISE_FLOPS + (CN_FLOPS if fused else 0)
    dom_name = ("k_pwx<double, imag, 8> (SO+CALCNU+HERM, CN-x)" if fused
                else "k_pointwise<double> (SO+CALCNU+HERM)")
    achieved_tflops = dom_flops * NX * NY / (dom_ms * 1e-3) / 1e12
    # the FP64 roof measured on this GPU in this run (FMA-chain kernel, CUDA events)
    try:
        fp64_peak = sgpe.measure_fp64_rate(solver.stream)
        peak_source = "measured in this run: FP64 FMA-chain kernel (sgpe_measure_fp64_rate), CUDA events"
    except Exception as exc:  # keep the line; say why the nominal figure is used
        fp64_peak = FP64_PEAK_TFLOPS
        peak_source = "nominal FP64 (152 SMs x 2 DFMA/clk x 2 x 2.07 GHz); measurement failed: %s" % exc

    # precision form (complex64 state, FP64 reductions) on the same workload
    s32 = sgpe.Solver(2, NX, NY, dx=DX, precision="c64", device=dev)
    s32.set_params(sgpe.Physics(**PHYS))
    psi0_dev32 = psi0_dev.to(torch.complex64)
    ms32, en32, _ = timed_run(s32, psi0_dev32, args.steps, args.warmup)
    t32 = max_over_ranks(statistics.mean(ms32), dev)
    e64, e32 = en64[-1][5], en32[-1][5]
    reset(s32, psi0_dev32)
    kms32, kcnt32 = s32.profile_steps(NSTEPS, True)
    kavg32 = {names[i]: kms32[i] / max(int(kcnt32[i]), 1) for i in range(4) if int(kcnt32[i]) > 0}

    # FP64-accurate double-float form (FP32 pairs) on the same workload; its
    # final state after one benchmark step against the complex128 one
    sdf = sgpe.Solver(2, NX, NY, dx=DX, precision="cdf", device=dev)
    sdf.set_params(sgpe.Physics(**PHYS))
    msdf, endf, _ = timed_run(sdf, psi0_dev, args.steps, args.warmup)
    tdf = max_over_ranks(statistics.mean(msdf), dev)
    edf = endf[-1][5]
    for s_ in (solver, sdf):
        reset(s_, psi0_dev)
        s_.step_imag(NSTEPS)
    st64, stdf = solver.get_state(), sdf.get_state()
    state_err_df = float(np.linalg.norm((stdf - st64).ravel()) / np.linalg.norm(st64.ravel()))
    reset(sdf, psi0_dev)
    kmsdf, kcntdf = sdf.profile_steps(NSTEPS, True)
    kavgdf = {names[i]: kmsdf[i] / max(int(kcntdf[i]), 1) for i in range(4) if int(kcntdf[i]) > 0}

    # end to end through the C ABI with host buffers: pinned host state in,
    # 2000 steps, observables and the final state out, copies inside the timed region
    host_in = torch.from_numpy(psi0.astype(np.complex128)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        solver.set_state_host_ptr(host_in.data_ptr())
        solver.step_imag(NSTEPS)
        solver.energy_array()
        solver.get_state_host_ptr(host_out.data_ptr())
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_t = max_over_ranks(statistics.mean(e2e_ms), dev)
    nbytes_state = 3 * NX * NY * 16

    forms = extra_workloads(dev) if (rank == 0 and not args.no_extra) else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        ra, ta, cores = cpu_oracle_rate(CPU_SAMPLE_STEPS, 0)
        r1, t1, _ = cpu_oracle_rate(CPU_SINGLE_STEPS, 1)
        cpu = {"value": ra, "unit": METRIC, "cores": cores, "kind": "oracle",
               "sample": "%d time steps of the 256x256 workload (%.1f s, %d OpenMP threads)" % (CPU_SAMPLE_STEPS, ta,
                                                                                             cores),
               "single_thread": {"value": r1, "cores": 1,
                                 "sample": "%d time steps (%.1f s)" % (CPU_SINGLE_STEPS, t1)}}

    lps = solver.launches_per_step()
    # + the end-of-steps norm/scale launch of the two-launch 2D step, flush, scale reset, observables
    launches = NSTEPS * lps + (1 if lps == 2 else 0) + 3
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "time_steps_per_bench_step": NSTEPS,
        "config": bench_config(ws),
        "roofline": {"bound": "alu", "kernel": dom_name,
                     "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp64_peak, "traffic": HEAD_TRAFFIC_BYTES,
                     "peak_source": peak_source, "nominal_peak": FP64_PEAK_TFLOPS,
                     "flops_per_point": dom_flops, "avg_launch_ms": dom_ms},
        "kernels": {"avg_ms": kavg, "share": share, "dominant": dom},
        "hbm_view": hbm_view(value / ws * 192 / 1e9),
        "chosen": {"form": "complex64 state, FP64 reductions", "value": replica_value(point_steps, ws, t32),
                   "ms_per_step": t32, "energy_rel_err_vs_fp64": abs(e32 - e64) / abs(e64),
                   "speedup_vs_fp64": t_step / t32, "kernels_avg_ms": kavg32},
        "fp64_accurate": {"form": "double-float (FP32 pairs), FP64 reductions", "value": replica_value(point_steps, ws, tdf),
                          "ms_per_step": tdf, "energy_rel_err_vs_fp64": abs(edf - e64) / abs(e64),
                          "state_rel_err_vs_fp64": state_err_df, "speedup_vs_fp64": t_step / tdf,
                          "kernels_avg_ms": kavgdf},
        "energy": {"E_fp64": e64, "E_c64": e32, "E_cdf": edf, "E_profile_pass": e_prof[5]},
        "forms": forms,
        "cpu_baseline": cpu,
        "e2e": {"value": replica_value(point_steps, ws, e2e_t), "unit": METRIC, "h2d_bytes_per_step": nbytes_state,
                "d2h_bytes_per_step": nbytes_state + 16 * 8, "ms_per_step": e2e_t},
        "gpu_launches": args.steps * launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
