#!/usr/bin/env python3
"""Benchmark of the fused D2Q9 MRT pseudopotential update on GB300.

Workload (one bench "step"): a 2048 x 2048 periodic lattice holding a Carnahan-Starling
droplet (a = 1, b = 4, R = 1, T = 0.8 T_c, G = -1, kappa = 0.6, nu = 0.1, radius 200,
tanh width 2, Maxwell densities), advanced by INNER = 100 time steps through lb_step
followed by one FP64 diagnostics reduction (lb_reduce: mass, momentum, max |u|).
Populations are FP32 (two buffers of 151 MB each, larger than the 129 MB L2).

Printed: one JSON line (rank 0). `value` = MLUPS over all ranks (device-timed, inputs
resident); `e2e` = the same through the C ABI with host buffers (populations in from
pinned host memory, density field out to pinned host memory, every step);
`roofline` = the fused kernel's algorithmic bytes per launch / its live CUDA-event
duration against the measured HBM copy bandwidth; `fp64` = the same workload in FP64;
`cpu_baseline` = the FP64 numpy oracle on one host core over a bounded sample;
`batched` = the 512-droplet sweep in one persistent launch per step; `surrogate` = the
network trained on a converged batched sweep and the kappa it picks, checked by Laplace
runs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU (torchrun): every rank advances its own replica lattice (the path does not
shard); `value` = total lattice updates of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline, FP32 vs FP64 on GB300; batched droplets/sec at σ err ≤1%"
NX, NY, INNER = 2048, 2048, 100
WORKLOAD = ("D2Q9 MRT pseudopotential droplet 2048x2048 periodic, Carnahan-Starling T=0.8Tc, "
            "G=-1, kappa=0.6, nu=0.1, R=200; 100 LB steps + 1 FP64 reduction per bench step")
ALG_BYTES_PER_SITE = {"fp32": 72, "fp64": 144, "bf16": 36}   # 9 populations read + 9 written


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--inner", type=int, default=INNER)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variant", type=int, default=-1,
                    help="step-kernel variant (-1: chosen by the library's autotuner)")
    ap.add_argument("--rows", type=int, default=0, help="rows per CTA (0: library default)")
    ap.add_argument("--batch-steps", type=int, default=10000,
                    help="time steps of the 512-lattice batched sweep (0: skip it)")
    ap.add_argument("--batch-lattices", type=int, default=512)
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage leg")
    ap.add_argument("--no-splash", action="store_true", help="skip the splash leg")
    ap.add_argument("--splash-steps", type=int, default=40000,
                    help="splash time steps per grid point (40000 = t* 5.05 at D 400, U 0.05)")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate leg (converged sweep, training, checked kappa)")
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------------------

def bench_config(nx, ny, inner, world):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD, "nx": nx, "ny": ny, "lb_steps_per_step": inner,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (2 x 151 MB FP32 population buffers)"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha(prec: str = "fp32") -> str:
    h = hashlib.sha256()
    unit = {"fp32": "f32", "fp64": "f64", "bf16": "bf16"}[prec]
    for name in ("lb_device.cuh", "lb_step.cuh", f"lb_step_{unit}.cu", f"lb_step_{unit}_stage.cu"):
        with open(os.path.join(ROOT, "paper_1306_6445_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_value(name: str, key: str, prec: str):
    """A figure of a committed ncu summary (profiles/<name>.md, `key: value`), if the
    summary was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_v = re.search(rf"{key}:\s*([0-9.eE+]+)", text)
    if not (m_sha and m_v) or m_sha.group(1) != kernel_source_sha(prec):
        return None
    return float(m_v.group(1))


def profiled_kernel(prec: str):
    """The kernel named by the committed 2048^2 summary (`kernel: name`), or None."""
    path = os.path.join(ROOT, "profiles", f"fused_step_{prec}_2048sq.md")
    if not os.path.exists(path):
        return None
    m = re.search(r"^kernel:\s*(\S+)", open(path).read(), re.M)
    return m.group(1) if m else None


def profiled_traffic(prec: str):
    """DRAM bytes per fused-step launch of the 2048^2 workload from the committed ncu summary."""
    return profiled_value(f"fused_step_{prec}_2048sq", "dram_bytes_per_launch", prec)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, one line every 50 ms from a single
    `nvidia-smi -lms 50` process that runs only while the sampler is entered (the timed
    region)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._p = None
        self._t = None

    def _read(self):
        for line in self._p.stdout:
            parts = [x.strip() for x in line.strip().split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __enter__(self):
        try:
            self._p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.1)               # the first line is out before the region starts
        except Exception:
            self._p = None
        return self

    def __exit__(self, *exc):
        if self._p is not None:
            time.sleep(0.06)              # one more line covering the end of the region
            self._p.terminate()           # this object's own child process
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
            self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def droplet_setup(lbm, inputs, nx, ny):
    eos = lbm.cs_eos(0.8)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    rates = lbm.RateParams.from_viscosity(0.1)
    rho = inputs.droplet_density(nx, ny, 200.0 * min(nx, ny) / 2048.0, rl, rv)
    return eos, rates, rho


# --------------------------------------------------------------------------------------
# native arm
# --------------------------------------------------------------------------------------

def time_precision(lbm, torch, inputs, prec, nx, ny, inner, steps, warmup, dist, launch=None,
                   clocks=None, stochastic=False):
    eos, rates, rho = droplet_setup(lbm, inputs, nx, ny)
    # BF16 storage: shift by the vapour density (most sites of the droplet lattice)
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.6, rates=rates, prec=prec,
                      storage_shift=float(rho.min()), stochastic_rounding=stochastic)
    lat.set_rho_u(rho)
    if launch is not None and launch[0] >= 0:
        lbm.lb_set_launch(lat.ctx, launch[0], launch[1])
    else:
        # the library's own launch autotuner (state unchanged); 20 launches per timed run
        # separate candidates about 1 % apart, FP64 launches are 30x longer
        lat.autotune(3 if prec == "fp64" else 20)
    shape = lbm.lb_get_launch(lat.ctx)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        lat.step(inner)
        lat.reduce()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.__enter__()
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        lat.step(inner)
        ev[k][1].record(stream)
        lat.reduce()
    t1.record(stream)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.__exit__(None, None, None)
    if dist is not None:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    step_kernel_ms = sum(a.elapsed_time(b) for a, b in ev)
    launches = steps * (inner * lbm.lb_kernels_per_step(lat.ctx) + 3)
    lat.close()
    return total_ms, step_kernel_ms / (steps * inner), launches, shape


def fp64_alu_roofline(lbm, torch, sites, kern_ms):
    """The FP64 update against its ALU roof: FP64-pipe thread instructions per site (ncu
    count, committed summary) x sites / the step kernel's CUDA-event time, against the FP64
    FMA rate the library's probe measures on this GPU now (every FP64 add, multiply and FMA
    takes one issue slot of the same pipe)."""
    peak = lbm.lb_probe_fp64_fma_rate(torch.cuda.current_stream().cuda_stream, 4096)
    inst = profiled_value("fused_step_fp64_2048sq", "fp64_pipe_inst_per_site", "fp64")
    out = {"bound": "alu", "peak": round(peak / 1e9, 2), "unit": "G FP64 inst/s",
           "peak_source": "lb_probe_fp64_fma_rate (measured FP64 FMA rate)",
           "inst_per_site": inst, "achieved": None, "frac": None}
    if inst is not None:
        achieved = inst * sites / (kern_ms * 1e-3)
        out.update(achieved=round(achieved / 1e9, 2), frac=round(achieved / peak, 4))
    return out


def time_e2e(lbm, torch, inputs, nx, ny, inner, steps, warmup):
    """Through the C ABI with host buffers: each step copies the populations in from pinned
    host memory (lb_set_populations), runs `inner` steps and reads the density field back
    into pinned host memory (lb_get_rho)."""
    eos, rates, rho = droplet_setup(lbm, inputs, nx, ny)
    lat = lbm.Lattice(nx, ny, eos, -1.0, kappa=0.6, rates=rates, prec="fp32")
    lat.set_rho_u(rho)
    f_host = torch.empty((9, ny, nx), dtype=torch.float32, pin_memory=True)
    import numpy as np
    f_host.numpy()[...] = lat.populations()
    rho_host = torch.empty((ny, nx), dtype=torch.float64, pin_memory=True)
    rho_np = rho_host.numpy()
    bi, bo = f_host.numel() * 4, rho_host.numel() * 8

    def one():
        lbm.lb_set_populations(lat.ctx, f_host.data_ptr(), bi)
        lbm.lb_step(lat.ctx, inner)
        lbm.lb_get_rho(lat.ctx, rho_np)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    lat.close()
    assert np.isfinite(rho_np).all()
    return el, bi, bo


def batch_setup(lbm, inputs, draws):
    """Lattice descriptors and initial densities of sweep draws: CS a=1 b=4 R=1, G=-1,
    sigma_F=0.087, Maxwell initial densities."""
    descs, rhos = [], []
    for d in draws:
        eos = lbm.cs_eos(d["t_over_tc"])
        rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
        descs.append(lbm.LatticeDesc(d["side"], d["side"], eos, -1.0, kappa=d["kappa"],
                                     sigma_force=0.087,
                                     rates=lbm.RateParams(s_v=1.0 / d["tau_v"])))
        rhos.append(inputs.droplet_density(d["side"], d["side"], d["radius"], rl, rv))
    return descs, rhos


def batched_sweep(lbm, torch, inputs, n_lat, steps, seed=1306, sample=24, dist=None):
    """The batched Laplace-law sweep: n_lat periodic droplet lattices drawn with the given
    seed (side U{64..512 step 32}, R/side U[0.15, 0.35], T/Tc U[0.65, 0.95], kappa
    U[0, 0.95], tau_v U[0.6, 1.2]; CS a=1 b=4 R=1, G=-1, sigma_F=0.087, Maxwell initial
    densities, FP32) in one persistent launch per step replayed from CUDA graphs.

    throughput_10k: `steps` steps of every lattice, against `sample` of the lattices run one
    by one through lb_step (extrapolated to all).
    converged: every lattice runs for its own step budget (0.5 side^2, at least 8192;
    sweep.step_budget) and is retired when done, its surface tension averaged over its last
    2048 steps and checked against the same average at 3/4 of the budget (converged when
    they agree within 1 %); compared with one lattice per side run alone through lb_step
    under the same protocol (extrapolated by side), and with FP64 batched runs of one lattice
    each of sides 64, 128, 256, 384 and 512 (surface-tension error of the FP32 batch).

    Under torchrun the lattices are split across ranks (independent problems, no
    data-path communication, site counts balanced); every rank times its own batch and
    the whole-job rates use the slowest rank's time (weak scaling in lattices)."""
    import numpy as np
    from paper_1306_6445_gb300 import shard, sweep
    world = dist.get_world_size() if dist is not None else 1
    rank = dist.get_rank() if dist is not None else 0
    all_draws = inputs.batch_draws(n_lat, seed)
    mine = shard.assign([d["side"] ** 2 for d in all_draws], world)[rank]
    draws = [all_draws[i] for i in mine]
    descs, rhos = batch_setup(lbm, inputs, draws)
    radii = np.array([d["radius"] for d in draws])
    sides = np.array([d["side"] for d in draws])
    sites_all = sum(d["side"] ** 2 for d in all_draws)

    def slowest(el):
        if dist is not None:
            tt = torch.tensor([el], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        return el

    # ---- fixed step count (throughput)
    b = lbm.Batch(descs, prec="fp32")
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    # the library's batch autotuner, timed on these states (it restores them)
    variant, rows = b.autotune(3)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    b.step(steps)
    b.sync()
    el = slowest(time.perf_counter() - t0)
    meas = b.measure(radii)
    failed = int(shard.gather_rows(meas, mine, n_lat, dist)[:, 7].sum())
    launch = b.launch()
    b.close()
    rng = np.random.default_rng(seed + 1)
    pick = rng.choice(len(descs), size=min(sample, len(descs)), replace=False)
    t_seq = 0.0
    for i in pick:
        d = descs[i]
        lat = lbm.Lattice(d.nx, d.ny, d.eos, d.G, kappa=d.kappa, sigma_force=d.sigma_force,
                          rates=d.rates, prec="fp32")
        lat.set_rho_u(rhos[i])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lat.step(steps)
        lat.sync()
        t_seq += time.perf_counter() - t1
        lat.close()
    seq_per_lattice = t_seq / len(pick)
    throughput = {
        "steps": steps, "seconds": round(el, 4), "failed": failed,
        "droplets_per_s": round(n_lat / el, 2),
        "mlups": round(sites_all * steps / el / 1e6, 1),
        "sequential_droplets_per_s": round(world / seq_per_lattice, 2),
        "speedup_vs_sequential": round(seq_per_lattice * n_lat / (el * world), 2),
        "launch": launch, "autotuned": {"variant": variant, "rows": rows}}

    # ---- every lattice to its own converged budget
    budgets = np.array([sweep.step_budget(int(s)) for s in sides])
    b = lbm.Batch(descs, prec="fp32")
    for i, r in enumerate(rhos):
        b.set_rho_u(i, r)
    b.autotune(3)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    res = sweep.converged_readings(b, budgets, radii)
    torch.cuda.synchronize()
    el_c = slowest(time.perf_counter() - t0)
    b.close()
    rows_c = np.stack([res["theta"], res["converged"], res["failed"], res["steps"]], axis=1)
    table = shard.gather_rows(rows_c, mine, n_lat, dist)
    n_conv = int(table[:, 1].sum())
    lu_all = float(sum(d["side"] ** 2 * table[k, 3] for k, d in enumerate(all_draws)))
    n_ext = int(sum(table[k, 3] > sweep.step_budget(d["side"]) for k, d in enumerate(all_draws)))
    # one lattice per side alone through lb_step under the same protocol
    t_side = {}
    for s_ in sorted(set(sides.tolist())):
        i = int(np.flatnonzero(sides == s_)[0])
        d = descs[i]
        lat = lbm.Lattice(d.nx, d.ny, d.eos, d.G, kappa=d.kappa, sigma_force=d.sigma_force,
                          rates=d.rates, prec="fp32")
        lat.set_rho_u(rhos[i])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sweep.converged_single(lat, int(budgets[i]), float(radii[i]))
        t_side[s_] = time.perf_counter() - t1
        lat.close()
    # a lattice's time alone scales with its step count (extensions included)
    t_seq_c = float(sum(t_side[int(s_)] * res["steps"][i] / budgets[i]
                        for i, s_ in enumerate(sides)))
    # FP64 batched reference of one lattice each of five sides spanning the range
    err = None
    if rank == 0:
        ref_idx = []
        for s_ in (64, 128, 256, 384, 512):
            hits = [k for k, d in enumerate(all_draws) if d["side"] == s_]
            if hits:
                ref_idx.append(hits[0])
        rdraws = [all_draws[k] for k in ref_idx]
        rdescs, rrhos = batch_setup(lbm, inputs, rdraws)
        b64 = lbm.Batch(rdescs, prec="fp64")
        for i, r in enumerate(rrhos):
            b64.set_rho_u(i, r)
        r64 = sweep.converged_readings(b64, [sweep.step_budget(d["side"]) for d in rdraws],
                                       [d["radius"] for d in rdraws])
        b64.close()
        e = np.abs(table[ref_idx, 0] / r64["theta"] - 1.0)
        err = {"sides": [d["side"] for d in rdraws],
               "rel_err": [round(float(x), 6) for x in e],
               "max": round(float(e.max()), 6), "within_1pct": int((e <= 0.01).sum())}
    return {
        "lattices": n_lat, "sites": sites_all, "ranks": world,
        "throughput_10k": throughput,
        "converged": {
            "protocol": "per-lattice budget 0.5 side^2 steps (>= 8192), retired when done; "
                        "sigma = mean of the last 2048 steps, converged if within 1 % of the "
                        "same mean at 3/4 of the budget, else run on by half the budget "
                        "(at most twice) and compared with the previous reading",
            "extended": n_ext,
            "seconds": round(el_c, 3), "lattice_updates": lu_all,
            "mlups": round(lu_all / el_c / 1e6, 1),
            "converged": n_conv, "converged_fraction": round(n_conv / n_lat, 4),
            "failed": int(table[:, 2].sum()),
            "droplets_per_s_converged": round(n_conv / el_c, 2),
            "sequential_seconds_estimate": round(t_seq_c, 3),
            "speedup_vs_sequential": round(t_seq_c / el_c, 2),
            "sigma_rel_err_vs_fp64": err,
            "theta_median": float(np.median(table[table[:, 1] == 1, 0])) if n_conv else None},
    }


def bf16_error_table(lbm, inputs, n=256, steps=40000, window=2048):
    """Converged n^2 droplet (CS 0.8 T_c, R = 50, nu = 0.1, Maxwell initial densities):
    density ratio and Laplace surface tension (p_in - p_out) R, each averaged over 32 GPU
    readings (lb_measure_droplet) in the last `window` steps, max |v| and mass drift in FP32
    and BF16 storage (rho_s = vapour density; nearest and stochastic rounding) relative to
    FP64."""
    import numpy as np
    eos = lbm.cs_eos(0.8)
    rates = lbm.RateParams.from_viscosity(0.1)
    pv, pl, _ = lbm.lb_maxwell(eos, -1.0)
    rows = {}
    for name in ("fp64", "fp32", "bf16", "bf16_stochastic"):
        prec = name.split("_")[0]
        lat = lbm.Lattice(n, n, eos, -1.0, rates=rates, prec=prec, storage_shift=pv,
                          stochastic_rounding=name.endswith("stochastic"))
        lat.set_rho_u(inputs.droplet_density(n, n, 50.0, pl, pv))
        m0 = lat.reduce()
        lat.step(steps - window)
        acc = np.zeros(2)
        k = window // 64
        for _ in range(k):
            lat.step(64)
            d = lat.measure_droplet(50.0)
            acc += (d["rho_in"] / d["rho_out"], d["theta"])
        m1 = lat.reduce()
        lat.close()
        rows[name] = {"ratio": acc[0] / k, "theta": acc[1] / k, "umax": m1[3],
                      "mass_drift": (m1[0] - m0[0]) / m0[0]}
    ref = rows["fp64"]
    out = {}
    for name in ("fp32", "bf16", "bf16_stochastic"):
        r = rows[name]
        out[name] = {"ratio_rel_err": round(r["ratio"] / ref["ratio"] - 1, 5),
                     "sigma_rel_err": round(r["theta"] / ref["theta"] - 1, 5),
                     "umax_vs_fp64": round(r["umax"] / ref["umax"], 3),
                     "mass_drift": float(f"{r['mass_drift']:.3e}")}
    out["workload"] = (f"{n}^2 droplet, CS 0.8Tc, R=50, nu=0.1, {steps} steps, rho_s=rho_v; "
                       f"ratio and sigma averaged over the last {window} steps")
    return out


def surrogate_leg(lbm, torch, n_train=512):
    """The surrogate end to end: a converged batched Laplace sweep of n_train droplets
    (128^2, R = 32, 24000 steps, reading averaged over the last 2048), full-batch Adam
    training in the library's kernels, then kappa for the hardest targets (the smallest
    sigma per temperature, kappa near 0.93) checked by a plain Laplace run, against the
    Eq. 22 law calibrated by a kappa = 0 run."""
    import numpy as np
    from paper_1306_6445_gb300 import surrogate, sweep

    X = sweep.training_points(n_train)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Y = sweep.laplace_points(lbm, X)
    t_sweep = time.perf_counter() - t0
    ok = Y[:, 3] == 0
    t0 = time.perf_counter()
    net, losses = surrogate.fit(lbm, X[ok], Y[ok, :3])
    t_fit = time.perf_counter() - t0
    adam_steps = sum(s for s, _ in surrogate.SCHEDULE)
    # per-step time of the training kernels alone (graph replays, no host work between)
    t0 = time.perf_counter()
    net.train(1000, 1e-5)
    us_step = (time.perf_counter() - t0) / 1000 * 1e6
    g = np.array([(0.7, 0.7, 5e-4), (0.7, 1.1, 5e-4), (0.8, 0.7, 2.5e-4), (0.8, 1.1, 2.5e-4),
                  (0.9, 0.7, 9e-5), (0.9, 1.1, 9e-5)])
    res = surrogate.tune_kappa(lbm, net, g[:, 0], g[:, 1], g[:, 2], tol=0.02, max_rounds=0)
    s0 = surrogate.sweep_points(lbm, g[:, 0], np.zeros(len(g)), g[:, 1])
    s_law = surrogate.sweep_points(lbm, g[:, 0], 1 - g[:, 2] / s0, g[:, 1])
    e_net, e_law = np.abs(res["rel_err"]), np.abs(s_law / g[:, 2] - 1)
    return net, {
        "train_samples": int(ok.sum()), "sweep_seconds": round(t_sweep, 3),
        "sweep_droplets_per_s": round(n_train / t_sweep, 1),
        "fit_seconds": round(t_fit, 3), "adam_steps": adam_steps,
        "us_per_adam_step": round(us_step, 2),
        "train_samples_per_s": round(int(ok.sum()) / (us_step * 1e-6), 0),
        "final_loss": losses[-1],
        "checked_targets": len(g), "laplace_runs_per_target": float(res["runs"].mean()),
        "sigma_err_net_max": round(float(e_net.max()), 5),
        "sigma_err_law_max": round(float(e_law.max()), 5),
        "law_calibration_runs_per_target": 1,
    }


def splash_point(lbm, torch, net, nx, ny, D, We, Re, U, t_over_tc, steps):
    """One droplet-splash run at 4096 x 1024 (film 0.1 D), FP32, CS at t_over_tc T_c with
    sigma_F = 0.087; Re = U D / nu_L, nu_V = 20 nu_L switched at the mean phase density; the
    target surface tension follows from We = rho_L U^2 D / sigma, and kappa comes from the
    surrogate network, checked by one Laplace run (128^2). The run starts at t* = 0.05
    after the first contact (splash.T0) and goes on for `steps` steps or until the EOS
    branch is left (recorded). Reports the kernel rate and the spread radius."""
    from paper_1306_6445_gb300 import splash, surrogate

    eos = lbm.cs_eos(t_over_tc)
    rv, rl, _ = lbm.lb_maxwell(eos, -1.0)
    sigma_t = rl * U * U * D / We
    nu_l = U * D / Re
    tau_l = 3.0 * nu_l + 0.5
    res = surrogate.tune_kappa(lbm, net, t_over_tc, tau_l, sigma_t, tol=0.02, max_rounds=2)
    kappa = float(res["kappa"][0])
    film = 0.1 * D
    lat = splash.make_lattice(lbm, nx, ny, eos, -1.0, kappa, 0.087, D, film, U, nu_l,
                              20.0 * nu_l, 0.5 * (rl + rv), rl, rv)
    lat.autotune(3)
    stream = torch.cuda.current_stream()
    marks = {splash.steps_to(t, D, U): t for t in (0.25, 0.75, 1.0, 1.5, 1.75, 2.5, 5.0)
             if splash.steps_to(t, D, U) <= steps}
    stops = sorted(set(marks) | set(range(1000, steps, 1000)) | {steps})
    radii = {}
    done, failed, ms = 0, None, 0.0
    torch.cuda.synchronize()
    try:
        for stop in stops:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(stop - done)
            e1.record(stream)
            lat.sync()                      # an EOS-domain error surfaces here
            ms += e0.elapsed_time(e1)
            done = stop
            if done in marks:
                radii[marks[done]] = round(splash.spread_radius(lat.rho(), film, D, rl, rv), 4)
    except lbm.LBError as e:
        failed = f"{lbm.STATUS_NAMES.get(e.status, e.status)} between steps {done} and {stop}"
    launch = lbm.lb_get_launch(lat.ctx)
    lat.close()
    return {"We": We, "Re": Re, "t_over_tc": t_over_tc, "density_ratio": round(rl / rv, 2),
            "kappa_from_surrogate": round(kappa, 5),
            "sigma_target": sigma_t, "sigma_checked_rel_err": round(float(res["rel_err"][0]), 5),
            "laplace_runs": int(res["runs"][0]),
            "mlups": round(nx * ny * done / (ms * 1e-3) / 1e6, 1) if done else None,
            "steps_done": done, "breakdown": failed, "launch": launch,
            "t_star_end": round(splash.T0 + U * done / D, 3),
            "spread_radius_over_D_at_t_star": radii,
            "power_law_1p3_sqrt_t": {t: round(1.3 * t ** 0.5, 4) for t in radii}}


def splash_leg(lbm, torch, net, nx=4096, ny=1024, D=400.0, U=0.05, t_over_tc=0.65,
               steps=None, t_retry=0.70):
    """The droplet-splash workload at 4096 x 1024 over the grid We in {200, 800} x Re in
    {500, 1000} (D = 400, U = 0.05, CS at 0.65 T_c), each point `steps` steps long. A point
    that leaves the EOS branch before t* = 1.75 (the paper's last time) runs again at
    t_retry T_c, a higher vapour density and a lower density ratio; both runs are listed."""
    from paper_1306_6445_gb300 import splash

    steps = ARGS.splash_steps if steps is None else steps
    points = []
    for We in (200.0, 800.0):
        for Re in (500.0, 1000.0):
            p = splash_point(lbm, torch, net, nx, ny, D, We, Re, U, t_over_tc, steps)
            points.append(p)
            if p["breakdown"] and p["steps_done"] < splash.steps_to(1.75, D, U):
                points.append(splash_point(lbm, torch, net, nx, ny, D, We, Re, U, t_retry, steps))
    return {"workload": f"{nx}x{ny} splash, D={D:.0f}, film {0.1 * D:.0f}, CS {t_over_tc}Tc "
                        f"(points that leave the EOS branch before t*=1.75 again at "
                        f"{t_retry}Tc), U={U}, FP32, up to {steps} steps per point, start at "
                        f"t*=0.05",
            "points": points}


def host_cpu():
    """The host's logical core count and CPU model (lscpu's model name, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"host_cores": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_baseline(nx, ny, budget_s=20.0):
    """The FP64 numpy oracle, single thread, on the same droplet lattice: as many whole
    steps as fit in ~budget_s (at least one). Runs in a child process so the BLAS thread
    count can be pinned to one."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
import numpy as np
from oracle import eos as OE, lattice as OL
from paper_1306_6445_gb300 import inputs
nx, ny, budget = %d, %d, %f
eos = OE.cs_eos(0.8)
rv, rl, _ = OE.maxwell(eos, -1.0)
rho = inputs.droplet_density(nx, ny, 200.0 * min(nx, ny) / 2048.0, rl, rv)
f = OL.equilibrium(rho, 0 * rho, 0 * rho)
p = OL.Params(eos=eos, G=-1.0, kappa=0.6, rates=OL.Rates.from_viscosity(0.1))
t = time.perf_counter(); n = 0
while True:
    f = OL.step(f, p); n += 1
    if time.perf_counter() - t > budget: break
el = time.perf_counter() - t
print(json.dumps({"steps": n, "seconds": el, "mlups": nx * ny * n / el / 1e6}))
""" % (ROOT, nx, ny, budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": "MLUPS", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return dict({"value": round(d["mlups"], 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                 "sample": f"{d['steps']} FP64 steps of the full {nx}x{ny} lattice "
                           f"({d['seconds']:.1f} s, numpy, 1 thread)"}, **host_cpu())


def native(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1306_6445_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()
    from paper_1306_6445_gb300 import inputs, lbm

    nx, ny, inner, K, W = args.nx, args.ny, args.inner, args.steps, args.warmup
    sites = nx * ny
    clocks = ClockSampler(local)
    total_ms, kern_ms, launches, shape = time_precision(lbm, torch, inputs, "fp32", nx, ny,
                                                        inner, K, W, dist,
                                                        (args.variant, args.rows), clocks)
    t = torch.tensor([total_ms], device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    value = world * sites * inner * K / (max_ms * 1e-3) / 1e6

    hbm, peak_src = measured_peaks()
    alg = ALG_BYTES_PER_SITE["fp32"] * sites
    achieved = alg / (kern_ms * 1e-3) / 1e9
    kname = "k_pull_collide_stage<float>" if shape["variant"] >= 4 else "k_pull_collide<float>"
    # the committed capture counts only for the kernel it was taken on
    traffic = profiled_traffic("fp32") if profiled_kernel("fp32") == kname else None
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic,
            "kernel": kname, "launch": shape, "alg_bytes_per_launch": alg,
            "kernel_ms": round(kern_ms, 5), "peak_source": f"{peak_src} (copy bandwidth)"}

    # FP64 leg
    fk = max(args.fp64_steps, 1)
    f_total, f_kern, _, shape64 = time_precision(lbm, torch, inputs, "fp64", nx, ny, inner, fk, 1,
                                                 dist)
    alg64 = ALG_BYTES_PER_SITE["fp64"] * sites
    fp64 = {"value": round(sites * inner * fk / (f_total * 1e-3) / 1e6, 1), "unit": "MLUPS",
            "kernel_ms": round(f_kern, 5),
            "hbm_frac": round(alg64 / (f_kern * 1e-3) / 1e9 / hbm, 4), "launch": shape64,
            "roofline": fp64_alu_roofline(lbm, torch, sites, f_kern)}

    # BF16 storage leg: speed, and the error table of a converged droplet against FP64
    bf16 = None
    if not args.no_bf16:
        b_total, b_kern, _, shape16 = time_precision(lbm, torch, inputs, "bf16", nx, ny, inner,
                                                     max(K // 2, 1), 1, dist)
        alg16 = ALG_BYTES_PER_SITE["bf16"] * sites
        s_total, s_kern, _, shape16s = time_precision(lbm, torch, inputs, "bf16", nx, ny, inner,
                                                      max(K // 2, 1), 1, dist, stochastic=True)
        bf16 = {"value": round(sites * inner * max(K // 2, 1) / (b_total * 1e-3) / 1e6, 1),
                "unit": "MLUPS", "kernel_ms": round(b_kern, 5),
                "hbm_frac": round(alg16 / (b_kern * 1e-3) / 1e9 / hbm, 4), "launch": shape16,
                "stochastic_rounding": {
                    "value": round(sites * inner * max(K // 2, 1) / (s_total * 1e-3) / 1e6, 1),
                    "kernel_ms": round(s_kern, 5),
                    "hbm_frac": round(alg16 / (s_kern * 1e-3) / 1e9 / hbm, 4),
                    "launch": shape16s},
                "error_vs_fp64": bf16_error_table(lbm, inputs)}

    e2e = None
    if not args.no_e2e:
        el, bi, bo = time_e2e(lbm, torch, inputs, nx, ny, inner, K, min(W, 2))
        if dist is not None:                     # the slowest rank's wall time
            te = torch.tensor([el], device="cuda")
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            el = float(te.item())
        e2e = {"value": round(world * sites * inner * K / el / 1e6, 1), "unit": "MLUPS",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}

    batched = None
    if args.batch_steps > 0:
        batched = batched_sweep(lbm, torch, inputs, args.batch_lattices, args.batch_steps,
                                dist=dist)
    surr = splash = None
    if not args.no_surrogate:
        net, surr = surrogate_leg(lbm, torch)
        if not args.no_splash:
            splash = splash_leg(lbm, torch, net)
        net.close()
    if rank == 0:
        cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(nx, ny)
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(max_ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(nx, ny, inner, world),
            "roofline": roof, "fp64": fp64, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks.summary(), "bf16": bf16,
            "batched": batched,
            "surrogate": surr, "splash": splash,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# --------------------------------------------------------------------------------------

def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one host thread for numpy's BLAS: set before numpy is first imported
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from oracle import eos as OE
    from oracle import lattice as OL
    from paper_1306_6445_gb300 import inputs

    # bounded sample of the workload: the whole droplet lattice (the same lattice as the
    # native arm and its cpu_baseline), one LB step per bench step (about 1.3 s each at
    # 2048^2 on one host core)
    nx, ny = args.nx, args.ny
    eos = OE.cs_eos(0.8)
    rv, rl, _ = OE.maxwell(eos, -1.0)
    rho = inputs.droplet_density(nx, ny, 200.0 * min(nx, ny) / 2048.0, rl, rv)
    f = OL.equilibrium(rho, 0 * rho, 0 * rho)
    p = OL.Params(eos=eos, G=-1.0, kappa=0.6, rates=OL.Rates.from_viscosity(0.1))
    for _ in range(args.warmup):
        f = OL.step(f, p)
    t = time.perf_counter()
    for _ in range(args.steps):
        f = OL.step(f, p)
    el = time.perf_counter() - t
    v = nx * ny * args.steps / el / 1e6
    sample = f"{args.steps} FP64 steps of the full {nx}x{ny} droplet lattice (numpy, 1 thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(bench_config(args.nx, args.ny, args.inner,
                                    int(os.environ.get("WORLD_SIZE", "1"))),
                       sample=f"the full {nx}x{ny} lattice, 1 LB step per bench step"),
        "cpu_baseline": dict({"value": round(v, 4), "unit": "MLUPS", "cores": 1,
                              "kind": "oracle", "sample": sample}, **host_cpu()),
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


ARGS = None


def main():
    global ARGS
    args = parse()
    ARGS = args
    if args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
