"""Throughput of the frequency-dependent irradiation ray tracer on GB300.

One step traces every grid of the 3-D disk-plus-envelope workload through the C
ABI (rt_irradiate, then the FP64 energy reduction of Eqs. 33-35 on the device):
by default the 512 x 256 x 512 grid (r, theta, phi; 67.1 M cells), 79 frequency
bins, midplane tau550 = 1 and 100, seeded synthetic inputs. The metric is cell x
frequency-bin updates per second. The 256 x 128 x 256 four-grid step (tau550 = 0.1,
1, 10, 100) rides along as a secondary object. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference that exists
for this method) on a bounded sample of the same workload, on the host cores.
Under torchrun every rank traces its own replica of the workload (independent
grids, no data exchange); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
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

import synth  # noqa: E402

METRIC = "ray-traced cell·freq updates/s (plain vs MLP surrogate @≤1e-3 err); % roofline"
UNIT = "cell·nu updates/s"
# the disk-plus-envelope workloads: grid, bins, midplane optical depths, seed
WORKLOADS = {
    "c3": {"nr": 512, "ntheta": 256, "nphi": 512, "n_nu": 79, "taus": (1.0, 100.0), "seed": 2},
    "c2": {"nr": 256, "ntheta": 128, "nphi": 256, "n_nu": 79, "taus": (0.1, 1.0, 10.0, 100.0), "seed": 1},
}
NNU = 79
# the 256 x 128 x 256 grid of the steps after the tracer (dust temperature, kappa(nu, T)
# tracer, flux-limited diffusion) and of the secondary tracer object
NR, NTH, NPH = 256, 128, 256
# rt_opacity_table_kind values
TABLE_KINDS = ("nu", "nu_t_separable", "nu_t", "nu_t_rank2", "nu_t_low_rank")
# tracer kernels (RT_KERNEL_*)
KERNEL_KINDS = ("tile", "ray", "ray_chunked")


def workload_name(spec, taus):
    return (f"disk3d {spec['nr']}x{spec['ntheta']}x{spec['nphi']} (r,theta,phi), {spec['n_nu']} nu bins, "
            f"tau550 in {{{','.join(f'{t:g}' for t in taus)}}}, env+20% lognormal, T_dust U(20,1600), "
            f"seed {spec['seed']}")


# algorithmic bytes per cell of the flux-limited-diffusion step (each array read or
# written once per kernel; stencil neighbours from cache). Set-up: 28 (cell kernel:
# rho, T, q, E in; F, storage, rhs out) + 36 (faces: 3 in; w[3], s, 1/dg, b out) + 8
# (start-value copy); with multigrid also 10 (BF16 copies of s, w[3], 1/dg) + 16 (the
# Galerkin coarsening reads s, w[3]; the coarse levels are 1/8, 1/64, ... of that).
# Jacobi iteration: 24 (apply: p, s, w[3] in; q out) + 28 (update: d, p, q, r, 1/dg in;
# d, r out) + 16 (direction); per pass 40 (residual) + 12 (accumulate). Multigrid
# iteration: 24 (apply) + 24 (update: d, p, q, r in; d, r out) + 12 (direction: z, p in;
# p out) + 14 (restriction: b in FP32, 1/dg, s, w[3] in BF16) + 18 (prolongation: the
# same in, z out) + 8 (the coarser levels); per pass 36 (residual: b, s, w[3], x in; r,
# d, p out) + 52 (one V-cycle and the direction) + 12 (accumulate)
FLD_SETUP_B, FLD_PASS_B, FLD_ITER_B = 72, 52, 68
FLD_SETUP_MG_B, FLD_PASS_MG_B, FLD_ITER_MG_B = 98, 100, 100
# exp-class operations per (cell, bin) traced bin by bin: e^{-tau_in}. The absorbed
# fraction 1 - e^{-dtau} needs a second one only where dtau is not small.
EXP_PER_CELL_NU = 1
# bins with kappa_i N_max <= THIN_X (N_max the largest total column of the rays one
# warp traces) enter the tracer's power series instead (no exponential per cell)
THIN_X = 1.0
# FMA-pipe operations of the power series per cell (paired Horner form of
# kThinTerms = 10 terms: 2 K + 1), and per (cell, bin) traced bin by bin at the least
# (the exponent's FMA and the accumulation)
SERIES_FMA_PER_CELL = 21
EXACT_FMA_PER_PAIR = 2
# algorithmic bytes per cell of the tracer: rho, T_dust in, q_abs, a_rad out (FP32)
TRACE_BYTES_PER_CELL = 16
# the roofline fraction the tracer is meant to reach on its binding floor
ROOFLINE_TARGET = 0.6
PROFILE_DIR = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = ("rt_ray.cu", "rt_ray_mc.cu", "rt_ray.cuh", "rt_device.cuh", "rt_internal.cuh")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", default="fp32_kahan")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="c3",
                   help="c3: the 512x256x512 grid at tau550 = 1 and 100 (default); c2: the 256x128x256 "
                        "grid at tau550 = 0.1, 1, 10, 100")
    p.add_argument("--grids", default=None,
                   help="comma-separated tau550 values of the grids in one step (default: the workload's)")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the secondary tracer object (the other workload of WORKLOADS)")
    p.add_argument("--shape", default=None,
                   help="force the tracer shape 'kind,cells_per_lane,warps,min_blocks' (skips the autotuner)")
    p.add_argument("--precision-sweep", action="store_true",
                   help="instead of the throughput line: error of every precision mode against the "
                        "FP64 oracle on the 512x256x512, 79-bin disk at tau550 = 1 and 100")
    p.add_argument("--sweep-grid", default="512x256x512")
    p.add_argument("--batch", action="store_true",
                   help="instead of the throughput line of the 4-grid step: the 96-grid uneven "
                        "batch (one persistent launch per step, CUDA-graph replay)")
    p.add_argument("--cpu-table", action="store_true",
                   help="instead of the throughput line: oracle (1 core, all cores) and GPU throughput of "
                        "the 2-D disk, the 3-D disk at tau 1 and 100, and the 512x256x512 disk")
    p.add_argument("--no-fld", action="store_true", help="skip the flux-limited-diffusion leg")
    p.add_argument("--fld", action="store_true",
                   help="print only the flux-limited-diffusion leg (trace the tau = 1 disk of --fld-grid, then "
                        "time --steps FLD steps with its q_abs)")
    p.add_argument("--fld-grid", default="256x128x256")
    p.add_argument("--fld-dt", type=float, default=1e4, help="FLD time step (s); the paper's is 1e4")
    p.add_argument("--no-surrogate", action="store_true",
                   help="skip the learned-surrogate leg of the default line")
    p.add_argument("--surrogate", action="store_true",
                   help="print only the learned-surrogate leg (train, then time against the exact tracer)")
    p.add_argument("--lut", action="store_true",
                   help="print only the lookup-table comparator (against the exact tracer on the 512x256x512 grids)")
    p.add_argument("--sur-grid", default="512x256x512", help="grid the surrogate is timed on")
    p.add_argument("--sur-train-grid", default="256x128x128", help="geometry of the training fields")
    p.add_argument("--sur-steps", type=int, default=60000, help="Adam steps of the surrogate training")
    p.add_argument("--sur-reps", type=int, default=10, help="timed calls per mode")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workloads(spec, taus, seed_offset=0):
    return [synth.disk3d(spec["nr"], spec["ntheta"], spec["nphi"], n_nu=spec["n_nu"], tau550=t,
                         seed=spec["seed"] + seed_offset) for t in taus]


def step_taus(args, spec):
    return tuple(float(x) for x in args.grids.split(",")) if args.grids else tuple(spec["taus"])


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_summary_path(spec):
    return os.path.join(PROFILE_DIR, f"k_ray_disk3d_{spec['nr']}x{spec['ntheta']}x{spec['nphi']}_nu{spec['n_nu']}.md")


def traffic_from_profile(path: str, src_hash: str):
    """DRAM bytes per launch of the tracer from a committed ncu summary, only if it
    was taken on the current kernel source."""
    try:
        txt = open(path).read()
    except OSError:
        return None
    h = None
    t = None
    for line in txt.splitlines():
        if line.startswith("kernel_source_sha256:"):
            h = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_full_launch:"):
            t = float(line.split(":", 1)[1].strip())
    return t if (h == src_hash and t is not None) else None


def _warp_partition(w, shape):
    """Per warp of the warp-per-ray kernel: the cells it traces, the bins its thin
    series takes (bt: kappa_i N_max <= THIN_X, N_max the largest total column of its
    rays) and the end of its tier (bt2: kappa_i c_max <= THIN_X, c_max the largest
    column of one lane's C cells; the tier is used when it adds bins and either a thin
    row exists or it adds >= 4). A warp holds R = 32 / G rays of G lanes of C cells
    where 32 C cells hold a ray; for C <= 8 and rays of up to 64 C cells, two warps
    share a ray (each 32 C of its cells, N_max the ray's total). The chunked kernel
    (kind 2) counts per warp and chunk: 4 rays of 8 lanes, N_max the largest column at
    the chunk's end, and its last live bin (na: kappa_i N <= 127 ln 2 at the smallest
    column in front of a lane; the bins after it underflow and are skipped). Returns
    cells, bt, bt2 and na per unit (na a single value but for the chunked kernel)."""
    nr, c = w.grid.nr, shape[1]
    dust = w.tdust32() <= w.t_sub
    col = (np.where(dust, w.rho32().astype(np.float64), 0.0) * np.diff(w.grid.r_if)).reshape(-1, nr)
    kap = np.sort(w.kappa[w.kappa > 0])
    na = np.full(1, len(kap))
    if shape[0] == 2:   # chunked: 4 rays of 8 lanes per warp, chunks of 8 C cells
        L = 8 * c
        nch = -(-nr // L)
        nrays = col.shape[0]
        nw = -(-nrays // 4)
        colp = np.zeros((nw * 4, nch * L))
        colp[:nrays, :nr] = col
        valid = np.zeros((nw * 4, nch * L), dtype=bool)
        valid[:nrays, :nr] = True
        lane = colp.reshape(nw, 4, nch * 8, c).sum(axis=3)           # lane sums, chunks and lanes in ray order
        end = np.cumsum(lane, axis=2)
        start = (end - lane).reshape(nw, 4, nch, 8)
        end = end.reshape(nw, 4, nch, 8)
        nmax = end[..., 7].max(axis=1).reshape(-1)
        cmax = lane.reshape(nw, 4, nch, 8).max(axis=(1, 3)).reshape(-1)
        n0min = start.min(axis=(1, 3)).reshape(-1)
        cells = valid.reshape(nw, 4, nch, L).sum(axis=(1, 3)).reshape(-1)
        na = np.searchsorted(kap, 127.0 * np.log(2.0) / np.maximum(n0min, 1e-300), side="right")
    elif 32 * c < nr:   # two warps per ray
        half = np.zeros((col.shape[0], 2, 32 * c))
        half.reshape(col.shape[0], -1)[:, :nr] = col
        nmax = np.repeat(col.sum(axis=1), 2)
        cmax = half.reshape(col.shape[0], 2, 32, c).sum(axis=3).max(axis=2).reshape(-1)
        cells = np.array([min(32 * c, nr), nr - min(32 * c, nr)] * col.shape[0])
    else:
        g = 8 if 8 * c >= nr else (16 if 16 * c >= nr else 32)   # lanes per ray
        r = 32 // g                                               # rays per warp
        nrays = col.shape[0]
        pad = (-nrays) % r
        colp = np.concatenate([col, np.zeros((pad, nr))]).reshape(-1, r, nr)
        nmax = colp.sum(axis=2).max(axis=1)
        chunks = np.zeros((colp.shape[0], r, g * c))
        chunks[:, :, :nr] = colp
        cmax = chunks.reshape(colp.shape[0], r, g, c).sum(axis=3).max(axis=(1, 2))
        rays = np.full(len(nmax), r)
        rays[-1] = r - pad
        cells = rays * nr
    bt = np.searchsorted(kap, THIN_X / np.maximum(nmax, 1e-300), side="right")
    bc = np.searchsorted(kap, THIN_X / np.maximum(cmax, 1e-300), side="right")
    use = (bc > bt) & ((bt > 0) | (bc >= 4))
    bt2 = np.where(use, bc, bt)
    return cells, bt, bt2, na


def exact_exp_ops(w, shape):
    """Exponentials of one tracer launch on grid w that its series cannot replace:
    one per (cell, bin) beyond the warp's tier (bt2), one per (lane, bin) of the tier
    (the tier's bins are expanded about each lane's first column), none for the thin
    series. The tile kernel traces every (cell, bin) bin by bin."""
    if shape[0] not in (1, 2):
        return w.grid.ncells * int(np.count_nonzero(w.kappa > 0))
    cells, bt, bt2, na = _warp_partition(w, shape)
    return int(np.sum(np.maximum(na - bt2, 0) * cells) + 32 * np.sum(bt2 - bt))


def series_fma_ops(w, shape):
    """FMA-pipe operations of one tracer launch on grid w that its arithmetic needs at
    the least: the power series (SERIES_FMA_PER_CELL per cell) in every warp that
    sums some bin in it, and EXACT_FMA_PER_PAIR per (cell, bin) traced bin by bin."""
    if shape[0] not in (1, 2):
        return EXACT_FMA_PER_PAIR * exact_exp_ops(w, shape)
    cells, bt, bt2, na = _warp_partition(w, shape)
    return int(SERIES_FMA_PER_CELL * np.sum(cells[bt2 > 0]) + EXACT_FMA_PER_PAIR * np.sum(np.maximum(na - bt2, 0) * cells))


def roofline_summary(grids, hbm_peak_gbs, ex2_peak_gops, ffma_peak_gops, ex2_basis, ffma_basis):
    """The tracer's roofline object over the launches of one step.

    grids: one dict per grid of the step with the algorithmic work of one launch
    (bytes: 16 B per cell; ex2: exponentials outside the thin series; fma: FMA-pipe
    operations at the least; cell_nu) and its mean CUDA-event launch time launch_s.
    The headline is HBM (16 B per cell, the per-unit figure of the scope): achieved
    = bytes / launch time, frac = achieved / the measured copy bandwidth. Beside it
    the two other floors (MUFU ex2 at the measured ex2 rate, FP32 FMA at the measured
    FFMA rate) and the binding floor per grid (the largest of the three times) summed
    over the step, against the launch time, and the target fraction."""
    t_launch = sum(g["launch_s"] for g in grids)
    by = sum(g["bytes"] for g in grids)
    ex = sum(g["ex2"] for g in grids)
    fm = sum(g["fma"] for g in grids)
    t_h = [g["bytes"] / (hbm_peak_gbs * 1e9) for g in grids]
    t_m = [g["ex2"] / (ex2_peak_gops * 1e9) for g in grids]
    t_f = [g["fma"] / (ffma_peak_gops * 1e9) for g in grids]
    names = []
    t_bind = 0.0
    for h, m, f in zip(t_h, t_m, t_f):
        t_bind += max(h, m, f)
        names.append("hbm" if h >= max(m, f) else ("mufu" if m >= f else "fp32"))
    achieved = by / t_launch / 1e9
    bind_frac = t_bind / t_launch
    return {
        "bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": hbm_peak_gbs,
        "frac": achieved / hbm_peak_gbs,
        "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
        "avg_launch_ms": t_launch / len(grids) * 1e3, "algorithmic_bytes_per_launch": by / len(grids),
        "per_grid_launch_ms": [g["launch_s"] * 1e3 for g in grids],
        "mufu": {"exact_ex2_per_launch": ex / len(grids), "achieved_gops": ex / t_launch / 1e9,
                 "peak_gops": ex2_peak_gops, "frac": sum(t_m) / t_launch, "peak_basis": ex2_basis},
        "fp32": {"fma_ops_per_launch": fm / len(grids), "achieved_gops": fm / t_launch / 1e9,
                 "peak_gops": ffma_peak_gops, "frac": sum(t_f) / t_launch, "peak_basis": ffma_basis},
        "binding_floor": {"per_grid": names, "frac": bind_frac,
                          "floor_ms_per_launch": t_bind / len(grids) * 1e3},
        "target_frac": ROOFLINE_TARGET,
        "target_met": bool(bind_frac >= ROOFLINE_TARGET),
        "one_ex2_per_cell_nu": {"cell_nu_per_s": sum(g["cell_nu"] for g in grids) / t_launch,
                                "peak_cell_nu_per_s": ex2_peak_gops * 1e9,
                                "frac": sum(g["cell_nu"] for g in grids) / t_launch / (ex2_peak_gops * 1e9)}}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1001_3301_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and --impl reference)
# --------------------------------------------------------------------------
def oracle_sample(w, n_rays, nthreads):
    import oracle
    g = w.grid
    # evenly spaced rays across the whole grid (polar, disk and envelope alike)
    sel = np.linspace(0, g.ntheta * g.nphi - 1, n_rays).astype(np.int64)
    rho = w.rho32().reshape(-1, g.nr)[sel].astype(np.float64)
    td = w.tdust32().reshape(-1, g.nr)[sel].astype(np.float64)
    th = np.linspace(0.0, math.pi, n_rays + 1)
    t0 = time.perf_counter()
    oracle.irradiate(g.r_if, th, np.array([0.0, 2 * math.pi]), w.t_star, w.r_star, w.nu,
                     w.kappa, w.t_sub, rho, td, nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_baseline(ws, target_s=12.0):
    """The oracle on the step's own grids: evenly spaced rays of every grid, as many (and,
    when a grid's rays run out, as many passes over all of them) as fill about
    target_s seconds of OpenMP work on the host cores."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    probe_rays = min(1024, ws[0].grid.ntheta * ws[0].grid.nphi)   # enough to keep every thread busy
    dt = oracle_sample(ws[0], probe_rays, cores)
    per_grid = probe_rays * target_s / max(dt, 1e-3) / len(ws)   # rays per grid for target_s
    n_rays = [int(min(w.grid.ntheta * w.grid.nphi, max(64, per_grid))) for w in ws]
    full = min(w.grid.ntheta * w.grid.nphi for w in ws)
    passes = int(min(8, max(1, round(per_grid / full)))) if per_grid > full else 1
    dt = 0.0
    units = 0
    for _ in range(passes):
        for w, n in zip(ws, n_rays):
            dt += oracle_sample(w, n, cores)
            units += n * w.grid.nr * len(w.nu)
    desc = ", ".join(f"{n} rays of tau550={w.tau550:g}" for w, n in zip(ws, n_rays))
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} pass(es) over {desc} (evenly spaced, {ws[0].grid.nr} cells x {len(ws[0].nu)} bins "
                      f"each; {units:.3e} cell-nu updates, {dt:.1f} s, OpenMP over rays)"}


def run_cpu_table(args, local):
    """Oracle (1 core and all cores, bounded ray samples) and GPU tracer (full grid,
    autotuned) throughput per workload, as one table."""
    import torch
    import oracle
    from paper_1001_3301_gb300 import Tracer, probe_alu_rates
    torch.cuda.set_device(local)
    oracle.build()
    cores = oracle.max_threads()
    ex2_clk, ffma_clk, mhz = probe_alu_rates()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = ex2_clk * nsm * 2070e6
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs") or 6678.0)
    cases = [("C1 64x32x1 nu32 tau1", synth.disk2d()),
             ("C2 256x128x256 nu79 tau1", synth.disk3d(256, 128, 256, n_nu=79, tau550=1.0, seed=1)),
             ("C2 256x128x256 nu79 tau100", synth.disk3d(256, 128, 256, n_nu=79, tau550=100.0, seed=1)),
             ("C3 512x256x512 nu79 tau1", synth.disk3d(512, 256, 512, n_nu=79, tau550=1.0, seed=2))]
    rows = []
    for name, w in cases:
        nrays = w.grid.ntheta * w.grid.nphi
        row = {"workload": name}
        for label, nth in (("oracle_1core", 1), ("oracle_all_cores", cores)):
            n = min(nrays, 8 * nth)
            dt = oracle_sample(w, n, nth)
            n = int(min(nrays, max(n, n * 3.0 / max(dt, 1e-3))))  # about 3 s of work
            dt = oracle_sample(w, n, nth)
            row[label] = n * w.grid.nr * len(w.nu) / dt
        tr = Tracer.from_grid(w.grid)
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        r = torch.from_numpy(w.rho32()).cuda()
        t = torch.from_numpy(w.tdust32()).cuda()
        q, a = torch.empty_like(r), torch.empty_like(r)
        tr.autotune(r, t, q, a, reps=2)
        for _ in range(3):
            tr.irradiate(r, t, q, a)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            tr.irradiate(r, t, q, a)
        e1.record()
        torch.cuda.synchronize()
        t_s = e0.elapsed_time(e1) / args.steps * 1e-3
        v = w.grid.ncells * len(w.nu) / t_s
        t_floor = max(TRACE_BYTES_PER_CELL * w.grid.ncells / (hbm * 1e9),
                      exact_exp_ops(w, tr.tuning()) / peak)
        row.update(gpu=v, gpu_roofline_frac=t_floor / t_s, tuning=list(tr.tuning()))
        tr.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"mode": "cpu_table", "cores": cores, "ex2_per_sm_clk": ex2_clk, "ffma_per_sm_clk": ffma_clk,
                      "rows": rows}), flush=True)


# seconds of OpenMP oracle work per step of the reference arm
REF_STEP_S = 1.0


def time_dust_temperature(st, steps, stream, hbm, i_med):
    """rt_dust_temperature (E_R = 0) on every grid of a tracer set, fed by its a_rad:
    CUDA events over `steps` passes over the grids (their 8 bytes per cell exceed L2
    together), the mean time per grid against the measured copy bandwidth."""
    import torch
    t_out = [torch.empty(w.grid.shape, dtype=torch.float32, device="cuda") for w in st["ws"]]
    for _ in range(3):
        for i, tr in enumerate(st["tracers"]):
            tr.dust_temperature(st["a"][i], None, t_out[i])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for i, tr in enumerate(st["tracers"]):
            tr.dust_temperature(st["a"][i], None, t_out[i])
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) / (steps * len(st["ws"]))
    g = st["ws"][0].grid
    ncell = g.ncells
    out = {"workload": f"disk3d {g.nr}x{g.ntheta}x{g.nphi}, a_rad of the tracer, "
                       f"tau550 in {{{','.join(f'{w.tau550:g}' for w in st['ws'])}}}",
           "ms_per_grid": t_ms, "cells_per_s": ncell / (t_ms * 1e-3),
           "achieved_gbs": 8.0 * ncell / (t_ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm,
           "frac_of_hbm": 8.0 * ncell / (t_ms * 1e-3) / 1e9 / hbm,
           "median_t_k": float(t_out[i_med].median())}
    del t_out
    return out


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on the GPU arm's workload: per step an evenly
    spaced sample of rays of every grid of the step, as many as fill about REF_STEP_S
    seconds of OpenMP work (the same sampling as the cpu_baseline leg)."""
    if rank != 0:
        return
    spec = WORKLOADS[args.workload]
    taus = step_taus(args, spec)
    ws = workloads(spec, taus)
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    nrays = ws[0].grid.ntheta * ws[0].grid.nphi
    probe = min(2048, nrays)
    dt = oracle_sample(ws[0], probe, cores)
    n_rays = int(min(nrays, max(256, probe * REF_STEP_S / max(dt, 1e-3) / len(ws))))
    for _ in range(max(args.warmup, 0)):
        for w in ws:
            oracle_sample(w, n_rays, cores)
    dt = 0.0
    for _ in range(args.steps):
        for w in ws:
            dt += oracle_sample(w, n_rays, cores)
    units = args.steps * sum(n_rays * w.grid.nr * len(w.nu) for w in ws)
    value = units / dt
    sample = (f"per step {n_rays} evenly spaced rays x {spec['nr']} cells x {spec['n_nu']} bins of each of the "
              f"{len(ws)} grids (OpenMP over rays)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(spec, taus), "sample_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def setup_tracers(ws, precision, shape_arg):
    """One context per grid, fields resident on the device, launch shape from the
    autotuner per grid (untimed) or forced."""
    import torch
    from paper_1001_3301_gb300 import Tracer
    tracers, rho, td, q, a = [], [], [], [], []
    for w in ws:
        tr = Tracer.from_grid(w.grid, precision)
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        tracers.append(tr)
        rho.append(torch.from_numpy(w.rho32()).cuda())
        td.append(torch.from_numpy(w.tdust32()).cuda())
        q.append(torch.empty(w.grid.shape, dtype=torch.float32, device="cuda"))
        a.append(torch.empty(w.grid.shape, dtype=torch.float32, device="cuda"))
    shapes = []
    for i, tr in enumerate(tracers):
        if shape_arg:
            tr.set_tuning(*shape_arg)
        else:
            tr.autotune(rho[i], td[i], q[i], a[i], reps=3)
        shapes.append(tuple(tr.tuning()))
    return {"tracers": tracers, "rho": rho, "td": td, "q": q, "a": a, "shapes": shapes, "ws": ws}


def time_step(st, steps, warmup, stream, dist=None, sampler=None):
    """Warm-up, then `steps` timed steps: every grid traced (rt_irradiate) and its FP64
    energy reduction enqueued (rt_energy_reduce). Returns the step time (max over
    ranks) and each grid's mean CUDA-event launch time of the tracer kernel."""
    import torch
    tr, rho, td, q, a = st["tracers"], st["rho"], st["td"], st["q"], st["a"]

    def step(ev=None):
        for i, t in enumerate(tr):
            if ev is not None:
                ev[i][0].record(stream)
            t.irradiate(rho[i], td[i], q[i], a[i])
            if ev is not None:
                ev[i][1].record(stream)
            t.energy_reduce()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in tr] for _ in range(steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if sampler is not None:
        sampler.__enter__()
        time.sleep(0.3)
    try:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for s in range(steps):
            step(evs[s])
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    finally:
        if sampler is not None:
            sampler.__exit__(None, None, None)
    ms = t_start.elapsed_time(t_end)
    launch_ms = [statistics.mean(evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(steps))
                 for i in range(len(tr))]
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms / steps, launch_ms


def tracer_roofline(st, launch_ms, ex2_peak, ffma_peak, hbm, ex2_basis, ffma_basis):
    grids = []
    for w, shape, lm in zip(st["ws"], st["shapes"], launch_ms):
        grids.append({"bytes": TRACE_BYTES_PER_CELL * w.grid.ncells, "ex2": exact_exp_ops(w, shape),
                      "fma": series_fma_ops(w, shape), "cell_nu": w.grid.ncells * len(w.nu),
                      "launch_s": lm * 1e-3})
    return roofline_summary(grids, hbm, ex2_peak, ffma_peak, ex2_basis, ffma_basis)


def close_tracers(st):
    if not st:
        return
    for tr in st["tracers"]:
        tr.close()
    st.clear()


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1001_3301_gb300 import probe_alu_rates

    spec = WORKLOADS[args.workload]
    taus = step_taus(args, spec)
    ws = workloads(spec, taus, seed_offset=rank)
    stream = torch.cuda.current_stream()
    shape_arg = tuple(int(x) for x in args.shape.split(",")) if args.shape else None
    prim = setup_tracers(ws, args.precision, shape_arg)
    prim_shapes = list(prim["shapes"])
    units_per_step = sum(w.grid.ncells * len(w.nu) for w in ws)
    clk = ClockSampler(local)
    ms_per_step, launch_ms = time_step(prim, args.steps, args.warmup, stream, dist, sampler=clk)
    value = world * units_per_step / (ms_per_step * 1e-3)

    # energy and input check of the last step (untimed read of what the step reduced)
    energies = [tr.energy_last() for tr in prim["tracers"]]
    max_energy_err = max(abs(e.rel_err) for e in energies)

    # roofline of the tracer kernel: HBM headline, MUFU and FP32 floors, binding floor
    ex2_clk, ffma_clk, probe_mhz = probe_alu_rates()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or probe_mhz
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks.get("hbm_gbs") or 6678.0)
    ex2_peak = ex2_clk * nsm * mhz * 1e6 / 1e9     # Gop/s of ex2 (also the temperature-table leg's bound)
    ffma_peak = ffma_clk * nsm * mhz * 1e6 / 1e9   # Gop/s of FFMA
    ex2_basis = f"measured {ex2_clk:.2f} ex2/SM/clk x {nsm} SMs x {mhz:.0f} MHz"
    ffma_basis = f"measured {ffma_clk:.1f} FFMA/SM/clk x {nsm} SMs x {mhz:.0f} MHz"
    src_hash = kernel_source_hash()
    roofline = tracer_roofline(prim, launch_ms, ex2_peak, ffma_peak, hbm, ex2_basis, ffma_basis)
    kinds = {s[0] for s in prim_shapes}
    roofline.update({"traffic": traffic_from_profile(profile_summary_path(spec), src_hash),
                     "kernel": "k_ray" if kinds <= {1, 2} else ("k_trace" if kinds == {0} else "k_ray/k_trace"),
                     "ffma_per_sm_clk": ffma_clk, "ex2_per_sm_clk": ex2_clk, "kernel_source_sha256": src_hash})

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        tracers = prim["tracers"]
        h_rho = [torch.from_numpy(w.rho32()).pin_memory() for w in ws]
        h_td = [torch.from_numpy(w.tdust32()).pin_memory() for w in ws]
        h_q = [torch.empty(w.grid.shape, dtype=torch.float32).pin_memory() for w in ws]
        h_a = [torch.empty(w.grid.shape, dtype=torch.float32).pin_memory() for w in ws]
        for i, tr in enumerate(tracers):  # allocates the staging buffers (untimed)
            tr.irradiate_host(h_rho[i], h_td[i], h_q[i], h_a[i])
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            # the step's grids in flight together (copies of one grid overlap the
            # trace and copies of the others), then every grid's outputs on the host
            for i, tr in enumerate(tracers):
                tr.irradiate_host_async(h_rho[i], h_td[i], h_q[i], h_a[i])
            for tr in tracers:
                tr.host_wait()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        nbytes = sum(4 * w.grid.ncells for w in ws)
        e2e = {"value": world * units_per_step * args.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
               "entry_point": "rt_irradiate_host_async + rt_host_wait (pinned host buffers)"}
        del h_rho, h_td, h_q, h_a

    # the dust-temperature update on the primary grids (their a_rad from the last step)
    temp_c3 = None
    if rank == 0 and args.workload == "c3":
        temp_c3 = time_dust_temperature(prim, args.steps, stream, hbm, 0)

    # the other workload's tracer step (rank 0), and the 256 x 128 x 256 tau = 1 grid
    # that the steps after the tracer run on
    sec = None
    sec_st = None
    c2 = prim if args.workload == "c2" else None
    if rank == 0 and not args.no_secondary:
        other = "c2" if args.workload == "c3" else "c3"
        ospec = WORKLOADS[other]
        if other == "c3":   # free the primary grids first
            close_tracers(prim)
            torch.cuda.empty_cache()
            c2 = None
        sec_st = setup_tracers(workloads(ospec, ospec["taus"]), args.precision, None)
        s_ms, s_launch = time_step(sec_st, args.steps, args.warmup, stream)
        s_units = sum(w.grid.ncells * len(w.nu) for w in sec_st["ws"])
        s_roof = tracer_roofline(sec_st, s_launch, ex2_peak, ffma_peak, hbm, ex2_basis, ffma_basis)
        s_roof["traffic"] = traffic_from_profile(profile_summary_path(ospec), src_hash)
        sec = {"workload": workload_name(ospec, ospec["taus"]), "value": s_units / (s_ms * 1e-3), "unit": UNIT,
               "ms_per_step": s_ms, "steps": args.steps, "launch_shapes": [list(x) for x in sec_st["shapes"]],
               "energy_max_rel_err": max(abs(t.energy_last().rel_err) for t in sec_st["tracers"]),
               "roofline": s_roof}
        if other == "c2":
            c2 = sec_st
    if rank == 0 and c2 is None and not (args.no_fld and args.no_secondary):
        c2 = setup_tracers(workloads(WORKLOADS["c2"], (1.0,)), args.precision, None)
    i1 = 0
    if c2:
        i1 = next((i for i, w in enumerate(c2["ws"]) if w.tau550 == 1.0), 0)

    # the dust-temperature update (Eq. 16) on the 256 x 128 x 256 grids, fed by their
    # a_rad (timed on its own, 8 bytes per cell against HBM); beside it the same on the
    # 512 x 256 x 512 grids (measured before they were freed)
    temp = None
    if rank == 0 and c2:
        for i, tr in enumerate(c2["tracers"]):
            tr.irradiate(c2["rho"][i], c2["td"][i], c2["q"][i], c2["a"][i])
        temp = time_dust_temperature(c2, args.steps, stream, hbm, i1)
    if temp_c3 is not None:
        temp = dict(temp or {}, on_512x256x512=temp_c3)

    # the tracer with temperature-dependent tables (24 temperatures) on the tau = 1 grid:
    # the synthetic table (one species whose abundance depends on T: it separates, the
    # one-column tracer with a per-cell column weight), two- to four-species tables (rank
    # two to four: that many columns per ray) and a full-rank one (per-bin scans)
    tdep = None
    if rank == 0 and c2:
        from paper_1001_3301_gb300 import Tracer
        w1 = c2["ws"][i1]
        tg = synth.t_grid(24)
        ri, ti = c2["rho"][i1], c2["td"][i1]
        qt, at = torch.empty_like(ri), torch.empty_like(ri)
        units = w1.grid.ncells * len(w1.nu)
        tdep = {"workload": f"disk3d {NR}x{NTH}x{NPH}, {NNU} bins x 24 temperatures, tau550 = {w1.tau550:g}"}
        for name, table in (("separable", synth.kappa_synth_t), ("two_species", synth.kappa_synth_t2),
                            ("three_species", synth.kappa_synth_t3), ("four_species", synth.kappa_synth_t4),
                            ("full_rank", synth.kappa_synth_t_full)):
            trt = Tracer.from_grid(w1.grid)
            trt.set_opacity_table_t(w1.nu, tg, table(w1.nu, tg), w1.t_sub)
            trt.set_star(w1.t_star, w1.r_star)
            sh_t = trt.autotune(ri, ti, qt, at, reps=2)
            for _ in range(3):
                trt.irradiate(ri, ti, qt, at)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                trt.irradiate(ri, ti, qt, at)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms = e0.elapsed_time(e1) / args.steps
            ach = EXP_PER_CELL_NU * units / (t_ms * 1e-3) / 1e9
            _, _, et = trt.irradiate(ri, ti, qt, at, energy=True)
            tdep[name] = {"table_kind": TABLE_KINDS[trt.table_kind()], "ms": t_ms,
                          "cell_nu_per_s": units / (t_ms * 1e-3),
                          "roofline": {"bound": "alu", "unit": "Gop/s (MUFU ex2, one per cell-nu)", "achieved": ach,
                                       "peak": ex2_peak, "frac": ach / ex2_peak},
                          "launch_shape": list(sh_t), "energy_rel_err": et.rel_err}
            trt.close()
        del qt, at

    # one implicit flux-limited-diffusion step (Eqs. 7-15) on the tau = 1 grid, with
    # that grid's q_abs as the source
    fld_line = None
    if rank == 0 and c2 and not args.no_fld:
        fld_line = run_fld(args, c2["tracers"][i1], c2["ws"][i1], c2["rho"][i1], c2["q"][i1], stream)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(ws)
    for st in (prim, sec_st, c2):
        close_tracers(st)
    torch.cuda.empty_cache()
    sur = None
    if rank == 0 and world == 1 and not args.no_surrogate:
        sur = run_surrogate(args, local)
        sur["lut_comparator"] = run_lut(args, local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded disk+envelope density, uniform dust temperatures, synthetic kappa_nu)",
            "config": {"workload": workload_name(spec, taus), "precision": args.precision,
                       "grids_per_step": len(ws), "cells_per_step": sum(w.grid.ncells for w in ws),
                       "nu_bins": spec["n_nu"],
                       "step": "per grid: rt_irradiate (tracer kernel) + rt_energy_reduce (FP64 energy reduction)",
                       "launch_shapes": [{"kernel": KERNEL_KINDS[sh[0]], "cells_per_lane": sh[1], "warps": sh[2],
                                          "min_blocks_per_sm": sh[3]} for sh in prim_shapes],
                       "l2": f"no flush: inputs+outputs {16 * sum(w.grid.ncells for w in ws) / 1e6:.0f} MB per step "
                             f"exceed the 129 MB L2",
                       "replicas_per_rank": 1},
            "roofline": roofline,
            "cpu_baseline": base,
            "e2e": e2e,
            "gpu_launches": 2 * len(ws) * args.steps,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                       "reasons": clocks["reasons"]},
            "energy_max_rel_err": max_energy_err,
            "secondary": sec,
            "dust_temperature": temp,
            "tdep": tdep,
            "fld": fld_line,
            "surrogate": sur,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


SUR_TAUS = (0.1, 0.3, 1.0, 3.0, 10.0, 30.0, 100.0)
SUR_TOL = 1e-3


def _dims(spec):
    return tuple(int(x) for x in spec.split("x"))


def run_surrogate(args, local):
    """The learned surrogate (8 -> 128 -> 128 -> 1 SiLU network on the tensor cores):
    trained on cells the exact tracer traced on seven optical depths (0.1-100) of the
    disk, then timed against the exact tracer on the surrogate grid (tau550 = 1,
    seed 2): gated by its trust map (validate = 0), the network alone (validate = 2),
    and judged by the exact tracer (validate = 1) for its error."""
    import torch
    from paper_1001_3301_gb300 import Tracer, probe_alu_rates, probe_tensor_rates
    torch.cuda.set_device(local)
    nr, nth, nph = _dims(args.sur_train_grid)
    trs = []
    t0 = time.perf_counter()
    train_w = [synth.disk3d(nr, nth, nph, n_nu=NNU, tau550=t, seed=10 + i) for i, t in enumerate(SUR_TAUS)]
    t_gen = time.perf_counter() - t0
    tr_train = Tracer.from_grid(train_w[0].grid)
    tr_train.set_opacity_table(train_w[0].nu, train_w[0].kappa, train_w[0].t_sub)
    tr_train.set_star(train_w[0].t_star, train_w[0].r_star)
    rho_t = [torch.from_numpy(w.rho32()).cuda() for w in train_w]
    td_t = [torch.from_numpy(w.tdust32()).cuda() for w in train_w]
    st = tr_train.surrogate_train(rho_t, td_t, n_samples=20_000_000, batch=8192, steps=args.sur_steps,
                                  lr=1e-3, seed=1)
    del rho_t, td_t
    path = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"rt_surrogate_{os.getpid()}.bin")
    tr_train.surrogate_save(path)
    tr_train.close()

    nr, nth, nph = _dims(args.sur_grid)
    w = synth.disk3d(nr, nth, nph, n_nu=NNU, tau550=1.0, seed=2)
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    tr.surrogate_load(path)
    os.remove(path)
    rho = torch.from_numpy(w.rho32()).cuda()
    td = torch.from_numpy(w.tdust32()).cuda()
    q_ex = torch.empty_like(rho)
    a_ex = torch.empty_like(rho)
    q_s = torch.empty_like(rho)
    a_s = torch.empty_like(rho)
    shape = tr.autotune(rho, td, q_ex, a_ex, reps=2)
    _, _, e = tr.irradiate(rho, td, q_ex, a_ex, energy=True)
    _, _, vst = tr.irradiate_surrogate(rho, td, q_s, a_s, err_tol=SUR_TOL, validate=1)
    _, _, gst = tr.irradiate_surrogate(rho, td, q_s, a_s, err_tol=SUR_TOL, validate=0)
    # error of the gated result against the exact tracer where a cell absorbs > 1e-12 L*
    g = w.grid
    dom = torch.from_numpy(np.outer(np.diff(g.phi_if), np.cos(g.theta_if[:-1]) - np.cos(g.theta_if[1:]))).cuda()
    d3 = torch.from_numpy((g.r_if[1:] ** 3 - g.r_if[:-1] ** 3) / 3.0).cuda()
    mask = (q_ex.double() * dom[:, :, None] * d3[None, None, :]) > 1e-12 * e.l_star
    rel = ((q_s.double() - q_ex.double()).abs() / q_ex.double().clamp_min(1e-300))[mask]
    gate_max = float(rel.max()) if rel.numel() else 0.0
    gate_over = int((rel > SUR_TOL).sum()) if rel.numel() else 0

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.sur_reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.sur_reps

    with ClockSampler(local) as clk:
        time.sleep(0.2)
        t_ex = timed(lambda: tr.irradiate(rho, td, q_ex, a_ex))
        t_gate = timed(lambda: tr.irradiate_surrogate(rho, td, q_s, a_s, err_tol=SUR_TOL, validate=0, stats=False))
        t_net = timed(lambda: tr.irradiate_surrogate(rho, td, q_s, a_s, err_tol=SUR_TOL, validate=2, stats=False))
    clocks = clk.summary()
    rates = probe_tensor_rates()
    ex2_clk, _, probe_mhz = probe_alu_rates()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks["sm_mhz"] or probe_mhz
    n = g.ncells
    # MUFU work of the network per cell: 256 SiLU = 256 ex2 + 256 rcp; the clock
    # cycles one SM needs for it at the measured rates bound the network alone
    clk_per_cell = 256.0 / ex2_clk + 256.0 / rates["rcp_f32"]
    peak_cells = nsm * mhz * 1e6 / clk_per_cell
    tr.close()
    return {
        "workload": f"disk3d {nr}x{nth}x{nph}, {NNU} nu bins, tau550 = 1, seed 2; trained on "
                    f"{args.sur_train_grid} x {len(SUR_TAUS)} optical depths 0.1-100",
        "err_tol": SUR_TOL,
        "exact": {"ms": t_ex, "cells_per_s": n / (t_ex * 1e-3), "cell_nu_per_s": n * NNU / (t_ex * 1e-3),
                  "launch_shape": list(shape)},
        "gated": {"ms": t_gate, "cells_per_s": n / (t_gate * 1e-3),
                  "equiv_cell_nu_per_s": n * NNU / (t_gate * 1e-3), "speedup_vs_exact": t_ex / t_gate,
                  "fallback_frac": gst["n_fallback"] / max(gst["n_dust"], 1),
                  "max_rel_err_vs_exact": gate_max, "cells_over_tol": gate_over,
                  "judged_cells": int(mask.sum()), "energy_rel_err": gst["rel_err"]},
        "network_only": {"ms": t_net, "cells_per_s": n / (t_net * 1e-3),
                         "equiv_cell_nu_per_s": n * NNU / (t_net * 1e-3), "speedup_vs_exact": t_ex / t_net},
        "validate": {"answered_frac": 1 - vst["n_fallback"] / max(vst["n_dust"], 1),
                     "max_rel_err": vst["max_rel_err"], "mean_rel_err": vst["mean_rel_err"]},
        "train": {"n_train": st["n_train"], "n_val": st["n_val"], "steps": args.sur_steps, "batch": 8192,
                  "val_rms_ln_g": st["val_rms"], "val_max_ln_g": st["val_max"], "train_ms": st["train_ms"],
                  "field_generation_s": t_gen},
        "roofline": {"bound": "alu", "unit": "cells/s (MUFU: 256 ex2 + 256 rcp per cell)",
                     "achieved": n / (t_net * 1e-3), "peak": peak_cells, "frac": n / (t_net * 1e-3) / peak_cells,
                     "peak_basis": f"measured {ex2_clk:.1f} ex2 and {rates['rcp_f32']:.1f} rcp /SM/clk x {nsm} SMs x {mhz:.0f} MHz",
                     "tensor_mac_per_cell": 36864, "umma_mac_per_sm_clk": rates["umma_n128_mac"]},
        "clocks": clocks,
    }


def run_lut(args, local):
    """The lookup-table comparator (rt_lut_build, rt_irradiate_lut) against the exact
    tracer on the 512 x 256 x 512 grids at tau550 = 1 and 100: time per launch, the
    warp-slots that fell back to the per-bin sum, and the largest relative error of q_abs
    and a_rad against the exact tracer in the cells that absorb more than 1e-12 L*."""
    import torch
    from paper_1001_3301_gb300 import Tracer
    torch.cuda.set_device(local)
    spec = WORKLOADS["c3"]
    out = {"err_tol": SUR_TOL}

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for tau in spec["taus"]:
        w = synth.disk3d(spec["nr"], spec["ntheta"], spec["nphi"], n_nu=spec["n_nu"], tau550=tau, seed=spec["seed"])
        g = w.grid
        tr = Tracer.from_grid(g)
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        rho = torch.from_numpy(w.rho32()).cuda()
        td = torch.from_numpy(w.tdust32()).cuda()
        q_ex, a_ex = torch.empty_like(rho), torch.empty_like(rho)
        q_l, a_l = torch.empty_like(rho), torch.empty_like(rho)
        shape = tr.autotune(rho, td, q_ex, a_ex, reps=2)
        t0 = time.perf_counter()
        tr.lut_build(SUR_TOL)
        t_build = time.perf_counter() - t0
        _, _, e_ex = tr.irradiate(rho, td, q_ex, a_ex, energy=True)
        _, _, e_l, fb = tr.irradiate_lut(rho, td, q_l, a_l, energy=True, stats=True)
        dom = torch.from_numpy(np.outer(np.diff(g.phi_if), np.cos(g.theta_if[:-1]) - np.cos(g.theta_if[1:]))).cuda()
        d3 = torch.from_numpy((g.r_if[1:] ** 3 - g.r_if[:-1] ** 3) / 3.0).cuda()
        mask = (q_ex.double() * dom[:, :, None] * d3[None, None, :]) > 1e-12 * e_ex.l_star
        rq = ((q_l.double() - q_ex.double()).abs() / q_ex.double().clamp_min(1e-300))[mask]
        ra = ((a_l.double() - a_ex.double()).abs() / a_ex.double().abs().clamp_min(1e-300))[mask]
        t_ex = timed(lambda: tr.irradiate(rho, td, q_ex, a_ex), args.sur_reps)
        t_l = timed(lambda: tr.irradiate_lut(rho, td, q_l, a_l), args.sur_reps)
        slots = g.ntheta * g.nphi // max(1, 32 // (8 if 8 * shape[1] >= g.nr else (16 if 16 * shape[1] >= g.nr else 32)))
        out[f"tau{tau:g}"] = {
            "exact_ms": t_ex, "lut_ms": t_l, "speedup_vs_exact": t_ex / t_l,
            "lut_cell_nu_per_s": g.ncells * len(w.nu) / (t_l * 1e-3),
            "fallback_warp_slots": fb, "fallback_frac": fb / max(slots, 1),
            "max_rel_err_q_vs_exact": float(rq.max()), "max_rel_err_a_vs_exact": float(ra.max()),
            "cells_over_tol": int((rq > SUR_TOL).sum()), "judged_cells": int(mask.sum()),
            "e_abs_rel_diff": abs(e_l.e_abs - e_ex.e_abs) / e_ex.l_star, "build_s": t_build,
            "launch_shape": list(shape)}
        tr.close()
        del rho, td, q_ex, a_ex, q_l, a_l, mask, rq, ra
        torch.cuda.empty_cache()
    return out


def bf16_round(x):
    """Round float64 values to bfloat16 (through float32, nearest-even)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def run_precision_sweep(args, local):
    """Errors of q_abs, a_rad and the energy sums of every precision mode (scan in
    FP64, compensated FP32, plain FP32; opacity table in FP32 or BF16) against the
    FP64 oracle, in the cells that absorb more than 1e-12 L*."""
    import torch
    import oracle
    from paper_1001_3301_gb300 import Tracer
    torch.cuda.set_device(local)
    oracle.build()
    nr, nth, nph = (int(x) for x in args.sweep_grid.split("x"))
    rows = []
    for tau in (1.0, 100.0):
        w = synth.disk3d(nr, nth, nph, n_nu=NNU, tau550=tau, seed=2)
        rho = torch.from_numpy(w.rho32()).cuda()
        td = torch.from_numpy(w.tdust32()).cuda()
        t0 = time.perf_counter()
        orc = oracle.irradiate_workload(w, nthreads=oracle.max_threads())
        t_orc = time.perf_counter() - t0
        orc_b = oracle.irradiate_workload(w, kappa=bf16_round(w.kappa), nthreads=oracle.max_threads())
        mask = orc.p_abs > 1e-12 * orc.l_star
        for prec in ("fp64", "fp32_kahan", "fp32_plain"):
            for bf16 in (False, True):
                tr = Tracer.from_grid(w.grid, prec)
                tr.set_opacity_table(w.nu, w.kappa, w.t_sub, kappa_bf16=bf16)
                tr.set_star(w.t_star, w.r_star)
                q = torch.empty_like(rho)
                a = torch.empty_like(rho)
                if prec != "fp64":  # the shape a user gets (FP64 has one kernel family, minutes per sweep)
                    tr.autotune(rho, td, q, a, reps=2)
                q, a, e = tr.irradiate(rho, td, q, a, energy=True)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                reps = 3
                ev[0].record()
                for _ in range(reps):
                    tr.irradiate(rho, td, q, a)
                ev[1].record()
                torch.cuda.synchronize()
                ms = ev[0].elapsed_time(ev[1]) / reps
                qh, ah = q.double().cpu().numpy(), a.double().cpu().numpy()
                row = {"tau550": tau, "scan": prec, "kappa_table": "bf16" if bf16 else "fp32",
                       "ms": ms, "cell_nu_per_s": w.grid.ncells * NNU / (ms * 1e-3),
                       "tuning": tr.tuning(), "cells_in_mask": int(mask.sum())}
                for ref_name, ref in (("vs_fp64_oracle", orc), ("vs_oracle_same_table", orc_b if bf16 else orc)):
                    rq = np.abs(qh[mask] - ref.q_abs[mask]) / ref.q_abs[mask]
                    ra = np.abs(ah[mask] - ref.a_rad[mask]) / np.abs(ref.a_rad[mask])
                    row[ref_name] = {"q_max": float(rq.max()), "q_p999": float(np.quantile(rq, 0.999)),
                                     "a_max": float(ra.max()), "a_p999": float(np.quantile(ra, 0.999)),
                                     "e_abs_rel": abs(e.e_abs - ref.e_abs) / ref.l_star,
                                     "energy_closure": e.rel_err}
                rows.append(row)
                tr.close()
                del q, a
        rows.append({"tau550": tau, "oracle_seconds": t_orc, "oracle_cores": oracle.max_threads()})
        del rho, td, orc, orc_b
        torch.cuda.empty_cache()
    print(json.dumps({"mode": "precision_sweep", "grid": args.sweep_grid, "nu_bins": NNU,
                      "mask": "cells absorbing > 1e-12 L*", "rows": rows}), flush=True)


def run_batch(args, local):
    """cell-nu updates/s of the 96-grid batch (Nr 64-512, Ntheta 32-256, Nphi 1/64/128,
    32/79/128 bins, tau550 log-uniform 0.1-100), one graph replay per step."""
    import torch
    from paper_1001_3301_gb300 import Batch, Tracer
    torch.cuda.set_device(local)
    specs = synth.batch_specs(96, seed=3)
    trs, rho, td, q, a = [], [], [], [], []
    units = 0
    for sp in specs:
        w = synth.disk3d(sp["nr"], sp["ntheta"], sp["nphi"], n_nu=sp["n_nu"], tau550=sp["tau550"],
                         seed=sp["seed"])
        tr = Tracer.from_grid(w.grid, args.precision)
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        trs.append(tr)
        rho.append(torch.from_numpy(w.rho32()).cuda())
        td.append(torch.from_numpy(w.tdust32()).cuda())
        q.append(torch.empty_like(rho[-1]))
        a.append(torch.empty_like(rho[-1]))
        units += w.grid.ncells * len(w.nu)
    b = Batch(trs)
    shape = b.autotune(rho, td, q, a, reps=2)
    for _ in range(args.warmup):
        b.run(rho, td, q, a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(args.steps):
            b.run(rho, td, q, a)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    es = b.energy()
    # the same grids one launch each (rt_irradiate, autotuned per shape class)
    for tr, r, t, qq, aa in zip(trs, rho, td, q, a):
        tr.autotune(r, t, qq, aa, reps=1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        for tr, r, t, qq, aa in zip(trs, rho, td, q, a):
            tr.irradiate(r, t, qq, aa)
    e1.record()
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1) / args.steps
    b.close()
    for tr in trs:
        tr.close()
    print(json.dumps({"mode": "batch", "grids": len(specs), "cells": sum(x.numel() for x in rho),
                      "cell_nu_per_step": units, "ms_per_step": ms, "value": units / (ms * 1e-3),
                      "unit": UNIT, "tuning": shape, "steps": args.steps,
                      "per_grid_launches_ms": ms_single, "per_grid_launches_value": units / (ms_single * 1e-3),
                      "energy_max_rel_err": max(abs(e.rel_err) for e in es),
                      "clocks": clk.summary()}), flush=True)


def run_fld(args, tr, w, rho, q, stream):
    """Time one implicit flux-limited-diffusion step (Eqs. 7-15) on the grid of ``tr``
    with ``q`` (the tracer's q_abs) as source: gas temperature and old E_R from
    ``synth.fld_fields``, the paper's outer boundary T0 = 14.7 K (Sect. 3.1.2),
    c_v = 1e8 erg/(g K), tol 1e-5. HBM-bound: FLD_SETUP_B + FLD_PASS_B per pass +
    FLD_ITER_B per iteration bytes per cell."""
    import torch
    tg_, e_, _ = synth.fld_fields(w.grid, seed=1)
    t_gas = torch.from_numpy(tg_.astype(np.float32)).cuda()
    e_old = torch.from_numpy(e_.astype(np.float32)).cuda()
    e_new = torch.empty_like(e_old)
    dt_s, c_v, t_bg = args.fld_dt, 1e8, 14.7
    for _ in range(max(1, min(args.warmup, 2))):
        _, fst = tr.fld_step(rho, t_gas, q, e_old, dt_s, c_v, t_bg, e_new=e_new, tol=1e-5, max_iter=20000)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, fst = tr.fld_step(rho, t_gas, q, e_old, dt_s, c_v, t_bg, e_new=e_new, tol=1e-5, max_iter=20000)
    e1.record(stream)
    torch.cuda.synchronize()
    f_ms = e0.elapsed_time(e1) / args.steps
    ncell = w.grid.ncells
    mg = fst["levels"] > 1
    sb, pb, ib = (FLD_SETUP_MG_B, FLD_PASS_MG_B, FLD_ITER_MG_B) if mg else (FLD_SETUP_B, FLD_PASS_B, FLD_ITER_B)
    nbytes = (sb + pb * fst["passes"] + ib * fst["iterations"]) * ncell
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks.get("hbm_gbs") or 6678.0)
    g = w.grid
    return {"workload": f"disk3d {g.nr}x{g.ntheta}x{g.nphi}, tau550 = {w.tau550:g}, dt = {dt_s:g} s, "
                        f"c_v = {c_v:g}, T_bg = {t_bg:g} K, tol = 1e-5",
            "ms_per_step": f_ms, "iterations": fst["iterations"], "passes": fst["passes"],
            "rel_change": fst["rel_change"], "ms_per_iteration": f_ms / max(1, fst["iterations"]),
            "preconditioner": f"aggregation multigrid, {fst['levels']} levels" if mg else "Jacobi",
            "cells_per_s": ncell / (f_ms * 1e-3),
            "roofline": {"bound": "hbm", "unit": "GB/s", "achieved": nbytes / (f_ms * 1e-3) / 1e9,
                         "peak": hbm, "frac": nbytes / (f_ms * 1e-3) / 1e9 / hbm,
                         "bytes_per_cell": f"{sb} + {pb} x {fst['passes']} passes + "
                                           f"{ib} x {fst['iterations']} iterations"}}


def run_fld_only(args, local):
    """--fld: trace the tau = 1 disk of --fld-grid, then time the FLD step on it."""
    import torch
    from paper_1001_3301_gb300 import Tracer
    torch.cuda.set_device(local)
    nr, nth, nph = _dims(args.fld_grid)
    w = synth.disk3d(nr, nth, nph, n_nu=NNU, tau550=1.0, seed=1)
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    rho = torch.from_numpy(w.rho32()).cuda()
    td = torch.from_numpy(w.tdust32()).cuda()
    q, _, _ = tr.irradiate(rho, td)
    out = run_fld(args, tr, w, rho, q, torch.cuda.current_stream())
    tr.close()
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.batch:
        if rank == 0:
            run_batch(args, local)
        return
    if args.precision_sweep:
        if rank == 0:
            run_precision_sweep(args, local)
        return
    if args.cpu_table:
        if rank == 0:
            run_cpu_table(args, local)
        return
    if args.surrogate:
        if rank == 0:
            print(json.dumps({"mode": "surrogate", **run_surrogate(args, local)}), flush=True)
        return
    if args.lut:
        if rank == 0:
            print(json.dumps({"mode": "lut_comparator", **run_lut(args, local)}), flush=True)
        return
    if args.fld:
        if rank == 0:
            print(json.dumps({"mode": "fld", **run_fld_only(args, local)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
