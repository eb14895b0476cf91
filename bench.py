#!/usr/bin/env python
"""Benchmark of the discrete-ordinates CT dose solve on GB300.

One step = one complete forward solve of the water-cylinder workload
(64x64x32 voxels, S8, P3, 19 groups, one cone-beam source): Siddon ray trace
and first-collision source, source iteration of the collided problem with
octant wavefront sweeps until the relative change of the scalar fluence is
below 1e-6 in every group, particle balance.  The metric is phase-space cell
updates per second: voxels x directions x groups x sweeps, divided by the
device time of the whole step.  Inputs are resident in HBM before the timed
region; the working set (four 160 MB moment arrays) is larger than L2.

After the headline line's own fields the line carries the other workloads of
the same metric, each solved after the timed region: the S16 abdomen, the
batched axial scan (64 views + 16 extra cylinders), the differentiable
abdomen (forward and adjoint solves), the paper's S_N x P_N scan and its
Table 6 meshes, and diamond against step differencing; each with its own
sweep roofline and, where stored FP64 oracle values exist, its error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on all host cores on a bounded
sample of the same workload (the complete solve of its highest-energy group:
ray trace, first-collision source and source iteration to the same
tolerance).  Under torchrun every rank solves its own view of an axial scan
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space cell updates/s (voxel*angle*group)"
UNIT = "cell_updates/s"
WORKLOAD = "water_cylinder"
WORKLOAD_DESC = ("35 cm water cylinder, 64x64x32 mesh (0.55x0.55x0.5 cm), fan 40 deg x 4 cm cone-beam "
                 "source at 54 cm, 19 groups 10-120 keV, S8 (80 directions), P3, FP32 sweep, tol 1e-6")
TOL = 1e-6

# DRAM traffic (read + write) of one full sweep of the water cylinder per sweep
# schedule (tile_x, tile_y, directions per block, kernel): a stored figure
# from one `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` capture,
# valid only for the kernel source it was taken on (keyed by its SHA-1), and
# reported as null once that source changes.
SWEEP_TRAFFIC = {
    (16, 16, 10, 1): (2246.4e6, "sweep_impl.cuh", "592eff4d10129e1bde8b55aecdf9fbf52f768e8c"),
    (16, 16, 5, 1): (1687.6e6, "sweep_impl.cuh", "592eff4d10129e1bde8b55aecdf9fbf52f768e8c"),
    (16, 8, 10, 3): (2534.9e6, "sweep_chain.cuh", "3502773d12d37fb58b50dbc1187553785b1df685"),
    (8, 8, 10, 4): (3338.1e6, "sweep_flow.cuh", "19e106b753eb9e515798e72f9e5fe72303e29839"),
    (16, 8, 10, 7): (2806.1e6, "sweep_flow.cuh", "19e106b753eb9e515798e72f9e5fe72303e29839"),
    (8, 8, 10, 7): (3000.1e6, "sweep_flow.cuh", "19e106b753eb9e515798e72f9e5fe72303e29839"),
    (16, 16, 10, 7): (2619.2e6, "sweep_flow.cuh", "19e106b753eb9e515798e72f9e5fe72303e29839"),
}

# sweep kernel by the library's sweep_kernel code
SWEEP_KERNELS = {1: "k_sweep", 3: "k_sweep_chain", 4: "k_sweep_flow",
                 5: "k_split_m2d + k_sweep_flow<split> + k_split_d2m", 7: "k_sweep_flow<face warp>",
                 8: "k_m2d_tc + k_sweep_flow<split> + k_d2m_tc"}

# FP32 lanes per SM and SMs of a GB300 (the ALU roofline of the CUDA-core sweep)
FP32_LANES_PER_SM = 128
SMS = 152


def _sha1(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def _r(x, sig=4):
    """x with every float rounded to `sig` significant digits (compact JSON)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}") if math.isfinite(x) else x
    if isinstance(x, dict):
        return {k: _r(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_r(v, sig) for v in x]
    return x


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def leading_groups(p, k):
    """The first k (highest-energy) groups of problem p as a problem of their
    own.  Scattering only goes down in energy, so these groups do not depend
    on the rest: their solve is exactly the first k groups of p's solve."""
    srcs = [dataclasses.replace(s, spectrum=None if s.spectrum is None else s.spectrum[:k]) for s in p.sources]
    return dataclasses.replace(p, sigma_t=p.sigma_t[:, :k].copy(), sigma_s=p.sigma_s[:, :, :k, :k].copy(),
                               k_dep=p.k_dep[:, :k].copy(), e_mid=p.e_mid[:k].copy(), sources=srcs)


def oracle_solve_sample(p, groups, threads):
    """Time the FP64 oracle's forward solve (ray trace, first-collision source,
    Gauss-Seidel source iteration to TOL) of the first `groups` groups of p on
    `threads` host threads (0: all).  Returns (cell updates/s, cell updates,
    seconds, threads used); the sweeps per group are left in
    oracle_solve_sample.iters."""
    from oracle import solver as osv
    from oracle import transport as tr
    used = tr.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    q = leading_groups(p, groups)
    t0 = time.perf_counter()
    sol = osv.solve(q, tol=TOL)
    el = time.perf_counter() - t0
    cells = q.V * q.n_angles * sum(sol.iters)
    oracle_solve_sample.iters = list(sol.iters)
    return cells / el, cells, el, used


def sweep_roofline(p, r, sm_mhz, hbm_peak):
    """Roofline of the sweep of one solve record: achieved FP32 TFLOP/s of the
    algorithmic flops (4M + 8 per cell update) over the sweep time against
    the FP32 FMA peak, and the algorithmic bytes (moments read and written
    once, material and density) against the measured HBM bandwidth."""
    M = (p.legendre + 1) ** 2
    cells = r["cell_updates"]
    sweep_s = r["ms_sweep"] / 1e3
    fpu = 4 * M + 8
    bpu = (2 * M * p.G * p.V * 4 + 5 * p.V) / (p.V * p.n_angles * p.G)
    tf = fpu * cells / sweep_s / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    gbs = bpu * cells / sweep_s / 1e9
    return {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "ms_per_sweep": r["ms_sweep"] / max(1, r["iterations"]), "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak}


def _max_rel(a, b):
    import numpy as np
    a, b = np.atleast_2d(a).astype(np.float64), np.atleast_2d(b).astype(np.float64)
    worst = 0.0
    for x, y in zip(a, b):
        sel = np.abs(y) > 1e-6 * np.abs(y).max()
        worst = max(worst, float((np.abs(x[sel] - y[sel]) / np.abs(y[sel])).max()))
    return worst


def golden_parity(name, phi, dose, phi_u=None, phi_c=None):
    """Error of a solve's total fluence [G][V] and dose [V] (and, if given,
    its uncollided and collided fluence) against the FP64 oracle values
    stored for seeded voxels of workload `name` (largest relative error over
    groups on values above 1e-6 of the group's maximum) and against the
    stored per-group fluence totals; None if none stored."""
    import numpy as np
    gold = os.path.join(ROOT, "tests", "golden", f"{name}_samples.npz")
    if not os.path.exists(gold):
        return None
    ref = np.load(gold)
    idx = ref["voxels"]
    out = {"voxels": int(idx.size), "max_rel_phi": _max_rel(phi[:, idx], ref["phi"]),
           "max_rel_dose": _max_rel(dose[idx], ref["dose"]),
           "max_rel_group_totals": float(np.abs(phi.astype(np.float64).sum(axis=1) / ref["phi_total"] - 1.0).max()),
           "tolerance": 1e-4}
    if phi_u is not None:
        out["max_rel_phi_u"] = _max_rel(phi_u[:, idx], ref["phi_u"])
    if phi_c is not None:
        out["max_rel_phi_c"] = _max_rel(phi_c[:, idx], ref["phi_c"])
    return out


def ray_visits(p, src):
    """Voxel visits of the uncollided ray trace of one point source (the work
    of the ray-trace kernel): for each voxel centre, 1 + the grid planes its
    ray crosses between the mesh entry and the centre (a tie where the ray
    crosses two planes at once counts twice, so this slightly over-counts)."""
    import numpy as np
    X, Y, Z = p.centres()
    T = np.stack([X, Y, Z], axis=1)
    S = np.asarray(src.pos, np.float64)
    o = np.asarray(p.origin, np.float64)
    sp = np.array([p.dx, p.dy, p.dz])
    n = np.array([p.nx, p.ny, p.nz])
    d = T - S
    lo, hi = o, o + n * sp
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - S) / d
        t2 = (hi - S) / d
    tmin = np.where(d != 0, np.minimum(t1, t2), -np.inf).max(axis=1)
    E = S + (tmin[:, None] + 1e-9) * d
    iE = np.clip(np.floor((E - o) / sp), 0, n - 1)
    iT = np.clip(np.floor((T - o) / sp), 0, n - 1)
    return int((1 + np.abs(iT - iE).sum(axis=1)).sum())


def _schedule(t):
    return {k: t[k] for k in ("tile_x", "tile_y", "angles_per_block", "sweep_kernel")}


def _timed_solve(DoctorsProblem, p, stream, tune=True):
    """Autotune (or not), solve once to warm up, then time one solve."""
    d = DoctorsProblem(p, stream=stream, tol=TOL, max_iters=500)
    t = d.autotune() if tune else None
    d.solve()
    return d, d.solve(), t


def bench_abdomen(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak):
    """The S16 abdomen (128x128x48, 0.25 cm, 19 groups, P3, one cone-beam
    projection): one autotuned solve, its sweep roofline, the ray trace's
    voxel visits and the error against stored FP64 oracle samples."""
    p = ph.config_problem("abdomen")
    d, r, t = _timed_solve(DoctorsProblem, p, stream)
    par = golden_parity("abdomen", d.fluence_host(2), d.dose_host(p.k_dep), d.fluence_host(0), d.fluence_host(1))
    d.close()
    return {"ms_per_solve": r["ms_total"], "cell_updates_per_s": r["cell_updates"] / (r["ms_total"] / 1e3),
            "iterations": r["iterations"], "converged": bool(r["converged"]), "schedule": _schedule(t),
            "roofline": sweep_roofline(p, r, sm_mhz, hbm_peak),
            "raytrace": {"voxel_visits": ray_visits(p, p.sources[0]), "ms_first_collision": r["ms_raytrace"]},
            "parity": par}


def bench_batched(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak):
    """Axial-scan batch: 64 views on the water-cylinder mesh plus 16 extra
    cylinders (6 x 48^3, 5 x 64x64x32, 5 x 96x96x32), solved as one
    graph-captured batch and, for comparison, one instance at a time.  The
    first view is the headline workload's problem, so its fluence and dose
    are checked against the stored FP64 oracle samples; the 64 views'
    summed dose is checked against one solve with all 64 sources (the
    problem is linear in its sources)."""
    import numpy as np
    from paper_1811_12391_gb300.solver import solve_batch
    base = ph.config_problem("water_cylinder")
    views = ph.axial_scan_sources(base, 64)
    inst = [base.with_sources([v]) for v in views] + ph.extra_cylinders()
    ds = [DoctorsProblem(q, stream=stream, tol=TOL, max_iters=500) for q in inst]
    ds[0].autotune()
    solve_batch(ds)                      # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = solve_batch(ds)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    view_dose = torch.zeros(base.V, dtype=torch.float64, device="cuda")
    for d in ds[:64]:
        view_dose += d.dose(base.k_dep)
    par = golden_parity("water_cylinder", ds[0].fluence_host(2), ds[0].dose_host(base.k_dep))
    e0.record(stream)
    for d in ds:
        d.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    cells = sum(r["cell_updates"] for r in res)
    for d in ds:
        d.close()
    sup = DoctorsProblem(base.with_sources(views), stream=stream, tol=TOL, max_iters=500)
    sup.solve()
    sup_dose = sup.dose(base.k_dep)
    sup.close()
    sel = sup_dose.abs() > 1e-6 * sup_dose.abs().max()
    superposition = float(((view_dose - sup_dose).abs()[sel] / sup_dose.abs()[sel]).max().item())
    flops = sum((4 * (q.legendre + 1) ** 2 + 8) * r["cell_updates"] for q, r in zip(inst, res))
    tf = flops / (ms_batch / 1e3) / 1e12
    peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    return {"instances": len(inst), "ms_batch": ms_batch, "ms_one_at_a_time": ms_single,
            "speedup_vs_one_at_a_time": ms_single / ms_batch,
            "cell_updates_per_s": cells / (ms_batch / 1e3),
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "note": "sweep flops of all instances over the batch's whole device time"},
            "iterations_max": max(r["iterations"] for r in res), "converged": all(r["converged"] for r in res),
            "parity": {"view0": par, "max_rel_summed_dose_vs_superposed_solve": superposition}}


def bench_differentiable(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak):
    """The differentiable abdomen (S8, P3, 19 groups, 32 views): the forward
    solve and the adjoint solve that gives the gradients of the liver-ROI
    mean dose with respect to the 32 view weights, 19 spectrum weights and
    every voxel density, against stored FP64 oracle gradients."""
    import numpy as np
    p = ph.config_problem("differentiable_abdomen")
    d, r, t = _timed_solve(DoctorsProblem, p, stream)
    roi = torch.as_tensor(p.roi / p.roi.sum(), device="cuda")
    d.roi_gradients(p.k_dep, roi)
    g = d.roi_gradients(p.k_dep, roi)
    par = None
    gold = os.path.join(ROOT, "tests", "golden", "differentiable_abdomen_gradients.npz")
    if os.path.exists(gold):
        ref = np.load(gold)
        gd = g["density"].cpu().numpy()
        idx = ref["voxels"]
        big = np.abs(ref["d_density"]) > 1e-4 * float(ref["d_density_max"])
        par = {"J": abs(g["J"] / float(ref["J"]) - 1.0),
               "d_weights": _max_rel(g["weights"].cpu().numpy(), ref["d_weights"]),
               "d_spectrum": _max_rel(g["spectrum"].cpu().numpy(), ref["d_spectrum"]),
               "d_density_sampled": float((np.abs(gd[idx] - ref["d_density"]) / np.abs(ref["d_density"]))[big].max()),
               "voxels": int(idx.size)}
    d.close()
    return {"ms_forward": r["ms_total"], "ms_adjoint": g["result"]["ms_total"],
            "iterations": [r["iterations"], g["result"]["iterations"]],
            "cell_updates_per_s": r["cell_updates"] / (r["ms_total"] / 1e3), "schedule": _schedule(t),
            "roofline": sweep_roofline(p, r, sm_mhz, hbm_peak), "parity": par}


def bench_sn_pn_scan(torch, DoctorsProblem, ph, stream):
    """The paper's S_N x P_N scan (Table 2) on its coarse water workload:
    64x64x16 mesh, 7 groups (10-100 keV), one isotropic point source, S2, S4,
    S6, S8 with P0 and P1, each autotuned and timed on one solve."""
    out = {}
    for L in (0, 1):
        for sn in (2, 4, 6, 8):
            p = ph.paper_water(sn=sn, L=L)
            d, r, t = _timed_solve(DoctorsProblem, p, stream)
            out[f"S{sn}P{L}"] = {"ms": r["ms_total"], "iters": r["iterations"], "kernel": t["sweep_kernel"],
                                 "cups": r["cell_updates"] / (r["ms_total"] / 1e3)}
            d.close()
    return out


# the paper's GPU runtimes for its water phantom, S6 P0, 7 groups (Table 6;
# one GK110 die of a GTX Titan Z, the paper's phantom and cross sections):
# context for the same-shaped synthetic runs, not a target
PAPER_TABLE6_GPU_S = {"paper_water_coarse_sp": 2.8, "paper_water_coarse_ct": 3.2,
                      "paper_water_fine_sp": 66.8, "paper_water_fine_ct": 364.4}


def bench_paper_workloads(torch, DoctorsProblem, ph, stream):
    """The paper's own water-phantom runs at its mesh sizes and settings
    (64x64x16 and 256x256x64, S6 P0, 7 groups; one point source or 16 cone
    beams), each autotuned and timed on one solve."""
    out = {}
    for name, paper_s in PAPER_TABLE6_GPU_S.items():
        p = ph.config_problem(name)
        d, r, t = _timed_solve(DoctorsProblem, p, stream)
        out[name.replace("paper_water_", "")] = {"ms": r["ms_total"], "cups": r["cell_updates"] / (r["ms_total"] / 1e3),
                                                 "kernel": t["sweep_kernel"], "paper_gpu_s": paper_s}
        d.close()
    return out


def bench_diamond(torch, DoctorsProblem, ph, stream):
    """Diamond against step differencing on the full-size water cylinder: each
    scheme autotuned (diamond runs on the dataflow kernel only) and timed on
    one solve, with the largest relative difference of the two schemes'
    per-group collided fluence integrals."""
    rec, sums = {}, {}
    for diff, label in ((0, "step"), (1, "diamond")):
        p = ph.config_problem("water_cylinder")
        p.differencing = diff
        d, r, t = _timed_solve(DoctorsProblem, p, stream)
        sums[diff] = d.fluence_host(1).astype("float64").sum(axis=1)
        rec[label] = {"ms": r["ms_total"], "ms_per_sweep": r["ms_sweep"] / max(1, r["iterations"]),
                      "iters": r["iterations"], "balance_rel": r["balance_rel"]}
        d.close()
    rec["max_rel_group_integral_diff"] = float(abs(sums[1] / sums[0] - 1).max())
    return rec


def run_reference(args, rank, world):
    """The oracle on all host cores: each step the complete solve of the
    workload's highest-energy group."""
    from synth import phantoms as ph
    if rank != 0:
        return
    p = ph.config_problem(WORKLOAD)
    for _ in range(args.warmup):
        oracle_solve_sample(p, 1, 0)
    cells = secs = 0.0
    used = 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, c, el, used = oracle_solve_sample(p, 1, 0)
        cells += c
        secs += el
    wall = time.perf_counter() - t0
    value = cells / secs
    sample = (f"each step: the FP64 oracle's complete solve of group 0 of the {p.nx}x{p.ny}x{p.nz} workload "
              f"(ray trace, first-collision source, source iteration to {TOL:g}; {p.n_angles} directions) on "
              f"{used} host threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baselines(p, ph, seconds):
    """The oracle on this host, in the same run: the complete solve of the
    first groups of the workload on all host threads and on one thread
    (groups added until about `seconds` of work), and the complete solve of
    the 16^3 tiny cube (all four groups) both ways."""
    out = {}
    for label, threads in (("all_cores", 0), ("one_core", 1)):
        k, rec = 1, None
        while k <= p.G:
            v, c, el, used = oracle_solve_sample(p, k, threads)
            rec = {"value": v, "cores": used, "groups": k, "seconds": el, "iterations": oracle_solve_sample.iters}
            if el >= seconds / 4 or threads == 1:
                break
            k *= 2
        out[label] = rec
    tiny = ph.config_problem("tiny_cube")
    out["tiny_cube_full_solve_s"] = {}
    for label, threads in (("all_cores", 0), ("one_core", 1)):
        v, c, el, used = oracle_solve_sample(tiny, tiny.G, threads)
        out["tiny_cube_full_solve_s"][label] = el
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="omit the other workloads (the headline fields are unchanged)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1811_12391_gb300.build import build as build_lib
    build_lib()
    from paper_1811_12391_gb300 import sharding
    from paper_1811_12391_gb300.solver import DoctorsProblem
    from synth import phantoms as ph

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = ph.config_problem(WORKLOAD)
    if world > 1:   # every rank solves its own block of the views of an axial scan
        p = p.with_sources(sharding.my_items(ph.axial_scan_sources(p, world), rank, world))
    hbm_peak, peak_kind = measured_peaks()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = DoctorsProblem(p, stream=stream, tol=TOL, max_iters=500)
        tuning = d.autotune()
        for _ in range(args.warmup):
            d.solve()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local).start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [d.solve() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if world > 1:
            dist.barrier()
        ms_max = sharding.max_time(e0.elapsed_time(e1), device="cuda")
        cells = sum(r["cell_updates"] for r in res)
        value = world * cells / (ms_max / 1e3)
        launches = int(sum(r["launches"] for r in res))
        sweeps = sum(r["iterations"] for r in res)
        ms_sweep = sum(r["ms_sweep"] for r in res)
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0

        # end to end through the C-ABI with host buffers (copies inside the
        # timed region): materials and densities in, total fluence and dose
        # out, every step, through pinned host buffers
        k_dep = np.ascontiguousarray(p.k_dep)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        mat_h, rho_h = pin(p.mat), pin(p.density)
        phi = torch.empty((p.G, p.V), dtype=torch.float32).pin_memory().numpy()
        dose = torch.empty(p.V, dtype=torch.float64).pin_memory().numpy()
        t0 = time.perf_counter()
        e2e_cells = 0.0
        for _ in range(args.steps):
            d.set_materials(mat_h, rho_h, p.sigma_t, p.sigma_s)
            d.set_sources(p.sources)
            r = d.solve()
            d.fluence_host(2, out=phi)
            d.dose_host(k_dep, out=dose)
            e2e_cells += r["cell_updates"]
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        h2d = p.V * 1 + p.V * 4
        d2h = phi.nbytes + dose.nbytes
        # the last end-to-end solve against stored FP64 oracle values
        parity = golden_parity(WORKLOAD, phi, dose, d.fluence_host(0), d.fluence_host(1)) if world == 1 else None

        # adjoint (backward) solve: gradients of the mean dose in a central region
        adjoint = None
        if not args.no_extra:
            roi = np.zeros(p.V)
            roi.reshape(p.nz, p.ny, p.nx)[p.nz // 2 - 2:p.nz // 2 + 2, p.ny // 2 - 4:p.ny // 2 + 4,
                                          p.nx // 2 - 4:p.nx // 2 + 4] = 1.0 / 256.0
            roi = torch.as_tensor(roi, device="cuda")
            d.solve()
            g = d.roi_gradients(p.k_dep, roi)
            g = d.roi_gradients(p.k_dep, roi)
            adjoint = {"ms": g["result"]["ms_total"], "iters": g["result"]["iterations"],
                       "gradients": "view weights, spectrum, densities"}
        d.close()

        # the axial scan's instances sharded over the ranks: each rank solves
        # its contiguous block one at a time; the 64 views' doses (one mesh)
        # are summed across ranks in FP64
        sharded = None
        if world > 1 and not args.no_extra:
            base = ph.config_problem(WORKLOAD)
            inst = [base.with_sources([v]) for v in ph.axial_scan_sources(base, 64)] + ph.extra_cylinders()
            mine = sharding.block(len(inst), rank, world)
            view_dose = torch.zeros(base.V, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            dist.barrier()
            t0 = time.perf_counter()
            sh_cells = 0.0
            for i in mine:
                q = DoctorsProblem(inst[i], stream=stream, tol=TOL, max_iters=500)
                rr = q.solve()
                sh_cells += rr["cell_updates"]
                if i < 64:
                    view_dose += q.dose(base.k_dep)
                q.close()
            torch.cuda.synchronize()
            ms_sh = sharding.max_time(1e3 * (time.perf_counter() - t0), device="cuda")
            sharding.sum_dose(view_dose)
            tot = torch.tensor([sh_cells], dtype=torch.float64, device="cuda")
            dist.all_reduce(tot)
            sharded = {"instances": len(inst), "ms_max_over_ranks": ms_sh,
                       "cell_updates_per_s": float(tot.item()) / (ms_sh / 1e3),
                       "summed_view_dose": float(view_dose.sum().item())}

        plain = batched = abdomen = diff_abd = scan = paper = diamond = None
        if not args.no_extra and world == 1:
            # the plain single-instance solve: tile-stage kernel, default schedule, no autotuning
            q = DoctorsProblem(p, stream=stream, tol=TOL, max_iters=500, sweep_kernel=1)
            q.solve()
            rp = q.solve()
            q.close()
            plain = {"kernel": "k_sweep (tile stages, 16x16 tiles, whole octants per CTA)",
                     "ms": rp["ms_total"], "ms_per_sweep": rp["ms_sweep"] / rp["iterations"],
                     "timed_solve_speedup": rp["ms_total"] / (ms_max / args.steps)}
            abdomen = bench_abdomen(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak)
            batched = bench_batched(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak)
            diff_abd = bench_differentiable(torch, DoctorsProblem, ph, stream, sm_mhz, hbm_peak)
            scan = bench_sn_pn_scan(torch, DoctorsProblem, ph, stream)
            paper = bench_paper_workloads(torch, DoctorsProblem, ph, stream)
            diamond = bench_diamond(torch, DoctorsProblem, ph, stream)

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    M = (p.legendre + 1) ** 2
    # algorithmic work of one sweep: per cell update 2M flops (moments ->
    # direction), 2M (direction -> moments) and 8 for the step solve; bytes:
    # read the moment source and write the moments once, plus material/density
    # (a sweep of the iteration's active groups only: converged leading groups
    # are not swept again, so the work is counted per cell update)
    flops_per_update = 4 * M + 8
    flops_per_sweep = flops_per_update * p.V * p.n_angles * p.G
    bytes_per_sweep = 2 * M * p.G * p.V * 4 + 5 * p.V
    bytes_per_update = bytes_per_sweep / (p.V * p.n_angles * p.G)
    sweep_s = ms_sweep / 1e3
    sec_per_sweep = sweep_s / sweeps
    achieved_tflops = flops_per_update * cells / sweep_s / 1e12
    achieved_gbs = bytes_per_update * cells / sweep_s / 1e9
    alu_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    key = (tuning["tile_x"], tuning["tile_y"], tuning["angles_per_block"], tuning["sweep_kernel"])
    traffic = None
    if key in SWEEP_TRAFFIC:
        tbytes, fname, sha = SWEEP_TRAFFIC[key]
        if _sha1(os.path.join(ROOT, "paper_1811_12391_gb300", "csrc", fname)) == sha:
            traffic = tbytes
    cpu = cpu_baselines(p, ph, args.cpu_seconds) if world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC, "voxels": p.V,
                   "directions": p.n_angles, "groups": p.G, "moments": M,
                   "sweeps_per_step": sweeps / args.steps, "l2": "inputs larger than L2 (4 x 160 MB moment arrays)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": f"{SWEEP_KERNELS.get(tuning['sweep_kernel'], '?')} (the launches of one sweep)",
                     "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / alu_peak,
                     "peak_kind": f"FP32 FMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_mhz:.0f} MHz",
                     "traffic": traffic,
                     "traffic_source": "stored ncu dram bytes of one sweep, keyed by the kernel source's SHA-1",
                     "algorithmic_flops_per_sweep": flops_per_sweep,
                     "algorithmic_bytes_per_sweep": bytes_per_sweep, "ms_per_sweep": 1e3 * sec_per_sweep,
                     "flops_per_cell_update": flops_per_update,
                     "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_kind": peak_kind + " (MEASURED_PEAKS.json)"}},
        "cpu_baseline": None if cpu is None else {
            "value": cpu["all_cores"]["value"], "unit": UNIT, "cores": cpu["all_cores"]["cores"], "kind": "oracle",
            "sample": (f"the FP64 oracle's complete solve of groups 0-{cpu['all_cores']['groups'] - 1} of the same "
                       f"workload (ray trace, first-collision source, source iteration to {TOL:g}) in "
                       f"{cpu['all_cores']['seconds']:.1f} s on {cpu['all_cores']['cores']} host threads"),
            "one_core": _r(cpu["one_core"]), "tiny_cube_full_solve_s": _r(cpu["tiny_cube_full_solve_s"])},
        "e2e": {"value": world * e2e_cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "parity": _r(parity),
        "gpu_launches": launches,
        "clocks": clocks,
        "autotune": _r(tuning),
        "adjoint": _r(adjoint),
        "plain_single_instance_solve": _r(plain),
        "axial_scan_sharded": _r(sharded),
        "paper_table6_workloads": _r(paper),
        "diamond_difference": _r(diamond),
        "sn_pn_scan_paper_water_coarse": _r(scan),
        "differentiable_abdomen": _r(diff_abd),
        "axial_scan_batch": _r(batched),
        "abdomen_s16": _r(abdomen),
    }
    print(json.dumps(line, separators=(",", ":")), flush=True)


if __name__ == "__main__":
    main()
