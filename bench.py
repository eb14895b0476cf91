#!/usr/bin/env python
"""Benchmark of the discrete-ordinates CT dose solve on GB300.

One step = one complete forward solve of the workload (Siddon ray trace and
first-collision source, source iteration of the collided problem with octant
wavefront sweeps until the relative change of the scalar fluence is below
1e-6 in every group, particle balance).  The metric is phase-space cell
updates per second: voxels x directions x groups x sweeps, divided by the
device time of the whole step.  Inputs are resident in HBM before the timed
region; the working set (four 160 MB moment arrays) is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (whole-mesh sweeps of one group).  Under torchrun
every rank solves its own view of an axial scan (weak scaling, no data-path
collective); rank 0 prints one JSON line.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space cell updates/s (voxel*angle*group)"
UNIT = "cell_updates/s"
WORKLOAD = "water_cylinder"
WORKLOAD_DESC = ("35 cm water cylinder, 64x64x32 mesh (0.55x0.55x0.5 cm), fan 40 deg x 4 cm cone-beam "
                 "source at 54 cm, 19 groups 10-120 keV, S8 (80 directions), P3, FP32 sweep, tol 1e-6")

# DRAM traffic (read + write) of one full sweep of this workload (the stage
# launches of one iteration) per sweep schedule (tile_x, tile_y,
# directions per block, kernel), from `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum` (profiles/k_sweep*_water_cylinder.md);
# valid only for the kernel source it was taken on.
SWEEP_TRAFFIC = {
    (16, 16, 10, 1): (2246.4e6, "sweep_impl.cuh", "592eff4d10129e1bde8b55aecdf9fbf52f768e8c"),
    (16, 16, 5, 1): (1687.6e6, "sweep_impl.cuh", "592eff4d10129e1bde8b55aecdf9fbf52f768e8c"),
    (16, 16, 10, 2): (2121.9e6, "sweep_tc.cu", "79ec5703826b205c1bdc9d4f7ff57c205fec428a"),
    (16, 8, 10, 3): (2534.9e6, "sweep_chain.cuh", "3502773d12d37fb58b50dbc1187553785b1df685"),
    (8, 8, 10, 4): (3154.0e6, "sweep_flow.cuh", "6057ed04a3eed69e65ed21239fae6fc7df83e2ca"),
}

# sweep kernel by the library's sweep_kernel code
SWEEP_KERNELS = {1: "k_sweep", 2: "k_sweep_tc", 3: "k_sweep_chain", 4: "k_sweep_flow",
                 5: "k_split_m2d + k_sweep_flow<split> + k_split_d2m", 6: "k_sweep_flow<two planes per step>"}

# FP32 lanes per SM and SMs of a GB300 (the ALU roofline of the CUDA-core sweep)
FP32_LANES_PER_SM = 128
SMS = 152


def _sha1(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


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


def oracle_sample(p, seconds=12.0):
    """Time the FP64 oracle's whole-mesh sweeps of group 0 of the workload
    (single-threaded C); returns (cell updates/s, sweeps, seconds)."""
    import numpy as np
    from oracle import quadrature as quad
    from oracle import transport as tr

    dirs, w, R, Mop, Dop = quad.angular_operators(p.sn, p.legendre)
    M = Mop.shape[1]
    sigt = p.density.astype(np.float64) * p.sigma_t[p.mat, 0]
    rng = np.random.default_rng(0)
    src = rng.uniform(0.0, 1.0, size=(M, p.V))
    tr.sweep((p.nx, p.ny, p.nz), (p.dx, p.dy, p.dz), dirs, w, Mop, Dop, sigt, src)   # load + warm
    n = 0
    t0 = time.perf_counter()
    while True:
        tr.sweep((p.nx, p.ny, p.nz), (p.dx, p.dy, p.dz), dirs, w, Mop, Dop, sigt, src)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    cells = n * p.V * dirs.shape[0]
    return cells / el, n, el


def bench_batched(torch, DoctorsProblem, ph, stream):
    """Axial-scan batch: 64 views on the water-cylinder mesh plus 16 extra
    cylinders (6 x 48^3, 5 x 64x64x32, 5 x 96x96x32), solved as one
    graph-captured batch and, for comparison, one instance at a time."""
    from paper_1811_12391_gb300.solver import solve_batch
    base = ph.config_problem("water_cylinder")
    inst = [base.with_sources([v]) for v in ph.axial_scan_sources(base, 64)] + ph.extra_cylinders()
    ds = [DoctorsProblem(q, stream=stream, tol=1e-6, max_iters=500) for q in inst]
    for d in ds[:1]:
        d.autotune()
    solve_batch(ds)                      # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = solve_batch(ds)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    dose_sum = float(sum(d.dose(q.k_dep).sum().item() for d, q in zip(ds, inst)))
    e0.record(stream)
    single = [d.solve() for d in ds]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1)
    cells = sum(r["cell_updates"] for r in res)
    for d in ds:
        d.close()
    return {"instances": len(inst), "ms_batch": ms_batch, "ms_one_at_a_time": ms_single,
            "speedup_vs_single_instance_solves": ms_single / ms_batch,
            "cell_updates_per_s": cells / (ms_batch / 1e3), "summed_dose": dose_sum,
            "iterations_max": max(r["iterations"] for r in res),
            "converged": all(r["converged"] for r in res)}


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


def bench_configs(torch, DoctorsProblem, ph, stream):
    """The other full-size workloads, each autotuned and timed on one solve
    after a warm-up: the S16 abdomen (one cone-beam projection), the 64-view
    axial scan superposed into one solve, and the differentiable abdomen
    (S8, 32 views) whose adjoint solve gives the gradients of the liver-ROI
    mean dose with respect to the view weights, the spectrum and every voxel
    density."""
    import numpy as np
    out = {}
    for name in ("abdomen", "axial_scan", "differentiable_abdomen"):
        p = ph.config_problem(name)
        d = DoctorsProblem(p, stream=stream, tol=1e-6, max_iters=500)
        tune = d.autotune()
        d.solve()
        r = d.solve()
        rec = {"voxels": p.V, "directions": p.n_angles, "groups": p.G, "sources": len(p.sources),
               "ms_per_solve": r["ms_total"], "cell_updates_per_s": r["cell_updates"] / (r["ms_total"] / 1e3),
               "iterations": r["iterations"], "converged": bool(r["converged"]),
               "schedule": {k: tune[k] for k in ("tile_x", "tile_y", "angles_per_block", "sweep_kernel")}}
        if name == "abdomen":
            rec["raytrace"] = {"rays_per_source": p.V, "voxel_visits_per_source": ray_visits(p, p.sources[0]),
                               "ms_first_collision": r["ms_raytrace"]}
        if name == "differentiable_abdomen":
            roi = torch.as_tensor(p.roi / p.roi.sum(), device="cuda")
            d.roi_gradients(p.k_dep, roi)
            g = d.roi_gradients(p.k_dep, roi)
            rec["adjoint_ms"] = g["result"]["ms_total"]
            rec["adjoint_iterations"] = g["result"]["iterations"]
            rec["gradients"] = {"view_weights": int(g["weights"].numel()), "spectrum": int(g["spectrum"].numel()),
                                "densities": int(g["density"].numel())}
        d.close()
        out[name] = rec
    return out


# the paper's GPU runtimes for its water phantom, S6 P0, 7 groups (Table 6;
# one GK110 die of a GTX Titan Z, the paper's phantom and cross sections):
# context for the same-shaped synthetic runs, not a target
PAPER_TABLE6_GPU_S = {"paper_water_coarse_sp": 2.8, "paper_water_coarse_ct": 3.2,
                      "paper_water_fine_sp": 66.8, "paper_water_fine_ct": 364.4}


def bench_paper_workloads(torch, DoctorsProblem, ph, stream):
    """The paper's own water-phantom runs at its mesh sizes and settings
    (64x64x16 and 256x256x64, S6 P0, 7 groups; one point source or 16 cone
    beams), each autotuned and timed on one solve after a warm-up."""
    out = {}
    for name, paper_s in PAPER_TABLE6_GPU_S.items():
        p = ph.config_problem(name)
        d = DoctorsProblem(p, stream=stream, tol=1e-6, max_iters=500)
        tune = d.autotune()
        d.solve()
        r = d.solve()
        out[name] = {"voxels": p.V, "directions": p.n_angles, "groups": p.G, "sources": len(p.sources),
                     "ms_per_solve": r["ms_total"], "cell_updates_per_s": r["cell_updates"] / (r["ms_total"] / 1e3),
                     "iterations": r["iterations"], "converged": bool(r["converged"]),
                     "sweep_kernel": tune["sweep_kernel"], "paper_gpu_s_context": paper_s}
        d.close()
    return out


def bench_diamond(torch, DoctorsProblem, ph, stream):
    """Diamond against step differencing on the 16^3 cube (S4 P1, 4 groups)
    and the full-size water cylinder: each scheme autotuned (diamond runs on
    the dataflow kernel only) and timed on one solve after a warm-up, with
    the largest relative difference of the two schemes' per-group collided
    fluence integrals."""
    out = {}
    for name in ("tiny_cube", "water_cylinder"):
        rec = {}
        sums = {}
        for diff, label in ((0, "step"), (1, "diamond")):
            p = ph.config_problem(name)
            p.differencing = diff
            d = DoctorsProblem(p, stream=stream, tol=1e-6, max_iters=500)
            tune = d.autotune()
            d.solve()
            r = d.solve()
            sums[diff] = d.fluence_host(1).astype("float64").sum(axis=1)
            rec[label] = {"ms_per_solve": r["ms_total"], "ms_per_sweep": r["ms_sweep"] / max(1, r["iterations"]),
                          "iterations": r["iterations"], "converged": bool(r["converged"]),
                          "balance_rel": r["balance_rel"],
                          "cell_updates_per_s": r["cell_updates"] / (r["ms_total"] / 1e3),
                          "schedule": {k: tune[k] for k in ("tile_x", "tile_y", "angles_per_block", "sweep_kernel")}}
            d.close()
        rec["max_rel_group_integral_diff"] = float(abs(sums[1] / sums[0] - 1).max())
        out[name] = rec
    return out


def run_reference(args, rank, world):
    from synth import phantoms as ph
    if rank != 0:
        return
    p = ph.config_problem(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample(p, seconds=0.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, n, el = oracle_sample(p, seconds=0.0)
        vals.append((v, n, el))
    wall = time.perf_counter() - t0
    total_cells = sum(v * el for v, n, el in vals)
    value = total_cells / sum(el for _, _, el in vals)
    sample = (f"{args.steps} whole-mesh FP64 sweeps of group 0 ({p.nx}x{p.ny}x{p.nz} voxels x "
              f"{p.n_angles} directions each) by the single-threaded oracle")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_DESC},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="omit the adjoint, batched-scan and other-workload measurements (the headline line is unchanged)")
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
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = DoctorsProblem(p, stream=stream, tol=1e-6, max_iters=500)
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
        parity = None
        gold = os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_samples.npz")
        if world == 1 and os.path.exists(gold):
            # the last end-to-end solve against FP64 oracle values stored for 600
            # seeded voxels (largest relative error over groups, on values above
            # 1e-6 of the group's maximum) and the per-group fluence totals
            ref = np.load(gold)
            idx = ref["voxels"]

            def max_rel(a, b):
                a, b = np.atleast_2d(a).astype(np.float64), np.atleast_2d(b).astype(np.float64)
                worst = 0.0
                for x, y in zip(a, b):
                    sel = np.abs(y) > 1e-6 * np.abs(y).max()
                    worst = max(worst, float((np.abs(x[sel] - y[sel]) / np.abs(y[sel])).max()))
                return worst

            parity = {"reference": "FP64 oracle, tests/golden/" + os.path.basename(gold), "voxels": int(idx.size),
                      "max_rel_phi": max_rel(phi[:, idx], ref["phi"]), "max_rel_dose": max_rel(dose[idx], ref["dose"]),
                      "max_rel_group_totals": float(np.abs(phi.astype(np.float64).sum(axis=1) / ref["phi_total"]
                                                          - 1.0).max()),
                      "tolerance": 1e-4}

        # adjoint (backward) solve of the mean dose in a central region
        adjoint = None
        if not args.no_extra:
            roi = np.zeros(p.V)
            roi.reshape(p.nz, p.ny, p.nx)[p.nz // 2 - 2:p.nz // 2 + 2, p.ny // 2 - 4:p.ny // 2 + 4,
                                          p.nx // 2 - 4:p.nx // 2 + 4] = 1.0 / 256.0
            roi = torch.as_tensor(roi, device="cuda")
            d.solve()
            g = d.roi_gradients(p.k_dep, roi)
            g = d.roi_gradients(p.k_dep, roi)
            adjoint = {"ms_per_solve": g["result"]["ms_total"], "iterations": g["result"]["iterations"],
                       "gradients": "view weights, spectrum, densities"}
        d.close()
        plain = None
        if not args.no_extra:
            # the plain single-instance solve: tile-stage kernel, default schedule, no autotuning
            q = DoctorsProblem(p, stream=stream, tol=1e-6, max_iters=500, sweep_kernel=1)
            q.solve()
            rp = q.solve()
            q.close()
            plain = {"kernel": "k_sweep (tile stages, default 16x16 tiles, whole octants per CTA)",
                     "ms_per_solve": rp["ms_total"], "ms_per_sweep": rp["ms_sweep"] / rp["iterations"],
                     "speedup_of_the_timed_solve": rp["ms_total"] / (ms_max / args.steps)}
        batched = None if (args.no_extra or world > 1) else bench_batched(torch, DoctorsProblem, ph, stream)
        others = None if (args.no_extra or world > 1) else bench_configs(torch, DoctorsProblem, ph, stream)
        paper = None if (args.no_extra or world > 1) else bench_paper_workloads(torch, DoctorsProblem, ph, stream)
        diamond = None if (args.no_extra or world > 1) else bench_diamond(torch, DoctorsProblem, ph, stream)

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
    hbm_peak, peak_kind = measured_peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    key = (tuning["tile_x"], tuning["tile_y"], tuning["angles_per_block"], tuning["sweep_kernel"])
    traffic = None
    if key in SWEEP_TRAFFIC:
        tbytes, fname, sha = SWEEP_TRAFFIC[key]
        if _sha1(os.path.join(ROOT, "paper_1811_12391_gb300", "csrc", fname)) == sha:
            traffic = tbytes
    cpu_v, cpu_n, cpu_s = oracle_sample(p, seconds=args.cpu_seconds) if world == 1 else (None, 0, 0)
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
                     "traffic": traffic, "algorithmic_flops_per_sweep": flops_per_sweep,
                     "algorithmic_bytes_per_sweep": bytes_per_sweep, "ms_per_sweep": 1e3 * sec_per_sweep,
                     "flops_per_cell_update": flops_per_update,
                     "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_kind": peak_kind + " (MEASURED_PEAKS.json)"}},
        "cpu_baseline": None if cpu_v is None else {
            "value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{cpu_n} whole-mesh FP64 sweeps of group 0 of the same workload in {cpu_s:.1f} s"},
        "e2e": {"value": world * e2e_cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "parity": parity,
        "gpu_launches": launches,
        "clocks": clocks,
        "autotune": tuning,
        "adjoint": adjoint,
        "plain_single_instance_solve": plain,
        "batched_axial_scan": batched,
        "other_workloads": others,
        "paper_workloads": paper,
        "diamond_difference": diamond,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
