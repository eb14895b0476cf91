"""Command line: solve a named synthetic workload and print the report.

  python -m paper_1811_12391_gb300 <workload> [--iters N] [--tol T] [--tile X Y] [--ab K] [--kernel 0..8]
                                   [--sn N] [--legendre L] [--device-loop] [--diamond] [--adjoint]
                                   [--autotune] [--repeat R]

Workloads: tiny_cube, water_cylinder, abdomen, axial_scan, differentiable_abdomen
(see synth/phantoms.py).  Used as the profiled command in profiles/.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser(prog="python -m paper_1811_12391_gb300")
    ap.add_argument("workload")
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--tile", type=int, nargs=2, default=(0, 0))
    ap.add_argument("--ab", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0, help="sweep kernel: 0 default, 1 CUDA-core, 3 chained CUDA-core, 4 dataflow, 5 dataflow with split "
                    "transforms, 7 dataflow with a face warp, 8 split transforms on the tensor cores")
    ap.add_argument("--sn", type=int, default=None, help="quadrature order (tiny_cube, water_cylinder, abdomen)")
    ap.add_argument("--legendre", type=int, default=None, help="Legendre order (tiny_cube, water_cylinder, abdomen)")
    ap.add_argument("--device-loop", action="store_true",
                    help="run the source iteration as one CUDA graph with a device-side while loop")
    ap.add_argument("--diamond", action="store_true", help="diamond differencing (dataflow sweep)")
    ap.add_argument("--adjoint", action="store_true",
                    help="after each solve, the adjoint solve and all gradients of the mean dose in a central box")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args()
    from paper_1811_12391_gb300.build import build
    build()
    from paper_1811_12391_gb300.solver import DoctorsProblem
    from synth import phantoms as ph

    p = ph.config_problem(args.workload, sn=args.sn, L=args.legendre)
    if args.diamond:
        p.differencing = 1
    d = DoctorsProblem(p, tol=args.tol, max_iters=args.iters, tile=tuple(args.tile), angles_per_block=args.ab,
                       sweep_kernel=args.kernel, device_loop=int(args.device_loop))
    if args.autotune:
        print(json.dumps({"autotune": d.autotune()}), flush=True)
    roi = None
    if args.adjoint:
        import numpy as np
        import torch
        box = np.zeros(p.V)
        box.reshape(p.nz, p.ny, p.nx)[p.nz // 2 - 2:p.nz // 2 + 2, p.ny // 2 - 4:p.ny // 2 + 4,
                                      p.nx // 2 - 4:p.nx // 2 + 4] = 1.0
        roi = torch.as_tensor(box / box.sum(), device="cuda")
    for _ in range(args.repeat):
        r = d.solve(allow_not_converged=True)
        print(json.dumps(r), flush=True)
        if roi is not None:
            g = d.roi_gradients(p.k_dep, roi)
            print(json.dumps({"adjoint": g["result"], "J": g["J"]}), flush=True)
    d.close()


if __name__ == "__main__":
    main()
