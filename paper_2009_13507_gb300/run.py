"""Run the split-step solver on one synthetic grid from the command line.

    python -m paper_2009_13507_gb300.run --dim 2 --n 256 --precision c64 --steps 64

Builds the state (a seeded random-phase Gaussian in 2D, a jittered Gaussian in
1D), advances it --steps time steps in imaginary (default) or real time with the
library's graph-replayed step, and prints the observables and the wall time as
one JSON line. The physics defaults are those of the 2D 256 x 256 benchmark
workload (c0 = 50, c2 = 1, Rashba gamma = 0.8, Omega = 0.5, dt = 2e-4).
Meant for quick checks and for profiler captures of a small, fixed case.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dim", type=int, default=2, choices=(1, 2))
    ap.add_argument("--n", type=int, default=256, help="points per axis")
    ap.add_argument("--dx", type=float, default=0.05)
    ap.add_argument("--precision", default="c128", choices=("c128", "c64", "cdf"))
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--real", action="store_true", help="real-time steps (default: imaginary time)")
    ap.add_argument("--c0", type=float, default=50.0)
    ap.add_argument("--c2", type=float, default=1.0)
    ap.add_argument("--so-type", type=int, default=1)
    ap.add_argument("--gamma", type=float, default=0.8)
    ap.add_argument("--omega", type=float, default=0.5)
    ap.add_argument("--dt", type=float, default=2e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--renorm", type=int, default=None, choices=(0, 1, 2),
                    help="renormalisation mode (default: 1 in imaginary time, 0 in real time)")
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import inputs as I
    from . import sgpe

    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    ny = n if args.dim == 2 else 1
    if args.dim == 2:
        psi0 = I.gaussian_phase_2d(n, n, args.dx, args.dx, seed=args.seed)
    else:
        psi0 = I.gaussian_jitter_1d(n, args.dx, seed=args.seed)
    dtype = torch.complex64 if args.precision == "c64" else torch.complex128
    s = sgpe.Solver(args.dim, n, ny, dx=args.dx, precision=args.precision, device=dev)
    s.set_params(sgpe.Physics(c0=args.c0, c2=args.c2, so_type=args.so_type, gamma=args.gamma, omega=args.omega,
                              dt=args.dt, renorm=(0 if args.real else 1) if args.renorm is None else args.renorm))
    s.load_state(torch.from_numpy(psi0.astype(np.complex128)).to(dev).to(dtype))
    s.synchronize()
    t0 = time.perf_counter()
    if args.real:
        s.step_real(args.steps)
    else:
        s.step_imag(args.steps)
    obs = s.energy()
    wall = time.perf_counter() - t0
    out = {"dim": args.dim, "n": n, "precision": args.precision, "steps": args.steps,
           "mode": "real" if args.real else "imag", "wall_s": wall,
           "point_steps_per_s": n * ny * args.steps / wall, "observables": obs}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
