"""Helpers shared by the GPU parity tests: build a GPU solver and an oracle
problem from the same parameters and compare results."""
import numpy as np

from oracle import oracle as O
from paper_2009_13507_gb300 import sgpe


def make_pair(dim, nx, ny=1, dx=0.05, dy=None, precision="c128", **phys):
    dy = dx if dy is None else dy
    prob = O.Problem(dim=dim, nx=nx, ny=ny if dim == 2 else 1, dx=dx, dy=dy, **phys)
    s = sgpe.Solver(dim, nx, ny, dx=dx, dy=dy, precision=precision)
    s.set_params(sgpe.Physics(**phys))
    return prob, s


def relerr(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def obs_relerr(gpu: dict, orc: dict, keys=("N+", "N0", "N-", "N", "E", "mu", "rms+", "rms0", "rms-", "rms")):
    worst = 0.0
    for k in keys:
        ref = orc[k]
        den = max(abs(ref), 1e-300)
        worst = max(worst, abs(gpu[k] - ref) / den)
    return worst
