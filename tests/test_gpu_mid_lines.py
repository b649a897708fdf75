"""2D grids whose lines have 257..1024 points: the register kernels with 16- and
32-point lane chunks (the fused head k_pwx<R, IMAG, 16|32> and the y sweep
k_cny_reg<R, IMAG, 16|32>, including the two-blocks-per-SM head for 512-point
rows) against the FP64 CPU oracle, in every precision, imaginary and real time;
and the real-time quench of the 512 x 512 precision workload from a prepared
ground state against the oracle.

Bars: complex128 and double-float 1e-10 normwise relative for the state and
relative for each observable; complex64 (FP32 state and sweeps, FP64
reductions) a stated bound on the same measures."""
import functools

import numpy as np
import pytest

from gpu_util import make_pair, obs_relerr, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu

PHYS_2D = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
# (nx, ny, dx, dy): chunk lengths (x, y) = (16, 16), (16, 32), (32, 2), (2, 32)
GRIDS = [(512, 512, 0.04, 0.04), (300, 700, 0.05, 0.05), (1024, 40, 0.02, 0.3), (40, 1000, 0.3, 0.02)]
NSTEPS = 24
TOL = {"c128": 1e-10, "cdf": 1e-10, "c64": 2e-5}


@functools.lru_cache(maxsize=None)
def _oracle_run(nx, ny, dx, dy, imag):
    prob = O.Problem(dim=2, nx=nx, ny=ny, dx=dx, dy=dy, **PHYS_2D)
    psi = I.gaussian_phase_2d(nx, ny, dx, dy, seed=nx + ny)
    ref = O.step(prob, psi, NSTEPS, imag)
    return prob, psi, ref, O.observables(prob, ref)


@pytest.mark.parametrize("precision", ["c128", "cdf", "c64"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "%dx%d" % g[:2])
def test_full_steps_mid_length_lines(grid, imag, precision):
    nx, ny, dx, dy = grid
    prob, psi, ref, oref = _oracle_run(nx, ny, dx, dy, imag)
    _, s = make_pair(2, nx, ny, dx=dx, dy=dy, precision=precision, **PHYS_2D)
    s.set_state(psi)
    (s.step_imag(NSTEPS) if imag else s.step_real(NSTEPS))
    tol = TOL[precision]
    assert relerr(s.get_state(), ref) < tol
    assert obs_relerr(s.energy(), oref) < tol


@functools.lru_cache(maxsize=None)
def _quench_case():
    """The real-time quench of the precision workload: 512 x 512, dx = 0.04, the
    2D physics (c0 = 50, c2 = 1, Rashba gamma = 0.8); ground state with Omega = 0.5
    prepared by 3000 FP64 imaginary-time steps on the GPU (the same bits then go to
    the oracle and to every precision), then Omega -> 0 and 100 real-time steps at
    dt = 1e-4 (the oracle needs a few seconds for them)."""
    n, dx = 512, 0.04
    prep = sgpe.Solver(2, n, n, dx=dx)
    prep.set_params(sgpe.Physics(**PHYS_2D))
    prep.set_state(I.gaussian_phase_2d(n, n, dx, dx, seed=0))
    prep.step_imag(3000)
    ground = prep.get_state()
    phys = dict(PHYS_2D, omega=0.0, dt=1e-4, renorm=0)
    prob = O.Problem(dim=2, nx=n, ny=n, dx=dx, dy=dx, **phys)
    ref = O.step(prob, ground, 100, False)
    return phys, prob, ground, ref, O.observables(prob, ground), O.observables(prob, ref)


@pytest.mark.parametrize("precision,tol_state,tol_obs", [("c128", 1e-10, 1e-10), ("cdf", 1e-10, 1e-10),
                                                         ("c64", 1e-5, 2e-6)])
def test_quench_against_oracle(precision, tol_state, tol_obs):
    phys, prob, ground, ref, o0, oref = _quench_case()
    n = prob.nx
    s = sgpe.Solver(2, n, n, dx=prob.dx, precision=precision)
    s.set_params(sgpe.Physics(**phys))
    s.set_state(ground)
    s.step_real(100)
    o = s.energy()
    assert relerr(s.get_state(), ref) < tol_state
    assert abs(o["E"] - oref["E"]) < tol_obs * abs(oref["E"])
    assert abs(o["N"] - oref["N"]) < tol_obs
    # the drift the oracle itself shows over the 100 steps (explicit-Euler SO grows the norm)
    assert abs(oref["N"] - o0["N"]) < 1e-6
