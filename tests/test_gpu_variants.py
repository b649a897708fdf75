"""The two step options against the FP64 oracle, through the C ABI: Strang
splitting (params.split = 1) and the SO substep by Crank-Nicolson
(params.so_mode = 1, the unitary variant; the GPU rotates each line into the
eigenbasis of its spin matrix and solves scalar skew-tridiagonal lines, the
oracle eliminates the 3x3 block-tridiagonal system in the original basis).

Bars as for the plain step: complex128 and double-float 1e-13 per substep and
1e-10 for whole steps; complex64 a stated bound."""
import ctypes

import numpy as np
import pytest

from gpu_util import make_pair, obs_relerr, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu

PHYS_2D = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
PHYS_1D = dict(c0=10.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2, dt=1e-4, renorm=1)
SUB_TOL = {"c128": 1e-13, "cdf": 1e-12, "c64": 2e-6}
STEP_TOL = {"c128": 1e-10, "cdf": 1e-10, "c64": 2e-5}


def _rand(prob, seed, env=6.0):
    cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)
    return I.random_state(prob.shape, seed, cell, envelope=env)


@pytest.mark.parametrize("precision", ["c128", "cdf", "c64"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which", ["so_cn", "so_cn_rev"])
@pytest.mark.parametrize("dim,nx,ny,so", [(1, 101, 1, 1), (1, 64, 1, 2), (1, 300, 1, 3), (2, 37, 29, 1),
                                          (2, 40, 33, 2), (2, 45, 19, 3), (2, 300, 260, 1)])
def test_so_cn_substep(dim, nx, ny, so, which, imag, precision):
    phys = dict(c0=5.0, c2=0.7, so_type=so, gamma=0.9, omega=0.3, dt=0.05, renorm=1, so_mode=1)
    prob, s = make_pair(dim, nx, ny, dx=0.15, dy=0.2, precision=precision, **phys)
    psi = _rand(prob, 11 + so + nx)
    s.set_state(psi)
    s.substep(which, imag)
    assert relerr(s.get_state(), O.substep(prob, psi, which, imag)) < SUB_TOL[precision]


CASES = [(2, 64, 48, 0.15), (2, 300, 200, 0.05), (1, 256, 1, 0.05), (1, 700, 1, 0.04)]


@pytest.mark.parametrize("precision", ["c128", "cdf", "c64"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("split,so_mode", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd_%dx%d" % c[:3])
def test_full_steps(case, split, so_mode, imag, precision):
    dim, nx, ny, dx = case
    phys = dict(PHYS_2D if dim == 2 else PHYS_1D, split=split, so_mode=so_mode)
    prob, s = make_pair(dim, nx, ny, dx=dx, precision=precision, **phys)
    psi = I.gaussian_phase_2d(nx, ny, dx, dx, seed=nx) if dim == 2 else I.gaussian_jitter_1d(nx, dx, seed=nx)
    s.set_state(psi)
    n = 30
    (s.step_imag(n) if imag else s.step_real(n))
    ref = O.step(prob, psi, n, imag)
    tol = STEP_TOL[precision]
    assert relerr(s.get_state(), ref) < tol
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < tol


def test_graph_replay_and_omega_table():
    """70 steps (two 32-step graph replays and 6 single steps) equal 70 single
    calls bit for bit; a per-step Omega(t) table in real time matches the oracle."""
    import torch
    phys = dict(PHYS_2D, split=1, so_mode=1)
    prob, s = make_pair(2, 40, 33, dx=0.2, **phys)
    psi = _rand(prob, 5)
    s.set_state(psi)
    s.step_imag(70)
    a = s.get_state()
    s.set_state(psi)
    for _ in range(70):
        s.step_imag(1)
    assert np.array_equal(a, s.get_state())
    phys["renorm"] = 0
    prob, s = make_pair(2, 48, 40, dx=0.15, **phys)
    om = 0.5 * np.cos(np.linspace(0, 3, 40)) + 0.1 * I.uniform(4, 40)
    psi = I.gaussian_phase_2d(48, 40, 0.15, 0.15, seed=6)
    s.set_state(psi)
    s.step_real(40, torch.tensor(om, dtype=torch.float64, device="cuda:0"))
    assert relerr(s.get_state(), O.step(prob, psi, 40, False, omega_t=om)) < 1e-10


@pytest.mark.parametrize("precision,tol", [("c128", 1e-12), ("cdf", 5e-11), ("c64", 5e-5)])
def test_so_cn_real_time_norm(precision, tol):
    """Real time with gamma != 0: the Crank-Nicolson SO keeps the norm (every
    substep unitary) over 2000 steps of the 2D workload physics on 128 x 128 to
    round-off (double-float: 2000 steps of ~2^-48 rounding, measured 6.3e-12;
    complex64: the FP32 LU factors of the skew lines and the FP32 rotations leave
    ~5e-9 a step, measured 1.1e-5 over the run); the explicit-Euler SO grows it."""
    n, dx = 128, 0.1
    psi = I.gaussian_phase_2d(n, n, dx, dx, seed=3)
    drift = {}
    for so_mode in (1, 0):
        phys = dict(PHYS_2D, renorm=0, so_mode=so_mode, dt=1e-3)
        _, s = make_pair(2, n, n, dx=dx, precision=precision, **phys)
        s.set_state(psi)
        s.step_real(2000)
        drift[so_mode] = s.energy()["N"] - 1.0
    assert abs(drift[1]) < tol
    assert drift[0] > 1e-6


def test_options_outside_their_range_are_refused():
    import torch
    s = sgpe.Solver(2, 2048, 8, dx=0.05)
    with pytest.raises(sgpe.SgpeError) as e:
        s.set_params(sgpe.Physics(**dict(PHYS_2D, so_mode=1)))
    assert e.value.status == sgpe.EUNSUPPORTED
    s.set_params(sgpe.Physics(**dict(PHYS_2D, split=1)))  # Strang alone works on long lines
    with pytest.raises(sgpe.SgpeError) as e:
        s.set_params(sgpe.Physics(**dict(PHYS_2D, split=2)))
    assert e.value.status == sgpe.EINVAL
    prob, s2 = make_pair(2, 40, 32, dx=0.2, **dict(PHYS_2D, renorm=0, so_mode=1))
    s2.set_state(I.gaussian_phase_2d(40, 32, 0.2, 0.2, seed=1))
    with pytest.raises(sgpe.SgpeError) as e:
        s2.loss_grad(np.full(4, 0.5), np.zeros((32, 40)))
    assert e.value.status == sgpe.EUNSUPPORTED
    ms, cnt = np.zeros(4), np.zeros(4, dtype=np.int32)
    assert s2.lib.sgpe_profile_steps(s2.ctx, 2, 1, ms.ctypes.data, cnt.ctypes.data) == sgpe.EUNSUPPORTED
    with pytest.raises(sgpe.SgpeError) as e:
        sgpe.BatchSolver([dict(dim=1, nx=64, dx=0.1, gamma=0.5, so_type=1, split=1)])
    assert e.value.status == sgpe.EUNSUPPORTED
    torch.cuda.synchronize()


def test_strang_converges_at_second_order_on_the_gpu():
    """The GPU's Strang + Crank-Nicolson SO real-time propagation of a linear
    problem (c0 = c2 = 0) against the dense matrix exponential: error ratio ~4
    per halving of dt (Lie with the Euler SO: ~2)."""
    import scipy.linalg as sla
    nx, ny, dx = 10, 9, 0.5
    base = dict(c0=0.0, c2=0.0, so_type=1, gamma=0.7, omega=0.6, renorm=0)
    psi = I.gaussian_phase_2d(nx, ny, dx, dx, seed=4)
    # the dense Hamiltonian from the oracle pins' construction
    import test_oracle_pins as T
    prob = O.Problem(dim=2, nx=nx, ny=ny, dx=dx, dy=dx, **base)
    exact = (sla.expm(-1j * 0.4 * T.h_linear_dense(prob)) @ psi.ravel()).reshape(psi.shape)
    errs = {}
    for split, so_mode in ((0, 0), (1, 1)):
        e = []
        for dt in (0.02, 0.01):
            _, s = make_pair(2, nx, ny, dx=dx, **dict(base, dt=dt, split=split, so_mode=so_mode))
            s.set_state(psi)
            s.step_real(int(round(0.4 / dt)))
            e.append(relerr(s.get_state(), exact))
        errs[(split, so_mode)] = e
    lie, strang = errs[(0, 0)], errs[(1, 1)]
    assert 1.8 < lie[0] / lie[1] < 2.2
    assert 3.8 < strang[0] / strang[1] < 4.2
