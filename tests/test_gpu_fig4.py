"""Fig. 4 of the paper: dynamical stability of the ground states after a small
quench of c0, by real-time propagation for 200 time units with the GPU solver.

(a) 1D SO-coupled ferromagnetic state (c0 = 885, c2 = -4.1, gamma p_x Sigma_x,
gamma = 0.5; DX = 0.05 on 640 points), c0 -> 920 at t = 0, DT = DX^2 * 0.05.
(b) 2D polar Rashba state (c0 = 482, c2 = 15, gamma = 0.5; DX = DY = 0.1 on
161 x 161), c0 -> 500 at t = 0, DT = DX^2 * 0.025.
The ground states come from imaginary time in complex128 (the (-1, 0, +1)
vortex initial state in 2D); the long real-time runs use the FP64-accurate
double-float form. The paper states that the component densities at t = 50,
100, 150, 200 stay close to the imaginary-time ones; checked here as a bound on
the relative L2 change of each rho_j (the quench makes them breathe by a few per
cent), with the norm growing only by the explicit-Euler SO law and the energy
following it. The first 100 real-time steps are
checked against the oracle; the unitary SO variant (Crank-Nicolson) keeps the
norm to round-off over the same 2D run."""
import numpy as np
import pytest

from gpu_util import make_pair, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SQ2 = np.sqrt(2.0)


def _ground_1d():
    n, dx = 640, 0.05
    phys = dict(c0=885.0, c2=-4.1, so_type=1, gamma=0.5, omega=0.0, dt=0.00025, renorm=1)
    _, s = make_pair(1, n, 1, dx=dx, **phys)
    x = I.grid_x(n, dx)
    env = np.exp(-x**2 / 72.0)
    psi = np.stack([np.full(n, 0.5), np.full(n, -1 / SQ2), np.full(n, 0.5)]) * np.exp(0.5j * x) * env
    s.set_state(psi[:, None, :] / np.sqrt(np.sum(abs(psi) ** 2) * dx))
    s.step_imag(120000)
    return s.get_state(), phys, n, 1, dx


def _ground_2d():
    n, dx = 161, 0.1
    phys = dict(c0=482.0, c2=15.0, so_type=1, gamma=0.5, omega=0.0, dt=0.0005, renorm=1)
    _, s = make_pair(2, n, n, dx=dx, **phys)
    s.set_state(I.vortex_state_2d(n, n, dx, dx, (-1, 0, 1), width=3.0))
    s.step_imag(60000)
    return s.get_state(), phys, n, n, dx


def _quench(ground, phys, nx, ny, dx, c0_new, dt, so_mode=0, t_end=200.0, precision="cdf"):
    dim = 2 if ny > 1 else 1
    q = dict(phys, c0=c0_new, dt=dt, renorm=0, so_mode=so_mode)
    prob, s = make_pair(dim, nx, ny, dx=dx, precision=precision, **q)
    s.set_state(ground)
    rho0 = np.abs(ground) ** 2
    E0 = s.energy()["E"]
    per = int(round(50.0 / dt))
    out = []
    for k in range(int(round(t_end / 50.0))):
        s.step_real(per)
        o = s.energy()
        rho = np.abs(s.get_state()) ** 2
        change = [float(np.linalg.norm(rho[j] - rho0[j]) / np.linalg.norm(rho0[j])) for j in range(3)]
        out.append((50.0 * (k + 1), change, o["E"], o["N"]))
    return prob, E0, out


@pytest.mark.parametrize("dim", [1, 2])
def test_fig4_quench_is_stable(dim):
    if dim == 1:
        ground, phys, nx, ny, dx = _ground_1d()
        c0_new, dt = 920.0, dx * dx * 0.05
    else:
        ground, phys, nx, ny, dx = _ground_2d()
        c0_new, dt = 500.0, dx * dx * 0.025
    # the first real-time steps of the quench against the oracle (complex128)
    q = dict(phys, c0=c0_new, dt=dt, renorm=0)
    prob, s = make_pair(dim, nx, ny, dx=dx, **q)
    s.set_state(ground)
    s.step_real(100)
    assert relerr(s.get_state(), O.step(prob, ground, 100, False)) < 1e-10
    prob, E0, hist = _quench(ground, phys, nx, ny, dx, c0_new, dt)
    g50 = hist[0][3] - 1.0
    for t, change, E, N in hist:
        print("\n%dD t = %5.1f  rho change %s  E = %.6f (E0 %.6f)  N - 1 = %.2e" % (
            dim, t, ["%.4f" % c for c in change], E, E0, N - 1.0))
        # the densities breathe after the quench (a few per cent) but stay close to the ground state's
        assert max(change) < 0.1
        # explicit-Euler SO: the norm grows by dt^2 |H_SO psi|^2 a step, a constant rate for a
        # state that stays close to stationary (measured 4.3e-4 (1D), 1.1e-3 (2D) per 50 time units)
        assert 0.0 < g50 < 2e-3
        assert abs((N - 1.0) - g50 * t / 50.0) < 0.05 * g50 * t / 50.0
        # the energy follows the norm (kinetic, trap and SO terms ~ N, interaction ~ N^2)
        assert abs(E - E0) < (2.5 * (N - 1.0) + 1e-4) * E0


def test_fig4_2d_with_unitary_so():
    """The same 2D quench (t = 50) with the SO substep by Crank-Nicolson: the norm
    stays 1 to round-off while the densities stay as close as with the Euler SO."""
    ground, phys, nx, ny, dx = _ground_2d()
    dt = dx * dx * 0.025
    _, E0, hist = _quench(ground, phys, nx, ny, dx, 500.0, dt, so_mode=1, t_end=50.0)
    _, _, hist_e = _quench(ground, phys, nx, ny, dx, 500.0, dt, so_mode=0, t_end=50.0)
    t, change, E, N = hist[-1]
    print("\nCN-SO t = 50: rho change %s, N - 1 = %.2e, E %.6f (E0 %.6f); Euler SO N - 1 = %.2e" % (
        change, N - 1.0, E, E0, hist_e[-1][3] - 1.0))
    assert abs(N - 1.0) < 1e-10
    assert max(change) < 0.1
    assert np.allclose(change, hist_e[-1][1], rtol=0.05, atol=1e-3)
    assert abs(E - E0) < 5e-4 * E0   # with the norm kept, the energy is kept too (splitting error)
