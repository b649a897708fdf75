"""The paper's converged energies (Table 3: convergence with the space step;
Table 4: SO-coupled and 2D spinor energies) reproduced by the GPU solver
(complex128), from the printed parameters, in imaginary time to convergence.

The second-order central first difference of the SO terms (and the 3-point
Laplacian) make the grid energies approach the continuum as O(dx^2): at DX =
0.05 the 1D energies sit 2e-5 above the printed ones, at DX = 0.4 up to 4e-3.
The paper's own values converge faster in DX, so its stencil differs from this
reading; the checks are therefore (i) the O(dx^2) convergence itself, (ii) the
Richardson extrapolation of the two finest grids against the printed converged
value (to its 5 decimals), (iii) the printed 4-decimal Table 4 values at their
own DX. Initial states: the 1D SO spinor ansatz of the oracle pins, and in 2D
the vortex states of Sec. 4 ((-1, 0, +1) polar, (0, +1, +2) ferro for Rashba;
the opposite charges for Dresselhaus). The first steps of each 2D run are also
checked against the oracle."""
import os

import numpy as np
import pytest

from gpu_util import make_pair, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SQ2 = np.sqrt(2.0)
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    rows = []
    for line in open(os.path.join(HERE, "golden", "tables_3_4.txt")):
        if line.strip() and not line.startswith("#"):
            t, dim, ph, c0, c2, g, dx, E = line.split()
            rows.append((t, int(dim), ph, float(c0), float(c2), float(g), float(dx), float(E)))
    return rows


GOLD = _golden()


def _printed(table, dim, phase, gamma, dx):
    for t, d, ph, c0, c2, g, h, E in GOLD:
        if t == table and d == dim and ph == phase and g == gamma and h == dx:
            return E
    raise KeyError((table, dim, phase, gamma, dx))


def _coupling(dim, phase):
    for t, d, ph, c0, c2, g, h, E in GOLD:
        if d == dim and ph == phase:
            return c0, c2
    raise KeyError((dim, phase))


def _initial(dim, phase, n, dx, gamma, so_type=1):
    if dim == 1:
        x = I.grid_x(n, dx)
        w = 4.0 if phase == "polar" else 6.0
        env = np.exp(-x**2 / (2 * w * w))
        if phase == "polar":
            psi = np.stack([1j * np.sin(gamma * x) / SQ2, -np.cos(gamma * x), 1j * np.sin(gamma * x) / SQ2]) * env
        else:
            psi = np.stack([np.full(n, 0.5), np.full(n, -1 / SQ2), np.full(n, 0.5)]) * np.exp(1j * gamma * x) * env
        return psi[:, None, :] / np.sqrt(np.sum(abs(psi) ** 2) * dx)
    sign = 1 if so_type == 1 else -1  # Rashba: upper signs of Sec. 4; Dresselhaus: lower
    if gamma == 0.0:
        return I.vortex_state_2d(n, n, dx, dx, (0, 0, 0), width=3.0, amplitudes=(0.5, 1.0, 0.5))
    charges = (-sign, 0, sign) if phase == "polar" else (0, sign, 2 * sign)
    return I.vortex_state_2d(n, n, dx, dx, charges, width=3.0)


def _ground(dim, phase, gamma, dx, dt, so_type=1, renorm=1, mag=0.0, check_oracle=False):
    """Imaginary time to convergence (|dE| / E < 1e-10 over tau = 2) on the GPU."""
    c0, c2 = _coupling(dim, phase)
    n = int(round(32.0 / dx)) if dim == 1 else int(round(16.0 / dx)) + 1
    phys = dict(c0=c0, c2=c2, so_type=so_type if gamma else 0, gamma=gamma, omega=0.0, dt=dt, renorm=renorm,
                mag=mag)
    prob, s = make_pair(dim, n, n if dim == 2 else 1, dx=dx, **phys)
    psi = _initial(dim, phase, n, dx, gamma, so_type)
    s.set_state(psi)
    if check_oracle:
        s.step_imag(100)
        assert relerr(s.get_state(), O.step(prob, psi, 100, True)) < 1e-10
    chunk = max(200, int(round(2.0 / dt)))
    e_old, steps = None, 0
    while steps * dt < 80.0:
        s.step_imag(chunk)
        steps += chunk
        o = s.energy()
        if e_old is not None and steps * dt > 10.0 and abs(o["E"] - e_old) < 1e-10 * o["E"]:
            break
        e_old = o["E"]
    return o


@pytest.mark.parametrize("phase", ["ferro", "polar"])
@pytest.mark.parametrize("dim", [1, 2])
def test_table3_convergence_and_limit(dim, phase):
    dxs = (0.4, 0.2, 0.1, 0.05)
    E = {dx: _ground(dim, phase, 0.5, dx, dx * dx * 0.1, check_oracle=(dim == 2 and dx == 0.1))["E"] for dx in dxs}
    printed = {dx: _printed("T3", dim, phase, 0.5, dx) for dx in (0.4, 0.2, 0.1)}
    limit = E[0.05] - (E[0.1] - E[0.05]) / 3.0
    print("\n%dD %s: GPU %s  printed %s  Richardson %.6f  printed limit %.5f" % (
        dim, phase, {k: round(v, 6) for k, v in E.items()}, printed, limit, _printed("T3", dim, phase, 0.5, 0)))
    ratio = (E[0.2] - E[0.1]) / (E[0.1] - E[0.05])
    # O(dx^2): ratio 4 asymptotically; the 1D polar state is not yet asymptotic at
    # DX = 0.2 (measured 6.1; its DX = 0.1 / 0.05 step is the Richardson pair)
    assert 3.0 < ratio < 7.0
    assert abs(limit - _printed("T3", dim, phase, 0.5, 0)) < 3e-5
    for dx in (0.2, 0.1):
        # the grid values lie above the converged one by the O(dx^2) stencil error
        assert 0.0 < E[dx] - limit < 2e-2 * dx * dx


@pytest.mark.parametrize("so_type", [1, 2])
@pytest.mark.parametrize("phase", ["ferro", "polar"])
def test_table4_2d_so_energies(phase, so_type):
    """Table 4, 2D SO-coupled column at DX = 0.1, DT = 0.0005: Rashba and
    Dresselhaus give the same energy (printed once); the ferro state's
    magnetisation is printed as m = 0.0468."""
    o = _ground(2, phase, 0.5, 0.1, 0.0005, so_type=so_type)
    printed = _printed("T4", 2, phase, 0.5, 0.1)
    print("\n2D %s so_type %d: E = %.6f (printed %.4f), m = %.5f" % (phase, so_type, o["E"], printed, o["mag"]))
    assert abs(o["E"] - printed) < 2.5e-4
    if phase == "ferro":
        assert abs(abs(o["mag"]) - 0.0468) < 2e-3


@pytest.mark.parametrize("phase", ["ferro", "polar"])
def test_table4_1d_so_energies(phase):
    o = _ground(1, phase, 0.5, 0.05, 0.00025)
    printed = _printed("T4", 1, phase, 0.5, 0.05)
    print("\n1D %s: E = %.6f (printed %.4f)" % (phase, o["E"], printed))
    assert abs(o["E"] - printed) < 1e-4


@pytest.mark.parametrize("phase", ["ferro", "polar"])
def test_table4_2d_spinor_without_so(phase):
    """Table 4, 2D spinor column at m = 0 (no SO, fixed magnetisation, Eq. (DJ))."""
    o = _ground(2, phase, 0.0, 0.1, 0.0005, renorm=2, mag=0.0)
    printed = _printed("T4", 2, phase, 0.0, 0.1)
    print("\n2D %s spinor: E = %.6f (printed %.4f)" % (phase, o["E"], printed))
    assert abs(o["E"] - printed) < 2.5e-4
