"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix
(arXiv:2009.13507). None of these re-types the oracle's own formulas: each
compares it with an independent construction (dense linear algebra, scipy's
expm, the equations of motion Eqs. (1)-(2), closed-form energies, identities,
or the energies printed in Table 4)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2009_13507_gb300 import inputs as I

SQ2 = np.sqrt(2.0)
# Spin-1 matrices, Eq. (smat)
SX = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=complex) / SQ2
SY = 1j * np.array([[0, -1, 0], [1, 0, -1], [0, 1, 0]], dtype=complex) / SQ2
SZ = np.diag([1.0, 0.0, -1.0]).astype(complex)


def d1(n, h):
    """Central first difference with zero ghosts."""
    return (np.eye(n, k=1) - np.eye(n, k=-1)) / (2 * h)


def d2(n, h):
    return (np.eye(n, k=1) - 2 * np.eye(n) + np.eye(n, k=-1)) / h**2


def grid_ops(prob):
    """Dense single-component operators on the flattened grid (index iy*nx + ix)."""
    nx, ny = prob.nx, (prob.ny if prob.dim == 2 else 1)
    x = I.grid_x(nx, prob.dx)
    if prob.dim == 1:
        Dx, Lap = d1(nx, prob.dx), d2(nx, prob.dx)
        V = np.diag(0.5 * prob.wx**2 * x**2)
        return dict(Dx=Dx, Dy=None, Lap=Lap, V=V, n=nx)
    y = I.grid_x(ny, prob.dy)
    Ix, Iy = np.eye(nx), np.eye(ny)
    Dx = np.kron(Iy, d1(nx, prob.dx))
    Dy = np.kron(d1(ny, prob.dy), Ix)
    Lap = np.kron(Iy, d2(nx, prob.dx)) + np.kron(d2(ny, prob.dy), Ix)
    V = np.diag((0.5 * prob.wx**2 * x[None, :] ** 2 + 0.5 * prob.wy**2 * y[:, None] ** 2).ravel())
    return dict(Dx=Dx, Dy=Dy, Lap=Lap, V=V, n=nx * ny)


def h_so_dense(prob):
    """gamma p_x Sigma (1D) or gamma (eta p_y Sigma_x - p_x Sigma_y) (2D), p = -i D (Sec. 2)."""
    g = grid_ops(prob)
    n = g["n"]
    if prob.so_type == 0:
        return np.zeros((3 * n, 3 * n), dtype=complex)
    px = -1j * g["Dx"]
    if prob.dim == 1:
        S = {1: SX, 2: SY, 3: SZ}[prob.so_type]
        return prob.gamma * np.kron(S, px)
    eta = {1: 1.0, 2: -1.0, 3: 0.0}[prob.so_type]
    py = -1j * g["Dy"]
    return prob.gamma * (eta * np.kron(SX, py) - np.kron(SY, px))


def h_linear_dense(prob, omega=None):
    """Linear part of Eqs. (1)-(2): -1/2 Lap + V + Omega Sigma_x + H_SO."""
    g = grid_ops(prob)
    om = prob.omega if omega is None else omega
    H = np.kron(np.eye(3), -0.5 * g["Lap"] + g["V"]) + om * np.kron(SX, np.eye(g["n"]))
    return H + h_so_dense(prob)


def gp_rhs(prob, psi, omega=None):
    """Right-hand side of Eqs. (1)-(2) at every point (the Hamiltonian applied to psi)."""
    n = psi[0].size
    v = psi.reshape(3, n)
    lin = (h_linear_dense(prob, omega) @ v.ravel()).reshape(3, n)
    pp, p0, pm = v
    rp, r0, rm = abs(pp) ** 2, abs(p0) ** 2, abs(pm) ** 2
    rho = rp + r0 + rm
    c0, c2 = prob.c0, prob.c2
    out = np.empty_like(v)
    out[0] = lin[0] + (c0 * rho + c2 * (rp - rm + r0)) * pp + c2 * p0**2 * np.conj(pm)
    out[2] = lin[2] + (c0 * rho + c2 * (rm - rp + r0)) * pm + c2 * p0**2 * np.conj(pp)
    out[1] = lin[1] + (c0 * rho + c2 * (rp + rm)) * p0 + 2 * c2 * pp * pm * np.conj(p0)
    return out.reshape(psi.shape)


def rand_state(prob, seed, envelope=8.0):
    cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)
    return I.random_state(prob.shape, seed, cell, envelope=envelope)


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


# ---------------------------------------------------------------------------
# Crank-Nicolson sweeps (LU / LUX / LUY): dense solve of the same system
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [5, 17, 33, 64])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dt", [1e-3, 0.2])
def test_cn_line_matches_dense_solve(oracle, n, imag, dt):
    prob = oracle.Problem(dim=1, nx=n, dx=0.1, dt=dt)
    psi = rand_state(prob, 11 + n)
    out = oracle.substep(prob, psi, "cn_x", imag)
    z = dt if imag else 1j * dt
    # i psi_t = -1/2 psi_xx  ->  (I + z/2 H) psi' = (I - z/2 H) psi,  H = -1/2 D2
    H = -0.5 * d2(n, prob.dx)
    M = np.eye(n) + 0.5 * z * H
    ref = np.stack([np.linalg.solve(M, (np.eye(n) - 0.5 * z * H) @ psi[j, 0]) for j in range(3)])[:, None, :]
    assert relerr(out, ref) < 1e-13


@pytest.mark.parametrize("imag", [True, False])
def test_cn_y_matches_dense_solve(oracle, imag):
    prob = oracle.Problem(dim=2, nx=6, ny=9, dx=0.2, dy=0.15, dt=0.05)
    psi = rand_state(prob, 5)
    z = prob.dt if imag else 1j * prob.dt
    H = -0.5 * d2(prob.ny, prob.dy)
    M, N = np.eye(prob.ny) + 0.5 * z * H, np.eye(prob.ny) - 0.5 * z * H
    ref = np.einsum("ab,jbx->jax", np.linalg.solve(M, N), psi)
    assert relerr(oracle.substep(prob, psi, "cn_y", imag), ref) < 1e-13
    H = -0.5 * d2(prob.nx, prob.dx)
    M, N = np.eye(prob.nx) + 0.5 * z * H, np.eye(prob.nx) - 0.5 * z * H
    ref = np.einsum("ab,jyb->jya", np.linalg.solve(M, N), psi)
    assert relerr(oracle.substep(prob, psi, "cn_x", imag), ref) < 1e-13


# ---------------------------------------------------------------------------
# HERM (Appendix A): exponential of the frozen matrix A, derivative = Eqs. (1)-(2)
# ---------------------------------------------------------------------------
def test_herm_is_matrix_exponential(oracle):
    prob = oracle.Problem(dim=1, nx=7, dx=0.3, c2=-1.7, omega=0.9, dt=0.07)
    psi = rand_state(prob, 3, envelope=0.0) * 2.0
    for imag in (True, False):
        z = prob.dt if imag else 1j * prob.dt
        out = oracle.substep(prob, psi, "herm", imag)
        Ot = prob.omega / SQ2
        for i in range(prob.nx):
            pp, p0, pm = psi[:, 0, i]
            a = prob.c2 * np.conj(pm) * p0 + Ot
            b = prob.c2 * np.conj(p0) * pp + Ot
            A = np.array([[0, a, 0], [np.conj(a), 0, b], [0, np.conj(b), 0]])
            ref = sla.expm(-z * A) @ psi[:, 0, i]
            assert np.allclose(out[:, 0, i], ref, rtol=0, atol=1e-13 * np.linalg.norm(ref))


def test_herm_derivative_is_offdiagonal_gp_terms(oracle):
    """d/dt of the HERM update at t = 0 equals -i times the curly-bracket and Rabi terms of Eqs. (1)-(2)."""
    prob = oracle.Problem(dim=1, nx=9, dx=0.3, c2=1.3, omega=0.6, dt=1e-5)
    psi = rand_state(prob, 21, envelope=0.0)
    fwd = oracle.substep(prob, psi, "herm", False)
    # central difference in t: real-time updates with +dt and -dt
    back = oracle.substep(oracle.Problem(**{**prob.__dict__, "dt": -prob.dt}), psi, "herm", False)
    deriv = (fwd - back) / (2 * prob.dt)  # = -i A psi
    pp, p0, pm = psi[:, 0, :]
    Om = prob.omega / SQ2
    terms = np.stack([prob.c2 * p0**2 * np.conj(pm) + Om * p0,
                      2 * prob.c2 * pp * pm * np.conj(p0) + Om * (pp + pm),
                      prob.c2 * p0**2 * np.conj(pp) + Om * p0])[:, None, :]
    assert relerr(deriv, -1j * terms) < 1e-8


def test_herm_unitary_in_real_time_and_identity_at_zero_coupling(oracle):
    prob = oracle.Problem(dim=2, nx=5, ny=4, dx=0.3, dy=0.3, c2=4.0, omega=1.1, dt=0.3)
    psi = rand_state(prob, 8, envelope=0.0)
    out = oracle.substep(prob, psi, "herm", False)
    assert np.allclose(np.sum(abs(out) ** 2, axis=0), np.sum(abs(psi) ** 2, axis=0), rtol=1e-14, atol=0)
    prob0 = oracle.Problem(dim=2, nx=5, ny=4, dx=0.3, dy=0.3, c2=0.0, omega=0.0, dt=0.3)
    assert np.array_equal(oracle.substep(prob0, psi, "herm", True), psi)


# ---------------------------------------------------------------------------
# CALCNU: derivative = square-bracket terms of Eqs. (1)-(2); real time keeps rho_j
# ---------------------------------------------------------------------------
def test_calcnu_derivative_and_density_invariance(oracle):
    prob = oracle.Problem(dim=2, nx=6, ny=5, dx=0.4, dy=0.5, c0=7.0, c2=-2.5, wx=1.3, wy=0.7, dt=1e-5)
    psi = rand_state(prob, 4, envelope=0.0) * 1.5
    fwd = oracle.substep(prob, psi, "calcnu", False)
    back = oracle.substep(oracle.Problem(**{**prob.__dict__, "dt": -prob.dt}), psi, "calcnu", False)
    deriv = (fwd - back) / (2 * prob.dt)
    pp, p0, pm = psi
    rp, r0, rm = abs(pp) ** 2, abs(p0) ** 2, abs(pm) ** 2
    rho = rp + r0 + rm
    x = I.grid_x(prob.nx, prob.dx)[None, :]
    y = I.grid_x(prob.ny, prob.dy)[:, None]
    V = 0.5 * (prob.wx**2 * x**2 + prob.wy**2 * y**2)
    terms = np.stack([(V + prob.c0 * rho + prob.c2 * (rp - rm + r0)) * pp,
                      (V + prob.c0 * rho + prob.c2 * (rp + rm)) * p0,
                      (V + prob.c0 * rho + prob.c2 * (rm - rp + r0)) * pm])
    assert relerr(deriv, -1j * terms) < 1e-8
    big = oracle.Problem(**{**prob.__dict__, "dt": 0.37})
    out = oracle.substep(big, psi, "calcnu", False)
    assert np.allclose(abs(out), abs(psi), rtol=1e-14, atol=0)


# ---------------------------------------------------------------------------
# SO (Appendix A Eqs. (p1)-(p2)): H_SO against the operator built from the spin
# matrices of Eq. (smat); Euler step identity in real time
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,so", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_so_operator_matches_spin_matrices(oracle, dim, so):
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=11, dx=0.2, so_type=so, gamma=0.7, dt=1e-3)
    else:
        prob = oracle.Problem(dim=2, nx=6, ny=5, dx=0.2, dy=0.3, so_type=so, gamma=0.7, dt=1e-3)
    psi = rand_state(prob, 30 + so, envelope=0.0)
    H = h_so_dense(prob)
    assert np.allclose(H, H.conj().T)
    ref = (H @ psi.ravel()).reshape(psi.shape)
    assert relerr(oracle.apply_hso(prob, psi), ref) < 1e-13
    # the substep itself: psi - z H psi
    for imag in (True, False):
        z = prob.dt if imag else 1j * prob.dt
        assert relerr(oracle.substep(prob, psi, "so", imag), psi - z * ref) < 1e-14


def test_so_real_time_norm_growth_law(oracle):
    prob = oracle.Problem(dim=2, nx=8, ny=7, dx=0.2, dy=0.2, so_type=1, gamma=0.9, dt=0.01)
    psi = rand_state(prob, 9)
    out = oracle.substep(prob, psi, "so", False)
    hpsi = oracle.apply_hso(prob, psi)
    n0, n1, nh = (np.sum(abs(a) ** 2) for a in (psi, out, hpsi))
    assert abs(n1 - (n0 + prob.dt**2 * nh)) < 1e-14 * n1


# ---------------------------------------------------------------------------
# Energy functional Eq. (energy): its gradient is the GP Hamiltonian, Eqs. (1)-(2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2])
def test_energy_gradient_is_gp_rhs(oracle, dim):
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=8, dx=0.3, c0=3.0, c2=-1.2, so_type=1, gamma=0.6, omega=0.8)
    else:
        prob = oracle.Problem(dim=2, nx=5, ny=4, dx=0.3, dy=0.4, c0=3.0, c2=1.7, so_type=1, gamma=0.6,
                              omega=0.8, wx=1.2, wy=0.9)
    cell = prob.dx * (prob.dy if dim == 2 else 1.0)
    psi = rand_state(prob, 17, envelope=0.0)
    rhs = gp_rhs(prob, psi)
    eps = 1e-6
    flat = psi.ravel()
    G = np.zeros_like(flat)
    for k in range(flat.size):
        e = []
        for d in (eps, -eps, 1j * eps, -1j * eps):
            q = flat.copy()
            q[k] += d
            e.append(oracle.observables(prob, q.reshape(psi.shape))["E"])
        G[k] = ((e[0] - e[1]) + 1j * (e[2] - e[3])) / (4 * eps)  # = dE/dpsi^*
    assert relerr(G / cell, rhs.ravel()) < 1e-7


def test_energy_of_linear_problem_is_rayleigh_quotient(oracle):
    prob = oracle.Problem(dim=2, nx=7, ny=6, dx=0.3, dy=0.25, so_type=2, gamma=0.4, omega=0.3)
    psi = rand_state(prob, 2)
    H = h_linear_dense(prob)
    cell = prob.dx * prob.dy
    E = np.real(np.vdot(psi.ravel(), H @ psi.ravel())) * cell
    assert abs(oracle.observables(prob, psi)["E"] - E) < 1e-12 * abs(E)


# ---------------------------------------------------------------------------
# RENORM (Eqs. (DJ2), (DJ)): the rescaled state satisfies Eq. (noma)
# ---------------------------------------------------------------------------
def test_renorm_fixes_norm_and_magnetisation(oracle):
    prob = oracle.Problem(dim=1, nx=40, dx=0.2, renorm=2, mag=0.37)
    psi = rand_state(prob, 6) * 1.7
    o = oracle.observables(prob, oracle.substep(prob, psi, "renorm", True))
    assert abs(o["N"] - 1) < 1e-14 and abs(o["mag"] - 0.37) < 1e-14
    prob.renorm = 1
    o = oracle.observables(prob, oracle.substep(prob, psi, "renorm", True))
    assert abs(o["N"] - 1) < 1e-14


# ---------------------------------------------------------------------------
# Whole steps: unitarity in real time, closed-form ground-state energies
# ---------------------------------------------------------------------------
def test_real_time_norm_conserved_without_so(oracle):
    prob = oracle.Problem(dim=2, nx=24, ny=20, dx=0.3, dy=0.3, c0=20.0, c2=-1.0, omega=0.7, dt=2e-3, renorm=0)
    psi = I.gaussian_phase_2d(24, 20, 0.3, 0.3, seed=3)
    out = oracle.step(prob, psi, 300, imag=False)
    assert abs(np.sum(abs(out) ** 2) / np.sum(abs(psi) ** 2) - 1) < 1e-13


def _ground(oracle, prob, nsteps, seed=1):
    if prob.dim == 1:
        psi = I.gaussian_phase_2d(prob.nx, 1, prob.dx, prob.dx, seed)[:, :1, :]
        psi = psi / np.sqrt(np.sum(abs(psi) ** 2) * prob.dx)
    else:
        psi = I.gaussian_phase_2d(prob.nx, prob.ny, prob.dx, prob.dy, seed)
    out = oracle.step(prob, psi, nsteps, imag=True)
    return oracle.observables(prob, out)["E"]


@pytest.mark.parametrize("so,gamma,omega,closed", [
    (0, 0.0, 0.0, 0.5),             # harmonic oscillator
    (1, 0.5, 0.0, 0.5 - 0.125),     # gamma p_x Sigma_x: shift -gamma^2/2
    (2, 0.5, 0.0, 0.5 - 0.125),     # gamma p_x Sigma_y
    (3, 0.5, 0.0, 0.5 - 0.125),     # gamma p_x Sigma_z
    (0, 0.0, 0.2, 0.5 - 0.2),       # Rabi: eigenvalues of Omega Sigma_x are 0, +-Omega
    (1, 0.5, 0.2, 0.5 - 0.125 - 0.2),  # both (they commute)
])
def test_1d_linear_ground_state_energy(oracle, so, gamma, omega, closed):
    prob = oracle.Problem(dim=1, nx=128, dx=0.1, dt=4e-3, so_type=so, gamma=gamma, omega=omega)
    E = _ground(oracle, prob, 15000)
    lam = np.linalg.eigvalsh(h_linear_dense(prob))[0]
    # split-step fixed point vs exact discrete ground state: O(dt^2), 4.7e-6 at dt = 4e-3
    assert abs(E - lam) < 1e-5
    assert abs(E - closed) < 4e-3       # discrete vs continuum (O(dx^2))


@pytest.mark.parametrize("so,closed", [(0, 1.0), (3, 1.0 - 0.5**2 / 2), (1, None)])
def test_2d_linear_ground_state_energy(oracle, so, closed):
    prob = oracle.Problem(dim=2, nx=24, ny=24, dx=0.4, dy=0.4, dt=4e-3, so_type=so, gamma=0.5)
    E = _ground(oracle, prob, 15000)
    lam = np.linalg.eigvalsh(h_linear_dense(prob))[0]
    assert abs(E - lam) < 2e-5
    if closed is not None:
        assert abs(E - closed) < 2e-2


def _table4_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "table4.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            ph, c0, c2, g, m, rn, E = line.split()
            rows.append((ph, float(c0), float(c2), float(g), float(m), int(rn), float(E)))
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("row", _table4_rows(), ids=lambda r: "%s-g%s-m%s" % (r[0], r[3], r[4]))
def test_table4_energies(oracle, row):
    """Converged 1D energies of Table 4 (printed to 4 decimals). Initial states:
    Gaussians; for the SO column the spinor ansatz of the supplement
    (polar: (i sin(gx)/sqrt2, -cos(gx), i sin(gx)/sqrt2); ferro: (1/2, -1/sqrt2, 1/2) e^{igx})."""
    ph, c0, c2, g, m, rn, E_paper = row
    nx, dx, dt = 640, 0.05, 0.00025
    prob = oracle.Problem(dim=1, nx=nx, dx=dx, dt=dt, c0=c0, c2=c2, so_type=1 if g else 0, gamma=g,
                          renorm=rn, mag=m)
    x = I.grid_x(nx, dx)
    w = 4.0 if ph == "polar" else 6.0
    env = np.exp(-x**2 / (2 * w * w))
    if g == 0:
        psi = I.gaussian_jitter_1d(nx, dx, 0, amp=(0.0 if m == 0 else 1e-3), width=w)
        nsteps = 40000
    else:
        if ph == "polar":
            psi = np.stack([1j * np.sin(g * x) / SQ2, -np.cos(g * x), 1j * np.sin(g * x) / SQ2]) * env
        else:
            psi = np.stack([np.full(nx, 0.5), np.full(nx, -1 / SQ2), np.full(nx, 0.5)]) * np.exp(1j * g * x) * env
        psi = psi[:, None, :] / np.sqrt(np.sum(abs(psi) ** 2) * dx)
        nsteps = 24000
    out = oracle.step(prob, psi, nsteps, imag=True)
    o = oracle.observables(prob, out)
    assert abs(o["N"] - 1) < 1e-12
    if rn == 2:
        assert abs(o["mag"] - m) < 1e-12
    # 4 printed decimals; the second-order SO stencil adds ~6e-5 at DX = 0.05
    assert abs(o["E"] - E_paper) < 1e-4


def _table3_1d_converged():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "tables_3_4.txt")):
        if line.strip() and not line.startswith("#"):
            t, dim, ph, c0, c2, g, dx, E = line.split()
            if t == "T3" and dim == "1" and float(dx) == 0.0:
                rows[ph] = (float(c0), float(c2), float(g), float(E))
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("phase", ["ferro", "polar"])
def test_table3_1d_converged_energy(oracle, phase):
    """Table 3's converged 1D SO energies (5 printed decimals) from the oracle on its
    own grids: DX = 0.1 and 0.05 on [-16, 16), DT = DX^2 / 10 (the imaginary-time
    step of Sec. 4), each run to |dE| < 1e-10 E over tau = 2. The R5 stencils leave
    an O(dx^2) error (DT scales with it), so the Richardson value E_0.05 -
    (E_0.1 - E_0.05) / 3 is the continuum one; it must reach the printed value to
    its last decimal, and both grid energies lie above it."""
    c0, c2, g, E_paper = _table3_1d_converged()[phase]
    threads = min(4, os.cpu_count() or 1)
    E = {}
    try:
        oracle.set_threads(threads)
        for dx in (0.1, 0.05):
            nx, dt = int(round(32.0 / dx)), dx * dx * 0.1
            prob = oracle.Problem(dim=1, nx=nx, dx=dx, dt=dt, c0=c0, c2=c2, so_type=1, gamma=g, renorm=1)
            x = I.grid_x(nx, dx)
            w = 4.0 if phase == "polar" else 6.0
            env = np.exp(-x**2 / (2 * w * w))
            if phase == "polar":
                psi = np.stack([1j * np.sin(g * x) / SQ2, -np.cos(g * x), 1j * np.sin(g * x) / SQ2]) * env
            else:
                psi = np.stack([np.full(nx, 0.5), np.full(nx, -1 / SQ2), np.full(nx, 0.5)]) * np.exp(1j * g * x) * env
            psi = psi[:, None, :] / np.sqrt(np.sum(abs(psi) ** 2) * dx)
            chunk, steps, e_old = int(round(2.0 / dt)), 0, None
            while steps * dt < 60.0:
                psi = oracle.step(prob, psi, chunk, imag=True)
                steps += chunk
                e = oracle.observables(prob, psi)["E"]
                if e_old is not None and steps * dt > 10.0 and abs(e - e_old) < 1e-10 * e:
                    break
                e_old = e
            assert abs(e - e_old) < 1e-10 * e  # converged in imaginary time
            E[dx] = e
    finally:
        oracle.set_threads(1)
    limit = E[0.05] - (E[0.1] - E[0.05]) / 3.0
    assert abs(limit - E_paper) < 3e-5
    assert E[0.1] > E[0.05] > limit


# ---------------------------------------------------------------------------
# rms sizes (LENGTH / RADIUS) and the chemical potential: closed forms and the
# GP Hamiltonian built independently from the spin matrices
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2])
def test_rms_of_displaced_gaussians_closed_form(oracle, dim):
    """Component j is a_j exp(-|r - r_j|^2 / (2 s_j^2)): its density is a Gaussian
    of variance s_j^2/2 per axis centred at r_j, so <r^2>_j = |r_j|^2 + d s_j^2/2
    whatever a_j. Different amplitudes, centres and widths per component catch a
    missing 1/N_j, a shifted origin and mixed-up components; the total rms is the
    N_j-weighted mean with N_j = a_j^2 (pi s_j^2)^(d/2). The grid sum of a Gaussian
    well inside the grid equals the integral to rounding."""
    amp = np.array([1.7, 0.6, 1.1])
    cen = np.array([[0.9, -0.4], [-0.3, 0.7], [0.2, 0.5]])
    wid = np.array([0.8, 1.3, 1.0])
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=400, dx=0.05)
        x = I.grid_x(400, 0.05)
        psi = np.stack([amp[j] * np.exp(-(x - cen[j, 0]) ** 2 / (2 * wid[j] ** 2)) for j in range(3)])[:, None, :]
        r2 = cen[:, 0] ** 2 + wid ** 2 / 2
    else:
        prob = oracle.Problem(dim=2, nx=160, ny=150, dx=0.1, dy=0.11)
        x = I.grid_x(160, 0.1)[None, :]
        y = I.grid_x(150, 0.11)[:, None]
        psi = np.stack([amp[j] * np.exp(-((x - cen[j, 0]) ** 2 + (y - cen[j, 1]) ** 2) / (2 * wid[j] ** 2))
                        for j in range(3)])
        r2 = cen[:, 0] ** 2 + cen[:, 1] ** 2 + wid ** 2
    o = oracle.observables(prob, psi.astype(complex))
    for j, k in enumerate(("rms+", "rms0", "rms-")):
        assert abs(o[k] - np.sqrt(r2[j])) < 1e-12 * np.sqrt(r2[j])
    Nj = amp ** 2 * (np.pi * wid ** 2) ** (dim / 2)
    tot = np.sqrt(np.sum(Nj * r2) / np.sum(Nj))
    assert abs(o["rms"] - tot) < 1e-12 * tot
    for j, k in enumerate(("N+", "N0", "N-")):
        assert abs(o[k] - Nj[j]) < 1e-12 * Nj[j]


@pytest.mark.parametrize("dim", [1, 2])
def test_mu_times_norm_is_expectation_of_gp_hamiltonian(oracle, dim):
    """mu N = Re <psi, H_GP psi> for any state, H_GP the right-hand side of
    Eqs. (1)-(2) assembled from dense operators (gp_rhs): the quartic terms
    enter twice, the quadratic ones once. Unnormalised random states with every
    term switched on catch a missing 1/N or E_int in place of 2 E_int."""
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=30, dx=0.25, c0=6.0, c2=-1.4, so_type=1, gamma=0.7, omega=0.45)
    else:
        prob = oracle.Problem(dim=2, nx=9, ny=7, dx=0.35, dy=0.3, c0=6.0, c2=2.1, so_type=2, gamma=0.7, omega=0.45,
                              wx=1.1, wy=0.8)
    cell = prob.dx * (prob.dy if dim == 2 else 1.0)
    psi = rand_state(prob, 41, envelope=0.0) * 1.9
    o = oracle.observables(prob, psi)
    Nt = np.sum(abs(psi) ** 2) * cell
    h = np.real(np.vdot(psi.ravel(), gp_rhs(prob, psi).ravel())) * cell
    assert abs(o["N"] - Nt) < 1e-13 * Nt
    assert abs(o["mu"] * Nt - h) < 1e-12 * abs(h)
    # and E itself differs from mu N by the interaction energy alone
    assert abs((o["mu"] * Nt - o["E"]) - o["E_int"]) < 1e-12 * abs(h)


def test_mu_is_the_eigenvalue_of_the_interacting_ground_state(oracle):
    """At the imaginary-time fixed point H_GP psi = mu psi (mu the Lagrange
    multiplier of the norm): the oracle's mu leaves a residual of the size of
    the splitting error, while the energy per particle E (different from mu
    when c0, c2 != 0) does not."""
    prob = oracle.Problem(dim=1, nx=96, dx=0.15, dt=1e-3, c0=10.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2)
    psi = I.gaussian_jitter_1d(96, 0.15, seed=3, amp=1e-2)
    # tau = 20: converged; the fixed point of the Lie splitting is O(dt) from the
    # eigenstate (residual 7.6e-4 at dt = 1e-3, 3.1e-4 at dt = 5e-4)
    out = oracle.step(prob, psi, 20000, imag=True)
    o = oracle.observables(prob, out)
    Hpsi = gp_rhs(prob, out)
    nrm = np.linalg.norm(out.ravel())
    res_mu = np.linalg.norm((Hpsi - o["mu"] * out).ravel()) / nrm
    res_E = np.linalg.norm((Hpsi - o["E"] * out).ravel()) / nrm
    assert o["mu"] - o["E"] > 0.5          # repulsive: mu = E + E_int/N well above E
    assert res_mu < 2e-3 * abs(o["mu"])
    assert res_E > 100 * res_mu


@pytest.mark.parametrize("dim", [1, 2])
def test_rms_of_linear_ground_state(oracle, dim):
    """Noninteracting harmonic ground state: <x^2> = 1/2 per axis, so rms = 1/sqrt2
    in 1D and 1 in 2D in the continuum (closed form, O(dx^2) grid error), and on
    the grid the dense eigenvector's sum r^2 |v|^2 / sum |v|^2 of the lowest
    eigenvalue of the discrete Hamiltonian (same value in every component)."""
    # rms is first order in the state's O(dt) distance from the eigenvector
    # (7e-4 relative at dt = 4e-3 in 1D): a small dt for a 1e-4 comparison
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=128, dx=0.1, dt=2.5e-4)
        closed, nsteps = np.sqrt(0.5), 40000
    else:
        prob = oracle.Problem(dim=2, nx=24, ny=24, dx=0.4, dy=0.4, dt=2.5e-4)
        closed, nsteps = 1.0, 40000
    if dim == 1:
        psi = I.gaussian_phase_2d(prob.nx, 1, prob.dx, prob.dx, 1)[:, :1, :]
        psi = psi / np.sqrt(np.sum(abs(psi) ** 2) * prob.dx)
    else:
        psi = I.gaussian_phase_2d(prob.nx, prob.ny, prob.dx, prob.dy, 1)
    out = oracle.step(prob, psi, nsteps, imag=True)
    o = oracle.observables(prob, out)
    g = grid_ops(prob)
    w, v = np.linalg.eigh(-0.5 * g["Lap"] + g["V"])
    x = I.grid_x(prob.nx, prob.dx)
    if dim == 1:
        r2 = x ** 2
    else:
        r2 = (x[None, :] ** 2 + I.grid_x(prob.ny, prob.dy)[:, None] ** 2).ravel()
    dense = np.sqrt(np.sum(r2 * abs(v[:, 0]) ** 2) / np.sum(abs(v[:, 0]) ** 2))
    for k in ("rms+", "rms0", "rms-", "rms"):
        assert abs(o[k] - dense) < 1e-4 * dense
        assert abs(o[k] - closed) < (2e-3 if dim == 1 else 3e-2) * closed


@pytest.mark.parametrize("imag", [True, False])
def test_oracle_threads_do_not_change_results(oracle, imag):
    """The oracle's point and line loops on several OpenMP threads give bitwise the
    same state and observables as on one (every grid sum stays sequential)."""
    prob = oracle.Problem(dim=2, nx=70, ny=45, dx=0.15, dy=0.2, c0=30.0, c2=-1.0, so_type=1, gamma=0.6,
                          omega=0.4, dt=1e-3, renorm=1)
    psi = I.gaussian_phase_2d(70, 45, 0.15, 0.2, seed=12)
    try:
        oracle.set_threads(1)
        a = oracle.step(prob, psi, 15, imag)
        oa = oracle.observables(prob, a)
        for n in (2, 5):
            assert oracle.set_threads(n) == n
            b = oracle.step(prob, psi, 15, imag)
            assert np.array_equal(a, b)
            assert oracle.observables(prob, b) == oa
    finally:
        oracle.set_threads(1)


# ---------------------------------------------------------------------------
# SO by Crank-Nicolson (unitary variant) and Strang splitting
# ---------------------------------------------------------------------------
def _cayley(H, z):
    n = H.shape[0]
    return np.linalg.solve(np.eye(n) + 0.5 * z * H, np.eye(n) - 0.5 * z * H)


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,so", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_so_cn_is_dense_cayley_transform(oracle, dim, so, imag):
    """The CN-treated SO substep against (I + z/2 H)^{-1} (I - z/2 H) built from dense
    operators: 1D H = H_SO of the spin matrices (the operator pinned above); 2D
    H_x = -gamma Sigma_y p_x and H_y = gamma eta Sigma_x p_y (whose sum is that
    H_SO), x lines first (y first in the reverse order)."""
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=13, dx=0.2, so_type=so, gamma=0.9, dt=0.05)
    else:
        prob = oracle.Problem(dim=2, nx=7, ny=6, dx=0.2, dy=0.25, so_type=so, gamma=0.9, dt=0.05)
    psi = rand_state(prob, 50 + so, envelope=0.0)
    z = prob.dt if imag else 1j * prob.dt
    Hso = h_so_dense(prob)
    if dim == 1:
        ref = (_cayley(Hso, z) @ psi.ravel()).reshape(psi.shape)
        assert relerr(oracle.substep(prob, psi, "so_cn", imag), ref) < 1e-13
        return
    g = grid_ops(prob)
    eta = {1: 1.0, 2: -1.0, 3: 0.0}[so]
    Hx = -prob.gamma * np.kron(SY, -1j * g["Dx"])
    Hy = prob.gamma * eta * np.kron(SX, -1j * g["Dy"])
    assert np.allclose(Hx + Hy, Hso, atol=1e-14)
    Mx, My = _cayley(Hx, z), _cayley(Hy, z)
    v = psi.ravel()
    assert relerr(oracle.substep(prob, psi, "so_cn", imag), (My @ (Mx @ v)).reshape(psi.shape)) < 1e-13
    assert relerr(oracle.substep(prob, psi, "so_cn_rev", imag), (Mx @ (My @ v)).reshape(psi.shape)) < 1e-13


@pytest.mark.parametrize("dim", [1, 2])
def test_so_cn_real_time_conserves_the_norm(oracle, dim):
    """With the SO substep by Crank-Nicolson every substep of a real-time step is
    unitary (Cayley transforms, phases, HERM), so the norm is conserved to
    round-off with gamma != 0; the explicit-Euler SO grows it instead."""
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=96, dx=0.15, c0=20.0, c2=-1.0, so_type=1, gamma=0.8, omega=0.4,
                              dt=2e-3, renorm=0, so_mode=1)
        psi = I.gaussian_jitter_1d(96, 0.15, seed=8, amp=0.05)
    else:
        prob = oracle.Problem(dim=2, nx=24, ny=20, dx=0.3, dy=0.3, c0=20.0, c2=-1.0, so_type=1, gamma=0.8,
                              omega=0.4, dt=2e-3, renorm=0, so_mode=1)
        psi = I.gaussian_phase_2d(24, 20, 0.3, 0.3, seed=8)
    n0 = np.sum(abs(psi) ** 2)
    for split in (0, 1):
        prob.split = split
        out = oracle.step(prob, psi, 300, imag=False)
        assert abs(np.sum(abs(out) ** 2) / n0 - 1) < 1e-12
    prob.so_mode, prob.split = 0, 0
    out = oracle.step(prob, psi, 300, imag=False)
    assert np.sum(abs(out) ** 2) / n0 - 1 > 1e-6


@pytest.mark.parametrize("dim", [1, 2])
def test_strang_splitting_is_second_order(oracle, dim):
    """Linear problem (c0 = c2 = 0, SO, Rabi, trap) in real time on a small grid:
    the exact propagator exp(-i H T) of the same discrete Hamiltonian (dense
    matrix exponential). Lie splitting with the Euler SO converges at first
    order in dt (error ratio ~2 per halving); Strang splitting with the
    Crank-Nicolson SO (every factor symmetric) at second order (ratio ~4)."""
    # gamma p_x Sigma_y does not commute with the Rabi term Omega Sigma_x; in 1D the
    # second-order CN error of the kinetic term hides Lie's first-order term above
    # dt ~ 2e-3, so the 1D orders are read at smaller steps
    if dim == 1:
        prob = oracle.Problem(dim=1, nx=24, dx=0.3, so_type=2, gamma=0.7, omega=0.6, renorm=0)
        psi = I.gaussian_jitter_1d(24, 0.3, seed=4, amp=0.2)
        dts = (0.00125, 0.000625)
    else:
        prob = oracle.Problem(dim=2, nx=10, ny=9, dx=0.5, dy=0.5, so_type=1, gamma=0.7, omega=0.6, renorm=0)
        psi = I.gaussian_phase_2d(10, 9, 0.5, 0.5, seed=4)
        dts = (0.02, 0.01)
    T = 0.4
    exact = (sla.expm(-1j * T * h_linear_dense(prob)) @ psi.ravel()).reshape(psi.shape)

    def err(split, so_mode, dt):
        p = oracle.Problem(**{**prob.__dict__, "dt": dt, "split": split, "so_mode": so_mode})
        return relerr(oracle.step(p, psi, int(round(T / dt)), imag=False), exact)

    lie = [err(0, 0, dt) for dt in dts]
    strang = [err(1, 1, dt) for dt in dts]
    assert 1.8 < lie[0] / lie[1] < 2.2
    assert 3.8 < strang[0] / strang[1] < 4.2
    assert strang[1] < lie[1] / 10
    if dim == 2:
        # Strang with the explicit-Euler SO stays first order
        euler = [err(1, 0, dt) for dt in dts]
        assert 1.8 < euler[0] / euler[1] < 2.2
