"""Pins of the oracle adjoint (oracle/adjoint.py): its differentiable forward
equals the C oracle's real-time steps, and its gradients equal central finite
differences of the C oracle's loss."""
import numpy as np
import pytest

from paper_2009_13507_gb300 import inputs as I

torch = pytest.importorskip("torch")


def _c_loss(O, prob, psi0, omega_t, rho_tgt):
    psi = O.step(prob, psi0, len(omega_t), imag=False, omega_t=omega_t)
    rho = np.sum(np.abs(psi) ** 2, axis=0)
    cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)
    return cell * np.sum((rho - rho_tgt) ** 2)


def _case(O, dim):
    if dim == 2:
        prob = O.Problem(dim=2, nx=20, ny=16, dx=0.35, dy=0.4, c0=15.0, c2=-1.5, so_type=1, gamma=0.7,
                         omega=0.5, wx=1.1, wy=0.9, dt=1e-2, renorm=0)
        psi0 = I.gaussian_phase_2d(20, 16, 0.35, 0.4, seed=2)
        tgt = I.gaussian_target(20, 16, 0.35, 0.4, seed=3)
    else:
        prob = O.Problem(dim=1, nx=48, dx=0.2, c0=20.0, c2=0.8, so_type=2, gamma=0.6, omega=0.4, wx=1.2,
                         dt=1e-2, renorm=0)
        psi0 = I.gaussian_jitter_1d(48, 0.2, seed=4, amp=0.05)
        tgt = I.gaussian_target(48, 1, 0.2, 0.2, seed=5)
    omega_t = 0.5 + 0.3 * np.sin(np.arange(24) * 0.7)
    return prob, psi0, omega_t, tgt


@pytest.mark.parametrize("dim", [1, 2])
def test_torch_forward_matches_c_oracle(oracle, dim):
    from oracle import adjoint as A
    prob, psi0, om, _ = _case(oracle, dim)
    ref = oracle.step(prob, psi0, len(om), imag=False, omega_t=om)
    got = A.final_psi(prob, psi0, om)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("dim", [1, 2])
def test_gradient_matches_central_differences(oracle, dim):
    from oracle import adjoint as A
    prob, psi0, om, tgt = _case(oracle, dim)
    L, g_om, g_wx, g_wy, _ = A.loss_and_grad(prob, psi0, om, tgt)
    assert abs(L - _c_loss(oracle, prob, psi0, om, tgt)) < 1e-13 * abs(L)
    h = 1e-4
    for n in (0, 5, len(om) - 1):
        op, omn = om.copy(), om.copy()
        op[n] += h
        omn[n] -= h
        fd = (_c_loss(oracle, prob, psi0, op, tgt) - _c_loss(oracle, prob, psi0, omn, tgt)) / (2 * h)
        assert abs(fd - g_om[n]) <= 1e-5 * max(abs(fd), 1e-2 * abs(g_om).max()), (n, fd, g_om[n])
    for name, g in (("wx", g_wx),) + ((("wy", g_wy),) if dim == 2 else ()):
        pp, pm = oracle.Problem(**prob.__dict__), oracle.Problem(**prob.__dict__)
        setattr(pp, name, getattr(prob, name) + h)
        setattr(pm, name, getattr(prob, name) - h)
        fd = (_c_loss(oracle, pp, psi0, om, tgt) - _c_loss(oracle, pm, psi0, om, tgt)) / (2 * h)
        assert abs(fd - g) <= 1e-5 * abs(fd), (name, fd, g)


@pytest.mark.parametrize("dim", [1, 2])
def test_vjp_matches_central_differences(oracle, dim):
    """The vector-Jacobian product for a random cotangent lam (L = Re sum conj(lam)
    psi_N): directional derivatives of the C oracle's L along a random complex
    direction of psi_0 (dL = Re sum conj(g_0) d), along single Omega_n and along wx
    / wy, by central differences."""
    from oracle import adjoint as A
    prob, psi0, om, _ = _case(oracle, dim)
    cell = prob.dx * (prob.dy if dim == 2 else 1.0)
    lam = I.random_state(psi0.shape, 77, cell)
    d = I.random_state(psi0.shape, 78, cell)

    def c_L(p, psi, omv):
        out = oracle.step(p, psi, len(omv), imag=False, omega_t=omv)
        return float(np.real(np.sum(np.conj(lam) * out)))

    psiN, g0, gom, gwx, gwy = A.vjp(prob, psi0, om, lam)
    assert np.linalg.norm(psiN - oracle.step(prob, psi0, len(om), imag=False, omega_t=om)) < 1e-13 * np.linalg.norm(psiN)
    h = 1e-5
    fd = (c_L(prob, psi0 + h * d, om) - c_L(prob, psi0 - h * d, om)) / (2 * h)
    an = float(np.real(np.sum(np.conj(g0) * d)))
    assert abs(fd - an) < 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g0) * np.linalg.norm(d)), (fd, an)
    for n in (0, len(om) // 2, len(om) - 1):
        op, omn = om.copy(), om.copy()
        op[n] += h
        omn[n] -= h
        fd = (c_L(prob, psi0, op) - c_L(prob, psi0, omn)) / (2 * h)
        assert abs(fd - gom[n]) <= 1e-6 * max(abs(fd), 1e-2 * abs(gom).max()), (n, fd, gom[n])
    for name, g in (("wx", gwx),) + ((("wy", gwy),) if dim == 2 else ()):
        pp, pm = oracle.Problem(**prob.__dict__), oracle.Problem(**prob.__dict__)
        setattr(pp, name, getattr(prob, name) + h)
        setattr(pm, name, getattr(prob, name) - h)
        fd = (c_L(pp, psi0, om) - c_L(pm, psi0, om)) / (2 * h)
        assert abs(fd - g) <= 1e-6 * max(abs(fd), 1e-3), (name, fd, g)
