"""FP64 oracle of the gradient of a final-density loss through the real-time
split-step propagator (arXiv:2009.13507, Sec. 3 and Appendix A).

TEST INFRASTRUCTURE: only the tests import this module.

The real-time step (z = i dt) is restated here with plain PyTorch CPU tensor
operations in complex128 -- SO (Eqs. (p1)-(p2), central differences, zero
ghosts), CALCNU, HERM through the eigenvector matrices of Eq. (11), and the
Crank-Nicolson sweeps as dense solves of the tridiagonal systems -- so that
torch.autograd yields the exact derivative of the discrete propagator
(discretise-then-differentiate). The loss is
    L = dx dy sum_r (rho_N(r) - rho_tgt(r))^2,   rho = sum_j |psi_j|^2,
and the gradient is taken with respect to the per-step Rabi strengths Omega_n
and the trap frequencies (wx, wy), V = (wx^2 x^2 + wy^2 y^2)/2.
The forward is pinned to the C oracle (sgpe_oracle.c) by the tests.
"""
from __future__ import annotations

import math

import numpy as np
import torch

SQ2 = math.sqrt(2.0)


def _grid(n, h):
    return (torch.arange(n, dtype=torch.float64) - n // 2) * h


def _shift_plus(f, axis):
    """f at index i+1 along axis (zero past the end)."""
    n = f.shape[axis]
    z = torch.zeros_like(f.narrow(axis, 0, 1))
    return torch.cat([f.narrow(axis, 1, n - 1), z], dim=axis)


def _shift_minus(f, axis):
    n = f.shape[axis]
    z = torch.zeros_like(f.narrow(axis, 0, 1))
    return torch.cat([z, f.narrow(axis, 0, n - 1)], dim=axis)


def _d1(f, axis, h):
    return (_shift_plus(f, axis) - _shift_minus(f, axis)) / (2.0 * h)


def h_so(prob, psi):
    """H_SO psi of Sec. 2 (same options and readings as the C oracle)."""
    pp, p0, pm = psi[0], psi[1], psi[2]
    g, gt = prob.gamma, prob.gamma / SQ2
    zero = torch.zeros_like(p0)
    if prob.so_type == 0 or g == 0.0:
        return torch.stack([zero, zero, zero])
    dx = lambda f: _d1(f, 1, prob.dx)
    if prob.dim == 1:
        if prob.so_type == 1:
            return torch.stack([-1j * gt * dx(p0), -1j * gt * (dx(pp) + dx(pm)), -1j * gt * dx(p0)])
        if prob.so_type == 2:
            return torch.stack([-gt * dx(p0), gt * (dx(pp) - dx(pm)), gt * dx(p0)])
        return torch.stack([-1j * g * dx(pp), zero, 1j * g * dx(pm)])
    eta = {1: 1.0, 2: -1.0, 3: 0.0}[prob.so_type]
    dy = lambda f: _d1(f, 0, prob.dy)
    fp = -1j * gt * (eta * dy(p0) + 1j * dx(p0))
    fm = -1j * gt * (eta * dy(p0) - 1j * dx(p0))
    g0 = -1j * gt * (-1j * dx(pp) + 1j * dx(pm) + eta * dy(pp) + eta * dy(pm))
    return torch.stack([fp, g0, fm])


def _cn_matrix(n, h, z):
    """(I - bt L)^{-1} (I + bt L), bt = z/(4 h^2), L = tridiag(1, -2, 1)."""
    L = (torch.diag(torch.ones(n - 1, dtype=torch.complex128), 1) - 2 * torch.eye(n, dtype=torch.complex128)
         + torch.diag(torch.ones(n - 1, dtype=torch.complex128), -1))
    bt = z / (4.0 * h * h)
    I = torch.eye(n, dtype=torch.complex128)
    return torch.linalg.solve(I - bt * L, I + bt * L)


class RealTimePropagator:
    """Real-time steps of one grid (prob: oracle.Problem), differentiable in (Omega_n, wx, wy)."""

    def __init__(self, prob):
        self.prob = prob
        z = 1j * prob.dt
        ny = prob.ny if prob.dim == 2 else 1
        self.Mx = _cn_matrix(prob.nx, prob.dx, z)
        self.My = _cn_matrix(ny, prob.dy, z) if prob.dim == 2 else None
        self.x = _grid(prob.nx, prob.dx)[None, :]
        self.y = _grid(ny, prob.dy)[:, None] if prob.dim == 2 else torch.zeros(1, 1, dtype=torch.float64)
        self.cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)

    def step(self, psi, omega, wx, wy):
        p, dt = self.prob, self.prob.dt
        z = 1j * dt
        # SO, Eqs. (p1)-(p2)
        psi = psi - z * h_so(p, psi)
        # CALCNU
        rp, r0, rm = (psi.real ** 2 + psi.imag ** 2)
        rho = rp + r0 + rm
        V = 0.5 * (wx * wx * self.x ** 2 + (wy * wy * self.y ** 2 if p.dim == 2 else 0.0))
        mup = V + p.c0 * rho + p.c2 * (rp - rm + r0)
        mu0 = V + p.c0 * rho + p.c2 * (rp + rm)
        mum = V + p.c0 * rho + p.c2 * (rm - rp + r0)
        psi = torch.stack([torch.exp(-z * mup) * psi[0], torch.exp(-z * mu0) * psi[1], torch.exp(-z * mum) * psi[2]])
        # HERM, Eq. (11): psi <- V diag(exp(-z lambda)) V^{-1} psi
        pp, p0, pm = psi[0], psi[1], psi[2]
        Ot = omega / SQ2
        a = p.c2 * torch.conj(pm) * p0 + Ot
        b = p.c2 * torch.conj(p0) * pp + Ot
        C = torch.sqrt(a.real ** 2 + a.imag ** 2 + b.real ** 2 + b.imag ** 2)
        s = 1.0 / (2.0 * C * C)
        u1 = (torch.conj(a) * pp + C * p0 + b * pm) * s
        u2 = (2.0 * torch.conj(b) * pp - 2.0 * a * pm) * s
        u3 = (torch.conj(a) * pp - C * p0 + b * pm) * s
        e1, e3 = torch.exp(-z * C), torch.exp(z * C)
        psi = torch.stack([a * e1 * u1 + b * u2 + a * e3 * u3,
                           C * e1 * u1 - C * e3 * u3,
                           torch.conj(b) * e1 * u1 - torch.conj(a) * u2 + torch.conj(b) * e3 * u3])
        # Crank-Nicolson along x, then y
        psi = psi @ self.Mx.T
        if p.dim == 2:
            psi = torch.einsum("ab,jbx->jax", self.My, psi)
        return psi

    def loss(self, psi0, omega_t, wx, wy, rho_tgt):
        psi = torch.as_tensor(np.asarray(psi0), dtype=torch.complex128)
        for n in range(omega_t.shape[0]):
            psi = self.step(psi, omega_t[n], wx, wy)
        rho = (psi.real ** 2 + psi.imag ** 2).sum(0)
        return self.cell * ((rho - rho_tgt) ** 2).sum(), psi


def loss_and_grad(prob, psi0, omega_t, rho_tgt):
    """L and dL/dOmega_n (n = 0..len-1), dL/dwx, dL/dwy as float64 numpy values."""
    prop = RealTimePropagator(prob)
    om = torch.tensor(np.asarray(omega_t, dtype=np.float64), requires_grad=True)
    wx = torch.tensor(float(prob.wx), dtype=torch.float64, requires_grad=True)
    wy = torch.tensor(float(prob.wy), dtype=torch.float64, requires_grad=True)
    tgt = torch.as_tensor(np.asarray(rho_tgt, dtype=np.float64).reshape(prob.ny if prob.dim == 2 else 1, prob.nx))
    L, psi = prop.loss(psi0, om, wx, wy, tgt)
    gom, gwx, gwy = torch.autograd.grad(L, (om, wx, wy), allow_unused=True)
    gwy = torch.zeros(()) if gwy is None else gwy
    return float(L.detach()), gom.numpy(), float(gwx), float(gwy), psi.detach().numpy()


def final_psi(prob, psi0, omega_t):
    prop = RealTimePropagator(prob)
    psi = torch.as_tensor(np.asarray(psi0), dtype=torch.complex128)
    with torch.no_grad():
        for n in range(len(omega_t)):
            psi = prop.step(psi, float(omega_t[n]), float(prob.wx), float(prob.wy))
    return psi.numpy()


def vjp(prob, psi0, omega_t, lam):
    """The propagator's vector-Jacobian product for a final-state cotangent lam:
    with L = Re sum conj(lam) psi_N (so that dL/dpsi_N = lam in the convention
    g = dL/dRe + i dL/dIm), returns psi_N, dL/dpsi_0 (same convention),
    dL/dOmega_n, dL/dwx, dL/dwy."""
    prop = RealTimePropagator(prob)
    p0 = torch.tensor(np.asarray(psi0), dtype=torch.complex128, requires_grad=True)
    om = torch.tensor(np.asarray(omega_t, dtype=np.float64), requires_grad=True)
    wx = torch.tensor(float(prob.wx), dtype=torch.float64, requires_grad=True)
    wy = torch.tensor(float(prob.wy), dtype=torch.float64, requires_grad=True)
    lt = torch.as_tensor(np.asarray(lam), dtype=torch.complex128)
    psi = p0
    for n in range(om.shape[0]):
        psi = prop.step(psi, om[n], wx, wy)
    L = (torch.conj(lt) * psi).real.sum()
    g0, gom, gwx, gwy = torch.autograd.grad(L, (p0, om, wx, wy), allow_unused=True)
    gwy = torch.zeros(()) if gwy is None else gwy
    return psi.detach().numpy(), g0.numpy(), gom.numpy(), float(gwx), float(gwy)
