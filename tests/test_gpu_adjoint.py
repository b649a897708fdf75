"""Differentiation form: the GPU hand-written adjoint of the real-time
propagator against the oracle adjoint (exact derivative of the discrete
propagator) and against central finite differences of the GPU loss."""
import numpy as np
import pytest

from gpu_util import make_pair
from oracle import adjoint as A
from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu


def _small(dim, precision="c128"):
    if dim == 2:
        phys = dict(c0=15.0, c2=-1.5, so_type=1, gamma=0.7, omega=0.5, wx=1.1, wy=0.9, dt=1e-2, renorm=0)
        prob, s = make_pair(2, 20, 16, dx=0.35, dy=0.4, precision=precision, **phys)
        psi0 = I.gaussian_phase_2d(20, 16, 0.35, 0.4, seed=2)
        tgt = I.gaussian_target(20, 16, 0.35, 0.4, seed=3)
    else:
        phys = dict(c0=20.0, c2=0.8, so_type=2, gamma=0.6, omega=0.4, wx=1.2, dt=1e-2, renorm=0)
        prob, s = make_pair(1, 48, 1, dx=0.2, precision=precision, **phys)
        psi0 = I.gaussian_jitter_1d(48, 0.2, seed=4, amp=0.05)
        tgt = I.gaussian_target(48, 1, 0.2, 0.2, seed=5)
    om = 0.5 + 0.3 * np.sin(np.arange(24) * 0.7)
    return prob, s, psi0, tgt, om


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("K", [1, 5, 24])
def test_adjoint_matches_oracle_gradient(dim, K):
    prob, s, psi0, tgt, om = _small(dim)
    L_ref, g_om, g_wx, g_wy, psiN = A.loss_and_grad(prob, psi0, om, tgt)
    s.set_state(psi0)
    L, dom, dw = s.loss_grad(om, tgt, checkpoint_every=K)
    assert abs(L - L_ref) < 1e-12 * abs(L_ref)
    d = dom.cpu().numpy()
    assert np.max(np.abs(d - g_om)) < 1e-9 * np.max(np.abs(g_om))
    assert abs(dw[0] - g_wx) < 1e-9 * abs(g_wx)
    if dim == 2:
        assert abs(dw[1] - g_wy) < 1e-9 * abs(g_wy)
    got = s.get_state()  # the bound state ends as psi_N
    assert np.linalg.norm(got - psiN) < 1e-11 * np.linalg.norm(psiN)


def test_adjoint_precision_form_error():
    prob, s, psi0, tgt, om = _small(2, precision="c64")
    L_ref, g_om, g_wx, g_wy, _ = A.loss_and_grad(prob, psi0, om, tgt)
    s.set_state(psi0)
    L, dom, dw = s.loss_grad(om, tgt, checkpoint_every=6)
    assert abs(L - L_ref) < 1e-5 * abs(L_ref)
    assert np.max(np.abs(dom.cpu().numpy() - g_om)) < 2e-3 * np.max(np.abs(g_om))
    assert abs(dw[0] - g_wx) < 2e-3 * abs(g_wx)


def test_autograd_function_backward():
    import torch
    prob, s, psi0, tgt, om = _small(2)
    omt = torch.tensor(om, dtype=torch.float64, device="cuda:0", requires_grad=True)
    w = torch.tensor([1.1, 0.9], dtype=torch.float64, device="cuda:0", requires_grad=True)
    p0 = torch.from_numpy(psi0).to("cuda:0")
    loss = sgpe.rabi_trap_loss(omt, w, s, p0, torch.from_numpy(tgt).to("cuda:0"), 6)
    loss.backward()
    L_ref, g_om, g_wx, g_wy, _ = A.loss_and_grad(prob, psi0, om, tgt)
    assert abs(loss.item() - L_ref) < 1e-12 * L_ref
    assert np.max(np.abs(omt.grad.cpu().numpy() - g_om)) < 1e-9 * np.max(np.abs(g_om))
    assert np.allclose(w.grad.cpu().numpy(), [g_wx, g_wy], rtol=1e-9, atol=0)


def test_differentiation_workload_against_central_differences():
    """The differentiation workload: 256 x 256, dx = 0.05, real time, 500 steps
    at dt = 2e-4, Omega_n = 0.5, checkpoint every 50 steps, Gaussian target;
    gradients against central differences of the (FP64) GPU loss at h = 1e-4."""
    import torch
    phys = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, wx=1.0, wy=1.0, dt=2e-4, renorm=0)
    n, nsteps = 256, 500
    s = sgpe.Solver(2, n, n, dx=0.05)
    s.set_params(sgpe.Physics(**phys))
    psi0 = I.gaussian_phase_2d(n, n, 0.05, 0.05, seed=0)
    tgt = I.gaussian_target(n, n, 0.05, 0.05, seed=7)
    om = np.full(nsteps, 0.5)

    def loss(omv, wx=1.0, wy=1.0):
        s.set_params(sgpe.Physics(**dict(phys, wx=wx, wy=wy)))
        s.set_state(psi0)
        s.step_real(nsteps, torch.tensor(omv, dtype=torch.float64, device="cuda:0"))
        rho = np.sum(np.abs(s.get_state()) ** 2, axis=0)
        return 0.05 * 0.05 * np.sum((rho - tgt) ** 2)

    s.set_state(psi0)
    L, dom, dw = s.loss_grad(om, tgt, checkpoint_every=50)
    d = dom.cpu().numpy()
    assert abs(L - loss(om)) < 1e-12 * L
    h = 1e-4
    # central differences carry a round-off floor of about eps * L / h
    floor = 100 * np.finfo(float).eps * L / h
    for k in (0, 123, 250, 400, 499):
        op, omn = om.copy(), om.copy()
        op[k] += h
        omn[k] -= h
        fd = (loss(op) - loss(omn)) / (2 * h)
        assert abs(fd - d[k]) < 1e-4 * abs(fd) + floor, (k, fd, d[k], floor)
    fdx = (loss(om, wx=1.0 + h) - loss(om, wx=1.0 - h)) / (2 * h)
    fdy = (loss(om, wy=1.0 + h) - loss(om, wy=1.0 - h)) / (2 * h)
    assert abs(fdx - dw[0]) < 1e-4 * abs(fdx) + floor
    assert abs(fdy - dw[1]) < 1e-4 * abs(fdy) + floor


@pytest.mark.parametrize("n,nsteps,tol_om", [(64, 50, 1e-3), (160, 20, 5e-3)])
def test_adjoint_precision_form_moderate_size(n, nsteps, tol_om):
    """The complex64 adjoint (FP32 state, FP64 gradient sums) against the oracle
    adjoint with the workload's physics (c0 = 50, c2 = 1, Rashba gamma = 0.8) and a
    varying Omega(t), checkpoint every 10 steps: its error against the exact FP64
    derivative is the stated error of the form. Measured on GB300: 64 x 64, 50
    real-time steps: loss 1.6e-6, dL/dOmega 7.0e-4 of its largest entry, dL/dw
    1.0e-5; 160 x 160 (the forward y sweeps on row tiles), 20 steps: loss 9.9e-7,
    dL/dOmega 2.2e-3, dL/dw 3.5e-6 (complex128 there: 1.9e-8 for dL/dOmega)."""
    phys = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, wx=1.0, wy=1.0, dt=1e-3, renorm=0)
    dx = 0.2
    prob, s = make_pair(2, n, n, dx=dx, precision="c64", **phys)
    psi0 = I.gaussian_phase_2d(n, n, dx, dx, seed=6)
    tgt = I.gaussian_target(n, n, dx, dx, seed=8)
    om = 0.5 + 0.2 * np.cos(np.arange(nsteps) * 0.3)
    L_ref, g_om, g_wx, g_wy, _ = A.loss_and_grad(prob, psi0, om, tgt)
    s.set_state(psi0)
    L, dom, dw = s.loss_grad(om, tgt, checkpoint_every=10)
    e_L = abs(L - L_ref) / abs(L_ref)
    e_om = np.max(np.abs(dom.cpu().numpy() - g_om)) / np.max(np.abs(g_om))
    e_w = max(abs(dw[0] - g_wx) / abs(g_wx), abs(dw[1] - g_wy) / abs(g_wy))
    print("complex64 adjoint vs oracle: loss %.2e, dL/dOmega %.2e, dL/dw %.2e" % (e_L, e_om, e_w))
    assert e_L < 1e-5
    assert e_om < tol_om
    assert e_w < 1e-3


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("K", [1, 5, 24])
def test_adjoint_step_random_cotangent(dim, K):
    """sgpe_adjoint_forward + sgpe_adjoint_step for a random final-state cotangent
    lam: dL/dpsi_0, dL/dOmega_n and dL/d(wx, wy) of L = Re sum conj(lam) psi_N
    against the oracle's vector-Jacobian product (exact derivative of the
    discrete propagator), complex128 at 1e-9."""
    import torch
    prob, s, psi0, _, om = _small(dim)
    cell = prob.dx * (prob.dy if dim == 2 else 1.0)
    lam = I.random_state(psi0.shape, 91 + K, cell)
    psiN, g0, gom, gwx, gwy = A.vjp(prob, psi0, om, lam)
    s.set_state(psi0)
    tape = s.adjoint_forward(om, checkpoint_every=K)
    assert np.linalg.norm(s.get_state() - psiN) < 1e-11 * np.linalg.norm(psiN)
    g, dom, dw = s.adjoint_step(tape, torch.from_numpy(lam).cuda())
    s.synchronize()
    assert np.linalg.norm(g.cpu().numpy() - g0) < 1e-9 * np.linalg.norm(g0)
    assert np.max(np.abs(dom.cpu().numpy() - gom)) < 1e-9 * np.max(np.abs(gom))
    assert abs(dw[0] - gwx) < 1e-9 * abs(gwx)
    if dim == 2:
        assert abs(dw[1] - gwy) < 1e-9 * abs(gwy)
    # the reverse leaves the bound state (psi_N) alone and can run again on the same tape
    g2, dom2, dw2 = s.adjoint_step(tape, torch.from_numpy(lam).cuda())
    s.synchronize()
    assert torch.equal(g2, g) and torch.equal(dom2, dom) and dw2 == dw
    assert np.linalg.norm(s.get_state() - psiN) < 1e-11 * np.linalg.norm(psiN)


def test_adjoint_step_precision_form():
    """complex64: the same products against the FP64 oracle, stated bound."""
    import torch
    prob, s, psi0, _, om = _small(2, precision="c64")
    lam = I.random_state(psi0.shape, 93, prob.dx * prob.dy)
    psiN, g0, gom, gwx, gwy = A.vjp(prob, psi0, om, lam)
    s.set_state(psi0)
    tape = s.adjoint_forward(om, checkpoint_every=6)
    g, dom, dw = s.adjoint_step(tape, torch.from_numpy(lam).cuda())
    s.synchronize()
    e_g = np.linalg.norm(g.cpu().numpy() - g0) / np.linalg.norm(g0)
    e_om = np.max(np.abs(dom.cpu().numpy() - gom)) / np.max(np.abs(gom))
    print("complex64 adjoint_step vs oracle: dpsi0 %.2e, dOmega %.2e" % (e_g, e_om))
    assert e_g < 1e-4 and e_om < 1e-3
    assert abs(dw[0] - gwx) < 1e-3 * abs(gwx)


def test_adjoint_step_needs_its_forward_pass():
    import torch
    prob, s, psi0, _, om = _small(2)
    s.set_state(psi0)
    tape = s.adjoint_forward(om, checkpoint_every=5)
    lam = torch.zeros((3, prob.ny, prob.nx), dtype=torch.complex128, device="cuda:0")
    fresh = dict(tape, ws=torch.zeros_like(tape["ws"]))
    with pytest.raises(sgpe.SgpeError) as e:
        s.adjoint_step(fresh, lam)
    assert e.value.status == sgpe.ESTATE
    with pytest.raises(sgpe.SgpeError) as e:
        s.adjoint_step(dict(tape, K=6), lam)
    assert e.value.status == sgpe.ESTATE


def test_propagate_real_any_loss():
    """propagate_real (a torch.autograd.Function on sgpe_adjoint_forward /
    sgpe_adjoint_step) under a loss written in torch by the caller, against
    torch.autograd through the oracle's differentiable propagator with the same
    loss: gradients w.r.t. psi_0, Omega(t) and (wx, wy)."""
    import torch
    prob, s, psi0, _, om = _small(2)
    cell = prob.dx * prob.dy

    def user_loss(psi):
        rho = psi.real ** 2 + psi.imag ** 2
        spin = (torch.conj(psi[0]) * psi[2]).real.sum() * cell
        return cell * (rho[1] ** 2).sum() + 0.3 * spin + cell * (rho[0] - rho[2]).sum() ** 2

    p0 = torch.from_numpy(psi0).cuda().requires_grad_(True)
    omt = torch.tensor(om, dtype=torch.float64, device="cuda:0", requires_grad=True)
    w = torch.tensor([prob.wx, prob.wy], dtype=torch.float64, device="cuda:0", requires_grad=True)
    L = user_loss(sgpe.propagate_real(p0, omt, w, s, 5))
    L.backward()
    prop = A.RealTimePropagator(prob)
    q0 = torch.from_numpy(psi0).requires_grad_(True)
    oq = torch.tensor(om, dtype=torch.float64, requires_grad=True)
    wq = torch.tensor([prob.wx, prob.wy], dtype=torch.float64, requires_grad=True)
    psi = q0
    for n in range(len(om)):
        psi = prop.step(psi, oq[n], wq[0], wq[1])
    Lr = user_loss(psi)
    Lr.backward()
    assert abs(L.item() - Lr.item()) < 1e-12 * abs(Lr.item())
    assert torch.linalg.norm(p0.grad.cpu() - q0.grad) < 1e-9 * torch.linalg.norm(q0.grad)
    assert torch.max(torch.abs(omt.grad.cpu() - oq.grad)) < 1e-9 * torch.max(torch.abs(oq.grad))
    assert torch.allclose(w.grad.cpu(), wq.grad, rtol=1e-9, atol=0)
