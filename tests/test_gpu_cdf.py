"""The double-float form (SGPE_CDF: every real part a pair of FP32 numbers,
~48 significant bits, all step arithmetic on the FP32 pipe) against the FP64
CPU oracle, through the C ABI; and the one-block 1D step loop that the
double-float and complex64 forms use on 1D grids.

It is held to the same bar as the complex128 form: 1e-10 normwise relative for
whole steps and observables; single substeps to 1e-12 (one substep's
double-float rounding, ~1e-14, well inside). Entry points that do not support
the form must say so (SGPE_EUNSUPPORTED)."""
import ctypes

import numpy as np
import pytest

from gpu_util import make_pair, obs_relerr, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu

SUBSTEPS = ["so", "calcnu", "herm", "cn_x", "cn_y", "renorm"]
PHYS_2D = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
PHYS_1D = dict(c0=10.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2, dt=1e-4, renorm=1)


def _rand(prob, seed, env=6.0):
    cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)
    return I.random_state(prob.shape, seed, cell, envelope=env)


def test_state_round_trip():
    """set_state splits complex128 into pairs; get_state joins them: exact to the
    pair's ~2^-48 relative resolution."""
    prob, s = make_pair(2, 40, 24, dx=0.2, precision="cdf", **PHYS_2D)
    psi = _rand(prob, 3)
    s.set_state(psi)
    back = s.get_state()
    assert back.dtype == np.complex128
    assert relerr(back, psi) < 1e-14


def test_load_state_from_device_complex128():
    import torch
    prob, s = make_pair(2, 48, 40, dx=0.15, precision="cdf", **PHYS_2D)
    psi = I.gaussian_phase_2d(48, 40, 0.15, 0.15, seed=2)
    s.load_state(torch.from_numpy(psi.astype(np.complex128)).cuda())
    s.step_imag(20)
    assert relerr(s.get_state(), O.step(prob, psi, 20, True)) < 1e-10


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which", SUBSTEPS)
@pytest.mark.parametrize("dim,nx,ny", [(2, 37, 29), (1, 101, 1)])
def test_substep_parity_cdf(dim, nx, ny, which, imag):
    if dim == 1 and which == "cn_y":
        pytest.skip("no y sweep in 1D")
    phys = dict(PHYS_2D if dim == 2 else PHYS_1D)
    phys["dt"] = 0.01
    prob, s = make_pair(dim, nx, ny, dx=0.2, precision="cdf", **phys)
    psi = _rand(prob, 100 + nx) * 3.0
    s.set_state(psi)
    s.substep(which, imag)
    assert relerr(s.get_state(), O.substep(prob, psi, which, imag)) < 1e-12


@pytest.mark.parametrize("imag", [True, False])
def test_full_step_parity_2d_cdf(imag):
    prob, s = make_pair(2, 64, 48, dx=0.15, precision="cdf", **PHYS_2D)
    psi = I.gaussian_phase_2d(64, 48, 0.15, 0.15, seed=1)
    s.set_state(psi)
    (s.step_imag(40) if imag else s.step_real(40))
    ref = O.step(prob, psi, 40, imag)
    assert relerr(s.get_state(), ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("nx,ny", [(512, 400), (386, 1024), (1023, 320), (320, 319)])
def test_tiled_grids_cdf(nx, ny, imag):
    """Double-float grids of 320..1024 points an axis on the kernels of long lines
    (319 rows: the register kernels):
    the pointwise kernel, the constant-factor x sweep with one or two warps a line,
    the row-tiled y sweep (one halo chunk), its norm partials and the finalize
    block; both time modes in turn, then the per-kernel profile."""
    prob, s = make_pair(2, nx, ny, dx=0.04, precision="cdf", **PHYS_2D)
    psi = _rand(prob, nx + 5 * ny, env=3.0)
    s.set_state(psi)
    (s.step_imag(3) if imag else s.step_real(3))
    ref = O.step(prob, psi, 3, imag)
    got = s.get_state()
    assert relerr(got, ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10
    s.set_state(psi)
    s.step_imag(2)
    s.step_real(1)
    ref2 = O.step(prob, O.step(prob, psi, 2, True), 1, False)
    assert relerr(s.get_state(), ref2) < 1e-10
    s.set_state(psi)
    s.profile_steps(3, imag=imag)
    assert relerr(s.get_state(), got) < 1e-13


@pytest.mark.parametrize("imag", [True, False])
def test_full_step_parity_1d_cdf(imag):
    prob, s = make_pair(1, 256, 1, dx=0.05, precision="cdf", **PHYS_1D)
    psi = I.gaussian_jitter_1d(256, 0.05, seed=0)
    s.set_state(psi)
    (s.step_imag(300) if imag else s.step_real(300))
    ref = O.step(prob, psi, 300, imag)
    assert relerr(s.get_state(), ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


def test_full_size_2d_config_cdf():
    """The 2D 256 x 256 imaginary-time workload, 40 steps, against the oracle."""
    prob, s = make_pair(2, 256, 256, dx=0.05, precision="cdf", **PHYS_2D)
    psi = I.gaussian_phase_2d(256, 256, 0.05, 0.05, seed=0)
    s.set_state(psi)
    s.step_imag(40)
    ref = O.step(prob, psi, 40, True)
    assert relerr(s.get_state(), ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


def test_cdf_tracks_complex128_over_a_long_run():
    """1000 imaginary-time steps: the double-float and complex128 forms agree
    far below the parity bar (their difference is rounding only)."""
    a = sgpe.Solver(2, 96, 80, dx=0.1, precision="cdf")
    b = sgpe.Solver(2, 96, 80, dx=0.1, precision="c128")
    psi = I.gaussian_phase_2d(96, 80, 0.1, 0.1, seed=5)
    for s in (a, b):
        s.set_params(sgpe.Physics(**PHYS_2D))
        s.set_state(psi)
        s.step_imag(1000)
    assert relerr(a.get_state(), b.get_state()) < 1e-11
    assert abs(a.energy()["E"] - b.energy()["E"]) < 1e-11 * abs(b.energy()["E"])


def test_real_time_norm_cdf():
    """500 real-time steps: without SO every substep is unitary and the norm is
    conserved to rounding; with SO (explicit Euler substep) the norm drifts by
    the method's own amount, which the double-float form reproduces."""
    psi = I.gaussian_phase_2d(128, 128, 0.1, 0.1, seed=7)
    for so in (0, 1):
        phys = dict(PHYS_2D, renorm=0, so_type=so)
        n = {}
        for prec in ("cdf", "c128"):
            s = sgpe.Solver(2, 128, 128, dx=0.1, precision=prec)
            s.set_params(sgpe.Physics(**phys))
            s.set_state(psi)
            n0 = s.energy()["N"]
            s.step_real(500)
            n[prec] = s.energy()["N"]
        if so == 0:
            assert abs(n["cdf"] - n0) < 1e-11
        assert abs(n["cdf"] - n["c128"]) < 1e-11


def test_real_time_omega_table_cdf():
    import torch
    phys = dict(PHYS_2D, renorm=0)
    prob, s = make_pair(2, 48, 40, dx=0.15, precision="cdf", **phys)
    psi = I.gaussian_phase_2d(48, 40, 0.15, 0.15, seed=4)
    om = 0.5 * np.cos(np.linspace(0, 3, 30)) + 0.1 * I.uniform(9, 30)
    s.set_state(psi)
    s.step_real(30, torch.tensor(om, dtype=torch.float64, device="cuda:0"))
    assert relerr(s.get_state(), O.step(prob, psi, 30, False, omega_t=om)) < 1e-10


@pytest.mark.parametrize("dim,nx,ny", [(2, 3, 3), (2, 33, 65), (1, 3, 1), (1, 1000, 1), (2, 2048, 3), (2, 3, 2048)])
def test_edge_sizes_cdf(dim, nx, ny):
    prob, s = make_pair(dim, nx, ny, dx=0.1, precision="cdf", **(PHYS_2D if dim == 2 else PHYS_1D))
    psi = _rand(prob, nx * 7 + ny, env=2.0)
    s.set_state(psi)
    s.step_imag(3)
    s.step_real(2)
    ref = O.step(prob, O.step(prob, psi, 3, True), 2, False)
    assert relerr(s.get_state(), ref) < 1e-10


def test_unsupported_entry_points_say_so():
    lib = sgpe.load()
    b = ctypes.c_void_p()
    inst = sgpe.Instance(2, 16, 16, 0.1, 0.1, sgpe.Physics(**PHYS_2D).c())
    rc = lib.sgpe_batch_create(ctypes.byref(b), 1, ctypes.byref(inst), sgpe.CDF, None)
    assert rc == sgpe.EUNSUPPORTED
    s = sgpe.Solver(2, 32, 32, dx=0.1, precision="cdf")
    s.set_params(sgpe.Physics(**dict(PHYS_2D, renorm=0)))
    size = ctypes.c_size_t()
    assert lib.sgpe_adjoint_workspace_bytes(s.ctx, 4, 2, ctypes.byref(size)) == sgpe.OK
    rc = lib.sgpe_adjoint_loss_grad(s.ctx, 4, None, None, 2, None, None, None, None)
    assert rc == sgpe.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["cdf", "c64", "c128"])
def test_1d_one_block_loop_split_calls(precision):
    """1D grids run the whole loop in one launch (one block in the FP32-pipe
    forms, one cluster in complex128); two calls of 7 steps continue exactly
    where one call of 14 goes (the pending scale and the step counter are
    handed over between calls)."""
    prob, s = make_pair(1, 200, 1, dx=0.06, precision=precision, **PHYS_1D)
    psi = I.gaussian_jitter_1d(200, 0.06, seed=4)
    s.set_state(psi)
    s.step_imag(14)
    a = s.get_state()
    s.set_state(psi)
    s.step_imag(7)
    s.step_imag(7)
    assert np.array_equal(a, s.get_state())


@pytest.mark.parametrize("precision", ["cdf", "c128"])
def test_1d_one_block_loop_omega_table(precision):
    import torch
    phys = dict(PHYS_1D, renorm=0)
    prob, s = make_pair(1, 256, 1, dx=0.05, precision=precision, **phys)
    psi = I.gaussian_jitter_1d(256, 0.05, seed=6)
    om = 0.3 * np.sin(np.linspace(0, 4, 80)) + 0.1 * I.uniform(11, 80)
    s.set_state(psi)
    s.step_real(80, torch.tensor(om, dtype=torch.float64, device="cuda:0"))
    assert relerr(s.get_state(), O.step(prob, psi, 80, False, omega_t=om)) < 1e-10


@pytest.mark.parametrize("imag", [True, False])
def test_1d_config_complex64(imag):
    """The 1D workload in the complex64 form (one-block loop): its error against
    the FP64 oracle after 2000 steps."""
    prob, s = make_pair(1, 256, 1, dx=0.05, precision="c64", **PHYS_1D)
    psi = I.gaussian_jitter_1d(256, 0.05, seed=0)
    s.set_state(psi)
    (s.step_imag(2000) if imag else s.step_real(2000))
    ref = O.step(prob, psi, 2000, imag)
    assert relerr(s.get_state(), ref) < 2e-5
    oe = O.observables(prob, ref)
    assert abs(s.energy()["E"] - oe["E"]) < 1e-5 * abs(oe["E"])


@pytest.mark.parametrize("precision", ["cdf", "c64", "c128"])
def test_2d_split_calls_continue_exactly(precision):
    """Two calls of 7 steps give bit for bit the state of one call of 14 on the
    two-launch 2D step: the end-of-steps kernel publishes the scale that the
    next head kernel would have derived from the same norm partials."""
    prob, s = make_pair(2, 96, 80, dx=0.1, precision=precision, **PHYS_2D)
    psi = I.gaussian_phase_2d(96, 80, 0.1, 0.1, seed=9)
    s.set_state(psi)
    s.step_imag(14)
    a = s.get_state()
    s.set_state(psi)
    s.step_imag(7)
    s.step_imag(7)
    assert np.array_equal(a, s.get_state())
