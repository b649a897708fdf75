"""GPU (libsgpe, sm_103a) against the FP64 CPU oracle, element by element on the
same seeded inputs, through the C ABI.

Tolerances: complex128 state -- 1e-13 normwise relative for one substep,
1e-10 for whole steps and observables (the FP64 parity bar); complex64 state --
its measured error against the FP64 oracle is asserted below a stated bound."""
import numpy as np
import pytest

from gpu_util import make_pair, obs_relerr, relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SUBSTEPS = ["so", "calcnu", "herm", "cn_x", "cn_y", "renorm"]


def _rand(prob, seed, env=6.0):
    cell = prob.dx * (prob.dy if prob.dim == 2 else 1.0)
    return I.random_state(prob.shape, seed, cell, envelope=env)


PHYS_2D = dict(c0=50.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
PHYS_1D = dict(c0=10.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2, dt=1e-4, renorm=1)


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which", SUBSTEPS)
@pytest.mark.parametrize("dim,nx,ny", [(2, 37, 29), (1, 101, 1)])
def test_substep_parity_fp64(dim, nx, ny, which, imag):
    if dim == 1 and which == "cn_y":
        pytest.skip("no y sweep in 1D")
    phys = dict(PHYS_2D if dim == 2 else PHYS_1D)
    phys["dt"] = 0.01  # large enough that every substep changes the state visibly
    prob, s = make_pair(dim, nx, ny, dx=0.2, **phys)
    psi = _rand(prob, 100 + nx) * 3.0
    s.set_state(psi)
    s.substep(which, imag)
    ref = O.substep(prob, psi, which, imag)
    assert relerr(s.get_state(), ref) < 1e-13


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which", ["cn_x", "cn_y"])
@pytest.mark.parametrize("bt", [0.02, 1.0, 50.0])
def test_cn_sweeps_across_bt(bt, which, imag):
    """CN sweeps for bt = dt/(4 dx^2) from small to large. The lanes' carry scan
    of the complex128 sweeps stops once the composed chunk factors are below
    2^-64: with 8-point chunks bt = 0.02 stops after one level, bt = 1 after
    three, bt = 50 runs all five (|fg| ~ 0.87). All must match the oracle's LU."""
    dx = 0.1
    phys = dict(PHYS_2D, dt=4.0 * dx * dx * bt)
    prob, s = make_pair(2, 200, 150, dx=dx, **phys)
    psi = _rand(prob, 17, env=3.0)
    s.set_state(psi)
    s.substep(which, imag)
    assert relerr(s.get_state(), O.substep(prob, psi, which, imag)) < 1e-13


# complex64: FP32 factors and state; the error grows with the condition of T (about 1 + 4 bt)
LONG_TOL = {("c128", 0.02): 1e-13, ("c128", 50.0): 1e-13, ("c128", 500.0): 1e-12,
            ("cdf", 0.02): 1e-12, ("cdf", 50.0): 1e-12, ("cdf", 500.0): 1e-11,
            ("c64", 0.02): 2e-6, ("c64", 50.0): 1e-4, ("c64", 500.0): 1e-3}


@pytest.mark.parametrize("precision", ["c128", "cdf", "c64"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which,nx,ny", [("cn_x", 1500, 7), ("cn_y", 7, 1500), ("cn_x", 4096, 3),
                                         ("cn_y", 3, 2100), ("cn_x", 1025, 3), ("cn_y", 4, 4095)])
@pytest.mark.parametrize("bt", [0.02, 50.0, 500.0])
def test_cn_long_lines(bt, which, nx, ny, imag, precision):
    """Lines longer than 1024 points: a group of ceil(n/512) warps per line, 16
    points a lane, the warps' chunk maps composed through shared memory (cut
    once negligible at small bt, all of them at bt = 50); ragged last warp and
    ragged last chunk (1025, 1500, 2100, 4095 points). The complex64 and
    double-float forms take the constant-factor solve with the start correction
    (its length: 10 points at bt = 0.02, 312 at bt = 50 in imaginary time, 442
    in real time); at bt = 500 the correction would exceed 512 points and they
    take the tables, as complex128 always does."""
    dx = 0.1
    phys = dict(PHYS_2D, dt=4.0 * dx * dx * bt)
    prob, s = make_pair(2, nx, ny, dx=dx, precision=precision, **phys)
    psi = _rand(prob, 29, env=3.0)
    s.set_state(psi)
    s.substep(which, imag)
    assert relerr(s.get_state(), O.substep(prob, psi, which, imag)) < LONG_TOL[(precision, bt)]


@pytest.mark.parametrize("precision", ["c64", "cdf"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("nx,ny", [(33, 1100), (64, 2048), (5, 1025), (70, 1300)])
@pytest.mark.parametrize("bt", [0.02, 0.3])
def test_cn_y_row_tiles(bt, nx, ny, imag, precision):
    """Columns longer than 1024 points in the constant-factor forms at small bt:
    the y sweep in row tiles of 32 columns x 128 rows with one (bt = 0.02) or two
    (bt = 0.3) halo chunks of 16 rows above and below; ragged last column tile
    (33, 70 and 5 columns), ragged last row tile (1100, 1025, 1300 rows), the
    start correction in the top tile. Then full steps in both time modes, whose
    norm partials come from the tiles (1024 of them per component at 64 x 2048:
    the wide finalize block)."""
    dy = 0.1
    phys = dict(PHYS_2D, dt=4.0 * dy * dy * bt)
    prob, s = make_pair(2, nx, ny, dx=0.1, dy=dy, precision=precision, **phys)
    psi = _rand(prob, 31 + nx, env=3.0)
    s.set_state(psi)
    s.substep("cn_y", imag)
    tol = {"c64": 5e-6, "cdf": 1e-12}[precision]
    assert relerr(s.get_state(), O.substep(prob, psi, "cn_y", imag)) < tol
    s.set_state(psi)
    (s.step_imag(3) if imag else s.step_real(3))
    ref = O.step(prob, psi, 3, imag)
    assert relerr(s.get_state(), ref) < (1e-5 if precision == "c64" else 1e-10)
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < (1e-5 if precision == "c64" else 1e-10)


@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("cdf", 1e-10), ("c64", 2e-5)])
@pytest.mark.parametrize("nx", [1025, 3000])
def test_1d_long_lines_full_steps(nx, precision, tol):
    """1D lines longer than 1024 points: the pointwise kernel, the warp-group x
    sweep with the step's norm partials (FP64 for complex128, double-float pairs
    otherwise) and the finalize block; imaginary then real time, with the
    observables."""
    prob, s = make_pair(1, nx, 1, dx=0.01, precision=precision, **PHYS_1D)
    psi = I.gaussian_jitter_1d(nx, 0.01, seed=nx)
    s.set_state(psi)
    s.step_imag(4)
    s.step_real(3)
    ref = O.step(prob, O.step(prob, psi, 4, True), 3, False)
    assert relerr(s.get_state(), ref) < tol
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < tol


@pytest.mark.parametrize("so", [0, 1, 2, 3])
@pytest.mark.parametrize("dim", [1, 2])
def test_so_variants_parity(dim, so):
    phys = dict(c0=5.0, c2=0.7, so_type=so, gamma=0.9, omega=0.3, dt=0.01, renorm=1)
    prob, s = make_pair(dim, 45, 19 if dim == 2 else 1, dx=0.15, dy=0.2, **phys)
    psi = _rand(prob, 7 + so)
    for imag in (True, False):
        s.set_state(psi)
        s.substep("so", imag)
        assert relerr(s.get_state(), O.substep(prob, psi, "so", imag)) < 1e-13


@pytest.mark.parametrize("imag", [True, False])
def test_full_step_parity_2d(imag):
    prob, s = make_pair(2, 64, 48, dx=0.15, **PHYS_2D)
    psi = I.gaussian_phase_2d(64, 48, 0.15, 0.15, seed=1)
    s.set_state(psi)
    n = 40
    if imag:
        s.step_imag(n)
    else:
        s.step_real(n)
    ref = O.step(prob, psi, n, imag)
    gpu = s.get_state()
    assert relerr(gpu, ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


@pytest.mark.parametrize("imag", [True, False])
def test_full_step_parity_1d_config(imag):
    """The 1D imaginary-time workload: Nx = 256, dx = 0.05, c0 = 10, c2 = -0.5,
    gamma p_x Sigma_x with gamma = 0.5, Omega = 0.2, dt = 1e-4, jittered Gaussian."""
    prob, s = make_pair(1, 256, 1, dx=0.05, **PHYS_1D)
    psi = I.gaussian_jitter_1d(256, 0.05, seed=0)
    s.set_state(psi)
    n = 300
    (s.step_imag(n) if imag else s.step_real(n))
    ref = O.step(prob, psi, n, imag)
    assert relerr(s.get_state(), ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


def test_full_size_2d_config_parity():
    """The 2D imaginary-time workload at its full size (256 x 256, dx = 0.05,
    c0 = 50, c2 = 1, Rashba gamma = 0.8, Omega = 0.5, dt = 2e-4, random-phase
    Gaussian), in the launch configuration the benchmark times (graph-replayed
    32-step blocks plus a remainder), for 40 steps against the oracle."""
    prob, s = make_pair(2, 256, 256, dx=0.05, **PHYS_2D)
    psi = I.gaussian_phase_2d(256, 256, 0.05, 0.05, seed=0)
    s.set_state(psi)
    s.step_imag(40)
    ref = O.step(prob, psi, 40, True)
    assert relerr(s.get_state(), ref) < 1e-10
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-10


def test_graph_replay_equals_single_steps():
    prob, s = make_pair(2, 40, 33, dx=0.2, **PHYS_2D)
    psi = _rand(prob, 77)
    s.set_state(psi)
    s.step_imag(70)  # two 32-step graph replays + 6 single steps
    a = s.get_state()
    s.set_state(psi)
    for _ in range(70):
        s.step_imag(1)
    b = s.get_state()
    assert np.array_equal(a, b)


def test_real_time_omega_table():
    import torch
    phys = dict(PHYS_2D)
    phys["renorm"] = 0
    prob, s = make_pair(2, 48, 40, dx=0.15, **phys)
    psi = I.gaussian_phase_2d(48, 40, 0.15, 0.15, seed=4)
    om = 0.5 * np.cos(np.linspace(0, 3, 50)) + 0.1 * I.uniform(9, 50)
    s.set_state(psi)
    s.step_real(50, torch.tensor(om, dtype=torch.float64, device="cuda:0"))
    ref = O.step(prob, psi, 50, False, omega_t=om)
    assert relerr(s.get_state(), ref) < 1e-10


@pytest.mark.parametrize("nx,ny", [(256, 300), (1026, 5)])
def test_real_time_omega_table_fused_kernels(nx, ny):
    """complex64 real-time steps with a per-step Omega(t) table on the kernels of long
    lines: a tiled grid (the y tiles move the step counter that indexes the table,
    no finalize block) and long rows (the finalize block moves it); 37 steps, a
    graph of 32 and 5 more, after imaginary-time steps that leave a pending scale."""
    import torch
    phys = dict(PHYS_2D)
    prob, s = make_pair(2, nx, ny, dx=0.05, precision="c64", **phys)
    psi = _rand(prob, nx + ny, env=2.0)
    om = 0.5 * np.cos(np.linspace(0, 3, 37)) + 0.1 * I.uniform(11, 37)
    s.set_state(psi)
    s.step_imag(3)
    s.step_real(37, torch.tensor(om, dtype=torch.float64, device="cuda:0"))
    ref = O.step(prob, O.step(prob, psi, 3, True), 37, False, omega_t=om)
    assert relerr(s.get_state(), ref) < 1e-5


@pytest.mark.parametrize("mag", [0.0, 0.3])
def test_fixed_magnetisation_renorm(mag):
    phys = dict(c0=30.0, c2=2.0, so_type=0, gamma=0.0, omega=0.0, dt=1e-3, renorm=2, mag=mag)
    prob, s = make_pair(1, 200, 1, dx=0.08, **phys)
    psi = I.gaussian_jitter_1d(200, 0.08, seed=2, amp=1e-2)
    s.set_state(psi)
    s.step_imag(200)
    ref = O.step(prob, psi, 200, True)
    assert relerr(s.get_state(), ref) < 1e-10
    o = s.energy()
    assert abs(o["N"] - 1) < 1e-12 and abs(o["mag"] - mag) < 1e-12


@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("cdf", 1e-10)])
def test_fixed_magnetisation_renorm_2d(precision, tol):
    """Eq. (DJ) on the two-launch 2D step, where the head kernel derives the
    per-component scale from the previous sweep's norm partials."""
    phys = dict(c0=30.0, c2=2.0, so_type=1, gamma=0.5, omega=0.0, dt=5e-4, renorm=2, mag=0.3)
    prob, s = make_pair(2, 64, 48, dx=0.15, precision=precision, **phys)
    psi = I.gaussian_phase_2d(64, 48, 0.15, 0.15, seed=3)
    s.set_state(psi)
    s.step_imag(60)
    ref = O.step(prob, psi, 60, True)
    assert relerr(s.get_state(), ref) < tol
    o = s.energy()
    assert abs(o["N"] - 1) < 1e-12 and abs(o["mag"] - 0.3) < 1e-12


@pytest.mark.parametrize("precision,nx,ny,tol", [("c64", 256, 300, 1e-5), ("cdf", 320, 384, 1e-10),
                                                  ("c64", 1026, 6, 1e-5)])
def test_fixed_magnetisation_renorm_tiled(precision, nx, ny, tol):
    """Eq. (DJ) on the kernels of long lines: a tiled complex64 grid (the fused head
    kernel forms the per-component scale from the y tiles' partials), a tiled
    double-float grid and complex64 long rows (the finalize block forms it). N and
    m are exact to the storage precision: 1e-12 in double-float, 1e-6 for the
    FP32-rounded complex64 state."""
    phys = dict(c0=30.0, c2=2.0, so_type=1, gamma=0.5, omega=0.0, dt=5e-4, renorm=2, mag=0.3)
    prob, s = make_pair(2, nx, ny, dx=0.05, precision=precision, **phys)
    psi = _rand(prob, 5 + nx, env=2.0)
    s.set_state(psi)
    s.step_imag(20)
    ref = O.step(prob, psi, 20, True)
    assert relerr(s.get_state(), ref) < tol
    o = s.energy()
    nt = 1e-6 if precision == "c64" else 1e-12
    assert abs(o["N"] - 1) < nt and abs(o["mag"] - 0.3) < nt


@pytest.mark.parametrize("dim,nx,ny", [(2, 3, 3), (2, 5, 7), (2, 17, 3), (2, 33, 65), (1, 3, 1), (1, 32, 1),
                                       (1, 33, 1), (1, 224, 1), (1, 256, 1), (1, 257, 1), (1, 1000, 1),
                                       (2, 1500, 4), (2, 2560, 3), (2, 4096, 3), (2, 3, 4096)])
def test_edge_sizes(dim, nx, ny):
    """Ragged and extreme grids. 1D complex128 lines of 32 (one CTA), 224, 256 (the largest) points run
    the one-cluster step loop; 257 and 1000 the three-launch path. 2D rows of 1500, 2560 and 4096 points
    take the long-line x sweep (warp groups) after the pointwise kernel."""
    prob, s = make_pair(dim, nx, ny, dx=0.1, **(PHYS_2D if dim == 2 else PHYS_1D))
    psi = _rand(prob, nx * 7 + ny, env=2.0)
    s.set_state(psi)
    s.step_imag(3)
    s.step_real(2)
    ref = O.step(prob, O.step(prob, psi, 3, True), 2, False)
    assert relerr(s.get_state(), ref) < 1e-10


def test_precision_form_error_is_small():
    """complex64 state and sweeps, FP64 reductions: error against the FP64 oracle."""
    prob, s = make_pair(2, 96, 80, dx=0.1, precision="c64", **PHYS_2D)
    psi = I.gaussian_phase_2d(96, 80, 0.1, 0.1, seed=5)
    s.set_state(psi)
    s.step_imag(200)
    ref = O.step(prob, psi, 200, True)
    assert relerr(s.get_state(), ref) < 2e-5
    oe = O.observables(prob, ref)
    assert abs(s.energy()["E"] - oe["E"]) / abs(oe["E"]) < 1e-5


@pytest.mark.parametrize("nx,ny", [(8192, 3), (2048, 5)])
def test_precision_form_max_line(nx, ny):
    """complex64 long rows: 8192 points (16-warp groups, one column per y tile) and 2048 (4-warp groups)."""
    prob, s = make_pair(2, nx, ny, dx=0.01, precision="c64", **PHYS_2D)
    psi = _rand(prob, 3, env=2.0)
    s.set_state(psi)
    s.step_real(2)
    assert relerr(s.get_state(), O.step(prob, psi, 2, False)) < 1e-5


@pytest.mark.parametrize("precision,tol", [("c64", 5e-6), ("cdf", 1e-12)])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("which", ["cn_x", "cn_y"])
def test_tiled_grid_sweeps(which, imag, precision, tol):
    """Single sweeps on a tiled grid (512 x 400: 64-row tiles, one halo chunk): the
    constant-factor x sweep with one warp a line and the row-tiled y sweep, against
    the oracle's Thomas solves."""
    prob, s = make_pair(2, 512, 400, dx=0.05, precision=precision, **PHYS_2D)
    psi = _rand(prob, 77, env=3.0)
    s.set_state(psi)
    s.substep(which, imag)
    assert relerr(s.get_state(), O.substep(prob, psi, which, imag)) < tol


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("nx,ny", [(256, 256), (160, 200), (384, 600), (512, 512), (1024, 386), (600, 1024), (385, 400),
                                   (128, 512)])
def test_precision_form_tiled_grids(nx, ny, imag):
    """complex64 grids of 129..1024 points an axis step on the kernels of long lines
    when the constant-factor form applies: even rows on the fused pointwise + x-sweep
    kernel (groups of one or two warps a line), which forms the pending scale from
    the row-tiled y sweep's norm partials (no finalize block); odd rows (385) on the
    pointwise kernel and the constant-factor x sweep, then the y tiles and the
    finalize block; 128-point rows take the register kernels.
    Full steps with the observables against the oracle, step calls of both time
    modes in turn (the pending scale handed between the two step paths), and the
    per-kernel profile."""
    prob, s = make_pair(2, nx, ny, dx=0.04, precision="c64", **PHYS_2D)
    psi = _rand(prob, nx * 3 + ny, env=3.0)
    s.set_state(psi)
    (s.step_imag(3) if imag else s.step_real(3))
    ref = O.step(prob, psi, 3, imag)
    got = s.get_state()
    assert relerr(got, ref) < 1e-5
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-5
    s.set_state(psi)
    s.step_imag(2)
    s.step_real(2)
    s.step_imag(1)
    ref2 = O.step(prob, O.step(prob, O.step(prob, psi, 2, True), 2, False), 1, True)
    assert relerr(s.get_state(), ref2) < 1e-5
    s.set_state(psi)
    s.profile_steps(3, imag=imag)
    assert relerr(s.get_state(), got) < 1e-6


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("nx,ny", [(1026, 5), (1500, 6), (2048, 4), (3000, 3), (4096, 3), (1501, 5)])
def test_precision_form_fused_long_rows(nx, ny, imag):
    """complex64 rows of 1025..2048 points, even: the pointwise substeps and the x
    sweep in one kernel (three warp groups of 3 or 4 warps, point pairs on FP32x2,
    slots past the row's end zero); 1501 points (odd), 3000 and 4096 take the
    separate kernels.
    Full steps with the observables against the oracle, then the per-kernel
    profile, which must advance the state exactly as the step does."""
    prob, s = make_pair(2, nx, ny, dx=0.02, precision="c64", **PHYS_2D)
    psi = _rand(prob, nx + 7 * ny, env=2.0)
    s.set_state(psi)
    (s.step_imag(3) if imag else s.step_real(3))
    ref = O.step(prob, psi, 3, imag)
    got = s.get_state()
    assert relerr(got, ref) < 1e-5
    assert obs_relerr(s.energy(), O.observables(prob, ref)) < 1e-5
    s.set_state(psi)
    s.profile_steps(3, imag=imag)
    assert relerr(s.get_state(), got) < 1e-6


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("nx,ny", [(9, 2048), (13, 1500), (8, 4100), (5, 2300)])
def test_precision_form_long_columns(nx, ny, imag):
    """complex64 columns longer than 1024 points: the y sweep's tiles of up to 4
    adjacent columns (32-byte row segments, a group of ceil(n/512) warps per
    column), ragged last tile (9 and 13 columns), ragged last warp (1500, 4100,
    2300: groups of 3, 9 and 5 warps, tiles of 1 to 4 columns)."""
    phys = dict(PHYS_2D, dt=4.0 * 0.01 * 0.01 * 0.5)
    prob, s = make_pair(2, nx, ny, dx=0.1, dy=0.01, precision="c64", **phys)
    psi = _rand(prob, nx + ny, env=2.0)
    s.set_state(psi)
    s.substep("cn_y", imag)
    assert relerr(s.get_state(), O.substep(prob, psi, "cn_y", imag)) < 2e-6
    s.set_state(psi)
    (s.step_imag(3) if imag else s.step_real(3))
    assert relerr(s.get_state(), O.step(prob, psi, 3, imag)) < 1e-5
