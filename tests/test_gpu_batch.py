"""Batched form (sgpe_batch_*): every instance of a batch of uneven grids and
parameters against the FP64 oracle run on that instance alone."""
import numpy as np
import pytest

from gpu_util import relerr
from oracle import oracle as O
from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu

PHYS_KEYS = ("c0", "c2", "so_type", "gamma", "omega", "wx", "wy", "dt", "renorm", "mag")


def _problem(spec):
    ph = spec["physics"]
    return O.Problem(dim=spec["dim"], nx=spec["nx"], ny=spec["ny"], dx=spec["dx"], dy=spec["dy"],
                     **{k: getattr(ph, k) for k in PHYS_KEYS})


def _initial(spec, seed):
    if spec["dim"] == 2:
        return I.gaussian_phase_2d(spec["nx"], spec["ny"], spec["dx"], spec["dy"], seed=seed)
    return I.gaussian_jitter_1d(spec["nx"], spec["dx"], seed=seed, amp=1e-2)


SMALL = [
    dict(dim=1, nx=37, dx=0.2, c0=5.0, c2=-0.5, so_type=1, gamma=0.5, omega=0.2, dt=2e-3),
    dict(dim=1, nx=128, dx=0.1, c0=20.0, c2=1.0, so_type=2, gamma=0.3, omega=0.0, dt=1e-3),
    dict(dim=1, nx=300, dx=0.05, c0=60.0, c2=0.7, so_type=3, gamma=0.9, omega=0.6, dt=1e-3),
    dict(dim=2, nx=40, ny=33, dx=0.3, c0=10.0, c2=-1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-3),
    dict(dim=2, nx=64, ny=64, dx=0.2, c0=30.0, c2=2.0, so_type=2, gamma=0.4, omega=0.1, dt=1e-3),
    dict(dim=2, nx=96, ny=70, dx=0.15, c0=50.0, c2=0.5, so_type=3, gamma=0.6, omega=0.9, dt=1e-3),
]


@pytest.mark.parametrize("tiles", [(0, 1), (2, 2)])
@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_small_uneven_batch_matches_oracle(precision, tiles):
    """Both x parts: the fused row kernel (0) and pointwise kernel + separate x sweep (2 warps per block)."""
    import torch
    bs = sgpe.BatchSolver(SMALL, precision=precision)
    bs.set_tiles(*tiles)
    states = [_initial(s, 10 + i) for i, s in enumerate(bs.specs)]
    bs.load_state(bs.pack(states))
    bs.step_imag(30)
    bs.step_real(10)
    obs = bs.energy()
    got = bs.states()
    tol_psi, tol_obs = (1e-10, 1e-10) if precision == "c128" else (1e-4, 1e-5)
    for i, spec in enumerate(bs.specs):
        prob = _problem(spec)
        ref = O.step(prob, O.step(prob, states[i], 30, True), 10, False)
        assert relerr(got[i], ref) < tol_psi, i
        ro = O.observables_array(prob, ref)
        for k in (0, 1, 2, 3, 5, 6, 7, 8, 9):
            assert abs(obs[i, k] - ro[k]) <= tol_obs * max(abs(ro[k]), 1e-3), (i, k, obs[i, k], ro[k])
    torch.cuda.synchronize()


TILED = [
    dict(dim=2, nx=256, ny=300, dx=0.05, c0=40.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4),
    dict(dim=2, nx=384, ny=256, dx=0.02, c0=20.0, c2=-1.0, so_type=2, gamma=0.5, omega=0.3, dt=2e-4),
    dict(dim=2, nx=257, ny=300, dx=0.05, c0=40.0, c2=1.0, so_type=1, gamma=0.8, omega=0.5, dt=2e-4),
    dict(dim=2, nx=100, ny=80, dx=0.15, c0=30.0, c2=0.5, so_type=3, gamma=0.6, omega=0.9, dt=1e-3),
    dict(dim=1, nx=400, dx=0.05, c0=60.0, c2=0.7, so_type=1, gamma=0.9, omega=0.6, dt=1e-3),
]


@pytest.mark.parametrize("tiles", [(0, 1), (2, 2)])
def test_tiled_instances_in_a_batch(tiles):
    """complex64 instances of 128..1024 points an axis with even rows take the tiled
    step inside the batch (the fused row kernel and the row tiles through work
    lists; one halo chunk at bt = 0.02, two at bt = 0.125), next to instances on the
    register path (odd rows, small grids, 1D) and with either x part of those."""
    bs = sgpe.BatchSolver(TILED, precision="c64")
    bs.set_tiles(*tiles)
    states = [_initial(s, 40 + i) for i, s in enumerate(bs.specs)]
    bs.load_state(bs.pack(states))
    bs.step_imag(20)
    bs.step_real(5)
    obs = bs.energy()
    got = bs.states()
    for i, spec in enumerate(bs.specs):
        prob = _problem(spec)
        ref = O.step(prob, O.step(prob, states[i], 20, True), 5, False)
        assert relerr(got[i], ref) < 1e-4, i
        ro = O.observables_array(prob, ref)
        for k in (0, 1, 2, 3, 5, 6, 7, 8, 9):
            assert abs(obs[i, k] - ro[k]) <= 1e-5 * max(abs(ro[k]), 1e-3), (i, k, obs[i, k], ro[k])


def test_batch_workload_sampled_against_oracle():
    """The batched workload at full size: 32 1D instances (nx ~ U{128..1024}) and
    32 2D instances (n ~ U{128..384}), (gamma, Omega, c0, c2) drawn per instance,
    autotuned line tiles; three instances (the largest 2D, the smallest 2D, the
    largest 1D) compared with the oracle after 12 imaginary-time steps."""
    table = I.batch_table(0)
    inst = []
    for t in table:
        d = dict(t)
        d.update(dx=0.05, dy=0.05, so_type=1, dt=(1e-4 if t["dim"] == 1 else 2e-4), renorm=1)
        inst.append(d)
    bs = sgpe.BatchSolver(inst, precision="c128")
    choice = bs.autotune(2)
    assert choice[0] in (0, 1, 2, 4) and choice[1] in (1, 2, 4)
    states = [_initial(s, 100 + i) for i, s in enumerate(bs.specs)]
    bs.load_state(bs.pack(states))
    bs.step_imag(12)
    obs = bs.energy()
    got = bs.states()
    two = [i for i, s in enumerate(bs.specs) if s["dim"] == 2]
    one = [i for i, s in enumerate(bs.specs) if s["dim"] == 1]
    pick = [max(two, key=lambda i: bs.specs[i]["nx"]), min(two, key=lambda i: bs.specs[i]["nx"]),
            max(one, key=lambda i: bs.specs[i]["nx"])]
    for i in pick:
        prob = _problem(bs.specs[i])
        ref = O.step(prob, states[i], 12, True)
        assert relerr(got[i], ref) < 1e-10, i
        assert abs(obs[i, 5] - O.observables(prob, ref)["E"]) < 1e-10 * abs(obs[i, 5])
    assert np.all(np.abs(obs[:, 3] - 1.0) < 1e-12)  # every instance renormalised


def test_batch_set_tiles_rejects_bad_shapes():
    bs = sgpe.BatchSolver(SMALL[:2], precision="c128")
    for x, y in ((3, 1), (0, 0), (8, 2), (-1, 1)):
        with pytest.raises(sgpe.SgpeError) as e:
            bs.set_tiles(x, y)
        assert e.value.status == sgpe.EINVAL
    bs.set_tiles(4, 4)
    n_sep = bs.launches_per_step()
    bs.set_tiles(0, 4)
    assert bs.launches_per_step() < n_sep  # the fused row kernel replaces the pointwise kernel


def test_batch_rejects_bad_instances():
    with pytest.raises(sgpe.SgpeError) as e:
        sgpe.BatchSolver([dict(dim=1, nx=2000, dx=0.1, dt=1e-3)])
    assert e.value.status == sgpe.EUNSUPPORTED
    with pytest.raises(sgpe.SgpeError) as e:
        sgpe.BatchSolver([dict(dim=2, nx=30, ny=30, dx=0.1, dt=-1.0)])
    assert e.value.status == sgpe.EINVAL
