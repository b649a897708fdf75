"""The seeded input generators (shared by both sides; no method arithmetic)."""
import numpy as np

from paper_2009_13507_gb300 import inputs as I


def test_splitmix64_reference_values():
    # First outputs of SplitMix64 from seed 0 (Steele, Lea, Flood 2014 reference generator)
    z = I.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    u = I.uniform(12345, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(u, I.uniform(12345, 100000))


def test_initial_states_are_normalised():
    a = I.gaussian_jitter_1d(256, 0.05, seed=0)
    assert a.shape == (3, 1, 256) and abs(np.sum(abs(a) ** 2) * 0.05 - 1) < 1e-13
    b = I.gaussian_phase_2d(64, 48, 0.1, 0.2, seed=1)
    assert b.shape == (3, 48, 64) and abs(np.sum(abs(b) ** 2) * 0.02 - 1) < 1e-13


def test_batch_table_ranges():
    t = I.batch_table(0)
    assert len(t) == 64
    for i, r in enumerate(t):
        if i < 32:
            assert r["dim"] == 1 and 128 <= r["nx"] <= 1024
        else:
            assert r["dim"] == 2 and 128 <= r["nx"] <= 384 and r["nx"] == r["ny"]
        assert 0 <= r["gamma"] <= 1 and 0 <= r["omega"] <= 1 and 1 <= r["c0"] <= 100 and -2 <= r["c2"] <= 2


def test_vortex_and_stripe_states():
    """The vortex initial states carry the imprinted angular momentum: the phase of
    component j winds L_j times around the origin; stripe states are real and
    even/odd in x as sin / cos."""
    n, h = 41, 0.4
    psi = I.vortex_state_2d(n, n, h, h, (-1, 0, 2))
    assert abs(np.sum(abs(psi) ** 2) * h * h - 1) < 1e-13
    x = I.grid_x(n, h)
    t = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    ix = np.rint(2.0 * np.cos(t) / h).astype(int) + n // 2
    iy = np.rint(2.0 * np.sin(t) / h).astype(int) + n // 2
    for j, L in enumerate((-1, 0, 2)):
        ph = np.angle(psi[j, iy, ix])
        wind = np.sum(np.angle(np.exp(1j * np.diff(np.append(ph, ph[0]))))) / (2 * np.pi)
        assert round(wind) == L
    s = I.stripe_state_2d(n, n, h, h, 0.5)
    assert np.allclose(s.imag, 0) and np.allclose(s[0], s[2])
    assert np.allclose(s[0][:, n // 2], 0) and abs(np.sum(abs(s) ** 2) * h * h - 1) < 1e-13
