"""Error paths of the C ABI on a GPU: bad parameters are rejected before any
launch, a non-finite state is reported by the next synchronising call, and
nothing traps."""
import ctypes

import numpy as np
import pytest

from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu


def _solver(**kw):
    s = sgpe.Solver(2, 32, 24, dx=0.1)
    s.set_params(sgpe.Physics(c0=10.0, c2=1.0, so_type=1, gamma=0.5, omega=0.3, dt=1e-3, **kw))
    return s


def test_bad_params_rejected():
    s = sgpe.Solver(2, 32, 24, dx=0.1)
    for bad in (dict(dt=0.0), dict(dt=-1.0), dict(so_type=5), dict(renorm=3), dict(renorm=2, mag=1.0),
                dict(c0=float("nan"))):
        kw = dict(dt=1e-3)
        kw.update(bad)
        with pytest.raises(sgpe.SgpeError) as e:
            s.set_params(sgpe.Physics(**kw))
        assert e.value.status == sgpe.EINVAL


def test_calls_out_of_order():
    s = sgpe.Solver(2, 32, 24, dx=0.1)
    with pytest.raises(sgpe.SgpeError) as e:
        s.step_imag(1)
    assert e.value.status == sgpe.ESTATE
    s.set_params(sgpe.Physics(dt=1e-3))
    with pytest.raises(sgpe.SgpeError) as e:
        s.step_imag(-1)
    assert e.value.status == sgpe.EINVAL
    assert s.lib.sgpe_substep(s.ctx, 9, 1, 0.0) == sgpe.EINVAL


def test_misaligned_buffers_rejected():
    s = sgpe.Solver(2, 32, 24, dx=0.1)
    rc = s.lib.sgpe_bind(s.ctx, ctypes.c_void_p(s.psi.data_ptr() + 8), ctypes.c_void_p(s.workspace.data_ptr()))
    assert rc == sgpe.EINVAL
    rc = s.lib.sgpe_bind(s.ctx, ctypes.c_void_p(s.psi.data_ptr()), ctypes.c_void_p(s.workspace.data_ptr() + 128))
    assert rc == sgpe.EINVAL


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_state_reported(bad):
    s = _solver(renorm=1)
    psi = np.ones((3, 24, 32), dtype=np.complex128) * 0.1
    psi[1, 5, 7] = bad
    s.set_state(psi)
    s.step_imag(3)
    with pytest.raises(sgpe.SgpeError) as e:
        s.energy()
    assert e.value.status == sgpe.ENONFINITE
    # the context stays usable: a finite state works again
    s.set_state(np.ones((3, 24, 32), dtype=np.complex128) * 0.1)
    s.step_imag(2)
    assert np.isfinite(s.energy()["E"])


def test_zero_steps_is_a_no_op():
    s = _solver()
    psi = np.full((3, 24, 32), 0.05 + 0.02j)
    s.set_state(psi)
    s.step_imag(0)
    s.step_real(0)
    assert np.array_equal(s.get_state(), psi)
