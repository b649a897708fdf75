"""sgpe_observables_noalloc: the observables for callers that cannot allocate
device memory (their scratch is a static array inside the library).

Checked through the C ABI against the regular entry point (sgpe_energy on a
context with a caller-provided workspace), on two calls in a row so that the
second call runs on scratch left over from the first. This file is collected
last on purpose; it also passes when run on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2009_13507_gb300 import inputs as I
from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu


def _case(dim, nx, ny, precision, seed, so_type=1):
    import torch
    phys = sgpe.Physics(c0=50.0, c2=1.0, so_type=so_type, gamma=0.8, omega=0.5, dt=2e-4, renorm=1)
    s = sgpe.Solver(dim, nx, ny, dx=0.1, precision=precision)
    s.set_params(phys)
    if dim == 2:
        psi = I.gaussian_phase_2d(nx, ny, 0.1, 0.1, seed=seed)
    else:
        psi = I.gaussian_jitter_1d(nx, 0.1, seed=seed)
    s.set_state(psi)
    s.step_imag(10)
    ref = s.energy_array()  # applies the pending scale: the bound state is now final
    out = torch.full((sgpe.NOBS,), float("nan"), dtype=torch.float64, device=s.device)
    return s, phys, ref, out


@pytest.mark.parametrize("dim,nx,ny,precision,so_type", [
    (2, 64, 48, "c128", 1), (2, 200, 150, "c64", 1), (2, 90, 70, "cdf", 2), (1, 300, 1, "c128", 1),
    (1, 257, 1, "cdf", 2), (1, 129, 1, "c64", 3)])
def test_noalloc_matches_energy_twice(dim, nx, ny, precision, so_type):
    """Every precision (the double-float state in its pair layout) and the 1D SO
    options gamma p_x Sigma_y and gamma p_x Sigma_z besides Sigma_x and 2D Rashba."""
    s, phys, ref, out = _case(dim, nx, ny, precision, seed=nx, so_type=so_type)
    lib = s.lib
    p = phys.c()
    prec = sgpe.PRECISIONS[precision]
    for call in range(2):
        out.fill_(float("nan"))
        rc = lib.sgpe_observables_noalloc(s.psi.data_ptr(), dim, nx, ny, s.dx, s.dy, prec, ctypes.byref(p),
                                          out.data_ptr(), ctypes.c_void_p(s.stream.cuda_stream))
        assert rc == sgpe.OK, lib.sgpe_last_error(None)
        s.stream.synchronize()
        got = out.cpu().numpy()
        # same kernel, same state: agreement within the FP64 parity tolerance
        den = np.maximum(np.abs(ref), 1e-300)
        assert np.all(np.abs(got - ref) <= 1e-10 * den + 1e-300), (call, got, ref)


def test_noalloc_rejects_grids_beyond_its_scratch():
    s, phys, ref, out = _case(2, 64, 48, "c128", seed=1)
    p = phys.c()
    # 4096 x 4096 needs 128 * 1024 reduction blocks: more than the static scratch holds
    rc = s.lib.sgpe_observables_noalloc(s.psi.data_ptr(), 2, 4096, 4096, 0.1, 0.1, sgpe.C128, ctypes.byref(p),
                                        out.data_ptr(), ctypes.c_void_p(s.stream.cuda_stream))
    assert rc == sgpe.EUNSUPPORTED
    assert b"static scratch" in s.lib.sgpe_last_error(None)
    rc = s.lib.sgpe_observables_noalloc(None, 2, 64, 48, 0.1, 0.1, sgpe.C128, ctypes.byref(p), out.data_ptr(),
                                        None)
    assert rc == sgpe.EINVAL
