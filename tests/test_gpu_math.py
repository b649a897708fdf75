"""The FP32 exp(x) - 1 of the complex64 CALCNU substep (a Cody-Waite reduction
and the Taylor series of expm1 on the reduced argument) against an FP64 truth
and against CUDA's expm1f, over the arguments the substep meets (dt mu of either
sign, small and large) and the special values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_13507_gb300 import sgpe

pytestmark = pytest.mark.gpu


def _ulps(y32, truth):
    """|y - truth| in units of the FP32 spacing at the true value."""
    spacing = np.spacing(np.abs(truth).astype(np.float32)).astype(np.float64)
    return np.abs(y32.astype(np.float64) - truth) / spacing


def test_expm1_within_two_ulps():
    rng = np.random.default_rng(1)
    n = 200_000
    x = np.concatenate([
        rng.uniform(-0.4, 0.4, n),                  # k = 0: the series alone
        rng.uniform(-20.0, 20.0, n),                # reduction with |k| <= 29
        rng.uniform(-87.0, 88.0, n // 2),           # up to the largest finite results
        np.linspace(-1e-6, 1e-6, 20_001),           # around zero
        10.0 ** rng.uniform(-40.0, -1.0, n // 4) * rng.choice([-1.0, 1.0], n // 4),  # tiny, incl. subnormal
        np.array([0.0, -0.0, 0.5 * np.log(2.0), -0.5 * np.log(2.0), np.log(2.0), 88.0, -87.0, -87.3, -100.0]),
    ]).astype(np.float32)
    y = sgpe.eval_expm1f(torch.from_numpy(x).cuda()).cpu().numpy()
    truth = np.expm1(x.astype(np.float64))
    assert np.all(np.isfinite(y))
    assert _ulps(y, truth).max() <= 2.0
    # CUDA's expm1f on the same arguments lies in the same band around the truth
    yc = torch.expm1(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.abs(y.astype(np.float64) - yc).max() <= np.max(3.0 * np.spacing(np.abs(truth).astype(np.float32)))
    assert (np.abs(y.astype(np.float64) - yc) / np.spacing(np.abs(truth).astype(np.float32))).max() <= 3.0


def test_expm1_special_values():
    x = np.array([np.nan, np.inf, -np.inf, 89.0, 1000.0, -1000.0], dtype=np.float32)
    y = sgpe.eval_expm1f(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.isnan(y[0])
    assert y[1] == np.inf and y[3] == np.inf and y[4] == np.inf
    assert y[2] == -1.0 and y[5] == -1.0


def test_expm1_rejects_bad_arguments():
    lib = sgpe.load()
    assert lib.sgpe_eval_expm1f(None, None, None, -1) == sgpe.EINVAL
    assert lib.sgpe_eval_expm1f(None, None, None, 4) == sgpe.EINVAL
    assert lib.sgpe_eval_expm1f(None, None, None, 0) == sgpe.OK
