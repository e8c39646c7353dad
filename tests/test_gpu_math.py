"""The record kernel's FP64 tangent of tracker angles, against 40-digit arithmetic.

Tracker lines are followed to the hull with slope tan(theta) (Sec. I: straight
lines from the trackers to the object).  For |theta| <= 0.25 rad the library
sums the Maclaurin series of tan to 11 terms and states a relative error of at
most 2.3e-16 there (about one unit in the last place); beyond, it calls the
CUDA library tan.  Both are checked
through the C ABI against mpmath at 40 significant digits.
"""
import mpmath
import numpy as np
import pytest
import torch

import paper_1802_01070_b300 as pct

pytestmark = pytest.mark.gpu


def _exact_tan(t):
    with mpmath.workdps(40):
        return np.array([float(mpmath.tan(mpmath.mpf(float(v)))) for v in t])


def _device_tan(t, dev):
    td = torch.from_numpy(t).to(dev)
    out = torch.empty_like(td)
    pct.pct_tan_angle(td, out)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def test_series_tangent_within_its_stated_bound(cuda_device):
    rng = np.random.default_rng(11)
    t = np.concatenate([rng.uniform(-0.25, 0.25, 20000), rng.normal(0, 0.005, 5000),
                        [0.25, -0.25, np.nextafter(0.25, 0), 1e-3, -1e-3, 1e-8, 5e-324, 0.0, -0.0]])
    got = _device_tan(t, cuda_device)
    want = _exact_tan(t)
    nz = want != 0
    rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    assert rel.max() <= 2.3e-16, rel.max()
    assert np.all(got[~nz] == 0.0)
    # odd function, and exact at zero
    assert np.array_equal(_device_tan(-t, cuda_device), -got)


def test_library_tangent_beyond_the_series_range(cuda_device):
    rng = np.random.default_rng(12)
    t = np.concatenate([rng.uniform(0.25, 1.4, 2000), -rng.uniform(0.25, 1.4, 2000)])
    t = t[np.abs(t) > 0.25]
    got = _device_tan(t, cuda_device)
    want = _exact_tan(t)
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() <= 4.5e-16, rel.max()
