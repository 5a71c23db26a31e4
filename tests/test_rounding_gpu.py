"""The FP32 path rounds its FP64 inputs to float on the integer pipes
(cher_round_to_float); it must give the IEEE round-to-nearest-even result
bit for bit, which the hardware conversion behind torch's cast provides."""
import numpy as np
import pytest

import paper_2006_14927_gb300 as P
from paper_2006_14927_gb300._binding import round_to_float

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(7)
    x = rng.normal(0.0, 1.0, 400_000) * 10.0 ** rng.uniform(-36, 36, 400_000)
    # exact halfway cases between neighbouring floats (ties to even) and
    # their neighbours one double ulp away
    f = rng.normal(0.0, 1.0, 100_000).astype(np.float32) * np.float32(1e3)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2.0
    ties = np.concatenate([mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)])
    # the workloads' magnitudes: heights, lengths, energies, times
    work = np.concatenate([rng.uniform(0, 1e5, 50_000), rng.uniform(0, 30, 50_000),
                           np.exp(rng.uniform(np.log(20), np.log(1e7), 50_000)),
                           rng.uniform(-1e6, 1e6, 50_000)])
    fmax = float(np.finfo(np.float32).max)
    edge = np.array([0.0, -0.0, 1.0, -1.0, fmax, -fmax, np.nextafter(fmax, np.inf), 3.5e38,
                     -1e39, 2.0 ** -126, -(2.0 ** -126), 2.0 ** 127, 1.5, 2.5,
                     float(np.float32(0.1)), 0.1, 1e-30, 123456789.123456789])
    return np.concatenate([x, ties, work, edge])


def test_rounding_matches_ieee_round_to_nearest_even():
    import torch
    P.build()
    x = torch.as_tensor(_inputs(), device="cuda")
    normal = x.abs() >= 2.0 ** -126
    zero = x == 0
    ours = round_to_float(x)
    ref = x.to(torch.float32)
    sel = normal | zero
    assert int(sel.sum()) > 850_000
    a = ours[sel].view(torch.int32).cpu().numpy()
    b = ref[sel].view(torch.int32).cpu().numpy()
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, (x[sel][bad[:5]].cpu().numpy(), a[bad[:5]], b[bad[:5]])


def test_rounding_flushes_below_the_smallest_normal_and_keeps_nan():
    import torch
    x = torch.tensor([1e-40, -1e-40, 2.0 ** -127, float("nan"), float("inf"), -float("inf")],
                     dtype=torch.float64, device="cuda")
    y = round_to_float(x).cpu().numpy()
    assert y[0] == 0.0 and y[1] == 0.0 and y[2] == 0.0
    assert np.signbit(y[1]) and not np.signbit(y[0])
    assert np.isnan(y[3]) and y[4] == np.inf and y[5] == -np.inf


def test_split_is_the_nearest_float_pair():
    """hi is the rounding above; lo is the float nearest to x - hi (computed
    here in FP64, where x - hi is exact), so hi + lo holds x to ~2^-48."""
    import torch
    from paper_2006_14927_gb300._binding import split_to_float
    rng = np.random.default_rng(11)
    # the magnitudes the FP32 path splits (heights above h_obs, times before
    # the front), exact ties, and values whose hi rounds up across a power of two
    x = np.concatenate([rng.uniform(-1e5, 1e5, 200_000), rng.uniform(0, 6e4, 200_000),
                        rng.normal(0, 1, 100_000) * 10.0 ** rng.uniform(-20, 20, 100_000),
                        np.nextafter(np.float64(2.0) ** np.arange(-30, 30), 0.0),
                        np.array([0.0, -0.0, 1.0, 3.0, -1e-30])])
    xt = torch.as_tensor(x, device="cuda")
    hi, lo = split_to_float(xt)
    hi, lo = hi.cpu().numpy(), lo.cpu().numpy()
    assert np.array_equal(hi.view(np.int32), xt.to(torch.float32).cpu().numpy().view(np.int32))
    r = x - hi.astype(np.float64)
    want = r.astype(np.float32)
    normal = (np.abs(want) >= np.float32(2.0 ** -126)) | (want == 0)
    assert normal.sum() > 490_000
    bad = np.nonzero((lo != want) & normal)[0]
    assert bad.size == 0, (x[bad[:5]], lo[bad[:5]], want[bad[:5]])
    big = np.abs(x) > 1.0
    err = np.abs(x - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(err[big] <= np.abs(x[big]) * 2.0 ** -47)
