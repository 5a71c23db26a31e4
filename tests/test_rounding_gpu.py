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
