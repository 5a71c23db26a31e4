"""Parity at the benchmark's full sizes for the two large workloads, in the
FP32 path and the launch shape the benchmark times: the 20 TeV shower at 60
degrees (1e8 steps, 100 spheres, tables 4000 x 256 to 75 degrees) and the
256-shower batch (2e8 steps in one persistent launch).

The oracle cannot redo 2e9 - 7e9 bunches, so it checks what it can compute
one by one: the bunch counts of 1e6 sampled steps (bit-exact), every bunch
of 300 sampled steps (200 with records, 100 drawn at random), whose
crossings must match the records the full launch wrote, and every bunch of
12 runs of 2000 consecutive steps traced with their own global indices
(ground point, time, direction, photons, wavelength); the rest is checked
through properties that hold at any size (the counters add up, the yield
kernel's counts of every step sum to the fused kernel's bunch counter,
nothing overflowed, no duplicate records).  Records are selected on the device after
packing, so the host never holds the full record buffers.
"""
import numpy as np
import pytest

import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, compare_hits, compare_yield, context, oracle_model, trace_blocks

pytestmark = pytest.mark.gpu

SEED = 0x5EED_1234_ABCD
# records per telescope that hold the densest telescope of each workload
CAP = {"inclined_20tev": 8_000_000, "batched_256": 12_000_000}
# the largest errors each run measured (read by whoever runs these tests in
# a script; pytest itself only checks them against the tolerances)
MEASURED = {}


def _rounded(tr: dict) -> dict:
    """A host sample as the FP32 path sees it (directions rounded to float)."""
    out = dict(tr)
    for k in ("ux", "uy", "uz"):
        out[k] = np.asarray(tr[k]).astype(np.float32).astype(np.float64)
    return out


@pytest.mark.parametrize("name", ["inclined_20tev", "batched_256"])
def test_full_size_sampled(name):
    import torch
    P.build()
    sc = workloads.WORKLOADS[name]()
    n = len(sc["tracks"]["x0"])
    M = oracle_model(sc)
    ctx = context(sc)
    dev = P.device_tracks(sc["tracks"], FP32, t_ref=sc["t_ref"])
    rng = np.random.default_rng(23)

    # bunch counts: the oracle on a sample, the two kernels on every step
    nb_g, w_g = ctx.segment_yield(dev, FP32)
    ys = np.sort(rng.choice(n, 1_000_000, replace=False))
    sub = _rounded({k: np.asarray(v)[ys] for k, v in sc["tracks"].items()})
    nb_o, w_o, _, _ = M.segment_yield(sub)
    ys_t = torch.as_tensor(ys, device=nb_g.device)
    dw_max = compare_yield(nb_o, nb_g[ys_t].cpu().numpy(), w_o, w_g[ys_t].cpu().numpy(), FP32)
    total_nb = int(nb_g.to(torch.int64).sum().item())
    del w_g

    out = ctx.alloc_hits(CAP[name], FP32)
    ctx.generate_propagate(dev, SEED, FP32, out)
    code, stats = ctx.sync_status(out)
    assert code == 0
    assert int(stats[0]) == n
    assert int(stats[3]) == total_nb
    assert int(stats[3]) == int(stats[4:9].sum())
    assert int(stats[10]) == 0
    assert int(out.count.sum().item()) == int(stats[9])

    # records packed on the device; the sampled steps' records come up
    pk = ctx.pack_records(out)
    off = pk["offset"]
    n_rec = int(off[-1].item())
    assert n_rec == int(stats[9])
    step = pk["key"] >> 32
    with_rec = torch.unique(step).cpu().numpy()
    hs = np.unique(np.concatenate([
        rng.choice(with_rec, min(200, len(with_rec)), replace=False),
        rng.choice(n, 100, replace=False)]))
    sel = torch.nonzero(torch.isin(step, torch.as_tensor(hs, device=step.device))).flatten()
    tel = torch.searchsorted(off[1:], sel, right=True)
    pos, tim = pk["pos"][sel].cpu().numpy(), pk["tim"][sel].cpu().numpy()
    rec = dict(tel=tel.cpu().numpy(), key=pk["key"][sel].cpu().numpy().view(np.uint64),
               x=pos[:, 0], y=pos[:, 1], cx=pos[:, 2], cy=pos[:, 3],
               t=tim[:, 0], zem=tim[:, 1], w=tim[:, 2], lam=tim[:, 3])
    order = np.lexsort((rec["key"], rec["tel"]))
    rec = {k: v[order] for k, v in rec.items()}
    assert len(np.unique(np.stack([rec["tel"], rec["key"].astype(np.int64)]), axis=1)[0]) \
        == len(rec["tel"])

    got = 0
    step_of = (rec["key"] >> np.uint64(32)).astype(np.int64)
    for i in hs.tolist():
        one = _rounded({k: np.asarray(v)[i:i + 1] for k, v in sc["tracks"].items()})
        o = M.bunches(one, SEED, track_base=int(i))
        m = step_of == i
        r = compare_hits(M, o, {k: v[m] for k, v in rec.items()}, FP32, track_base=int(i))
        got += r["n_common"]
    assert got > 100
    del out, pk, dev
    torch.cuda.synchronize()
    # every bunch of 12 runs of 2000 consecutive steps: positions, times,
    # directions, photons and wavelengths within the FP32 tolerances
    tb = trace_blocks(M, ctx, sc["tracks"], sc["t_ref"], SEED, FP32, rng)
    assert tb["n"] > 100_000
    assert tb["edge_status"] + tb["edge_hit"] < 0.01 * tb["n"]
    MEASURED[name] = dict(tb, max_dw_yield_1e6_steps=dw_max)
    ctx.close()
