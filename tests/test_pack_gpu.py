"""cher_pack_records: every telescope's records packed contiguously,
telescope after telescope, against the per-telescope buffers they come
from (the same records in the same order, counts clipped to the capacity),
in both precisions; a destination too small copies what fits and still
reports the total."""
import numpy as np
import pytest

import paper_2006_14927_gb300 as P
import workloads
from parity import FP32, FP64, context, gpu_hits, host_tracks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_packed_records_equal_the_per_telescope_buffers(prec):
    import torch
    P.build()
    sc = workloads.vertical_1tev(n=40_000)
    ctx = context(sc)
    code, stats, out = gpu_hits(ctx, host_tracks(sc, prec), sc["t_ref"], 5, prec, 3000)
    assert code == 0 or code == 6            # a small cap: some telescopes overflow
    cnt = np.minimum(out.count.cpu().numpy(), out.cap)
    assert cnt.max() == out.cap and cnt.min() < out.cap
    d = ctx.pack_records(out)
    torch.cuda.synchronize()
    off = d["offset"].cpu().numpy()
    assert off[0] == 0 and np.array_equal(np.diff(off), cnt)
    pos, tim, key = out.pos.cpu().numpy(), out.tim.cpu().numpy(), out.key.cpu().numpy()
    pp, tt, kk = d["pos"].cpu().numpy(), d["tim"].cpu().numpy(), d["key"].cpu().numpy()
    for k, c in enumerate(cnt):
        assert np.array_equal(pp[off[k]:off[k] + c], pos[k, :c])
        assert np.array_equal(tt[off[k]:off[k] + c], tim[k, :c])
        assert np.array_equal(kk[off[k]:off[k] + c], key[k, :c])
    # a destination with room for half: the first half, the full total
    half = int(off[-1]) // 2
    dst = {k: v[:half] if k != "offset" else torch.zeros_like(v) for k, v in d.items()}
    dst = {k: v.clone() for k, v in dst.items()}
    for v in (dst["pos"], dst["tim"], dst["key"]):
        v.zero_()
    ctx.pack_records(out, dst)
    torch.cuda.synchronize()
    assert int(dst["offset"][-1]) == int(off[-1])
    assert np.array_equal(dst["key"].cpu().numpy(), kk[:half])
    assert np.array_equal(dst["pos"].cpu().numpy(), pp[:half])
    ctx.close()
