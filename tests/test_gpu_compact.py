"""Standalone stable compaction of caller particle arrays through the C ABI
(o2pic_compact_particles): removed particles (x = NaN) are dropped and the
rest keep their order — checked bit-exactly against a boolean-mask filter."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _arrays(n, dead_frac, seed):
    rng = np.random.default_rng(seed)
    a = {k: rng.standard_normal(n).astype(np.float32) for k in ("x", "vx", "vy", "vz")}
    a["x"] = np.abs(a["x"])
    a["x"][rng.random(n) < dead_frac] = np.nan
    a["id"] = rng.permutation(n).astype(np.uint32)
    return a


@pytest.mark.parametrize("n,dead", [(0, 0.1), (1, 0.0), (1, 1.0), (5, 0.5), (8192, 0.3), (8193, 0.3),
                                    (100_003, 0.05), (3_000_000, 0.02), (200_000, 1.0)])
def test_compact_matches_mask_filter(n, dead):
    import torch
    from paper_0705_0497_gb300 import api
    a = _arrays(n, dead, n + 17)
    d = [torch.from_numpy(a[k] if k != "id" else a[k].view(np.int32)).cuda() for k in ("x", "vx", "vy", "vz", "id")]
    out = api.compact_particles(*d)
    keep = ~np.isnan(a["x"])
    for k, t in zip(("x", "vx", "vy", "vz", "id"), out):
        got = t.cpu().numpy()
        if k == "id":
            got = got.view(np.uint32)
        assert np.array_equal(got, a[k][keep]), k
