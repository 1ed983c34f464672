"""The tuner times configurations, proves they give identical results, and
caches the best one."""
import json

import pytest

from paper_2308_07173_gb300 import autotune
from paper_2308_07173_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_tune_small(gpu_lib, tmp_path):
    tr = W.oval_1500()
    m = torch.from_numpy(tr.sample_map(200_000, seed=41)).cuda()
    g = W.rng_for(42)
    q = torch.from_numpy(tr.raycast(*tr.random_pose(g), g)[::8].copy()).cuda()
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(m, q, 20, 1e-3, occupancies=(8, 16), rho_scales=(0.9, 1.1), warps=(2, 4), reps=3,
                        cache=cache)
    assert len(res["grid"]) == 8
    best = res["best"]
    assert best["ms"] == min(r["ms"] for r in res["grid"])
    assert autotune.lookup(cache, 20, m.shape[0], q.shape[0]) == json.loads(json.dumps(best))
    t = autotune.apply(m, best)
    i, d, c = t.knn_cov(q, 20, 1e-3)
    ref = gpu_lib.Target(m)
    i2, d2, c2 = ref.knn_cov(q, 20, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(i, i2) and torch.equal(c.view(torch.int32), c2.view(torch.int32))
    t.close()
    ref.close()
