"""The tuner times configurations of all six parameters (cell occupancy,
starting-radius scale, warps per block, queries per warp item, survivor
slots, per-query starting radius), proves they give identical results, and
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
    space = {"occupancy": (8.0, 16.0), "rho_scale": (0.9, 1.1), "warps": (2, 4), "tile": (16, 32),
             "slots": (0, 64), "probe": (1, 2)}
    res = autotune.tune(m, q, 20, 1e-3, space=space, rounds=1, reps=3, cache=cache)
    # every value of every parameter was timed at least once (and raised on a changed result)
    for name, values in space.items():
        assert {r[name] for r in res["grid"]} >= set(values), name
    best = res["best"]
    assert best["ms"] == min(r["ms"] for r in res["grid"])
    assert autotune.lookup(cache, 20, m.shape[0], q.shape[0]) == json.loads(json.dumps(best))
    t = autotune.apply(m, best)
    i, d, c = t.knn_cov(q, 20, 1e-3)
    ref = gpu_lib.Target(m)
    i2, d2, c2 = ref.knn_cov(q, 20, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(i, i2) and torch.equal(d.view(torch.int32), d2.view(torch.int32))
    assert torch.equal(c.view(torch.int32), c2.view(torch.int32))
    t.close()
    ref.close()


def test_tune_rejects_bad_values(gpu_lib):
    t = gpu_lib.Target(torch.from_numpy(W.uniform_box(1000, seed=3)).cuda())
    with pytest.raises(gpu_lib.PcError):
        t.set_tune(slots=48)
    with pytest.raises(gpu_lib.PcError):
        t.set_tune(probe=3)
    t.set_tune(slots=64, probe=2)
    t.close()


def test_tune_starts_from_a_given_configuration(gpu_lib):
    """The descent starts from `start` (the stored best when re-tuning):
    the first configuration timed is that one, and the best is never
    slower than it."""
    m = torch.from_numpy(W.uniform_box(60_000, seed=5)).cuda()
    q = torch.from_numpy(W.uniform_box(4000, seed=6)).cuda()
    start = {"occupancy": 16.0, "rho_scale": 1.1, "warps": 2, "tile": 32, "slots": 0, "probe": 1}
    res = autotune.tune(m, q, 12, 1e-3, space={"warps": (2, 4)}, rounds=1, reps=3, start=start)
    first = res["grid"][0]
    assert all(first[k] == v for k, v in start.items())
    assert res["best"]["ms"] <= first["ms"]
    assert res["best"]["occupancy"] == 16.0 and res["best"]["rho_scale"] == 1.1
