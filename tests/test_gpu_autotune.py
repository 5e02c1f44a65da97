"""The autotuner measuring on the GPU: it returns one of the candidates,
records every candidate's time, and a second tuner on the same cache answers
without measuring."""
import json

import numpy as np
import pytest

import oracle as O
from paper_1911_11906_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_band_width_and_workers_are_tuned_and_cached(tmp_path):
    from paper_1911_11906_gb300 import autotune as A
    path = str(tmp_path / "tune.json")
    b = A.best_band_width(196, route="fp64", candidates=(16, 32), tuner=A.Autotuner(path), reps=1)
    assert b in (16, 32)
    entries = json.load(open(path))["entries"]
    (val,) = [v for k, v in entries.items() if k.startswith("eig_band_width:")]
    assert set(val["seconds"]) == {"16", "32"} and all(s > 0 for s in val["seconds"].values())
    assert A.best_band_width(200, route="fp64", candidates=(16, 32), tuner=A.Autotuner(path)) == b
    probs = []
    for p in I.batched_problems(6):
        _, Acsr = O.assemble(p.mask, p.h)
        probs.append({"A": torch.from_numpy(np.ascontiguousarray(Acsr.dense().T)).cuda().t()})
    w = A.best_workers(probs, candidates=(2, 3), tuner=A.Autotuner(path))
    assert w in (2, 3)
    assert A.Autotuner(path).lookup("batched_workers", {"device": A._device_name(), "count": 6,
                                                        "n_max_bucket": A.size_bucket(max(p["A"].shape[0] for p in probs)),
                                                        "n_sum_bucket": A.size_bucket(sum(p["A"].shape[0] for p in probs)),
                                                        "mixed": 0}, (2, 3)) == w


def test_ozaki_schedule_is_tuned_cached_and_applied(tmp_path):
    """The slice-product schedule (raster group, digit width, tile width,
    cluster size) is measured over the candidates, cached, answered from the
    cache by a second tuner,
    and set on a context, whose products stay FP64-accurate."""
    from paper_1911_11906_gb300 import autotune as A
    import paper_1911_11906_gb300 as F
    path = str(tmp_path / "tune.json")
    sched = A.best_ozaki_schedule(640, groups=(0, 2), bits=(7, 8), tiles=(128, 256), clusters=(1, 2),
                                  tuner=A.Autotuner(path), reps=1)
    assert sched["ozaki_group"] in (0, 2) and sched["ozaki_bits"] in (7, 8) and sched["ozaki_tile_n"] in (128, 256)
    assert sched["ozaki_cluster"] in (1, 2)
    entries = json.load(open(path))["entries"]
    (val,) = [v for k, v in entries.items() if k.startswith("ozaki_schedule:")]
    assert set(val["seconds"]) == {f"{g}/{w}/{t}/{c}" for g in (0, 2) for w in (7, 8) for t in (128, 256)
                                   for c in (1, 2)}
    assert A.best_ozaki_schedule(700, groups=(0, 2), bits=(7, 8), tiles=(128, 256), clusters=(1, 2),
                                 tuner=A.Autotuner(path)) == sched
    ctx = F.Context()
    A.apply_schedule(ctx, sched)
    assert ctx.get_schedule("ozaki_group") == sched["ozaki_group"]
    assert ctx.get_schedule("ozaki_cluster") == sched["ozaki_cluster"]
    rng = np.random.default_rng(640)
    X = rng.standard_normal((640, 300))
    got = F.dgemm_ozaki(torch.from_numpy(X.T.copy()).cuda().t(), torch.from_numpy(X.T.copy()).cuda().t(),
                        trans_a=True, ctx=ctx).cpu().numpy()
    scale = np.abs(X).max(axis=0)[:, None] * np.abs(X).max(axis=0)[None, :] * 640
    assert np.max(np.abs(got - X.T @ X) / scale) <= 1e-15
