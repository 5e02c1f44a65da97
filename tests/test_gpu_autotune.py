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
