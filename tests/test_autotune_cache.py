"""Host side of the batched-launch autotuner: cache keys and the JSON cache (no GPU)."""
import json
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1611_04474_gb300 import workloads as W


@pytest.fixture
def autotune():
    from paper_1611_04474_gb300 import api, autotune

    try:
        api.load()
    except RuntimeError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(str(e))
    return autotune


def _fake_batch(systems, mode=1, ntypes=6):
    return SimpleNamespace(systems=systems, mode=mode, n=sum(s.n for s in systems),
                           ffs=[SimpleNamespace(ntypes=ntypes)], tuning=(0, 0))


def test_key_separates_what_decides_the_shape(autotune):
    systems = W.batch_of_systems(nsys=6, seed=3, n_range=(500, 3000))
    k = autotune.cache_key(_fake_batch(systems))
    assert k == autotune.cache_key(_fake_batch(systems))
    assert k != autotune.cache_key(_fake_batch(systems, mode=0))
    assert k != autotune.cache_key(_fake_batch(systems, ntypes=8))
    assert k != autotune.cache_key(_fake_batch(systems[:1]))


def test_regimes(autotune):
    systems = W.batch_of_systems(nsys=10, seed=7, n_range=(400, 6000))
    reg, small = autotune.regimes(_fake_batch(systems))
    dims = [np.floor(s.box / s.rc) for s in systems]
    assert reg == any(d.min() >= 3 for d in dims) and small == any(d.min() < 3 for d in dims)


def test_cache_hit_sets_tuning_without_measuring(autotune, tmp_path, monkeypatch):
    systems = W.batch_of_systems(nsys=4, seed=3, n_range=(500, 3000))
    b = _fake_batch(systems)
    path = tmp_path / "t.json"
    path.write_text(json.dumps({autotune.cache_key(b): {"tuning": [2, 1], "ms": {}}}))
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: pytest.fail("measured on a hit"))
    e = autotune.tune(b, cache_path=str(path))
    assert b.tuning == (2, 1) and not e["measured"]


def test_bad_cache_entries_are_remeasured(autotune, tmp_path, monkeypatch):
    systems = W.batch_of_systems(nsys=4, seed=3, n_range=(500, 3000))
    b = _fake_batch(systems)
    path = tmp_path / "t.json"
    path.write_text(json.dumps({autotune.cache_key(b): {"tuning": [9, 0]}}))
    monkeypatch.setattr(autotune, "measure", lambda *a, **k: ((3, 0), {"regular": [1, 1, 1, 0.5]}))
    e = autotune.tune(b, cache_path=str(path))
    assert e["measured"] and b.tuning == (3, 0)
    assert json.loads(path.read_text())[autotune.cache_key(b)]["tuning"] == [3, 0]


def test_fixed_tile_tunes_over_the_cluster_shapes_only(autotune):
    from paper_1611_04474_gb300 import api

    assert autotune.shapes_for(api.ACCUM_FIXED_TILE) == [0, 5]
    assert autotune.shapes_for(api.ACCUM_FIXED64) == list(range(api.BATCH_SHAPES))
