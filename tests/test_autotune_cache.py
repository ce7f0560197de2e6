"""Host logic of the batched kernel's autotuner (no GPU): the workload
signature and the JSON cache that lets a workload of the same class on the
same GPU model skip the timing."""
import json

import pytest

from paper_2404_08247_gb300 import autotune as A

torch = pytest.importorskip("torch")


def probs(n1, n2):
    return ([{"ndim": 1, "n": [n, 1, 1]} for n in n1] +
            [{"ndim": 2, "n": [n, n, 1]} for n in n2])


def test_signature_classes():
    a = A.signature(probs([100, 200], [32]), "mixed", "GPU-A")
    # cell totals within the same power-of-two bucket share the class
    assert A.signature(probs([110, 190], [32]), "mixed", "GPU-A") == a
    assert A.signature(probs([400, 200], [32]), "mixed", "GPU-A") != a
    assert A.signature(probs([100, 200], [32, 8]), "mixed", "GPU-A") != a
    assert A.signature(probs([100, 200], [32]), "fp64", "GPU-A") != a
    assert A.signature(probs([100, 200], [32]), "mixed", "GPU-B") != a
    assert A.signature(probs([], []), "mixed") == "mixed|1d:0:0|2d:0:0"


def test_cache_hit_skips_timing(tmp_path, monkeypatch):
    """A cached entry for this GPU model and workload class is returned as it
    is, marked cached, without creating a batch; an unreadable cache file
    counts as empty."""
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GPU-A")
    p = probs([100], [32])
    sig = A.signature(p, "mixed", "GPU-A")
    path = tmp_path / "tune.json"
    entry = {"tile2d": 2, "blocks_per_sm": 1, "timings_ms": {"2,1": 1.0}, "signature": sig}
    path.write_text(json.dumps({sig: entry}))
    res = A.tune([(q, None) for q in p], "mixed", cache_path=str(path))
    assert res == dict(entry, cached=True)
    path.write_text("{not json")
    assert A._load(str(path)) == {}


def test_cache_store_is_atomic_and_merges(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    A._store(path, {"a": {"tile2d": 0}})
    cache = A._load(path)
    cache["b"] = {"tile2d": 1}
    A._store(path, cache)
    assert A._load(path) == {"a": {"tile2d": 0}, "b": {"tile2d": 1}}
    assert [f.name for f in (tmp_path / "sub").iterdir()] == ["tune.json"]
