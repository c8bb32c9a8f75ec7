"""Host logic of the schedule autotuner: cache keys and the JSON cache."""
import json

from paper_2602_15883_b300 import autotune, synth


def test_key_separates_architectures_and_sizes():
    a = autotune.schedule_key(synth.config("tgv"), 262144, 65536, 32, "B300")
    b = autotune.schedule_key(synth.config("beltrami32"), 262144, 65536, 32, "B300")
    c = autotune.schedule_key(synth.config("tgv"), 2 * 262144, 65536, 32, "B300")
    d = autotune.schedule_key(synth.config("tgv"), 262144 + 1000, 65536, 32, "B300")
    assert len({a, b, c}) == 3
    assert a == d   # same log2 bucket


def test_cache_roundtrip(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("DPINN_AUTOTUNE_CACHE", str(p))
    assert autotune.load_cache() == {}
    autotune.store_cache("k1", {"jet_tiles": 8, "val_tiles": 0, "order": 0, "ms": 1.5})
    autotune.store_cache("k2", {"jet_tiles": 2, "val_tiles": 4, "order": 1, "ms": 2.5})
    data = json.loads(p.read_text())
    assert data["k1"]["jet_tiles"] == 8 and data["k2"]["order"] == 1
    p.write_text("not json")
    assert autotune.load_cache() == {}


def test_key_separates_precision_activation_and_build():
    from paper_2602_15883_b300 import autotune, synth
    base = synth.config("beltrami32")
    k = lambda cfg, build="b1": autotune.schedule_key(cfg, 262144, 65536, 32, "B300", build)
    assert k(base) != k(dict(base, precision=1))
    assert k(base) != k(dict(base, activation=1))
    assert k(base) != k(base, "b2")
    assert k(base) == k(dict(base))


def test_key_separates_searched_precisions():
    base = synth.config("beltrami32")
    k = lambda cfg, precisions=None: autotune.schedule_key(cfg, 262144, 65536, 32, "B300", "b1", precisions)
    assert k(base, (0, 1)) == k(dict(base, precision=1), (1, 0))   # the handle's own precision is not the key
    assert k(base, (0, 1)) != k(base) and k(base, (0, 1)) != k(dict(base, precision=1))
