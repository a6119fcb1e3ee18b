"""Host-side cache of autotuned launch shapes (paper_1105_2791_gb300/tuning.py): keys,
round trip, replacement and validation.  No GPU is needed."""
import json

import pytest

pytest.importorskip("torch")

from paper_1105_2791_gb300 import tuning as T


def _entry(**kw):
    e = {"chunk": 32, "legendre_maps": 8, "cubic_ctas": 512, "ms": 51.25}
    e.update(kw)
    return e


def test_key_names_every_deciding_parameter():
    k = T.tuning_key("NVIDIA GB300", 2000, 16, 2001, 4096, 4, 32, True, "pixel", False)
    assert k == "NVIDIA GB300|lmax=2000|P=16|grid=2001x4096|fp16x3|B=32|linear=pixel|mask=0"
    assert T.tuning_key("NVIDIA GB300", 2000, 16, 2001, 4096, 4, 32, False, "pixel", True).endswith(
        "|linear=off|mask=1")
    keys = {T.tuning_key("d", 500, P, 501, 1024, prec, B, True, "ring", False)
            for P in (10, 16) for prec in (0, 1, 4) for B in (8, 32)}
    assert len(keys) == 12


def test_store_load_round_trip_and_replace(tmp_path):
    path = str(tmp_path / "sub" / "tiles.json")
    assert T.load(path) == {}
    T.store(path, "a", _entry())
    T.store(path, "b", _entry(chunk=16, ms=3.5))
    data = T.load(path)
    assert set(data) == {"a", "b"} and data["b"]["chunk"] == 16 and data["b"]["ms"] == 3.5
    T.store(path, "a", _entry(legendre_maps=4))
    data = json.load(open(path))
    assert data["a"]["legendre_maps"] == 4 and data["b"]["chunk"] == 16
    assert [p.name for p in (tmp_path / "sub").iterdir()] == ["tiles.json"]   # no temporary left


def test_invalid_entries_are_not_used(tmp_path):
    assert T.valid_entry(_entry())
    assert not T.valid_entry({"chunk": 8})
    assert not T.valid_entry(_entry(cubic_ctas=0))
    assert not T.valid_entry(_entry(legendre_maps="x"))
    bad = tmp_path / "bad.json"
    bad.write_text("[1, 2]")
    with pytest.raises(ValueError):
        T.load(str(bad))
