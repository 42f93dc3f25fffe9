"""Host logic of the tuning table (no GPU): the choice among measured candidates, the
JSON round trip, lookups of absent configurations, and that other entries are kept."""
import json

from paper_1903_00548_gb300 import autotune as A


def test_choose_prefers_smallest_within_tolerance():
    assert A.choose({32: 9.0, 64: 9.1, 128: 8.0}) == 32          # 64 within 2 % of the top
    assert A.choose({32: 7.0, 64: 9.2, 128: 9.3}) == 64
    assert A.choose({32: 7.0, 64: 9.0, 128: 9.3}) == 128
    assert A.choose({16: 1.0}) == 16


def test_record_and_lookup_round_trip(tmp_path):
    path = str(tmp_path / "t.json")
    assert A.lookup("ribbon512", 512, 200, "mixed", path) is None
    A.record("ribbon512", 512, 200, "mixed", {32: 9.0, 64: 10.0}, {"device": "x"}, path)
    A.record("ribbon256_wide", 256, 200, "mixed", {16: 40.0}, {}, path)
    assert A.lookup("ribbon512", 512, 200, "mixed", path) == 64
    assert A.lookup("ribbon256_wide", 256, 200, "mixed", path) == 16
    assert A.lookup("ribbon512", 512, 100, "mixed", path) is None
    t = json.load(open(path))
    assert t[A.key("ribbon512", 512, 200, "mixed")]["energy_solves_per_s"] == {"32": 9.0, "64": 10.0}
