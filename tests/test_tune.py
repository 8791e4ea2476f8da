"""The autotuner's table and its JSON file, on the host (no GPU needed):
insert and replace per (device, kind, shape bucket), bucket lookup, the
file round trip, and rejection of malformed entries and files."""
import json
import os

import pytest

import paper_1209_5198_gb300 as gf2


@pytest.fixture
def lib():
    try:
        l = gf2.load()
    except ImportError as e:
        pytest.skip(str(e))
    gf2.tune_clear()
    yield l
    gf2.tune_clear()


def entry(device="GB300 sm152 cc10.3", bn=32768, bm=32768, panel_w=128, table_c=8, schedule=1, ms=12.5):
    e = gf2.TuneEntry()
    e.device = device.encode()
    e.kind = gf2.GF2_TUNE_DECOMPOSE
    e.bucket_n, e.bucket_m = bn, bm
    e.opts = gf2.Opts(panel_w=panel_w, table_c=table_c, schedule=schedule)
    e.ms = ms
    return e


def test_put_lookup_by_bucket_and_replace(lib):
    gf2.tune_put(entry())
    gf2.tune_put(entry(bn=1024, bm=2048, panel_w=64, table_c=4, schedule=0, ms=0.4))
    assert gf2.tune_count() == 2
    # 20000 x 30000 falls in the 32768 x 32768 bucket; 1000 x 1025 in 1024 x 2048
    got = gf2.tune_lookup("GB300 sm152 cc10.3", 20000, 30000)
    assert got is not None and got.opts.panel_w == 128 and got.opts.table_c == 8 and got.ms == 12.5
    got = gf2.tune_lookup("GB300 sm152 cc10.3", 1000, 1025)
    assert got is not None and (got.bucket_n, got.bucket_m) == (1024, 2048) and got.opts.panel_w == 64
    assert gf2.tune_lookup("GB300 sm152 cc10.3", 40000, 30000) is None  # 65536 x 32768: no entry
    assert gf2.tune_lookup("other device", 20000, 30000) is None
    assert gf2.tune_lookup("GB300 sm152 cc10.3", 1, 1) is None  # 64 x 64
    # the same slot is replaced, not duplicated
    gf2.tune_put(entry(schedule=3, ms=11.0))
    assert gf2.tune_count() == 2
    assert gf2.tune_lookup("GB300 sm152 cc10.3", 32768, 32768).opts.schedule == 3


@pytest.mark.parametrize("bad", [
    dict(bn=1000), dict(bm=32), dict(device=""), dict(device='a"b'), dict(device="a\\b"),
    dict(panel_w=96), dict(table_c=5), dict(schedule=9), dict(ms=-1.0),
])
def test_put_rejects_bad_entries(lib, bad):
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.tune_put(entry(**bad))
    assert e.value.status == gf2.GF2_ERR_ARG
    assert gf2.tune_count() == 0


def test_json_round_trip(lib, tmp_path):
    gf2.tune_put(entry())
    gf2.tune_put(entry(device="another GPU sm10 cc9.0", bn=64, bm=128, panel_w=64, table_c=4, schedule=0, ms=0.25))
    path = str(tmp_path / "tune.json")
    gf2.tune_save(path)
    doc = json.load(open(path))
    assert doc["gf2_tune"] == 1 and len(doc["entries"]) == 2
    first = doc["entries"][0]
    assert first["device"] == "GB300 sm152 cc10.3" and first["kind"] == "decompose"
    assert (first["bucket_n"], first["panel_w"], first["table_c"], first["schedule"]) == (32768, 128, 8, 1)
    gf2.tune_clear()
    assert gf2.tune_count() == 0
    gf2.tune_load(path)
    assert gf2.tune_count() == 2
    got = gf2.tune_lookup("another GPU sm10 cc9.0", 60, 100)
    assert got is not None and got.opts.table_c == 4 and abs(got.ms - 0.25) < 1e-9
    # a file written by another program with other key order and spacing loads too
    doc["entries"] = [dict(reversed(list(e.items()))) for e in doc["entries"]]
    doc["entries"][0]["schedule"] = 2
    json.dump(doc, open(path, "w"), indent=3)
    gf2.tune_load(path)  # merges: replaces the matching slots
    assert gf2.tune_count() == 2
    assert gf2.tune_lookup("GB300 sm152 cc10.3", 32768, 32768).opts.schedule == 2


@pytest.mark.parametrize("text", [
    "", "[]", '{"gf2_tune": 2, "entries": []}', '{"gf2_tune": 1}', '{"gf2_tune": 1, "entries": [{}]}',
    '{"gf2_tune": 1, "entries": [{"device": "x", "kind": "product", "bucket_n": 64, "bucket_m": 64}]}',
    '{"gf2_tune": 1, "entries": [{"device": "x", "kind": "decompose", "bucket_n": 100, "bucket_m": 64, "ms": 1}]}',
    '{"gf2_tune": 1, "entries": [{"device": "x", "kind": "decompose", "bucket_n": 64, "bucket_m": 64, '
    '"panel_w": 1.5, "ms": 1}]}',
    '{"gf2_tune": 1, "entries": []} trailing',
])
def test_load_rejects_malformed_files(lib, tmp_path, text):
    gf2.tune_put(entry())
    path = str(tmp_path / "bad.json")
    open(path, "w").write(text)
    with pytest.raises(gf2.Gf2Error) as e:
        gf2.tune_load(path)
    assert e.value.status == gf2.GF2_ERR_ARG
    assert gf2.tune_count() == 1  # nothing loaded, nothing lost


def test_load_missing_file(lib, tmp_path):
    with pytest.raises(gf2.Gf2Error):
        gf2.tune_load(str(tmp_path / "none.json"))
    assert not os.path.exists(str(tmp_path / "none.json"))
