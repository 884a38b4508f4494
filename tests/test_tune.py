"""Host logic of the run-time choices (include/cch.h, tuning): the size
buckets, the table and its JSON cache.  No GPU: entries are keyed by an
explicit GPU name and SM count."""
import json

import pytest

import paper_1508_05488_gb300 as cch

DEFAULTS = {"small_max": 16384, "stair_div": 16, "stair_min": 8192, "stair_max": 1 << 20,
            "a1_len_min": 4096, "cls_per_sm": 2}


@pytest.fixture(autouse=True)
def clean_table():
    cch.lib().cch_tune_clear()
    yield
    cch.lib().cch_tune_clear()


def test_buckets_are_floor_log2_of_points_per_set():
    b = cch.lib().cch_tune_bucket
    assert [b(n, 1) for n in (0, 1, 2, 3, 4, 1023, 1024, 20_000_000)] == [0, 0, 1, 1, 2, 9, 10, 24]
    assert b(4096 * 126_000, 4096) == 16 and b(100, 0) == 6


def test_defaults_when_no_entry_and_batch_default():
    p, found = cch.tune_get(cch.CCH_F64, False, 20, gpu="TestGPU", sms=10)
    assert not found and p == DEFAULTS
    p, found = cch.tune_get(cch.CCH_I32, True, 16, gpu="TestGPU", sms=10)
    assert not found and p == dict(DEFAULTS, a1_len_min=16384)


def test_set_get_save_load_round_trip(tmp_path):
    a = dict(DEFAULTS, small_max=4096, stair_div=32, stair_min=4096, stair_max=1 << 19, cls_per_sm=1)
    b = dict(DEFAULTS, a1_len_min=65536)
    cch.tune_set(a, cch.CCH_F64, False, 24, gpu='Test "GPU" \\ A', sms=152)
    cch.tune_set(b, cch.CCH_I32, True, 16, gpu="TestGPU", sms=10)
    path = str(tmp_path / "tune.json")
    assert cch.lib().cch_tune_save(path.encode()) == 0
    doc = json.load(open(path))                                   # plain JSON
    assert len(doc["entries"]) == 2 and {e["gpu"] for e in doc["entries"]} == {'Test "GPU" \\ A', "TestGPU"}
    cch.lib().cch_tune_clear()
    assert cch.tune_get(cch.CCH_F64, False, 24, gpu='Test "GPU" \\ A', sms=152)[1] is False
    assert cch.lib().cch_tune_load(path.encode()) == 0
    assert cch.tune_get(cch.CCH_F64, False, 24, gpu='Test "GPU" \\ A', sms=152) == (a, True)
    assert cch.tune_get(cch.CCH_I32, True, 16, gpu="TestGPU", sms=10) == (b, True)
    # the key is the whole tuple: another SM count, dtype, batch flag or bucket misses
    assert cch.tune_get(cch.CCH_I32, True, 16, gpu="TestGPU", sms=11)[1] is False
    assert cch.tune_get(cch.CCH_F64, True, 16, gpu="TestGPU", sms=10)[1] is False
    assert cch.tune_get(cch.CCH_I32, False, 16, gpu="TestGPU", sms=10)[1] is False
    assert cch.tune_get(cch.CCH_I32, True, 17, gpu="TestGPU", sms=10)[1] is False


@pytest.mark.parametrize("bad", [dict(small_max=0), dict(small_max=16385), dict(stair_div=0),
                                 dict(stair_min=1 << 21), dict(a1_len_min=2048), dict(a1_len_min=5000),
                                 dict(cls_per_sm=3)])
def test_invalid_choices_are_rejected(bad):
    with pytest.raises(cch.CchError) as e:
        cch.tune_set(dict(DEFAULTS, **bad), cch.CCH_F64, False, 10, gpu="TestGPU", sms=10)
    assert e.value.code == -1


@pytest.mark.parametrize("text", ['', '{"entries": [', '{"entries": [{"gpu": "G", "sms": 1}]}',
                                  '{"entries": [{"gpu": "G", "sms": 1, "dtype": 2, "batched": 0, "bucket": 3, '
                                  '"small_max": 0, "stair_div": 16, "stair_min": 1, "stair_max": 2, '
                                  '"a1_len_min": 4096, "cls_per_sm": 2}]}',
                                  '{"entries": [{"gpu": "G", "sms": 99999999999999999999}]}'])
def test_malformed_cache_is_rejected_and_changes_nothing(tmp_path, text):
    cch.tune_set(DEFAULTS, cch.CCH_F64, False, 5, gpu="Keep", sms=1)
    path = tmp_path / "bad.json"
    path.write_text(text)
    assert cch.lib().cch_tune_load(str(path).encode()) == -1
    assert cch.tune_get(cch.CCH_F64, False, 5, gpu="Keep", sms=1)[1] is True
    assert cch.lib().cch_tune_load(str(tmp_path / "missing.json").encode()) == -9
