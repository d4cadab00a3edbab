"""Host-side logic of the batched projection: argument checks of
mls_batch_create (made before any device call, so they run without a GPU)
and the autotuner's cache."""
import ctypes
import json

import pytest

from paper_2401_03365_gb300.batched import TuneCache, tune_key


@pytest.fixture(scope="module")
def lib():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi.lib()


def _create(lib, offsets, ks):
    off = (ctypes.c_int64 * len(offsets))(*offsets)
    kk = (ctypes.c_int32 * max(len(ks), 1))(*ks)
    h = ctypes.c_void_p()
    rc = lib.mls_batch_create(len(ks), off, kk, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("offsets, ks, code", [
    ([0], [], -1),                          # no clouds
    ([1, 10], [4], -1),                     # offsets[0] != 0
    ([0, 10, 10], [4, 4], -1),              # an empty cloud
    ([0, 10, 5], [4, 4], -1),               # offsets going back
    ([0, 10, 20], [4, 0], -2),              # k < 1
    ([0, 10, 20], [4, 65], -2),             # k > MLS_MAX_K
    ([0, 10, 15], [4, 6], -2),              # k > n_c
    ([0, 2**31], [8], -8),                  # a cloud beyond the index range
    ([0, 2**30, 2**31], [8, 8], -8),        # a total beyond the index range
])
def test_batch_create_rejects_bad_layouts(lib, offsets, ks, code):
    rc, h = _create(lib, offsets, ks)
    assert rc == code
    assert not h.value
    assert lib.mls_last_error().decode().startswith("mls_batch_create")


def test_batch_entry_points_reject_a_null_handle(lib):
    assert lib.mls_project_batched(None, None, None, None, None, 2, 1, None, None, None, None) == -1
    assert lib.mls_batch_replay(None, None) == -1
    assert lib.mls_batch_set_shape(None, 1, 128, 1) == -1
    assert lib.mls_batch_total(None) == -1
    assert lib.mls_batch_idx_offset(None, 0) == -1
    lib.mls_batch_destroy(None)


def test_tune_key_separates_device_fit_k_mix_and_size():
    base = tune_key("GB300", 2, "mixed", [16, 32, 64, 64], 1000)
    assert base == tune_key("GB300", 2, "mixed", [64, 16, 64, 32], 1000)     # order of clouds
    assert base == tune_key("GB300", 2, "mixed", [16, 32, 64, 64], 1020)     # same size class
    for other in (tune_key("B200", 2, "mixed", [16, 32, 64, 64], 1000),
                  tune_key("GB300", 1, "mixed", [16, 32, 64, 64], 1000),
                  tune_key("GB300", 2, "fp32", [16, 32, 64, 64], 1000),
                  tune_key("GB300", 2, "mixed", [16, 16, 64, 64], 1000),
                  tune_key("GB300", 2, "mixed", [16, 32, 64, 64], 5000)):
        assert other != base


def test_tune_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = TuneCache(path)
    assert c.get("x") is None
    c.put("x", (4, 128, 1), 1.5)
    assert TuneCache(path).get("x") == (4, 128, 1)
    assert json.load(open(path))["x"] == {"shape": [4, 128, 1], "ms": 1.5}


def test_tune_cache_ignores_a_corrupt_file(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    c = TuneCache(str(path))
    assert c.get("x") is None
    c.put("x", (1, 64, 4), 2.0)
    assert TuneCache(str(path)).get("x") == (1, 64, 4)
