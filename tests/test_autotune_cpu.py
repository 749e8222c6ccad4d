"""Host logic of the autotuner and of the tensor-core launch configuration,
on a machine without a GPU: cache keys, the JSON cache file (hits applied
without measuring, foreign or malformed files refused and left alone), and
argument checks.  Measuring needs a GPU (tests/test_gpu_autotune.py)."""
import json

import pytest

import paper_1707_00164_b300 as G
import workloads as wl


def _handle(n=600, seed=None, **over):
    w = wl.scaled(wl.C1, n)
    if seed is not None:
        w = wl.scaled(w, n, point_seed=seed)
    K = w.matrix()
    p = G.default_params(leaf_size=64, max_rank=32, tau=1e-5, kappa=16, budget=0.05, **over)
    return G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), p)


def _cache(path, entries, fmt="gofmm-autotune"):
    path.write_text(json.dumps({"format": fmt, "version": 1, "entries": entries}))


def test_config_defaults_and_validation():
    h = _handle()
    for prec in (G.PREC_TF32, G.PREC_BF16, G.PREC_BF16X3):
        assert G.get_tc_config(h, prec) == dict(piece=256, schedule=G.SCHED_FUSED, order=G.ORDER_CRITICAL)
    G.set_tc_config(h, G.PREC_BF16X3, 128, G.SCHED_STAGED, G.ORDER_LOCAL)
    assert G.get_tc_config(h, G.PREC_BF16X3) == dict(piece=128, schedule=G.SCHED_STAGED, order=G.ORDER_LOCAL)
    assert G.get_tc_config(h, G.PREC_BF16)["piece"] == 256  # per precision
    assert G.get_tc_config(h, G.PREC_TF32)["schedule"] == G.SCHED_FUSED
    G.set_tc_config(h, G.PREC_BF16, 128, G.SCHED_PAIR, G.ORDER_CRITICAL)
    assert G.get_tc_config(h, G.PREC_BF16)["schedule"] == G.SCHED_PAIR
    G.set_tc_config(h, G.PREC_BF16, 256, G.SCHED_HYBRID, G.ORDER_LOCAL)
    assert G.get_tc_config(h, G.PREC_BF16)["schedule"] == G.SCHED_HYBRID
    G.set_tc_config(h, G.PREC_BF16, 256, G.SCHED_FUSED, G.ORDER_SCHEDULE)
    assert G.get_tc_config(h, G.PREC_BF16)["order"] == G.ORDER_SCHEDULE
    G.set_tc_config(h, G.PREC_BF16, 256, G.SCHED_FUSED, G.ORDER_READY)
    assert G.get_tc_config(h, G.PREC_BF16)["order"] == G.ORDER_READY
    G.set_tc_config(h, G.PREC_BF16, 256, G.SCHED_FUSED, G.ORDER_LEVELS)
    assert G.get_tc_config(h, G.PREC_BF16)["order"] == G.ORDER_LEVELS
    for args in [(G.PREC_BF16, 64, 0, 0), (G.PREC_BF16, 256, 4, 0), (G.PREC_BF16, 256, 0, 5),
                 (G.PREC_FP32, 256, 0, 0), (G.PREC_FP64, 128, 0, 0)]:
        with pytest.raises(G.GofmmError) as e:
            G.set_tc_config(h, *args)
        assert e.value.code == G.ERR_ARG
    with pytest.raises(G.GofmmError):
        G.get_tc_config(h, G.PREC_FP32)


def test_keys_follow_structure_r_tiles_and_precision():
    # the key describes the shapes the kernels see (node sizes, ranks, near
    # and far lists), so another problem with other shapes gets another key
    h1, h1b, h2 = _handle(), _handle(), _handle(n=700)
    k = G.autotune_key([h1], [512], G.PREC_BF16X3)
    assert k == G.autotune_key([h1b], [512], G.PREC_BF16X3)  # same compression, same key
    assert k == G.autotune_key([h1], [385], G.PREC_BF16X3)  # same number of 128-column tiles
    assert k != G.autotune_key([h1], [384], G.PREC_BF16X3)
    assert k != G.autotune_key([h1], [512], G.PREC_BF16)
    assert k != G.autotune_key([h2], [512], G.PREC_BF16X3)
    kb = G.autotune_key([h1, h2], [512, 64], G.PREC_BF16X3)
    assert kb != k and kb != G.autotune_key([h2, h1], [64, 512], G.PREC_BF16X3)
    assert k.startswith("e") and kb.startswith("b") and len(k) == 17
    # the launch configuration is an output of tuning, not part of the key
    G.set_tc_config(h1, G.PREC_BF16X3, 128, G.SCHED_STAGED, G.ORDER_LOCAL)
    assert G.autotune_key([h1], [512], G.PREC_BF16X3) == k


def test_cache_hit_applies_the_stored_choice_without_measuring(tmp_path):
    h = _handle()
    key = G.autotune_key([h], [300], G.PREC_BF16X3)
    path = tmp_path / "tune.json"
    other = {"key": "e0000000000000000", "piece": 256, "schedule": 0, "order": 0}
    _cache(path, [other, {"key": key, "piece": 128, "schedule": 1, "order": 1, "candidates": []}])
    before = path.read_text()
    t = G.autotune(h, 300, G.PREC_BF16X3, str(path))
    assert t["from_cache"] and t["candidates"] == [] and t["key"] == key
    assert (t["piece"], t["schedule"], t["order"]) == (128, 1, 1)
    assert G.get_tc_config(h, G.PREC_BF16X3) == dict(piece=128, schedule=1, order=1)
    assert path.read_text() == before  # a hit writes nothing


def test_batch_cache_hit_sets_every_handle(tmp_path):
    hs = [_handle(), _handle(seed=5), _handle(n=900)]
    rs = [16, 200, 64]
    key = G.autotune_key(hs, rs, G.PREC_BF16)
    path = tmp_path / "tune.json"
    _cache(path, [{"key": key, "piece": 128, "schedule": 1, "order": 1}])
    t = G.autotune_batch(hs, rs, G.PREC_BF16, str(path))
    assert t["from_cache"] and t["piece"] == 128
    # the batch form (staged) and order come with the piece
    assert all(G.get_tc_config(h, G.PREC_BF16) == dict(piece=128, schedule=1, order=1) for h in hs)


def test_cache_hit_with_the_schedule_order(tmp_path):
    h = _handle()
    key = G.autotune_key([h], [512], G.PREC_TF32)
    path = tmp_path / "tune.json"
    _cache(path, [{"key": key, "piece": 256, "schedule": G.SCHED_HYBRID, "order": G.ORDER_SCHEDULE}])
    t = G.autotune(h, 512, G.PREC_TF32, str(path))
    assert t["from_cache"] and (t["schedule"], t["order"]) == (G.SCHED_HYBRID, G.ORDER_SCHEDULE)
    assert G.get_tc_config(h, G.PREC_TF32) == dict(piece=256, schedule=G.SCHED_HYBRID, order=G.ORDER_SCHEDULE)


def test_cache_miss_needs_a_gpu_and_leaves_the_file_alone(tmp_path):
    h = _handle()
    path = tmp_path / "tune.json"
    _cache(path, [{"key": "e0123456789abcdef", "piece": 128, "schedule": 0, "order": 0}])
    before = path.read_text()
    with pytest.raises(G.GofmmError) as e:
        G.autotune(h, 64, G.PREC_TF32, str(path))
    assert e.value.code == G.ERR_CUDA
    assert path.read_text() == before
    with pytest.raises(G.GofmmError) as e:
        G.autotune(h, 64, G.PREC_TF32, None)  # no cache: measuring is the only way
    assert e.value.code == G.ERR_CUDA


@pytest.mark.parametrize("text", [
    "not json at all",
    '{"format": "something-else", "entries": []}',
    '{"format": "gofmm-autotune", "entries": {}}',
    '{"format": "gofmm-autotune", "entries": [}',
    '{"format": "gofmm-autotune", "entries": []} trailing',
])
def test_foreign_or_malformed_cache_is_refused(tmp_path, text):
    h = _handle()
    path = tmp_path / "tune.json"
    path.write_text(text)
    with pytest.raises(G.GofmmError) as e:
        G.autotune(h, 64, G.PREC_BF16, str(path))
    assert e.value.code == G.ERR_ARG
    assert path.read_text() == text


def test_cache_entry_missing_fields_is_refused(tmp_path):
    h = _handle()
    key = G.autotune_key([h], [64], G.PREC_BF16)
    path = tmp_path / "tune.json"
    _cache(path, [{"key": key, "piece": 128}])
    with pytest.raises(G.GofmmError) as e:
        G.autotune(h, 64, G.PREC_BF16, str(path))
    assert e.value.code == G.ERR_ARG


def test_autotune_argument_checks(tmp_path):
    h = _handle()
    for prec, r in [(G.PREC_FP32, 64), (G.PREC_FP64, 64), (G.PREC_BF16, 0)]:
        with pytest.raises(G.GofmmError) as e:
            G.autotune(h, r, prec, None)
        assert e.value.code == G.ERR_ARG
