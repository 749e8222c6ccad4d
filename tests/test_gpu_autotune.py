"""Tensor-core launch configurations and the autotuner on the GPU.

Every configuration (task piece height 256 / 128; one fused launch, one
launch per stage, or one launch per stage on SM pairs with M = 256 MMAs;
tiles in critical-path or locality order) must give bitwise the same U:
the configurations cut and order tiles but never change a task's summation
order.  Parity with the FP64 oracle is then one comparison per precision
(the default configuration is compared in test_gpu_tensor.py; here the 128
piece is compared too, on a problem whose skeleton blocks are taller than
128 so that tasks really are cut)."""
import json

import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [G.PREC_TF32, G.PREC_BF16, G.PREC_BF16X3]
NAMES = {G.PREC_TF32: "tf32", G.PREC_BF16: "bf16", G.PREC_BF16X3: "bf16x3"}
TOL = {G.PREC_TF32: 5e-3, G.PREC_BF16: 2e-2, G.PREC_BF16X3: 1e-4}
CONFIGS = [(p, s, o) for p in (256, 128) for s in (G.SCHED_FUSED, G.SCHED_STAGED, G.SCHED_PAIR, G.SCHED_HYBRID)
           for o in (G.ORDER_CRITICAL, G.ORDER_LOCAL, G.ORDER_SCHEDULE, G.ORDER_READY, G.ORDER_LEVELS)]


def run(h, Wt, prec):
    Ut = torch.full_like(Wt, float("nan"))
    G.evaluate(h, Wt, Ut, prec)
    G.synchronize(h)
    return Ut.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tall():
    # leaves of 300 points and ranks up to 300: leaf, S2S and S2N blocks
    # taller than 128 (and than 256), r = 300 (three r-tiles, ragged)
    w = wl.scaled(wl.C3, 4800)
    h, st, K = both(w, leaf_size=300, max_rank=300, tau=1e-7)
    s = G.stats(h)
    assert s["max_rank"] > 256
    W = w.rhs(300)
    return h, st, K, W, O.evaluate(st, K, W)


@pytest.mark.parametrize("prec", PRECS, ids=[NAMES[p] for p in PRECS])
def test_every_configuration_gives_bitwise_the_same_result(tall, prec):
    h, st, K, W, ref = tall
    Wt = torch.from_numpy(W.astype(np.float32)).cuda()
    G.prepare(h, W.shape[1], prec)
    out = {}
    for cfg in CONFIGS:
        G.set_tc_config(h, prec, *cfg)
        assert G.get_tc_config(h, prec) == dict(piece=cfg[0], schedule=cfg[1], order=cfg[2])
        a = run(h, Wt, prec)
        b = run(h, Wt, prec)  # second call: graph replay
        assert np.array_equal(a, b), cfg
        out[cfg] = a
    base = out[CONFIGS[0]]
    assert np.all(np.isfinite(base))
    for cfg, u in out.items():
        assert np.array_equal(u, base), cfg
    assert rel(out[(128, G.SCHED_FUSED, G.ORDER_LOCAL)], ref) <= TOL[prec]
    G.set_tc_config(h, prec, 256, G.SCHED_FUSED, G.ORDER_CRITICAL)


def test_autotune_measures_applies_and_caches(tall, tmp_path):
    h, st, K, W, ref = tall
    prec = G.PREC_BF16X3
    path = tmp_path / "tune.json"
    t = G.autotune(h, 300, prec, str(path))
    assert not t["from_cache"] and len(t["candidates"]) == 16
    ms = [c["ms"] for c in t["candidates"]]
    assert all(m > 0 for m in ms)
    best = t["candidates"][int(np.argmin(ms))]
    assert (t["piece"], t["schedule"], t["order"]) == (best["piece"], best["schedule"], best["order"])
    assert G.get_tc_config(h, prec) == dict(piece=t["piece"], schedule=t["schedule"], order=t["order"])
    doc = json.loads(path.read_text())
    assert doc["format"] == "gofmm-autotune" and len(doc["entries"]) == 1
    e = doc["entries"][0]
    assert e["key"] == t["key"] and e["piece"] == t["piece"] and len(e["candidates"]) == 16
    # the tuned configuration evaluates correctly
    Wt = torch.from_numpy(W.astype(np.float32)).cuda()
    assert rel(run(h, Wt, prec), ref) <= 1e-4
    # a second tuning reads the cache back
    G.set_tc_config(h, prec, 256, G.SCHED_FUSED, G.ORDER_CRITICAL)
    t2 = G.autotune(h, 300, prec, str(path))
    assert t2["from_cache"] and (t2["piece"], t2["schedule"], t2["order"]) == (t["piece"], t["schedule"], t["order"])
    # another r-tile count is another entry
    G.autotune(h, 64, prec, str(path))
    assert len(json.loads(path.read_text())["entries"]) == 2


def test_batch_autotune_and_stale_batch(tmp_path):
    insts = wl.batching_instances(4)
    hs, Ws = [], []
    for w in insts:
        K = w.matrix()
        h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), G.default_params(**w.params()))
        G.prepare(h, w.r, G.PREC_BF16)
        hs.append(h)
        Ws.append(torch.from_numpy(w.rhs().astype(np.float32)).cuda())
    rs = [w.r for w in insts]
    singles = [run(h, W, G.PREC_BF16) for h, W in zip(hs, Ws)]
    t = G.autotune_batch(hs, rs, G.PREC_BF16, str(tmp_path / "b.json"))
    assert len(t["candidates"]) == 4 and t["piece"] in (128, 256)
    assert t["schedule"] in (G.SCHED_FUSED, G.SCHED_STAGED)
    assert all(G.get_tc_config(h, G.PREC_BF16)["piece"] == t["piece"] for h in hs)
    assert all(G.get_tc_config(h, G.PREC_BF16)["schedule"] == t["schedule"] for h in hs)
    b = G.Batch(hs, rs, G.PREC_BF16)
    Us = [torch.full_like(W, float("nan")) for W in Ws]
    b.evaluate(Ws, Us)
    torch.cuda.synchronize()
    for u, s in zip(Us, singles):
        assert np.array_equal(u.double().cpu().numpy(), s)
    # re-planning a handle makes the batch refuse to run
    other = 128 if t["piece"] == 256 else 256
    G.set_tc_config(hs[0], G.PREC_BF16, other)
    with pytest.raises(G.GofmmError) as e:
        b.evaluate(Ws, Us)
    assert e.value.code == G.ERR_ARG
    b.free()


def test_engine_in_flight_blocks_replanning():
    w = wl.scaled(wl.C1, 2000)
    K = w.matrix()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), G.default_params(leaf_size=64))
    G.prepare(h, 64, G.PREC_BF16)
    eng = G.Engine(G.PREC_BF16, 1 << 28)
    W = torch.from_numpy(w.rhs(64).astype(np.float32)).cuda()
    U = torch.empty_like(W)
    eng.submit(h, W, U)
    with pytest.raises(G.GofmmError) as e:
        G.set_tc_config(h, G.PREC_BF16, 128)
    assert e.value.code == G.ERR_ARG
    assert G.LIB.gofmm_free(h.ptr) == G.ERR_ARG  # nor freed while in flight
    G.set_tc_config(h, G.PREC_BF16, 256, G.SCHED_STAGED)  # same plan: allowed
    eng.drain()
    G.set_tc_config(h, G.PREC_BF16, 128)  # nothing in flight any more
    eng.free()
