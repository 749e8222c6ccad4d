"""Batching and serving engine: many evaluations in one grouped launch per
step.  Each request's result must be bitwise the single evaluation's (same
kernel, same tasks, same summation order), alone or in any mix, including
requests that join while others are mid-flight; admission waits for pool
memory."""
import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = G.PREC_BF16X3


def _instance(n, dim, h, seed, m=64, s=64):
    w = wl.Workload(f"inst{seed}", n, dim, "normal", wl.GAUSSIAN, h, 1e-2, leaf_size=m, max_rank=s, tau=1e-5,
                    kappa=16, budget=0.03, r=1, point_seed=seed, w_seed=seed + 500)
    K = w.matrix()
    hd = G.compress(G.Entries.gaussian(K.points, h, 1e-2),
                    G.default_params(leaf_size=m, max_rank=s, tau=1e-5, kappa=16, budget=0.03))
    G.prepare(hd, 256, PREC)
    return w, hd


@pytest.fixture(scope="module")
def instances():
    specs = [(3000, 3, 0.5, 1), (1111, 2, 0.3, 2), (5000, 6, 0.9, 3), (2048, 4, 0.7, 4), (700, 8, 1.0, 5)]
    return [_instance(*sp) for sp in specs]


def _single(hd, W):
    U = torch.empty_like(W)
    G.set_timing(hd, True)  # direct launches
    G.evaluate(hd, W, U, PREC)
    G.set_timing(hd, False)
    G.synchronize(hd)
    return U


def test_batch_of_uneven_instances_matches_single_evaluations(instances):
    rs = [16, 256, 100, 129, 37]
    Ws = [torch.from_numpy(w.rhs(r).astype(np.float32)).cuda() for (w, _), r in zip(instances, rs)]
    refs = [_single(hd, W) for (w, hd), W in zip(instances, Ws)]
    eng = G.Engine(PREC, 4 << 30)
    Us = [torch.full_like(W, float("nan")) for W in Ws]
    ids = [eng.submit(hd, W, U) for (w, hd), W, U in zip(instances, Ws, Us)]
    eng.drain()
    st = eng.stats()
    assert st["completed"] == len(ids) and st["max_active"] == len(ids)
    for U, ref in zip(Us, refs):
        assert torch.equal(U, ref)
    # and one of them against the oracle (same structure)
    w, hd = instances[1]
    h2, st2, K = both(w, leaf_size=64, max_rank=64, kappa=16)
    ref_o = O.evaluate(st2, K, w.rhs(256))
    got = Us[1].double().cpu().numpy()
    assert np.linalg.norm(got - ref_o) / np.linalg.norm(ref_o) <= 1e-4


def test_continuous_batching_result_is_the_same_alone_and_in_the_mix(instances):
    w, hd = instances[2]
    X = torch.from_numpy(w.rhs(200).astype(np.float32)).cuda()
    eng = G.Engine(PREC, 4 << 30)
    alone = torch.empty_like(X)
    eng.submit(hd, X, alone)
    eng.drain()
    # now in a mix: X joins after others started, more join while it runs
    eng2 = G.Engine(PREC, 4 << 30)
    others = []
    def add(k, r):
        wk, hk = instances[k]
        Wk = torch.from_numpy(wk.rhs(r).astype(np.float32)).cuda()
        Uk = torch.empty_like(Wk)
        eng2.submit(hk, Wk, Uk)
        others.append((Wk, Uk))
    add(0, 64)
    add(2, 300)          # same matrix as X, different W
    eng2.step()
    eng2.step()
    mixed = torch.full_like(X, float("nan"))
    xid = eng2.submit(hd, X, mixed)
    eng2.step()
    add(3, 17)
    for _ in range(3):
        eng2.step()
    add(4, 256)
    eng2.drain()
    assert eng2.poll(xid) == G.Engine.DONE
    assert torch.equal(mixed, alone)


def test_admission_waits_for_pool_memory(instances):
    w, hd = instances[0]
    Ws = [torch.from_numpy(wl.scaled(w, w.n, w_seed=s).rhs(128).astype(np.float32)).cuda() for s in range(4)]
    refs = [_single(hd, W) for W in Ws]
    eng_big = G.Engine(PREC, 4 << 30)
    U0 = torch.empty_like(Ws[0])
    eng_big.submit(hd, Ws[0], U0)
    eng_big.drain()
    # a pool that holds one request's workspace but not two
    ws = eng_big.workspace(hd, 128)
    eng = G.Engine(PREC, ws * 3 // 2 + (1 << 20))
    Us = [torch.empty_like(W) for W in Ws]
    for W, U in zip(Ws, Us):
        eng.submit(hd, W, U)
    eng.drain()
    st = eng.stats()
    assert st["completed"] == 4 and st["max_active"] == 1
    for U, ref in zip(Us, refs):
        assert torch.equal(U, ref)


def test_engine_errors(instances):
    w, hd = instances[4]
    W = torch.zeros((w.n, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GofmmError) as e:
        G.Engine(G.PREC_FP32, 1 << 30)
    assert e.value.code == G.ERR_UNSUPPORTED
    eng = G.Engine(G.PREC_TF32, 1 << 30)   # handle not prepared for TF32
    with pytest.raises(G.GofmmError) as e:
        eng.submit(hd, W, torch.empty_like(W))
    assert e.value.code == G.ERR_ARG
    small = G.Engine(PREC, 1 << 20)
    with pytest.raises(G.GofmmError) as e:
        small.submit(hd, W, torch.empty_like(W))
    assert e.value.code == G.ERR_NOMEM


@pytest.mark.parametrize("schedules", [(G.SCHED_FUSED,) * 5, (G.SCHED_STAGED,) * 5,
                                       (G.SCHED_FUSED, G.SCHED_STAGED, G.SCHED_FUSED, G.SCHED_HYBRID,
                                        G.SCHED_FUSED)], ids=["fused", "staged", "mixed"])
def test_static_batch_matches_single_evaluations_and_replays(instances, schedules):
    """All handles on the fused schedule: one dependency-driven launch runs
    every stage of every instance; otherwise one launch per stage step.
    Both give each instance's single evaluation bit for bit."""
    rs = [16, 256, 100, 129, 37]
    hs = [hd for _, hd in instances]
    for hd, sc in zip(hs, schedules):
        G.set_tc_config(hd, PREC, 256, sc, G.ORDER_LOCAL)
    Ws = [torch.from_numpy(w.rhs(r).astype(np.float32)).cuda() for (w, _), r in zip(instances, rs)]
    refs = [_single(hd, W) for hd, W in zip(hs, Ws)]
    B = G.Batch(hs, rs, PREC)
    fused = all(sc == G.SCHED_FUSED for sc in schedules)
    Us = [torch.full_like(W, float("nan")) for W in Ws]
    for _ in range(3):  # first call direct, later calls replay the captured graph
        for U in Us:
            U.fill_(float("nan"))
        B.evaluate(Ws, Us)
        torch.cuda.synchronize()
        assert B.info()["error"] == 0
        # kernels per call: a gather per instance + 1 fused GEMM launch, or one per stage step
        assert (B.info()["launches"] == len(hs) + 1) == fused
        for U, ref in zip(Us, refs):
            assert torch.equal(U, ref)


def test_fused_batch_of_more_than_64_instances():
    """More instances than one launch holds: one fused launch per 64, each
    instance bitwise its single evaluation."""
    hs, Ws = [], []
    for i in range(67):
        w = wl.Workload(f"b{i}", 300 + 7 * i, 3, "normal", wl.GAUSSIAN, 0.6, 1e-2, leaf_size=32, max_rank=32,
                        tau=1e-5, kappa=8, budget=0.03, r=1, point_seed=100 + i, w_seed=900 + i)
        K = w.matrix()
        hd = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift),
                        G.default_params(leaf_size=32, max_rank=32, tau=1e-5, kappa=8, budget=0.03))
        G.prepare(hd, 24, PREC)
        G.set_tc_config(hd, PREC, 128, G.SCHED_FUSED, G.ORDER_LOCAL)
        hs.append(hd)
        Ws.append(torch.from_numpy(w.rhs(1 + i % 24).astype(np.float32)).cuda())
    refs = [_single(hd, W) for hd, W in zip(hs, Ws)]
    B = G.Batch(hs, [W.shape[1] for W in Ws], PREC)
    Us = [torch.full_like(W, float("nan")) for W in Ws]
    B.evaluate(Ws, Us)
    torch.cuda.synchronize()
    assert B.info()["error"] == 0 and B.info()["launches"] == len(hs) + 2
    for U, ref in zip(Us, refs):
        assert torch.equal(U, ref)
    B.free()
