"""Tensor-core evaluation with the block entries generated inside the GEMM
kernel (GOFMM_CACHE_NONE): generator warps write each K-block chunk into
shared memory in the MMA layout (FP32 entry formula, rounded to TF32 / BF16
/ BF16 hi + lo) instead of copying cached tiles.  Checked against the FP64
oracle on the same structure with the per-precision tolerances of the
cached path, for every launch configuration (bitwise equal among
themselves), and in the serving engine (bitwise the same alone and in a mix
with cached-block matrices)."""
import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import abs_product, assert_same_structure, assert_tensor_close, both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {G.PREC_TF32: 5e-3, G.PREC_BF16: 2e-2, G.PREC_BF16X3: 1e-4}
PRECS = [G.PREC_TF32, G.PREC_BF16, G.PREC_BF16X3]
NAMES = {G.PREC_TF32: "tf32", G.PREC_BF16: "bf16", G.PREC_BF16X3: "bf16x3"}


def run(h, W, prec):
    Wt = torch.from_numpy(W.astype(np.float32)).cuda()
    Ut = torch.full_like(Wt, float("nan"))
    G.evaluate(h, Wt, Ut, prec)
    G.synchronize(h)
    return Ut.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def tol(prec, K, W):
    """Per-precision bound at a sum condition <= 25, scaled above it (as for
    cached blocks: relative rounding errors grow with || |K| |W| || / || K W ||)."""
    Kd = K.dense()
    kappa = float(np.linalg.norm(np.abs(Kd) @ np.abs(W)) / np.linalg.norm(Kd @ W))
    return TOL[prec] * max(1.0, kappa / 25.0)


CASES = [
    ("gauss6d_n8192_r300", wl.scaled(wl.C2, 8192), 300, dict(knn_exact_max=20000)),
    ("ragged_n1000_r37", wl.scaled(wl.C1, 1000), 37, dict(leaf_size=32)),
    ("imq_tall_n3000_m400", wl.scaled(wl.C3, 3000), 64, dict(leaf_size=400, max_rank=300, tau=1e-6)),
    ("single_leaf_n50_r7", wl.scaled(wl.C1, 50), 7, dict(leaf_size=64)),
    ("tiny_n9_r1", wl.scaled(wl.C1, 9), 1, dict(leaf_size=4, max_rank=2)),
]


@pytest.mark.parametrize("prec", PRECS, ids=[NAMES[p] for p in PRECS])
@pytest.mark.parametrize("name,w,r,over", CASES, ids=[c[0] for c in CASES])
def test_generated_blocks_match_oracle(name, w, r, over, prec):
    h, st, K = both(w, callback=False, cache_mode=G.CACHE_NONE, **over)
    assert_same_structure(h, st)
    W = w.rhs(r)
    ref = O.evaluate(st, K, W)
    U = run(h, W, prec)
    assert np.all(np.isfinite(U))
    assert rel(U, ref) <= tol(prec, K, W), rel(U, ref)
    # the generator rounds each FP32 entry to the mode's format, like the
    # cached tiles, so the same element-wise bound holds
    assert_tensor_close(U, ref, O.evaluate_abs(st, K, W), abs_product(K, W), prec)


def test_generated_blocks_every_configuration_bitwise_equal():
    # r = 520: five r-tiles, so the 128-row generator kernel runs four-r-tile
    # tiles (its stages hold four) beside a ragged single one
    w = wl.scaled(wl.C3, 3000)
    h, st, K = both(w, callback=False, cache_mode=G.CACHE_NONE, leaf_size=400, max_rank=300, tau=1e-6)
    W = w.rhs(520)
    prec = G.PREC_BF16X3
    G.prepare(h, 520, prec)
    out = []
    for piece in (256, 128):
        for sched in (G.SCHED_FUSED, G.SCHED_STAGED, G.SCHED_HYBRID):
            for order in (G.ORDER_CRITICAL, G.ORDER_LOCAL, G.ORDER_SCHEDULE, G.ORDER_READY, G.ORDER_LEVELS):
                G.set_tc_config(h, prec, piece, sched, order)
                out.append(run(h, W, prec))
    assert all(np.array_equal(o, out[0]) for o in out)
    ref = O.evaluate(st, K, W)
    assert rel(out[0], ref) <= TOL[prec]
    assert_tensor_close(out[0], ref, O.evaluate_abs(st, K, W), abs_product(K, W), prec)
    G.set_tc_config(h, prec, 128, G.SCHED_PAIR)
    with pytest.raises(G.GofmmError) as e:  # the pair kernel reads cached blocks only
        run(h, W, prec)
    assert e.value.code == G.ERR_UNSUPPORTED


def test_generated_and_cached_in_one_engine_mix():
    w1 = wl.scaled(wl.C2, 6000)
    w2 = wl.scaled(wl.C3, 5000)
    prec = G.PREC_BF16
    hs = []
    for w, cm in ((w1, G.CACHE_NONE), (w2, G.CACHE_BLOCKS)):
        K = w.matrix()
        ent = G.Entries.gaussian(K.points, w.bandwidth, w.shift) if w.kernel == wl.GAUSSIAN else \
            G.Entries.imq(K.points, w.bandwidth, w.shift)
        h = G.compress(ent, G.default_params(**w.params(), cache_mode=cm))
        G.prepare(h, 256, prec)
        hs.append(h)
    Ws = [torch.from_numpy(w1.rhs(100).astype(np.float32)).cuda(),
          torch.from_numpy(w2.rhs(256).astype(np.float32)).cuda()]
    alone = []
    for h, W in zip(hs, Ws):
        U = torch.empty_like(W)
        G.evaluate(h, W, U, prec)
        G.synchronize(h)
        alone.append(U.clone())
    eng = G.Engine(prec, 1 << 30)
    Us = [torch.full_like(W, float("nan")) for W in Ws]
    for h, W, U in zip(hs, Ws, Us):
        eng.submit(h, W, U)
    eng.drain()
    for a, b in zip(alone, Us):
        assert torch.equal(a, b)
    eng.free()
