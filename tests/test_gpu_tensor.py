"""Tensor-core evaluation (tcgen05: TF32, BF16, split BF16x3 with FP32
accumulation) against the FP64 oracle on the same structure.

Tolerances follow the operand rounding: each MMA input is rounded to the
mode's format (unit roundoff u: TF32 2^-11, BF16 2^-9; split BF16 keeps
about 2^-16 of the FP32 value) and the result passes through up to four
rounded stages (N2S, S2S, S2N, L2L), so the relative Frobenius error is a
few u times the condition of the sums, kappa = || |K| |W| || / || K W ||:
TF32 <= 5e-3, BF16 <= 2e-2, BF16x3 <= 1e-4 at kappa <= 25 (the Gaussian
cases), scaled by kappa / 25 above it (an inverse multiquadric with random
right-hand sides cancels much more: kappa 180 for one column)."""
import os

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


def sum_condition(K, W):
    """kappa = || |K| |W| ||_F / || K W ||_F (dense K; the test sizes allow it)."""
    Kd = K.dense()
    return float(np.linalg.norm(np.abs(Kd) @ np.abs(W)) / np.linalg.norm(Kd @ W))


def tol(prec, K, W):
    return TOL[prec] * max(1.0, sum_condition(K, W) / 25.0)


CASES = [
    ("c2_recipe_n8192_r300", wl.scaled(wl.C2, 8192), 300, dict(knn_exact_max=20000)),
    ("ragged_n1000_r37", wl.scaled(wl.C1, 1000), 37, dict(leaf_size=32, callback=False)),
    ("paper_far_n1024_r130", wl.scaled(wl.C1, 1024), 130, dict(leaf_size=32, far=O.FAR_PAPER, budget=0.05,
                                                               callback=False)),
    ("hss_n512_r5", wl.scaled(wl.C1, 512), 5, dict(leaf_size=32, budget=0.0, callback=False)),
    ("tall_blocks_n3000_m400", wl.scaled(wl.C3, 3000), 64, dict(leaf_size=400, max_rank=300, tau=1e-6)),
    # degenerate shapes: one leaf (no skeletons, no far field), one column,
    # fewer points than one MMA tile row block
    ("single_leaf_n50_r7", wl.scaled(wl.C1, 50), 7, dict(leaf_size=64, callback=False)),
    ("imq_angle_n777_r1", wl.scaled(wl.C3, 777), 1, dict(leaf_size=50, max_rank=40, distance=O.ANGLE, tau=1e-4)),
    ("tiny_n9_r3", wl.scaled(wl.C1, 9), 3, dict(leaf_size=4, max_rank=2, callback=False)),
]


@pytest.mark.parametrize("prec", PRECS, ids=[NAMES[p] for p in PRECS])
@pytest.mark.parametrize("name,w,r,over", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_evaluate_matches_oracle(name, w, r, over, prec):
    over = dict(over)
    cb = over.pop("callback", None)
    h, st, K = both(w, callback=cb, **over)
    assert_same_structure(h, st)
    W = w.rhs(r)
    ref = O.evaluate(st, K, W)
    U = run(h, W, prec)
    assert np.all(np.isfinite(U))
    assert rel(U, ref) <= tol(prec, K, W), (rel(U, ref), sum_condition(K, W))
    assert_tensor_close(U, ref, O.evaluate_abs(st, K, W), abs_product(K, W), prec)


def test_tensor_core_is_deterministic_and_r_independent():
    w = wl.scaled(wl.C1, 2000)
    h, st, K = both(w, leaf_size=64, callback=False)
    W = w.rhs(200)
    a = run(h, W, G.PREC_BF16X3)
    b = run(h, W, G.PREC_BF16X3)
    assert np.array_equal(a, b)
    c = run(h, W[:, :70], G.PREC_BF16X3)   # fewer columns after more: same values
    assert np.array_equal(c, a[:, :70])


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_rows.npz")


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle rows not generated")
@pytest.mark.parametrize("prec", PRECS, ids=[NAMES[p] for p in PRECS])
def test_full_size_tensor_core_against_oracle_rows(prec):
    g = np.load(GOLDEN)
    w = wl.C2
    K = w.matrix()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), G.default_params(**w.params()))
    W = torch.from_numpy(w.rhs(512).astype(np.float32)).cuda()
    U = torch.empty_like(W)
    G.evaluate(h, W, U, prec)
    G.synchronize(h)
    assert g["u_oracle"].shape[1] == 512   # every r-tile of the launch is compared
    got = U[torch.from_numpy(g["rows"]).cuda()].double().cpu().numpy()
    assert rel(got, g["u_oracle"]) <= TOL[prec]
    assert_tensor_close(got, g["u_oracle"], g["u_abs"], g["u_kabs"], prec)
    # the configuration the benchmark times (autotuned) and every other one
    # the tuner measured give bitwise this result at full size
    ref = U.clone()
    t = G.autotune(h, 512, prec, None)
    for cfg in [(t["piece"], t["schedule"], t["order"])] + [(c["piece"], c["schedule"], c["order"])
                                                            for c in t["candidates"][::3]]:
        G.set_tc_config(h, prec, *cfg)
        U.fill_(float("nan"))
        G.evaluate(h, W, U, prec)
        G.synchronize(h)
        assert torch.equal(U, ref), cfg


@pytest.mark.parametrize("prec", [G.PREC_FP32, G.PREC_BF16X3], ids=["fp32", "bf16x3"])
def test_graph_replay_matches_direct_launches(prec):
    """Repeated calls with the same buffers are replayed from a CUDA graph;
    the result must equal the directly launched sequence bit for bit."""
    w = wl.scaled(wl.C1, 1500)
    h, st, K = both(w, leaf_size=64, callback=False)
    W = torch.from_numpy(w.rhs(96).astype(np.float32)).cuda()
    U = torch.empty_like(W)
    G.set_timing(h, True)  # timing forces direct launches
    G.evaluate(h, W, U, prec)
    G.synchronize(h)
    ref = U.clone()
    G.set_timing(h, False)
    for _ in range(4):  # calls 2.. replay the captured graph
        U.fill_(float("nan"))
        G.evaluate(h, W, U, prec)
        G.synchronize(h)
        assert torch.equal(U, ref)


def test_trim_keeps_tensor_core_results_and_rebuilds_cuda_core_stores():
    w = wl.scaled(wl.C1, 1200)
    h, st, K = both(w, leaf_size=64, callback=False)
    W = w.rhs(40)
    a = run(h, W, G.PREC_BF16X3)
    b32 = run(h, W, G.PREC_FP32)
    G.trim(h)
    assert np.array_equal(run(h, W, G.PREC_BF16X3), a)   # tiles kept
    assert np.array_equal(run(h, W, G.PREC_FP32), b32)   # stores rebuilt on demand


GOLDEN_C3 = os.path.join(os.path.dirname(__file__), "golden", "imq4d_n131072_r2048_rows.npz")


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(GOLDEN_C3), reason="oracle rows not generated")
def test_precision_workload_every_mode_against_oracle_rows():
    """IMQ kernel, 4-D uniform points, N = 131072, m = 256, s = 512 (ranks up
    to 512: tasks split across two MMA N tiles), tau 1e-6, r = 2048: every
    mode against the oracle's FP64 rows (all 2048 columns, written by
    tests/golden/make_rows.py), element by element in the tensor modes."""
    g = np.load(GOLDEN_C3)
    w = wl.C3
    K = w.matrix()
    h = G.compress(G.Entries.imq(K.points, w.bandwidth, w.shift), G.default_params(**w.params()))
    assert G.stats(h)["skel_total"] == int(g["skel_total"])
    W = torch.from_numpy(w.rhs(w.r).astype(np.float32)).cuda()
    U = torch.empty_like(W)
    rows = torch.from_numpy(g["rows"]).cuda()
    cols = g["u_oracle"].shape[1]
    for prec, tol in [(G.PREC_FP32, 1e-5)] + [(p, TOL[p]) for p in PRECS]:
        U.fill_(float("nan"))
        G.evaluate(h, W, U, prec)
        G.synchronize(h)
        got = U[rows][:, :cols].double().cpu().numpy()
        assert rel(got, g["u_oracle"]) <= tol, (prec, rel(got, g["u_oracle"]))
        assert_tensor_close(got, g["u_oracle"], g["u_abs"], g["u_kabs"], prec)
