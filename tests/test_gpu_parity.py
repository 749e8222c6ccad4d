"""GPU evaluation against the FP64 oracle, element by element, on the same
seeded inputs.  The native and the oracle compressions are checked to be the
same structure first (bit-exact integer decisions), so K~ is the same linear
map on both sides and the two evaluations must agree up to rounding:
<= 1e-12 relative in FP64 mode, <= 1e-5 in FP32 mode (FP32 rounding of K,
W and P and FP32 accumulation over a few thousand terms, ~1e-6 expected)."""
import os

import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import assert_same_structure, assert_tensor_close, both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def gpu_eval(h, W, prec, dtype, ld_pad=0):
    n, r = W.shape
    Wb = torch.zeros((n, r + ld_pad), dtype=dtype, device="cuda")
    Ub = torch.full((n, r + ld_pad), float("nan"), dtype=dtype, device="cuda")
    Wb[:, :r] = torch.from_numpy(W).to(dtype)
    Wt, Ut = Wb[:, :r], Ub[:, :r]
    G.evaluate(h, Wt, Ut, prec)
    torch.cuda.synchronize()
    if ld_pad:
        assert torch.isnan(Ub[:, r:]).all()  # nothing written past r
    return Ut.cpu().double().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check(U, ref, tol):
    assert np.all(np.isfinite(U))
    assert rel(U, ref) <= tol, rel(U, ref)
    assert np.abs(U - ref).max() <= 10 * tol * np.abs(ref).max()


FP64_CASES = [
    ("c1_callback_r16", wl.C1, 16, dict()),
    ("ragged_n1000_r37", wl.scaled(wl.C1, 1000), 37, dict(leaf_size=32, callback=False)),
    ("paper_far_n1024", wl.scaled(wl.C1, 1024), 5, dict(leaf_size=32, far=O.FAR_PAPER, budget=0.05,
                                                         callback=False)),
    ("hss_n512", wl.scaled(wl.C1, 512), 3, dict(leaf_size=32, budget=0.0, callback=False)),
    ("imq_angle_r1", wl.scaled(wl.C3, 777), 1, dict(leaf_size=50, max_rank=40, distance=O.ANGLE,
                                                    tau=1e-4)),
    ("generated_n1000", wl.scaled(wl.C1, 1000), 37, dict(leaf_size=32, callback=False,
                                                          cache_mode=G.CACHE_NONE)),
    ("single_leaf", wl.scaled(wl.C1, 50), 7, dict(leaf_size=64, callback=False)),
    ("ann_6d_n3000", wl.scaled(wl.C2, 3000), 64, dict(knn_exact_max=1000, leaf_size=64, max_rank=64)),
]


@pytest.mark.parametrize("name,w,r,over", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_evaluate_matches_oracle(name, w, r, over):
    over = dict(over)
    cb = over.pop("callback", None)
    cm = over.pop("cache_mode", None)
    h, st, K = both(w, callback=cb, cache_mode=cm, **over)
    assert_same_structure(h, st)
    W = w.rhs(r)
    ref = O.evaluate(st, K, W)
    check(gpu_eval(h, W, G.PREC_FP64, torch.float64), ref, FP64_TOL)


@pytest.mark.parametrize("cache_mode", [G.CACHE_BLOCKS, G.CACHE_NONE])
def test_fp32_evaluate_matches_oracle(cache_mode):
    w = wl.scaled(wl.C2, 8192)
    h, st, K = both(w, cache_mode=cache_mode, knn_exact_max=20000)
    assert_same_structure(h, st)
    W = w.rhs(100)
    ref = O.evaluate(st, K, W)
    check(gpu_eval(h, W.astype(np.float32), G.PREC_FP32, torch.float32, ld_pad=3), ref, FP32_TOL)


def test_full_rank_and_no_far_field_are_exact_on_gpu():
    w = wl.scaled(wl.C1, 600)
    K = w.matrix()
    W = w.rhs(9)
    dense = K.dense() @ W
    h1, _, _ = both(w, leaf_size=32, tau=0.0, max_rank=600, n_sample=600, callback=False)
    check(gpu_eval(h1, W, G.PREC_FP64, torch.float64), dense, FP64_TOL)
    h2, st2, _ = both(w, leaf_size=32, budget=2.0, kappa=600, callback=False)
    assert not st2.far
    check(gpu_eval(h2, W, G.PREC_FP64, torch.float64), dense, FP64_TOL)


def test_repeatable_host_buffers_and_checkpoint(tmp_path):
    w = wl.scaled(wl.C1, 1000)
    h, st, K = both(w, leaf_size=32, callback=False)
    W = w.rhs(16)
    a = gpu_eval(h, W, G.PREC_FP64, torch.float64)
    b = gpu_eval(h, W, G.PREC_FP64, torch.float64)
    assert np.array_equal(a, b)  # deterministic: fixed summation order, no atomics
    Uh = np.zeros_like(W)
    G.evaluate_host(h, W, Uh, G.PREC_FP64)
    assert np.array_equal(Uh, a)
    path = str(tmp_path / "s.bin")
    G.export(h, path)
    h2 = G.import_(path, G.Entries.gaussian(K.points, w.bandwidth, w.shift))
    assert np.array_equal(gpu_eval(h2, W, G.PREC_FP64, torch.float64), a)


def test_evaluate_argument_errors():
    w = wl.scaled(wl.C1, 300)
    h, _, _ = both(w, leaf_size=32, callback=False)
    W = torch.zeros((300, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GofmmError) as e:
        G.evaluate(h, W, torch.zeros_like(W), G.PREC_FP64)
    assert e.value.code == G.ERR_UNSUPPORTED
    with pytest.raises(G.GofmmError) as e:
        G.evaluate(h, W, W, G.PREC_FP32)
    assert e.value.code == G.ERR_ARG


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_rows.npz")


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle rows not generated")
def test_full_size_fp32_against_oracle_rows():
    """The throughput workload at full size (N = 65536, r = 512, FP32), in the
    configuration bench.py times: sampled rows against the oracle's rows
    (written by tests/golden/make_c2_rows.py), and the symmetry of K~."""
    g = np.load(GOLDEN)
    w = wl.C2
    K = w.matrix()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), G.default_params(**w.params()))
    assert G.stats(h)["skel_total"] == int(g["skel_total"])
    W = torch.from_numpy(w.rhs(512).astype(np.float32)).cuda()
    U = torch.empty_like(W)
    G.evaluate(h, W, U, G.PREC_FP32)
    rows = torch.from_numpy(g["rows"]).cuda()
    got = U[rows][:, : g["u_oracle"].shape[1]].double().cpu().numpy()
    assert rel(got, g["u_oracle"]) <= FP32_TOL
    assert_tensor_close(got, g["u_oracle"], g["u_abs"], g["u_kabs"], G.PREC_FP32)  # row by row, all 512 columns
    # same rows as the oracle => same error against the exact product
    assert abs(rel(got, g["u_exact"]) - rel(g["u_oracle"], g["u_exact"])) <= 1e-4
    # K~ symmetric: V^T (K~ W) == (K~ V)^T W
    V = torch.from_numpy(wl.scaled(wl.C2, w.n, w_seed=99).rhs(512).astype(np.float32)).cuda()
    KV = torch.empty_like(V)
    G.evaluate(h, V, KV, G.PREC_FP32)
    lhs = (V.double().T @ U.double())
    rhs = (KV.double().T @ W.double())
    assert float(torch.linalg.norm(lhs - rhs) / torch.linalg.norm(lhs)) <= 1e-5


@pytest.mark.parametrize("prec,dt", [(G.PREC_FP64, np.float64), (G.PREC_FP32, np.float32),
                                     (G.PREC_BF16X3, np.float32)], ids=["fp64", "fp32", "bf16x3"])
def test_host_buffer_pipeline_is_bitwise_the_device_evaluation(prec, dt):
    """Host buffers with r >= 256 run over 128-column chunks with the copies
    overlapped; columns are independent, so the result equals the
    device-buffer evaluation bit for bit (ragged last chunk, padded host
    leading dimensions)."""
    w = wl.scaled(wl.C1, 3000)
    h, st, K = both(w, leaf_size=64, callback=False)
    r = 300
    W = w.rhs(r).astype(dt)
    Wt = torch.from_numpy(W).cuda()
    Ut = torch.empty_like(Wt)
    G.evaluate(h, Wt, Ut, prec)
    G.synchronize(h)
    ref = Ut.cpu().numpy()
    Wpad = np.zeros((w.n, r + 5), dtype=dt)
    Wpad[:, :r] = W
    Upad = np.full((w.n, r + 7), np.nan, dtype=dt)
    G.evaluate_host(h, Wpad[:, :r], Upad[:, :r], prec)
    assert np.array_equal(Upad[:, :r], ref)
    assert np.all(np.isnan(Upad[:, r:]))  # nothing written past r
    if prec == G.PREC_FP64:
        assert np.linalg.norm(Upad[:, :r] - O.evaluate(st, K, W)) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec,dt,r", [(G.PREC_FP64, np.float64, 300), (G.PREC_BF16X3, np.float32, 300),
                                       (G.PREC_BF16X3, np.float32, 37)], ids=["fp64", "bf16x3", "bf16x3_r37"])
def test_host_async_calls_in_flight_are_bitwise_the_device_evaluation(prec, dt, r):
    """Several asynchronous host-buffer calls in flight at once (the two
    device staging slots alternate; r = 300 runs the two-chunk pipeline,
    r = 37 one chunk), then a synchronous call: each U bitwise the
    device-buffer evaluation of its W, final after synchronize."""
    w = wl.scaled(wl.C1, 3000)
    h, st, K = both(w, leaf_size=64, callback=False)
    Ws = [torch.from_numpy(wl.scaled(wl.C1, 3000, w_seed=10 + i).rhs(r).astype(dt)).pin_memory() for i in range(3)]
    refs = []
    for W in Ws:
        Wd = W.cuda()
        Ud = torch.empty_like(Wd)
        G.evaluate(h, Wd, Ud, prec)
        G.synchronize(h)
        refs.append(Ud.cpu().numpy())
    Us = [torch.full_like(W, float("nan")).pin_memory() for W in Ws]
    for W, U in zip(Ws, Us):
        G.evaluate_host_async(h, W.numpy(), U.numpy(), prec)
    G.synchronize(h)
    for U, ref in zip(Us, refs):
        assert np.array_equal(U.numpy(), ref)
    Ux = np.full((w.n, r), np.nan, dtype=dt)
    G.evaluate_host(h, Ws[1].numpy(), Ux, prec)  # a synchronous call after asynchronous ones
    assert np.array_equal(Ux, refs[1])
