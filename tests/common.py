"""Shared test helpers: build the same compressed matrix with the native
library and with the oracle, and compare them."""
import numpy as np

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl


def native_entries(w: wl.Workload, K=None, callback=None):
    K = K if K is not None else w.matrix()
    use_cb = w.entries_via_callback if callback is None else callback
    if use_cb:
        return G.Entries.callback(w.n, K)
    if w.kernel == wl.GAUSSIAN:
        return G.Entries.gaussian(K.points, w.bandwidth, w.shift)
    return G.Entries.imq(K.points, w.bandwidth, w.shift)


_DIST = {O.GRAM_L2: G.DIST_GRAM_L2, O.ANGLE: G.DIST_ANGLE, O.LEXICOGRAPHIC: G.DIST_LEXICOGRAPHIC,
         O.RANDOM: G.DIST_RANDOM}
_FAR = {O.FAR_SYMMETRIC: G.FAR_SYMMETRIC, O.FAR_PAPER: G.FAR_PAPER}


def both(w: wl.Workload, callback=None, cache_mode=None, **over):
    """(native handle, oracle structure, K) for workload w with overrides."""
    K = w.matrix()
    prm = O.Params(**w.params(**over))
    nat = dict(leaf_size=prm.leaf_size, max_rank=prm.max_rank, tau=prm.tau, budget=prm.budget,
               kappa=prm.kappa, distance=_DIST[prm.distance], far_mode=_FAR[prm.far],
               n_centroid=prm.n_centroid, n_sample=prm.n_sample, seed=prm.seed,
               knn_exact_max=prm.knn_exact_max, ann_max_iter=prm.ann_max_iter,
               ann_target_recall=prm.ann_target_recall)
    if cache_mode is not None:
        nat["cache_mode"] = cache_mode
    h = G.compress(native_entries(w, K, callback), G.default_params(**nat))
    st = O.compress(K, w.n, prm)
    return h, st, K


def assert_same_structure(h, st, p_rtol=1e-8):
    s = G.structure(h)
    tree = st.tree
    assert s["depth"] == tree.depth
    assert np.array_equal(s["perm"], tree.perm)
    assert len(s["near"]) == len(st.near)
    for a, b in zip(s["near"], st.near):
        assert np.array_equal(a, b)
    nn = (2 << tree.depth) - 1
    for node in range(nn):
        assert np.array_equal(s["far"][node], st.far.get(node, np.zeros(0, dtype=np.int64))), node
    for node in range(1, nn):
        assert np.array_equal(s["skel"][node], st.skel[node]), node
        scale = max(1.0, np.abs(st.P[node]).max())
        assert np.abs(s["P"][node] - st.P[node]).max() <= p_rtol * scale, node
    return s


# ------------------------------------------------ tensor-precision bounds ---
# Relative bounds at a sum condition kappa = || |K| |W| || / || K~ W || <= 25,
# scaled by kappa / 25 above it (the rule of the whole-block Frobenius checks,
# applied here to every row with that row's own kappa).
TC_TOL = {G.PREC_FP32: 1e-5, G.PREC_TF32: 5e-3, G.PREC_BF16: 2e-2, G.PREC_BF16X3: 1e-4}
# Element-wise unit: |U - U_oracle|_ij <= c * (|P|, |K|, |W| evaluation)_ij,
# the oracle's Alg. 7 on absolute values (oracle.evaluate_abs).  To first
# order every stage (N2S, S2S, S2N, L2L) adds at most about 3 u in that
# scale: both MMA operands rounded to the mode's format (unit roundoff u:
# TF32 2^-11, BF16 2^-9) and the stage's output rounded again for the next
# stage; four stages give 12 u.  Split BF16x3 keeps x to about 2^-18 |x|
# (hi + lo) and drops lo*lo (2^-18), so four stages stay below 2^-14, and the
# FP32 accumulation of up to ~1000 MMA partial sums adds about 2^-14: 2^-13.
# (That scale carries |T| of every level, so at large N it is loose; the
# row check below is the sharp one.)
TC_ELEM = {G.PREC_TF32: 12 * 2.0 ** -11, G.PREC_BF16: 12 * 2.0 ** -9, G.PREC_BF16X3: 2.0 ** -13}


def abs_product(K, W):
    """|K| |W| from the dense matrix (test sizes only)."""
    return np.abs(K.dense()) @ np.abs(W)


def assert_tensor_close(U, ref, uabs, kabs, prec, kappa_ref=25.0):
    """Result U against the oracle's FP64 rows `ref`: element by element
    against the first-order rounding scale `uabs` (oracle.evaluate_abs of
    the same rows; tensor precisions only), and row by row in the relative
    norm, each row's bound scaled by its own sum condition
    || (|K| |W|)_i || / || ref_i || from `kabs` (rows of |K| |W|), so that one
    wrong row or tile cannot hide in the norm of the whole block."""
    U = np.asarray(U, dtype=np.float64)
    assert U.shape == ref.shape == uabs.shape == kabs.shape
    assert np.all(np.isfinite(U))
    err = np.abs(U - ref)
    # FP32 on the CUDA cores: no element-wise bound (its sums of thousands
    # of terms have a worst-case bound far above any useful tolerance)
    bound = TC_ELEM.get(prec, np.inf) * uabs
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float((err / np.maximum(bound, 1e-300)).max()))
    rn = np.linalg.norm(ref, axis=1)
    rerr = np.linalg.norm(U - ref, axis=1) / np.maximum(rn, 1e-300)
    rkappa = np.linalg.norm(kabs, axis=1) / np.maximum(rn, 1e-300)
    rtol = TC_TOL[prec] * np.maximum(1.0, rkappa / kappa_ref)
    worst = int(np.argmax(rerr / rtol))
    assert np.all(rerr <= rtol), (float(rerr[worst]), float(rtol[worst]), worst)
    return float((err / np.maximum(bound, 1e-300)).max()), float((rerr / rtol).max())
