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
