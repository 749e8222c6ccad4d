"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(not against the oracle itself): closed forms, library routines, the paper's
worked example, exact special cases and brute force."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.spatial

import oracle as O
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prm(**kw):
    base = dict(leaf_size=32, max_rank=64, tau=1e-5, kappa=32, budget=0.03)
    base.update(kw)
    return O.Params(**base)


class LinearKernel:
    """K = X X^T + shift I: Gram vectors are known in closed form,
    phi_i = [x_i, sqrt(shift) e_i]."""

    def __init__(self, X, shift):
        self.X, self.shift = X, shift

    def __call__(self, I, J):
        I = np.asarray(I).reshape(-1)
        J = np.asarray(J).reshape(-1)
        out = self.X[I] @ self.X[J].T
        out[I[:, None] == J[None, :]] += self.shift
        return out

    def diag(self, I):
        I = np.asarray(I).reshape(-1)
        return np.array([self(np.array([i]), np.array([i]))[0, 0] for i in I])


# ----------------------------------------------------------------- inputs ---
def test_splitmix64_published_vectors():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    out = O.sm_outputs(0, 0, 3)
    assert [int(v) for v in out] == [int(x, 16) for x in g["state0_outputs"]]


def test_entries_match_library_distance():
    w = wl.scaled(wl.C2, 300)
    K = w.matrix()
    X = w.points()
    D2 = scipy.spatial.distance.cdist(X, X, "sqeuclidean")
    ref = np.exp(-D2 / (2 * 0.8 ** 2)) + 1e-2 * np.eye(300)
    assert np.allclose(K.dense(), ref, rtol=1e-13, atol=1e-15)
    np.linalg.cholesky(K.dense())  # SPD
    w3 = wl.scaled(wl.C3, 200)
    K3 = w3.matrix()
    X3 = w3.points()
    ref3 = 1.0 / np.sqrt(1 + scipy.spatial.distance.cdist(X3, X3, "sqeuclidean") / 0.25) + 1e-2 * np.eye(200)
    assert np.allclose(K3.dense(), ref3, rtol=1e-13, atol=1e-15)


# -------------------------------------------------------------- distances ---
def test_gram_distances_closed_form():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((20, 4))
    K = LinearKernel(X, 0.5)
    Phi = np.hstack([X, math.sqrt(0.5) * np.eye(20)])
    i, j = np.meshgrid(np.arange(20), np.arange(20), indexing="ij")
    kij = K(np.arange(20), np.arange(20))
    d = O.distance_values(O.GRAM_L2, K.diag(i.ravel()).reshape(20, 20),
                          K.diag(j.ravel()).reshape(20, 20), kij)
    ref = np.linalg.norm(Phi[:, None, :] - Phi[None, :, :], axis=2)
    assert np.allclose(d, ref, atol=1e-12)
    a = O.distance_values(O.ANGLE, K.diag(i.ravel()).reshape(20, 20),
                          K.diag(j.ravel()).reshape(20, 20), kij)
    cos = (Phi @ Phi.T) / np.outer(np.linalg.norm(Phi, axis=1), np.linalg.norm(Phi, axis=1))
    assert np.allclose(a, 1 - cos ** 2, atol=1e-12)  # sin^2 of the angle


# ------------------------------------------------------------------- tree ---
@pytest.mark.parametrize("n,m", [(256, 16), (300, 32), (97, 8)])
def test_tree_on_a_line_is_interval_partition(n, m):
    """On 1-D points with a wide Gaussian the Gram-l2 distance grows with
    |x_i - x_j|, so Alg. 1 picks the two ends and the median split of
    d_ip - d_iq cuts the node into a left and a right interval."""
    rng = np.random.default_rng(1)
    X = rng.random((n, 1))
    K = wl.KernelMatrix(wl.GAUSSIAN, X, 2.0, 1e-3)
    prm = _prm(leaf_size=m)
    tree = O.build_tree(K, K.diag(np.arange(n)), n, prm)
    assert tree.depth == O.tree_depth(n, m)
    sizes = [tree.node_idx[tree.leaf_node(b)].size for b in range(tree.n_leaves)]
    assert max(sizes) <= m and max(sizes) - min(sizes) <= 1
    assert sorted(tree.perm.tolist()) == list(range(n))
    order = np.argsort(X[:, 0])
    rank = np.empty(n, dtype=int)
    rank[order] = np.arange(n)
    ivals = sorted((rank[tree.node_idx[tree.leaf_node(b)]].min(),
                    rank[tree.node_idx[tree.leaf_node(b)]].max(), sizes[b])
                   for b in range(tree.n_leaves))
    pos = 0
    for lo, hi, sz in ivals:  # contiguous, non-overlapping runs of the x order
        assert lo == pos and hi == pos + sz - 1
        pos += sz


# -------------------------------------------------------------------- kNN ---
def test_knn_exact_matches_kdtree():
    """For a Gaussian kernel the Gram-l2 distance is a monotone function of
    the Euclidean distance, so the Gram kNN must equal a k-d tree query."""
    w = wl.scaled(wl.C1, 1500)
    K = w.matrix()
    X = w.points()
    c, _ = O.knn_exact(K, K.diag(np.arange(1500)), np.arange(1500), 1500, 16, O.GRAM_L2)
    _, ref = scipy.spatial.cKDTree(X).query(X, k=16)
    assert np.array_equal(np.sort(c, axis=1), np.sort(ref, axis=1))
    assert np.all(c[:, 0] == np.arange(1500))  # an index is its own nearest


def test_ann_reaches_target_recall():
    w = wl.scaled(wl.C2, 6000)
    K = w.matrix()
    prm = _prm(leaf_size=128, kappa=16, knn_exact_max=1000, seed=5)
    knn, iters, recall = O.all_nearest_neighbors(K, K.diag(np.arange(6000)), 6000, prm)
    assert 1 <= iters <= prm.ann_max_iter
    assert recall >= prm.ann_target_recall or iters == prm.ann_max_iter
    _, ref = scipy.spatial.cKDTree(w.points()).query(w.points(), k=16)
    true_recall = np.mean([np.intersect1d(knn[i], ref[i]).size / 16 for i in range(6000)])
    assert abs(true_recall - recall) < 0.1   # the sampled estimate is honest
    X = w.points()
    d = np.linalg.norm(X[knn] - X[:, None, :], axis=2)
    assert np.all(np.diff(d, axis=1) >= -1e-12)  # lists ordered by distance
    assert all(len(set(row)) == 16 for row in knn)


# ------------------------------------------------------------- near / far ---
def _small_structure(n=512, **kw):
    w = wl.scaled(wl.C1, n)
    K = w.matrix()
    prm = _prm(**kw)
    return K, w, O.compress(K, n, prm)


def test_near_lists_self_symmetric_budget():
    K, w, st = _small_structure(1024, leaf_size=32, budget=0.05)
    B = int(math.floor(0.05 * 1024 / 32))
    nl = st.tree.n_leaves
    for b in range(nl):
        assert b in st.near[b]
        for a in st.near[b]:
            assert b in st.near[int(a)]
    # every list is its own ballot (<= B others) plus the leaves whose ballot
    # chose it, so the off-diagonal entries number at most 2 B per leaf
    counts = np.array([len(x) - 1 for x in st.near])
    assert counts.sum() <= 2 * B * nl and counts.min() >= 1
    _, _, st0 = _small_structure(512, budget=0.0)
    assert all(list(x) == [b] for b, x in enumerate(st0.near))


def test_far_lists_symmetric_and_partition_once():
    K, w, st = _small_structure(1024, leaf_size=32, budget=0.05)
    tree = st.tree
    nl = tree.n_leaves
    cover = np.zeros((nl, nl), dtype=int)
    for b in range(nl):
        cover[b, st.near[b]] += 1
    for x, lst in st.far.items():
        for y in lst:
            assert x in st.far[int(y)]
            lx, hx = O.leaves_under(tree, x)
            ly, hy = O.leaves_under(tree, int(y))
            cover[lx:hx, ly:hy] += 1
    assert np.all(cover == 1)


def test_fig2_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "fig2_far_lists.json")))
    L = g["depth"]
    n = 1 << L
    nodes = [None] * ((1 << (L + 1)) - 1)
    tree = O.Tree(n, L, nodes, np.arange(n), np.arange(n))
    near = [np.array([b]) for b in range(n)]
    far = O.find_far(tree, near)
    for h, lst in g["find_far"].items():
        assert sorted(far[int(h)]) == lst
    O.merge_far_node(far, g["alpha"])
    for h, lst in g["after_merge_at_alpha"].items():
        assert sorted(far[int(h)]) == lst


# ---------------------------------------------------------------------- ID ---
def test_pivoted_qr_matches_lapack_geqp3():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 40)) * rng.uniform(0.1, 10, 40)[None, :]
    perm, R, s, rdiag = O.pivoted_qr(A, 40, 0.0)
    Q2, R2, p2 = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert s == 40
    assert np.array_equal(perm, p2)
    assert np.allclose(rdiag, np.abs(np.diag(R2)), rtol=1e-10)
    assert np.allclose(np.abs(R), np.abs(R2), atol=1e-10 * abs(R2[0, 0]))


def test_id_reconstruction_bound():
    """|A - A[:, skel] P|_F <= sqrt(n - s) * |R_{s,s}| <= sqrt(n - s) tau |R_00|."""
    w = wl.scaled(wl.C1, 600)
    K = w.matrix()
    rows = np.arange(0, 600, 2)
    cols = np.arange(1, 600, 6)
    A = K(rows, cols)
    for tau in (1e-2, 1e-4, 1e-6):
        perm, R, s, rdiag = O.pivoted_qr(A, 100, tau)
        P = O.interpolation_matrix(perm, R, s)
        err = np.linalg.norm(A - A[:, perm[:s]] @ P)
        assert err <= math.sqrt(A.shape[1] - s) * tau * rdiag[0] * (1 + 1e-8)
        assert np.allclose(P[:, perm[:s]], np.eye(s))
        ref = np.abs(np.diag(scipy.linalg.qr(A, pivoting=True, mode="r")[0]))[:s]
        assert np.allclose(rdiag, ref, rtol=1e-8)


# ---------------------------------------------------- exact special cases ---
@pytest.mark.parametrize("n", [512, 600])
def test_full_rank_is_exact(n):
    """tau = 0 and s >= N/2: every P is a permutation, so K~ = K (§8-style
    exactness: the ID is exact at full rank)."""
    K, w, st = _small_structure(n, tau=0.0, max_rank=n, n_sample=n)
    W = w.rhs(r=5)
    U = O.evaluate(st, K, W)
    ref = K.dense() @ W
    assert np.linalg.norm(U - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [512, 600])
def test_no_far_field_is_exact(n):
    K, w, st = _small_structure(n, budget=2.0, kappa=n)  # B >= leaves - 1
    assert not st.far
    W = w.rhs(r=3)
    U = O.evaluate(st, K, W)
    ref = K.dense() @ W
    assert np.linalg.norm(U - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("far", [O.FAR_SYMMETRIC, O.FAR_PAPER])
def test_evaluate_equals_telescoped_assembly(far):
    """Alg. 7's recursions (N2S postorder, S2N preorder) must reproduce the
    H-matrix built block by block from the telescoped bases; HSS (budget 0)
    and FMM (budget 5 %) lists, same-level and cross-level far pairs."""
    for budget in (0.0, 0.05):
        K, w, st = _small_structure(512, budget=budget, far=far, tau=1e-3)
        Kt = O.assemble(st, K)
        Ui = O.evaluate(st, K, np.eye(512))
        assert np.abs(Kt - Ui).max() <= 1e-13 * np.abs(Kt).max()
        if far == O.FAR_SYMMETRIC:
            assert np.abs(Ui - Ui.T).max() <= 1e-13 * np.abs(Ui).max()


def test_eps2_falls_with_tau():
    """Fig. 5 behaviour: smaller tau gives smaller eps2 (x3 slack)."""
    w = wl.scaled(wl.C1, 1024)
    K = w.matrix()
    W = w.rhs(r=4)
    ref = K.dense() @ W
    errs = []
    for tau in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
        st = O.compress(K, 1024, _prm(tau=tau, max_rank=256))
        U = O.evaluate(st, K, W)
        errs.append(np.linalg.norm(U - ref) / np.linalg.norm(ref))
    for a, b in zip(errs, errs[1:]):
        assert b <= 3 * a
    assert errs[-1] < 1e-6 and errs[0] > 1e-3


@pytest.mark.slow
def test_c1_against_dense_brute_force():
    """The FP64 workload at N = 4096: the whole pipeline against dense K W,
    and the 100-row estimate of eps2 (§3) against the full one."""
    w = wl.C1
    K = w.matrix()
    st = O.compress(K, w.n, O.Params(**w.params()))
    W = w.rhs()
    U = O.evaluate(st, K, W)
    ref = K.dense() @ W
    full = np.linalg.norm(U - ref) / np.linalg.norm(ref)
    rows = wl.sample_rows(w.n)
    est = O.eps2(U[rows], O.dense_rows(K, rows, W))
    assert full < 1e-2            # s = 64 caps the rank below what tau asks
    assert 0.3 < est / full < 3.0


def test_path_restricted_rows_equal_full_evaluation():
    """evaluate_leaves follows the same tasks along root-to-leaf paths; it
    must reproduce the rows of the full Alg. 7 evaluation (HSS and FMM
    lists, cross-level far pairs)."""
    for far in (O.FAR_SYMMETRIC, O.FAR_PAPER):
        K, w, st = _small_structure(1024, leaf_size=32, budget=0.05, far=far)
        W = w.rhs(r=6)
        U = O.evaluate(st, K, W)
        got = O.evaluate_leaves(st, K, W, [0, 5, 31])
        for b, rows in got.items():
            idx = st.tree.node_idx[st.tree.leaf_node(b)]
            assert np.abs(rows - U[idx]).max() <= 1e-13 * np.abs(U).max()
