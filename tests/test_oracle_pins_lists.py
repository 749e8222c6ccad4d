"""Pins of the oracle's near-list ballot, neighbour-based row sampling and
centroid scores against hand-derived values and explicit Gram vectors (not
against the oracle itself), and of its algorithmic flop count against a
count made by hand on a tiny structure."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _line_tree(n, depth, leaf_of=None):
    """A Tree over indices 0..n-1 in order: leaf b holds a contiguous run, and
    every inner node the union of its children."""
    nl = 1 << depth
    per = n // nl
    nodes = [None] * ((1 << (depth + 1)) - 1)
    for b in range(nl):
        nodes[nl - 1 + b] = np.arange(b * per, (b + 1) * per, dtype=np.int64)
    for h in range(nl - 2, -1, -1):
        nodes[h] = np.concatenate([nodes[2 * h + 1], nodes[2 * h + 2]])
    lo = np.arange(n, dtype=np.int64) // per
    return O.Tree(n, depth, nodes, np.arange(n, dtype=np.int64), lo)


# ------------------------------------------------------- near-list ballot ---
def test_near_ballot_hand_tallied():
    """§2.2 Alg. 3 with the ballot and eq. (budget): votes descending, ties to
    the smaller leaf, at most floor(budget N / m) others, then symmetrised.
    The expected lists were tallied by hand (tests/golden/near_ballot.json)."""
    g = json.load(open(os.path.join(GOLDEN, "near_ballot.json")))
    tree = _line_tree(g["n"], 3)
    assert int(math.floor(g["budget"] * g["n"] / g["leaf_size"])) == 2
    prm = O.Params(leaf_size=g["leaf_size"], budget=g["budget"], kappa=4)
    near = O.leaf_near(tree, np.array(g["knn"], dtype=np.int64), prm)
    assert [x.tolist() for x in near] == g["near"]
    # each list is its own ballot plus the leaves whose ballot chose it
    for b, bal in enumerate(g["ballot"]):
        chosen_by = [a for a, other in enumerate(g["ballot"]) if b in other and a != b]
        assert sorted(set(bal) | set(chosen_by)) == g["near"][b]


def test_near_ballot_budget_limits():
    """Budget 0 keeps every leaf alone (HSS, §3 "0% budget"); a budget above
    the number of leaves admits every voted leaf (the plain neighbour rule,
    'alpha and beta near if alpha meets N(beta)')."""
    g = json.load(open(os.path.join(GOLDEN, "near_ballot.json")))
    tree = _line_tree(g["n"], 3)
    knn = np.array(g["knn"], dtype=np.int64)
    near0 = O.leaf_near(tree, knn, O.Params(leaf_size=2, budget=0.0, kappa=4))
    assert [x.tolist() for x in near0] == [[b] for b in range(8)]
    nearall = O.leaf_near(tree, knn, O.Params(leaf_size=2, budget=1.0, kappa=4))
    voted = [set() for _ in range(8)]
    for i, row in enumerate(knn):
        for j in row:
            if j >= 0:
                voted[i // 2].add(int(j) // 2)
    for b in range(8):
        for a in list(voted[b]):
            voted[a].add(b)
    assert [x.tolist() for x in nearall] == [sorted(v) for v in voted]


# --------------------------------------------------- importance sampling ---
def _sampling_case():
    """Node 1 (indices 0..7) of a 16-index tree of depth 3 and a kappa = 3
    neighbour table.  Out-of-node neighbour counts, tallied by hand:
    9: 3, 12: 3, 10: 2, 11: 1, 14: 1; so by decreasing count with ties to
    the smaller index the order is 9, 12, 10, 11, 14."""
    tree = _line_tree(16, 3)
    knn = np.full((16, 3), -1, dtype=np.int64)
    rows = {0: [0, 9, 12], 1: [1, 9, 12], 2: [2, 9, 3], 3: [3, 10, 2],
            4: [4, 10, 5], 5: [5, 14, 4], 6: [6, 12, 7], 7: [7, 6, 11]}
    for i, r in rows.items():
        knn[i] = r
    return tree, knn


def test_sample_rows_neighbour_prefix_hand_counted():
    """§2.2 skeletonization: I' starts with the neighbours of alpha outside
    alpha, most frequent first (ties to the smaller index)."""
    tree, knn = _sampling_case()
    got = O.sample_rows(tree, knn, 1, O.Params(max_rank=64, n_sample=4, kappa=3))
    assert got.tolist() == [9, 12, 10, 11]
    got = O.sample_rows(tree, knn, 1, O.Params(max_rank=2, n_sample=0, kappa=3))  # |I'| = 2 s
    assert got.tolist() == [9, 12, 10, 11]
    got = O.sample_rows(tree, knn, 1, O.Params(max_rank=64, n_sample=5, kappa=3))
    assert got.tolist() == [9, 12, 10, 11, 14]


def test_sample_rows_uniform_tail_outside_node():
    """Past the neighbours, I' is filled by draws without replacement from
    the rest of the complement: never an index of alpha nor a repeat; the
    size is min(N - |alpha|, n_sample)."""
    tree, knn = _sampling_case()
    got = O.sample_rows(tree, knn, 1, O.Params(max_rank=64, n_sample=7, kappa=3))
    assert got[:5].tolist() == [9, 12, 10, 11, 14]
    assert set(got[5:].tolist()) <= {8, 13, 15} and len(set(got.tolist())) == 7
    got = O.sample_rows(tree, knn, 1, O.Params(max_rank=64, n_sample=100, kappa=3))
    assert got[:5].tolist() == [9, 12, 10, 11, 14] and sorted(got[5:].tolist()) == [8, 13, 15]


def test_sample_rows_tail_is_uniform():
    """Over many seeds every index of the rest is drawn with probability
    (tail size) / (rest size): leaf 0 (heap node 7, indices 0..7) of a
    64-index tree, 5 neighbours, 51 others, 10 drawn."""
    tree = _line_tree(64, 3)
    knn = np.full((64, 3), -1, dtype=np.int64)
    for i, j in enumerate([9, 9, 12, 12, 10, 14, 11, 9]):
        knn[i] = [i, j, -1]
    outside = np.array([9, 12, 10, 11, 14])
    rest = np.setdiff1d(np.arange(8, 64), outside)
    trials = 3000
    hits = np.zeros(64)
    for seed in range(trials):
        got = O.sample_rows(tree, knn, 7, O.Params(max_rank=64, n_sample=15, kappa=3, seed=seed))
        assert got[:5].tolist() == [9, 12, 10, 11, 14]
        assert not np.isin(got, np.arange(8)).any() and len(set(got.tolist())) == 15
        hits[got[5:]] += 1
    p = 10 / rest.size
    freq = hits[rest] / trials
    assert np.abs(freq - p).max() < 5 * math.sqrt(p * (1 - p) / trials)
    assert hits[np.arange(8)].sum() == 0


# ------------------------------------------------------- centroid scores ---
class _Gram:
    """K = Phi Phi^T with explicit Gram vectors Phi (rows)."""

    def __init__(self, Phi):
        self.Phi = Phi

    def __call__(self, I, J):
        return self.Phi[np.asarray(I).reshape(-1)] @ self.Phi[np.asarray(J).reshape(-1)].T

    def diag(self, I):
        P = self.Phi[np.asarray(I).reshape(-1)]
        return np.einsum("ij,ij->i", P, P)


def _gram_case(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 3)) + rng.standard_normal(3)
    Phi = np.hstack([X, 0.7 * np.eye(n)])   # phi_i = [x_i, 0.7 e_i]: K = X X^T + 0.49 I
    return Phi, _Gram(Phi)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_centroid_scores_against_gram_vectors(seed):
    """§2.1: c = mean of sampled Gram vectors; Gram-l2 score = |phi_i - c|^2
    - |c|^2, angle score = sin^2 of the angle between phi_i and c."""
    Phi, K = _gram_case(seed)
    idx = np.arange(3, 37)
    C = np.array([5, 9, 17, 30, 33])
    c = Phi[C].mean(axis=0)
    diagK = K.diag(np.arange(Phi.shape[0]))
    s2 = O.centroid_scores(K, diagK, idx, C, O.GRAM_L2)
    assert np.allclose(s2, np.sum((Phi[idx] - c) ** 2, axis=1) - c @ c, atol=1e-12)
    sa = O.centroid_scores(K, diagK, idx, C, O.ANGLE)
    cos = (Phi[idx] @ c) / (np.linalg.norm(Phi[idx], axis=1) * np.linalg.norm(c))
    assert np.allclose(sa, 1 - cos ** 2, atol=1e-12)


@pytest.mark.parametrize("kind", [O.GRAM_L2, O.ANGLE])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_metric_split_against_gram_vectors(kind, seed):
    """Alg. 1 computed on explicit Gram vectors: p farthest from the centroid
    of the whole node (n_c >= |alpha| samples every index), q farthest from
    p, median split of d_ip - d_iq (left child ceil(n/2), ties by index)."""
    Phi, K = _gram_case(seed)
    n = Phi.shape[0]
    idx = np.arange(n, dtype=np.int64)
    c = Phi.mean(axis=0)
    if kind == O.GRAM_L2:
        dist = lambda A, b: np.linalg.norm(A - b, axis=1)  # noqa: E731
    else:
        def dist(A, b):
            cs = (A @ b) / (np.linalg.norm(A, axis=1) * np.linalg.norm(b))
            return 1 - cs ** 2
    p = int(np.argmax(dist(Phi, c)))
    dp = dist(Phi, Phi[p])
    q = int(np.argmax(dp))
    v = dp - dist(Phi, Phi[q])
    order = sorted(range(n), key=lambda i: (v[i], i))
    left = np.sort(order[:(n + 1) // 2])
    lc, rc = O.metric_split(K, K.diag(idx), idx, kind, 7, 0, n)
    assert lc.tolist() == left.tolist()
    assert rc.tolist() == np.setdiff1d(idx, left).tolist()


# ------------------------------------------------------------ flop count ---
def _tiny_structure():
    """Depth-1 tree of 10 indices (leaves of 6 and 4), skeletons of 2 and 3,
    the two leaves far from each other (budget 0)."""
    nodes = [np.arange(10), np.arange(6), np.arange(6, 10)]
    tree = O.Tree(10, 1, nodes, np.arange(10), np.array([0] * 6 + [1] * 4))
    P = {1: np.ones((2, 6)), 2: np.ones((3, 4))}
    skel = {1: np.array([0, 1]), 2: np.array([6, 7, 8])}
    st = O.Structure(O.Params(leaf_size=6), tree, np.zeros((10, 1), dtype=np.int64),
                     [np.array([0]), np.array([1])], {1: np.array([2]), 2: np.array([1])},
                     skel, P, {})
    return st


def test_flop_count_hand_counted():
    """Table 2 with the real shapes; the identity part of every P is a copy,
    not arithmetic: N2S = S2N = 2 r (2 (6 - 2) + 3 (4 - 3)) = 22 r,
    S2S = 2 r (2 * 3 + 3 * 2) = 24 r, L2L = 2 r (6 * 6 + 4 * 4) = 104 r."""
    f = O.flop_count(_tiny_structure(), 5)
    assert f == dict(n2s=22 * 5, s2s=24 * 5, s2n=22 * 5, l2l=104 * 5, total=(22 + 24 + 22 + 104) * 5)
