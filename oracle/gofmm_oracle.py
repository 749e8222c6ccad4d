"""Plain, slow, FP64 GOFMM: compression (tree, neighbours, near/far lists,
skeletons) and evaluation, written step by step from the paper.

TEST INFRASTRUCTURE -- only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module.

Every function names the passage it follows (section, algorithm, table or
equation of the paper).  Where the paper is silent or ambiguous the reading
taken is stated in the docstring; the same readings are listed in the design
notes of the repository.

Input: an entry routine ``K(I, J) -> ndarray`` (plus ``K.diag(I)``) -- the
only input the method needs (§1, problem statement).  Points are never seen.

Pinning (tests/test_oracle_pins*.py): dense brute force K.W, exactness at
full rank and with no far field, the explicitly assembled H-matrix of the
telescoping formula, symmetry, the Fig. 2 worked example of FindFar/MergeFar,
kNN against a k-d tree, pivoted QR against LAPACK GEQP3, the tree split on
1-D points, the eps2-versus-tau trend, a hand-tallied near-list ballot
(votes, ties, budget, symmetrisation), hand-counted importance-sampled rows
I' and the uniformity of their tail, the centroid scores and Alg. 1 split
recomputed on explicit Gram vectors (Gram-l2 and angle), and a hand-counted
flop tally.  Each of these pins fails when the corresponding step is
mutated (ballot or sampling order reversed, ties flipped, the self vote or
the node's own indices kept, a centroid-score term changed).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np
import scipy.linalg

# distance / partitioning modes (§2.1 "Three measures of distance", §3 list of
# partitionings)
GRAM_L2 = "kernel"      # d_ij^2 = K_ii + K_jj - 2 K_ij
ANGLE = "angle"         # d_ij = 1 - K_ij^2 / (K_ii K_jj)
LEXICOGRAPHIC = "lexicographic"
RANDOM = "random"

# far-list construction
FAR_SYMMETRIC = "symmetric"   # same-level dual traversal (symmetric K~)
FAR_PAPER = "paper"           # Alg. 4 FindFar + Alg. 5 MergeFar, literally

# purposes of the seeded random streams
_P_CENTROID = 1
_P_ANN_SPLIT = 2
_P_ANN_RECALL = 3
_P_SAMPLE = 4
_P_RANDOM_PERM = 5

# --------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea, Flood, "Fast
# splittable pseudorandom number generators", OOPSLA 2014).  The i-th output
# of a generator whose state starts at `key` is mix64(key + (i+1)*GAMMA).
# The method's random choices (centroid samples, random projections, row
# samples) are drawn from streams keyed by (seed, purpose, id).
# --------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sm_outputs(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream at `key`."""
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + (i + np.uint64(1)) * _GAMMA)


def stream_key(seed: int, purpose: int, sub: int) -> int:
    tag = (purpose << 40) | sub
    return int(sm_outputs(seed & 0xFFFFFFFFFFFFFFFF, tag, 1)[0])


def partial_shuffle(arr: np.ndarray, k: int, key: int) -> np.ndarray:
    """First k entries of a Fisher-Yates shuffle of `arr` driven by the
    stream `key`: step t swaps position t with t + (u_t mod (n - t))."""
    a = np.array(arr, copy=True)
    n = a.size
    k = min(k, n)
    u = sm_outputs(key, 0, k)
    for t in range(k):
        j = t + int(u[t] % np.uint64(n - t))
        a[t], a[j] = a[j], a[t]
    return a[:k]


# --------------------------------------------------------------------------
# Parameters and results
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    leaf_size: int = 64          # m
    max_rank: int = 64           # s (maximum skeleton size)
    tau: float = 1e-5            # adaptive ID tolerance
    kappa: int = 32              # neighbours per index
    budget: float = 0.03         # direct-evaluation budget (§2.2 eq. budget)
    distance: str = GRAM_L2
    far: str = FAR_SYMMETRIC
    n_centroid: int = 32         # n_c of the centroid sample (Alg. 1)
    n_sample: int = 0            # |I'| target; 0 means 2 * max_rank
    seed: int = 0
    knn_exact_max: int = 16384   # exhaustive kNN up to this N, else ANN
    ann_max_iter: int = 10       # §2.2: stop after 10 iterations ...
    ann_target_recall: float = 0.8  # ... or 80 % accuracy


@dataclasses.dataclass
class Tree:
    """Balanced binary tree in heap numbering (root 0, children 2h+1, 2h+2),
    all leaves at depth `depth`."""
    n: int
    depth: int
    node_idx: List[np.ndarray]   # sorted original indices of every node
    perm: np.ndarray             # tree position -> original index
    leaf_of: np.ndarray          # original index -> leaf number (0-based)

    @property
    def n_leaves(self) -> int:
        return 1 << self.depth

    def leaf_node(self, b: int) -> int:
        return (1 << self.depth) - 1 + b

    def level_nodes(self, lvl: int) -> range:
        return range((1 << lvl) - 1, (1 << (lvl + 1)) - 1)

    def offset(self, h: int) -> int:
        """First tree position of node h."""
        lvl = int(math.floor(math.log2(h + 1)))
        first_leaf = (h + 1 - (1 << lvl)) << (self.depth - lvl)
        off = 0
        for b in range(first_leaf):
            off += self.node_idx[self.leaf_node(b)].size
        return off


@dataclasses.dataclass
class Structure:
    params: Params
    tree: Tree
    knn: np.ndarray                      # (N, kappa) neighbour indices
    near: List[np.ndarray]               # per leaf number: sorted leaf numbers
    far: Dict[int, np.ndarray]           # heap id -> sorted heap ids
    skel: Dict[int, np.ndarray]          # heap id -> skeleton (original indices, pivot order)
    P: Dict[int, np.ndarray]             # heap id -> s x ncols interpolation matrix
    rdiag: Dict[int, np.ndarray]         # heap id -> |R_kk| of the pivoted QR (diagnostic)
    ann_iters: int = 0
    ann_recall: float = 1.0


# --------------------------------------------------------------------------
# §2.1 distances from three entries
# --------------------------------------------------------------------------
def distance_values(kind: str, kii, kjj, kij):
    """d_ij for the Gram-l2 distance (d^2 = K_ii + K_jj - 2 K_ij, clamped at 0
    before the square root) or the Gram-angle distance
    (d = 1 - K_ij^2 / (K_ii K_jj)), §2.1."""
    if kind == GRAM_L2:
        d2 = (kii + kjj) - 2.0 * kij
        return np.sqrt(np.maximum(d2, 0.0))
    if kind == ANGLE:
        return 1.0 - (kij * kij) / (kii * kjj)
    raise ValueError(kind)


def knn_key(kind: str, kii, kjj, kij):
    """Monotone stand-in for d_ij used to rank neighbours: the clamped d^2 for
    Gram-l2 (same order as d), d itself for the angle distance."""
    if kind == GRAM_L2:
        return np.maximum((kii + kjj) - 2.0 * kij, 0.0)
    if kind == ANGLE:
        return 1.0 - (kij * kij) / (kii * kjj)
    raise ValueError(kind)


def metric_of(distance: str) -> str:
    """Distance used wherever one is needed (neighbour search, splits): the
    angle distance when chosen, the Gram-l2 distance otherwise -- the
    lexicographic and random partitionings still need neighbours for the
    near lists and the row sampling (reading: §3 lists them as
    partitionings only)."""
    return ANGLE if distance == ANGLE else GRAM_L2


def tree_depth(n: int, m: int) -> int:
    """Reading of §2.1 "splitting terminates at leaf size m" for a complete
    tree: the depth is the smallest L with ceil(n / 2^L) <= m, and every node
    above depth L is split."""
    L = 0
    while -(-n // (1 << L)) > m:
        L += 1
    return L


def _median_split(idx: np.ndarray, v: np.ndarray):
    """medianSplit of Alg. 1: order by (v, original index); the left child
    takes the first ceil(n/2)."""
    order = np.lexsort((idx, v))
    half = -(-idx.size // 2)
    return np.sort(idx[order[:half]]), np.sort(idx[order[half:]])


def centroid_scores(K, diagK, idx, C, kind):
    """Distance of every index of the node to the sampled centroid
    c = (1/n_c) sum_{j in C} phi_j (§2.1, "Tree partitioning"), from entries
    only: d(i, c)^2 - |c|^2 = K_ii - (2/n_c) sum_{j in C} K_ij for the
    Gram-l2 distance (the constant |c|^2 is dropped: it does not move the
    argmax), and d(i, c) = 1 - (phi_i, c)^2 / (|phi_i|^2 |c|^2) with
    (phi_i, c) = (1/n_c) sum_j K_ij and |c|^2 = (1/n_c^2) sum_{j,k} K_jk for
    the angle distance."""
    nc = C.size
    Kc = K(idx, C)
    S = np.zeros(idx.size)
    for t in range(nc):
        S = S + Kc[:, t]
    kii = diagK[idx]
    if kind == GRAM_L2:
        score = kii - 2.0 * S / nc
    else:
        Kcc = K(C, C)
        acc = 0.0
        for t in range(nc):
            for u in range(nc):
                acc += Kcc[t, u]
        cc = acc / (nc * nc)
        a = S / nc
        score = 1.0 - (a * a) / (kii * cc)
    return score


def metric_split(K, diagK, idx, kind, seed, h, n_centroid):
    """Alg. 1 (metricSplit) with the sampled centroid of §2.1.

    The centroid is taken over n_c indices drawn from the node;
    p = argmax_i d(i, c) (`centroid_scores`), q = argmax_i d(i, p), split on
    d_ip - d_iq.  Ties of an argmax go to the smallest original index.
    """
    nc = min(n_centroid, idx.size)
    C = partial_shuffle(idx, nc, stream_key(seed, _P_CENTROID, h))
    kii = diagK[idx]
    score = centroid_scores(K, diagK, idx, C, kind)
    p = int(idx[int(np.argmax(score))])
    dp = distance_values(kind, kii, diagK[p], K(idx, [p])[:, 0])
    q = int(idx[int(np.argmax(dp))])
    dq = distance_values(kind, kii, diagK[q], K(idx, [q])[:, 0])
    return _median_split(idx, dp - dq)


def random_split(K, diagK, idx, kind, key):
    """Random projection split used by the neighbour search (§2.1, last
    paragraph): as Alg. 1 but p and q are drawn at random (q != p)."""
    n = idx.size
    u = sm_outputs(key, 0, 64)
    p = int(idx[int(u[0] % np.uint64(n))])
    t = 1
    q = p
    while q == p:
        if t >= u.size:
            u = np.concatenate([u, sm_outputs(key, u.size, 64)])
        q = int(idx[int(u[t] % np.uint64(n))])
        t += 1
    kii = diagK[idx]
    dp = distance_values(kind, kii, diagK[p], K(idx, [p])[:, 0])
    dq = distance_values(kind, kii, diagK[q], K(idx, [q])[:, 0])
    return _median_split(idx, dp - dq)


def build_tree(K, diagK, n: int, prm: Params, split=None) -> Tree:
    """PRE-order SPLI over a balanced binary tree (§2.2, Alg. 2 step 4).

    `split(idx, h)` overrides the splitter (used for the random projection
    trees of the neighbour search)."""
    L = tree_depth(n, prm.leaf_size)
    nodes: List[Optional[np.ndarray]] = [None] * ((1 << (L + 1)) - 1)
    nodes[0] = np.arange(n, dtype=np.int64)
    rank = None
    if prm.distance == RANDOM and split is None:
        rank = np.empty(n, dtype=np.int64)
        rank[partial_shuffle(np.arange(n, dtype=np.int64), n,
                             stream_key(prm.seed, _P_RANDOM_PERM, 0))] = np.arange(n)
    for lvl in range(L):
        for h in range((1 << lvl) - 1, (1 << (lvl + 1)) - 1):
            idx = nodes[h]
            if split is not None:
                lc, rc = split(idx, h)
            elif prm.distance == LEXICOGRAPHIC:
                half = -(-idx.size // 2)
                lc, rc = idx[:half], idx[half:]
            elif prm.distance == RANDOM:
                lc, rc = _median_split(idx, rank[idx].astype(np.float64))
            else:
                lc, rc = metric_split(K, diagK, idx, prm.distance, prm.seed, h,
                                      prm.n_centroid)
            nodes[2 * h + 1], nodes[2 * h + 2] = lc, rc
    leaves = nodes[(1 << L) - 1:]
    perm = np.concatenate(leaves).astype(np.int64)
    leaf_of = np.empty(n, dtype=np.int64)
    for b, lf in enumerate(leaves):
        leaf_of[lf] = b
    return Tree(n, L, nodes, perm, leaf_of)


# --------------------------------------------------------------------------
# §2.2 neighbour lists N(i)
# --------------------------------------------------------------------------
def _select_kappa(keys: np.ndarray, cols: np.ndarray, kappa: int):
    """Per row, the kappa smallest (key, col) pairs, ordered by (key, col)."""
    o1 = np.argsort(cols, axis=1, kind="stable")
    k1 = np.take_along_axis(keys, o1, axis=1)
    c1 = np.take_along_axis(cols, o1, axis=1)
    o2 = np.argsort(k1, axis=1, kind="stable")
    k2 = np.take_along_axis(k1, o2, axis=1)
    c2 = np.take_along_axis(c1, o2, axis=1)
    # equal columns carry equal keys, so duplicates are adjacent now
    keep = np.ones_like(c2, dtype=bool)
    keep[:, 1:] = c2[:, 1:] != c2[:, :-1]
    rank = np.cumsum(keep, axis=1) - 1
    sel = keep & (rank < kappa)
    rows = c2.shape[0]
    out_c = c2[sel].reshape(rows, kappa)
    out_k = k2[sel].reshape(rows, kappa)
    return out_c, out_k


def knn_exact(K, diagK, rows: np.ndarray, n: int, kappa: int, kind: str, block=512):
    """Exhaustive kappa-nearest neighbours (index i counts as its own nearest
    neighbour), ordered by (distance, index)."""
    rows = np.asarray(rows, dtype=np.int64)
    allj = np.arange(n, dtype=np.int64)
    out_c = np.empty((rows.size, kappa), dtype=np.int64)
    out_k = np.empty((rows.size, kappa))
    for b0 in range(0, rows.size, block):
        r = rows[b0:b0 + block]
        D = knn_key(kind, diagK[r][:, None], diagK[None, :], K(r, allj))
        part = np.argpartition(D, kappa - 1, axis=1)[:, :kappa]
        thr = np.take_along_axis(D, part, axis=1).max(axis=1)
        for t in range(r.size):
            cand = np.nonzero(D[t] <= thr[t])[0]
            o = np.lexsort((cand, D[t, cand]))[:kappa]
            out_c[b0 + t] = cand[o]
            out_k[b0 + t] = D[t, cand[o]]
    return out_c, out_k


def all_nearest_neighbors(K, diagK, n: int, prm: Params):
    """Neighbour search of Alg. 2 steps 1-3 and §2.2 ("Index nearest
    neighbor list"): exhaustive when n <= knn_exact_max; otherwise repeated
    random projection trees with exhaustive search inside each leaf, merged
    into the running kappa-best lists, until the recall on 100 sampled
    indices reaches the target or the iteration limit is hit.  Returns
    (neighbours, iterations, recall)."""
    kappa = min(prm.kappa, n)
    if n <= prm.knn_exact_max:
        c, _ = knn_exact(K, diagK, np.arange(n), n, kappa, metric_of(prm.distance))
        return c, 0, 1.0
    cur_c = np.full((n, kappa), -1, dtype=np.int64)
    cur_k = np.full((n, kappa), np.inf)
    sample = np.sort(partial_shuffle(np.arange(n, dtype=np.int64), min(100, n),
                                     stream_key(prm.seed, _P_ANN_RECALL, 0)))
    exact_c, _ = knn_exact(K, diagK, sample, n, kappa, metric_of(prm.distance))
    recall = 0.0
    it = 0
    for it in range(1, prm.ann_max_iter + 1):
        def split(idx, h, _it=it):
            return random_split(K, diagK, idx, metric_of(prm.distance),
                                stream_key(prm.seed, _P_ANN_SPLIT, (_it << 24) | h))
        tr = build_tree(K, diagK, n, prm, split=split)
        for b in range(tr.n_leaves):
            lf = tr.node_idx[tr.leaf_node(b)]
            D = knn_key(metric_of(prm.distance), diagK[lf][:, None], diagK[lf][None, :], K(lf, lf))
            # unfilled slots carry distinct placeholder ids >= n and an
            # infinite key, so they sort after every real candidate
            cc = np.where(cur_c[lf] < 0, n + np.arange(kappa)[None, :], cur_c[lf])
            cols = np.concatenate([cc, np.broadcast_to(lf, (lf.size, lf.size))], axis=1)
            keys = np.concatenate([cur_k[lf], D], axis=1)
            c, k = _select_kappa(keys, cols, kappa)
            c = np.where(c >= n, -1, c)
            cur_c[lf], cur_k[lf] = c, k
        hits = 0
        for t, i in enumerate(sample):
            hits += np.intersect1d(cur_c[i], exact_c[t]).size
        recall = hits / (sample.size * kappa)
        if recall >= prm.ann_target_recall:
            break
    return cur_c, it, recall


# --------------------------------------------------------------------------
# §2.2 near and far lists
# --------------------------------------------------------------------------
def leaf_near(tree: Tree, knn: np.ndarray, prm: Params) -> List[np.ndarray]:
    """Alg. 3 (LeafNear) with the ballot and budget of §2.2 eq. (budget), then
    symmetrised.

    Readings: a leaf is always near itself; each occurrence of an index of
    leaf a among the neighbours of the indices of leaf b is one vote for a;
    at most floor(budget * N / m) other leaves are admitted, in order of
    decreasing votes (ties to the smaller leaf number), only leaves with at
    least one vote are candidates; symmetrisation (a in Near(b) => b in
    Near(a)) runs after the budget and may exceed it."""
    nl = tree.n_leaves
    B = int(math.floor(prm.budget * tree.n / prm.leaf_size))
    near = []
    for b in range(nl):
        lf = tree.node_idx[tree.leaf_node(b)]
        nb = knn[lf].ravel()
        votes = np.bincount(tree.leaf_of[nb[nb >= 0]], minlength=nl)
        votes[b] = 0
        cand = np.nonzero(votes)[0]
        order = np.lexsort((cand, -votes[cand]))
        near.append(set([b]) | set(int(a) for a in cand[order[:B]]))
    for b in range(nl):
        for a in list(near[b]):
            near[a].add(b)
    return [np.array(sorted(s), dtype=np.int64) for s in near]


def far_symmetric(tree: Tree, near: List[np.ndarray]) -> Dict[int, np.ndarray]:
    """Far lists by a same-level dual traversal (reading of Algs. 4-5 that keeps
    K~ symmetric, §1 "GOFMM guarantees symmetry"): nodes X != Y on one level
    are far iff no leaf below X is near a leaf below Y while their parents
    are not far.  Far(X) contains Y iff Far(Y) contains X, and the near leaf
    pairs plus the far pairs cover every block of K exactly once."""
    L = tree.depth
    nl = tree.n_leaves
    nm = [None] * (L + 1)
    m = np.zeros((nl, nl), dtype=bool)
    for b in range(nl):
        m[b, near[b]] = True
    nm[L] = m
    for lvl in range(L - 1, -1, -1):
        c = nm[lvl + 1]
        k = c.shape[0] // 2
        nm[lvl] = (c[0::2, 0::2] | c[0::2, 1::2] | c[1::2, 0::2] | c[1::2, 1::2]).reshape(k, k)
    far: Dict[int, np.ndarray] = {}
    for lvl in range(1, L + 1):
        base = (1 << lvl) - 1
        cnt = 1 << lvl
        for x in range(cnt):
            ys = [y for y in range(cnt) if (not nm[lvl][x, y]) and nm[lvl - 1][x // 2, y // 2]]
            if ys:
                far[base + x] = np.array([base + y for y in ys], dtype=np.int64)
    return far


def leaves_under(tree: Tree, h: int):
    lvl = int(math.floor(math.log2(h + 1)))
    first = (h + 1 - (1 << lvl)) << (tree.depth - lvl)
    return first, first + (1 << (tree.depth - lvl))


def find_far(tree: Tree, near: List[np.ndarray]) -> Dict[int, set]:
    """Alg. 4 (FindFar) from the root for every leaf beta: a visited node that
    contains a leaf of Near(beta) is descended into, any other node joins
    Far(beta).  Returns the leaf lists before merging."""
    n_nodes = (1 << (tree.depth + 1)) - 1
    far = {h: set() for h in range(n_nodes)}

    def visit(beta_node, h, nearset):
        lo, hi = leaves_under(tree, h)
        if any(lo <= a < hi for a in nearset):
            if 2 * h + 1 < n_nodes:
                visit(beta_node, 2 * h + 1, nearset)
                visit(beta_node, 2 * h + 2, nearset)
        else:
            far[beta_node].add(h)

    for b in range(tree.n_leaves):
        visit(tree.leaf_node(b), 0, set(int(a) for a in near[b]))
    return far


def merge_far_node(far: Dict[int, set], h: int) -> None:
    """One MergeFar step (Alg. 5) at inner node h: Far(h) gains
    Far(l) & Far(r), which leaves both children."""
    both = far[2 * h + 1] & far[2 * h + 2]
    far[h] |= both
    far[2 * h + 1] -= both
    far[2 * h + 2] -= both


def far_paper(tree: Tree, near: List[np.ndarray]) -> Dict[int, np.ndarray]:
    """Alg. 4 for every leaf followed by Alg. 5 (MergeFar) in postorder from
    the root, literally."""
    far = find_far(tree, near)
    n_nodes = len(far)

    def merge(h):
        if 2 * h + 1 >= n_nodes:
            return
        merge(2 * h + 1)
        merge(2 * h + 2)
        merge_far_node(far, h)

    merge(0)
    return {h: np.array(sorted(s), dtype=np.int64) for h, s in far.items() if s}


# --------------------------------------------------------------------------
# §2.2 skeletonization: adaptive interpolative decomposition
# --------------------------------------------------------------------------
def pivoted_qr(A: np.ndarray, max_rank: int, tau: float):
    """Householder QR with column pivoting (Businger-Golub; the GEQP3 of
    §2.2), truncated adaptively.  At step k the remaining column with the
    largest residual norm (recomputed, ties to the smallest original column
    position) becomes pivot k.  The rank s is the number of pivots with
    |R_kk| > tau |R_00| (reading of "sigma_{s+1} < tau": relative, estimated
    by the pivoted-QR diagonal), at least 1 and at most
    min(max_rank, rows, cols).

    Returns (perm, R, s, rdiag): perm[k] = original position of pivot k,
    R = the first s rows of the triangularised matrix (all columns, pivot
    order), rdiag = |R_kk| for the accepted pivots."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    perm = np.arange(n)
    kmax = min(m, n, max_rank)
    rdiag = []
    r00 = 0.0
    s = 0
    for k in range(kmax):
        norms = np.sqrt(np.einsum("ij,ij->j", A[k:, k:], A[k:, k:]))
        mx = norms.max()
        cand = np.nonzero(norms == mx)[0]
        j = k + int(cand[np.argmin(perm[k + cand])])
        if j != k:
            A[:, [k, j]] = A[:, [j, k]]
            perm[[k, j]] = perm[[j, k]]
        rkk = float(mx)
        if k == 0:
            r00 = rkk
        elif rkk <= tau * r00:
            break
        x = A[k:, k].copy()
        alpha = -math.copysign(rkk, x[0]) if x[0] != 0 else -rkk
        v = x
        v[0] -= alpha
        vn2 = float(v @ v)
        if vn2 > 0.0:
            A[k:, k:] -= np.outer(v, (2.0 / vn2) * (v @ A[k:, k:]))
        A[k + 1:, k] = 0.0
        rdiag.append(rkk)
        s = k + 1
        if r00 == 0.0:
            break
    s = max(s, 1)
    return perm, np.triu(A[:s, :]), s, np.array(rdiag[:s])


def interpolation_matrix(perm: np.ndarray, R: np.ndarray, s: int) -> np.ndarray:
    """COEF (Table 2): P = [I | R11^{-1} R12] Pi^T by triangular solve, as an
    s x ncols matrix in the original column order (§2.2 low-rank
    approximation: K_{I beta} ~ K_{I skel} P_{skel beta})."""
    n = R.shape[1]
    P = np.zeros((s, n))
    P[np.arange(s), perm[:s]] = 1.0
    if n > s:
        R11 = R[:s, :s]
        if np.all(np.abs(np.diag(R11)) > 0):
            P[:, perm[s:]] = scipy.linalg.solve_triangular(R11, R[:s, s:], lower=False)
    return P


def sample_rows(tree: Tree, knn: np.ndarray, h: int, prm: Params) -> np.ndarray:
    """Neighbour-based importance sampling of the rows I' (§2.2).

    Reading: |I'| = min(N - |alpha|, n_sample) with n_sample = 2 s by
    default.  First the neighbours of alpha's indices that lie outside alpha,
    by decreasing number of occurrences (ties to the smaller index); the rest
    is drawn uniformly without replacement from the remaining complement
    (ascending list, partial Fisher-Yates on the node's stream)."""
    n = tree.n
    idx = tree.node_idx[h]
    target = prm.n_sample if prm.n_sample > 0 else 2 * prm.max_rank
    need = min(n - idx.size, target)
    inside = np.zeros(n, dtype=bool)
    inside[idx] = True
    nb = knn[idx].ravel()
    cnt = np.bincount(nb[nb >= 0], minlength=n)
    cnt[inside] = 0
    cand = np.nonzero(cnt)[0]
    order = np.lexsort((cand, -cnt[cand]))
    chosen = cand[order[:need]]
    if chosen.size < need:
        taken = inside.copy()
        taken[chosen] = True
        rest = np.nonzero(~taken)[0]
        extra = partial_shuffle(rest, need - chosen.size, stream_key(prm.seed, _P_SAMPLE, h))
        chosen = np.concatenate([chosen, extra])
    return chosen.astype(np.int64)


def skeletonize(K, tree: Tree, knn: np.ndarray, prm: Params):
    """Alg. 6 in postorder over every node except the root: ID of K_{I' beta}
    (leaf) or K_{I' [l~ r~]} (inner, columns = children's skeletons, so the
    skeletons nest, §2.2 telescoping)."""
    L = tree.depth
    skel, P, rd = {}, {}, {}
    for lvl in range(L, 0, -1):
        for h in tree.level_nodes(lvl):
            if lvl == L:
                cols = tree.node_idx[h]
            else:
                cols = np.concatenate([skel[2 * h + 1], skel[2 * h + 2]])
            rows = sample_rows(tree, knn, h, prm)
            A = K(rows, cols)
            perm, R, s, rdiag = pivoted_qr(A, prm.max_rank, prm.tau)
            skel[h] = cols[perm[:s]]
            P[h] = interpolation_matrix(perm, R, s)
            rd[h] = rdiag
    return skel, P, rd


def compress(K, n: int, prm: Params) -> Structure:
    """Alg. 2 (Compress) without the optional caching steps: the oracle's
    evaluation asks the entry routine for every block it needs."""
    diagK = K.diag(np.arange(n))
    knn, iters, recall = all_nearest_neighbors(K, diagK, n, prm)
    tree = build_tree(K, diagK, n, prm)
    near = leaf_near(tree, knn, prm)
    far = far_symmetric(tree, near) if prm.far == FAR_SYMMETRIC else far_paper(tree, near)
    skel, P, rd = skeletonize(K, tree, knn, prm)
    return Structure(prm, tree, knn, near, far, skel, P, rd, iters, recall)


# --------------------------------------------------------------------------
# Alg. 7 / Table 2: evaluation
# --------------------------------------------------------------------------
def evaluate(st: Structure, K, W: np.ndarray) -> np.ndarray:
    """U = K~ W in FP64 (Alg. 7): POST N2S, ANY S2S, PRE S2N, ANY L2L,
    each task exactly as Table 2 (u starts at zero; the S2N leaf task and
    L2L both accumulate into u)."""
    tree = st.tree
    L = tree.depth
    W = np.asarray(W, dtype=np.float64)
    r = W.shape[1]
    wt: Dict[int, np.ndarray] = {}
    # N2S, postorder
    for lvl in range(L, 0, -1):
        for h in tree.level_nodes(lvl):
            if lvl == L:
                wt[h] = st.P[h] @ W[tree.node_idx[h]]
            else:
                wt[h] = st.P[h] @ np.vstack([wt[2 * h + 1], wt[2 * h + 2]])
    # S2S
    ut = {h: np.zeros((st.skel[h].size, r)) for h in st.skel}
    for b, lst in st.far.items():
        for a in lst:
            ut[b] += K(st.skel[b], st.skel[a]) @ wt[a]
    # S2N, preorder
    U = np.zeros((tree.n, r))
    for lvl in range(1, L + 1):
        for h in tree.level_nodes(lvl):
            t = st.P[h].T @ ut[h]
            if lvl < L:
                sl = st.skel[2 * h + 1].size
                ut[2 * h + 1] += t[:sl]
                ut[2 * h + 2] += t[sl:]
            else:
                U[tree.node_idx[h]] += t
    # L2L
    for b in range(tree.n_leaves):
        rows = tree.node_idx[tree.leaf_node(b)]
        for a in st.near[b]:
            cols = tree.node_idx[tree.leaf_node(int(a))]
            U[rows] += K(rows, cols) @ W[cols]
    return U


def evaluate_leaves(st: Structure, K, W: np.ndarray, leaves) -> Dict[int, np.ndarray]:
    """Rows of U = K~ W belonging to the given leaves (leaf numbers), by the
    same tasks as `evaluate` restricted to what those rows read: N2S on every
    node, then S2S and S2N only along the root-to-leaf paths, then the leaf
    S2N and L2L.  Returns {leaf: rows of U in the leaf's index order}."""
    tree = st.tree
    L = tree.depth
    W = np.asarray(W, dtype=np.float64)
    r = W.shape[1]
    wt: Dict[int, np.ndarray] = {}
    for lvl in range(L, 0, -1):
        for h in tree.level_nodes(lvl):
            if lvl == L:
                wt[h] = st.P[h] @ W[tree.node_idx[h]]
            else:
                wt[h] = st.P[h] @ np.vstack([wt[2 * h + 1], wt[2 * h + 2]])
    out = {}
    for b in leaves:
        leaf = tree.leaf_node(int(b))
        path = []
        h = leaf
        while h > 0:
            path.append(h)
            h = (h - 1) // 2
        path.reverse()
        ut = None
        for depth_i, h in enumerate(path):
            cur = np.zeros((st.skel[h].size, r))
            for a in st.far.get(h, []):
                cur += K(st.skel[h], st.skel[int(a)]) @ wt[int(a)]
            if ut is not None:
                p = path[depth_i - 1]
                t = st.P[p].T @ ut
                sl = st.skel[2 * p + 1].size
                cur += t[:sl] if h == 2 * p + 1 else t[sl:]
            ut = cur
        rows = tree.node_idx[leaf]
        u = st.P[leaf].T @ ut if ut is not None else np.zeros((rows.size, r))
        for a in st.near[int(b)]:
            cols = tree.node_idx[tree.leaf_node(int(a))]
            u = u + K(rows, cols) @ W[cols]
        out[int(b)] = u
    return out


class AbsEntries:
    """|K(I, J)| entry by entry (diagonal too)."""

    def __init__(self, K):
        self.K = K

    def __call__(self, I, J):
        return np.abs(self.K(I, J))

    def diag(self, I):
        return np.abs(self.K.diag(I))


def evaluate_abs(st: Structure, K, W: np.ndarray) -> np.ndarray:
    """Rounding-error scale of the evaluation: Alg. 7 run on |P|, |K| and
    |W| (every interpolation matrix, every sampled block and the right-hand
    sides replaced by their entrywise absolute values).  Each task of
    Table 2 is a product of nonnegative factors, so the result bounds
    |P^T K P| |W| and |K_{ba}| |W| term by term; a product computed with unit
    roundoff u is then off by at most a small multiple of u times this value,
    element by element.  Test infrastructure for the tensor-precision bounds
    (no passage of the paper defines it)."""
    ast = dataclasses.replace(st, P={h: np.abs(P) for h, P in st.P.items()})
    return evaluate(ast, AbsEntries(K), np.abs(np.asarray(W, dtype=np.float64)))


def dense_rows(K, rows: np.ndarray, W: np.ndarray, block=256) -> np.ndarray:
    """Exact rows of K W by brute force."""
    n = W.shape[0]
    allj = np.arange(n)
    out = np.empty((rows.size, W.shape[1]))
    for b0 in range(0, rows.size, block):
        out[b0:b0 + block] = K(rows[b0:b0 + block], allj) @ W
    return out


def eps2(approx_rows: np.ndarray, exact_rows: np.ndarray) -> float:
    """Relative error of §3: |K~w - Kw|_F / |Kw|_F over the sampled rows."""
    return float(np.linalg.norm(approx_rows - exact_rows) / np.linalg.norm(exact_rows))


def tree_order(tree: Tree, h: int) -> np.ndarray:
    """Indices of node h in tree order (its leaves left to right)."""
    if 2 * h + 1 >= len(tree.node_idx):
        return tree.node_idx[h]
    return np.concatenate([tree_order(tree, 2 * h + 1), tree_order(tree, 2 * h + 2)])


def telescoped_basis(st: Structure, h: int) -> np.ndarray:
    """P_{h~ h} over all indices of node h (columns in tree order), formed
    explicitly by the telescoping expression (§2.2, eq. telescope):
    P_{a~a} = P_{a~[l~r~]} diag(P_{l~l}, P_{r~r})."""
    tree = st.tree
    if 2 * h + 1 >= (1 << (tree.depth + 1)) - 1:
        return st.P[h]
    Pl = telescoped_basis(st, 2 * h + 1)
    Pr = telescoped_basis(st, 2 * h + 2)
    return st.P[h] @ scipy.linalg.block_diag(Pl, Pr)


def assemble(st: Structure, K) -> np.ndarray:
    """The H-matrix K~ as a dense N x N array (original order): direct
    blocks K_{beta alpha} for near leaf pairs plus
    P_{b~b}^T K_{b~a~} P_{a~a} for every far pair (§2.2, Evaluation)."""
    tree = st.tree
    n = tree.n
    Kt = np.zeros((n, n))
    for b in range(tree.n_leaves):
        rows = tree.node_idx[tree.leaf_node(b)]
        for a in st.near[b]:
            cols = tree.node_idx[tree.leaf_node(int(a))]
            Kt[np.ix_(rows, cols)] += K(rows, cols)
    for b, lst in st.far.items():
        Pb = telescoped_basis(st, b)
        for a in lst:
            Pa = telescoped_basis(st, int(a))
            blk = Pb.T @ K(st.skel[b], st.skel[int(a)]) @ Pa
            Kt[np.ix_(tree_order(tree, b), tree_order(tree, int(a)))] += blk
    return Kt


def flop_count(st: Structure, r: int) -> dict:
    """Algorithmic flops per evaluation (Table 2 with the real block shapes):
    N2S/S2N count 2 s (ncols - s) r each -- P = [I | T] Pi^T, and its
    identity part is a copy, not arithmetic (§2.2, low-rank approximation
    and the cost paragraph after Alg. 7) -- S2S 2 s_b s_a r per far pair, L2L
    2 |b| |a| r per near pair."""
    tree = st.tree
    n2s = sum(2 * P.shape[0] * (P.shape[1] - P.shape[0]) * r for P in st.P.values())
    s2s = sum(2 * st.skel[b].size * st.skel[int(a)].size * r
              for b, lst in st.far.items() for a in lst)
    l2l = 0
    for b in range(tree.n_leaves):
        nb = tree.node_idx[tree.leaf_node(b)].size
        for a in st.near[b]:
            l2l += 2 * nb * tree.node_idx[tree.leaf_node(int(a))].size * r
    return dict(n2s=n2s, s2s=s2s, s2n=n2s, l2l=l2l, total=2 * n2s + s2s + l2l)
