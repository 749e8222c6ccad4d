"""Full-rank subtrees on the tensor cores.

A node whose rank equals its column count has P = Pi^T, a permutation (§2.2,
P = [I | R11^-1 R12] Pi^T with R12 empty), and when its children are full
rank too its skeleton weights w~ are rows of W itself.  The tensor-core plan
then drops the node's N2S task, and every slab that read w~ of such nodes
reads W in tree order instead, with its block's columns permuted when the
block tiles are made (a column map, zero where a leaf's rows end before its
chunk does) or, for generated blocks, the tree-order column list (only where
the leaves leave no padding inside the range).

Leaves of 31 and 32 points (N = 1000, m = 32) put padding between the leaves
in the chunk layout of W, so these cases reach the column maps with gaps:
  * tau = 0 and a rank cap above N / 2: every node is full rank (K~ = K);
  * tau = 0 and a rank cap of 40: the leaves are full rank, their parents
    (62-64 columns) are not, so the parents' N2S slabs [w~_l; w~_r] read two
    ragged leaves of W.
Each is checked against the FP64 oracle on the same structure, in every
tensor precision, with cached and with generated blocks."""
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
CASES = {
    "every_node_full_rank": dict(tau=0.0, max_rank=600, n_sample=600),
    "full_rank_leaves_only": dict(tau=0.0, max_rank=40),
}
_built = {}


def build(case, cache_mode):
    key = (case, cache_mode)
    if key not in _built:
        w = wl.scaled(wl.C1, 1000)
        h, st, K = both(w, leaf_size=32, callback=False, cache_mode=cache_mode, **CASES[case])
        _built[key] = (w, h, st, K)
    return _built[key]


def full_rank_nodes(s):
    """Nodes whose P is a permutation matrix (entries 0 and 1, one 1 per row
    and per column): square P with exact entries."""
    out = []
    for node, P in s["P"].items():
        P = np.asarray(P)
        sk = len(s["skel"][node])
        if P.size == 0 or P.size % sk:
            continue
        P = P.reshape(sk, -1)
        if P.shape[0] == P.shape[1] and np.all((P == 0) | (P == 1)) and np.all(P.sum(0) == 1) \
                and np.all(P.sum(1) == 1):
            out.append(node)
    return out


@pytest.mark.parametrize("prec", PRECS, ids=[NAMES[p] for p in PRECS])
@pytest.mark.parametrize("cache_mode", [G.CACHE_BLOCKS, G.CACHE_NONE], ids=["cached", "generated"])
@pytest.mark.parametrize("case", list(CASES))
def test_full_rank_subtrees_match_oracle(case, cache_mode, prec):
    w, h, st, K = build(case, cache_mode)
    s = assert_same_structure(h, st)
    sizes = np.diff(s["leaf_off"])
    assert np.any(sizes % 64 != 0)  # padding between leaves in the chunk layout of W
    depth = s["depth"]
    leaves = range((1 << depth) - 1, (2 << depth) - 1)
    fr = set(full_rank_nodes(s))
    assert all(b in fr for b in leaves)  # tau = 0, cap above the leaf size
    if case == "full_rank_leaves_only":
        assert not any(((1 << (depth - 1)) - 1) <= x < (1 << depth) - 1 for x in fr)
    W = w.rhs(37)
    ref = O.evaluate(st, K, W)
    if case == "every_node_full_rank":
        dense = K.dense() @ W  # full rank everywhere: K~ = K
        assert np.linalg.norm(ref - dense) <= 1e-10 * np.linalg.norm(dense)
    Wt = torch.from_numpy(W.astype(np.float32)).cuda()
    Ut = torch.full_like(Wt, float("nan"))
    G.evaluate(h, Wt, Ut, prec)
    G.synchronize(h)
    U = Ut.double().cpu().numpy()
    assert np.all(np.isfinite(U))
    kappa = float(np.linalg.norm(abs_product(K, W)) / np.linalg.norm(K.dense() @ W))
    rel = float(np.linalg.norm(U - ref) / np.linalg.norm(ref))
    assert rel <= TOL[prec] * max(1.0, kappa / 25.0), (rel, kappa)
    assert_tensor_close(U, ref, O.evaluate_abs(st, K, W), abs_product(K, W), prec)
