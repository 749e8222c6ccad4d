"""The element-wise and row-wise parity checks of the tensor precisions
(tests/common.py) catch the mistakes a norm over a whole block can hide: a
result within rounding passes; two rows exchanged, one r-tile of one row
lost, or one row off by a few percent fail.  The mistakes are planted in
the oracle's own result on the CPU."""
import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import TC_TOL, abs_product, assert_tensor_close


@pytest.fixture(scope="module")
def case():
    w = wl.scaled(wl.C2, 2048)
    K = w.matrix()
    st = O.compress(K, w.n, O.Params(**w.params(leaf_size=64, max_rank=64)))
    W = w.rhs(256)
    return st, O.evaluate(st, K, W), O.evaluate_abs(st, K, W), abs_product(K, W)


PRECS = [G.PREC_TF32, G.PREC_BF16, G.PREC_BF16X3]


@pytest.mark.parametrize("prec", PRECS)
def test_rounding_sized_noise_passes(case, prec):
    st, ref, ua, ka = case
    rng = np.random.default_rng(0)
    # a relative error a tenth of the row bound, in every element
    noise = 0.1 * TC_TOL[prec] * ref * rng.uniform(-1, 1, ref.shape)
    assert_tensor_close(ref + noise, ref, ua, ka, prec)


@pytest.mark.parametrize("prec", PRECS + [G.PREC_FP32])
def test_planted_mistakes_fail(case, prec):
    st, ref, ua, ka = case
    leaf = st.tree.node_idx[st.tree.leaf_node(3)]
    swapped = ref.copy()
    swapped[[leaf[0], leaf[1]]] = swapped[[leaf[1], leaf[0]]]     # a mis-scattered pair of rows
    lost_tile = ref.copy()
    lost_tile[leaf[5], 128:256] = 0.0                            # one r-tile of one row never written
    scaled = ref.copy()
    scaled[leaf[7]] *= 1.05                                      # one row 5 % off
    for bad in (swapped, lost_tile, scaled):
        with pytest.raises(AssertionError):
            assert_tensor_close(bad, ref, ua, ka, prec)
