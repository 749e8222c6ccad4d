"""The native host compression (C++) against the oracle (Python), on the same
seeded inputs: every integer decision (tree order, near and far lists,
skeletons) bit-exact, interpolation matrices within 1e-8."""
import pytest

import oracle as O
import workloads as wl
from common import assert_same_structure, both

CASES = [
    ("c1_callback_full", wl.C1, dict()),
    ("gauss_ragged_n1000_m32", wl.scaled(wl.C1, 1000), dict(leaf_size=32, callback=False)),
    ("gauss6d_n3000_ann", wl.scaled(wl.C2, 3000), dict(knn_exact_max=1000, leaf_size=64, max_rank=64)),
    ("imq_angle_n777", wl.scaled(wl.C3, 777), dict(leaf_size=50, max_rank=40, distance=O.ANGLE, tau=1e-4)),
    ("paper_far_n1024", wl.scaled(wl.C1, 1024), dict(leaf_size=32, far=O.FAR_PAPER, budget=0.05,
                                                     callback=False)),
    ("hss_budget0", wl.scaled(wl.C1, 512), dict(leaf_size=32, budget=0.0, callback=False)),
    ("lexicographic", wl.scaled(wl.C1, 600), dict(leaf_size=32, distance=O.LEXICOGRAPHIC,
                                                  callback=False)),
    ("random_order", wl.scaled(wl.C1, 600), dict(leaf_size=32, distance=O.RANDOM, callback=False)),
    ("single_leaf", wl.scaled(wl.C1, 50), dict(leaf_size=64, callback=False)),
]


@pytest.mark.parametrize("name,w,over", CASES, ids=[c[0] for c in CASES])
def test_native_compression_matches_oracle(name, w, over):
    over = dict(over)
    cb = over.pop("callback", None)
    h, st, K = both(w, callback=cb, **over)
    assert_same_structure(h, st)
