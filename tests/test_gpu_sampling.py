"""Compression with the sampled blocks K_{I'a} generated on the GPU
(gofmm_params.sample_device = 1; Alg. 2 steps 8-9 on the device, pivoted QR
and solve on the host in FP64).

The device accumulates squared distances in the host's order without fused
multiply-adds, and FP64 division and square root are correctly rounded on
both sides, so inverse-multiquadric entries are bitwise the host's and the
whole compression is identical.  The Gaussian's exp may differ from the
host's in the last bit; the tree, near and far lists do not depend on the
sampled blocks and must be identical, the skeletons may differ at
near-ties, and the evaluation of the compressed matrix is checked against
the oracle's evaluation of that same structure (1e-12, FP64) and against
dense K W."""
import copy

import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import assert_same_structure, both, native_entries

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def compress(w, sample_device, **over):
    p = w.params(**over)
    p["sample_device"] = sample_device
    return G.compress(native_entries(w, callback=False), G.default_params(**p))


def same(a, b):
    sa, sb = G.structure(a), G.structure(b)
    if not (np.array_equal(sa["perm"], sb["perm"]) and len(sa["near"]) == len(sb["near"])):
        return False, 0.0
    for x, y in zip(sa["near"], sb["near"]):
        if not np.array_equal(x, y):
            return False, 0.0
    for x, y in zip(sa["far"], sb["far"]):
        if not np.array_equal(x, y):
            return False, 0.0
    # fraction of nodes with the same skeleton; their P agree to rounding
    # (bitwise when the sampled entries are)
    eq = []
    for n in range(1, len(sa["skel"])):
        e = np.array_equal(sa["skel"][n], sb["skel"][n])
        if e:
            scale = max(1.0, float(np.abs(sa["P"][n]).max()))
            assert np.abs(sa["P"][n] - sb["P"][n]).max() <= 1e-8 * scale, n
        eq.append(e)
    return True, float(np.mean(eq))


def test_imq_device_sampling_is_bitwise_the_host_compression():
    w = wl.scaled(wl.C3, 6000)
    h_host = compress(w, 0, leaf_size=128, max_rank=96)
    h_dev = compress(w, 1, leaf_size=128, max_rank=96)
    lists_equal, frac = same(h_host, h_dev)
    assert lists_equal and frac == 1.0
    sa, sb = G.structure(h_host), G.structure(h_dev)
    assert all(np.array_equal(sa["P"][n], sb["P"][n]) for n in range(1, len(sa["skel"])))


def test_gaussian_device_sampling_parity_and_accuracy():
    w = wl.C1  # Gaussian, N = 4096, entries through the generator here
    h, st, K = both(w, callback=False)
    assert_same_structure(h, st)  # host sampling reproduces the oracle
    h_dev = compress(w, 1)
    lists_equal, frac = same(h, h_dev)
    assert lists_equal
    assert frac >= 0.9, frac  # skeletons may differ only at near-ties
    # the oracle's evaluation of exactly the device-sampled structure
    s = G.structure(h_dev)
    st_dev = copy.copy(st)
    st_dev.skel = {n: s["skel"][n] for n in range(1, len(s["skel"]))}
    st_dev.P = {n: s["P"][n] for n in range(1, len(s["skel"]))}
    W = w.rhs()
    ref = O.evaluate(st_dev, K, W)
    Wt = torch.from_numpy(W).cuda()
    Ut = torch.empty_like(Wt)
    G.evaluate(h_dev, Wt, Ut, G.PREC_FP64)
    G.synchronize(h_dev)
    U = Ut.cpu().numpy()
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) <= 1e-12
    # accuracy against dense K W matches the host-sampled compression
    exact = K.dense() @ W
    e_dev = np.linalg.norm(U - exact) / np.linalg.norm(exact)
    e_host = np.linalg.norm(O.evaluate(st, K, W) - exact) / np.linalg.norm(exact)
    assert e_dev <= 2.0 * e_host + 1e-12, (e_dev, e_host)
