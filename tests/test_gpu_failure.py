"""Failure detection without a GPU fault: every device-side wait of the
tensor-core kernels is bounded (about a second); a wait that runs out makes
the kernel record an error code and return, the host reads it through
gofmm_synchronize, and the context stays usable.  The failure is made with
a completion count that nothing reaches (no trap, no bad address, no endless
loop)."""
import time

import numpy as np
import pytest

import paper_1707_00164_b300 as G
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    w = wl.scaled(wl.C1, 1500)
    K = w.matrix()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift), G.default_params(leaf_size=64))
    W = torch.from_numpy(w.rhs(64).astype(np.float32)).cuda()
    ref = torch.empty_like(W)
    G.evaluate(h, W, ref, G.PREC_BF16X3)
    G.synchronize(h)
    G.debug_stall_next(h, G.PREC_BF16X3)
    U = torch.empty_like(W)
    t0 = time.time()
    G.evaluate(h, W, U, G.PREC_BF16X3)
    with pytest.raises(G.GofmmError) as e:
        G.synchronize(h)
    assert e.value.code == G.ERR_TIMEOUT
    assert time.time() - t0 < 60
    # the error was reported once; the handle and the context still work
    again = torch.full_like(W, float("nan"))
    G.evaluate(h, W, again, G.PREC_BF16X3)
    G.synchronize(h)
    assert torch.equal(again, ref)
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0
