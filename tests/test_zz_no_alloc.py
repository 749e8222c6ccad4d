"""gofmm_evaluate_static, the entry point for callers that may not allocate
device memory while running (for example a serving loop whose memory budget
is fixed at start-up: an allocation there could fail, and it synchronises the
device).  It must give the same result as gofmm_evaluate, call after call,
with its scratch in the library's fixed device array.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import paper_1707_00164_b300 as G
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def _handle(n=2000):
    w = wl.scaled(wl.C1, n)
    K = w.matrix()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift),
                   G.default_params(leaf_size=64, max_rank=64, tau=1e-5, budget=0.03))
    return w, h


@pytest.mark.parametrize("prec,dtype,tol", [(G.PREC_FP64, torch.float64, FP64_TOL),
                                            (G.PREC_FP32, torch.float32, FP32_TOL)])
def test_static_scratch_matches_evaluate_twice(prec, dtype, tol):
    w, h = _handle()
    r = 24
    G.prepare(h, r, prec)
    W = torch.from_numpy(w.rhs(r)).to("cuda", dtype)
    ref = torch.empty_like(W)
    G.evaluate(h, W, ref, prec)
    for _ in range(2):  # two calls in a row share (and reuse) the array
        U = torch.full_like(W, float("nan"))
        G.evaluate_static(h, W, U, prec)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm((U - ref).double()) / torch.linalg.norm(ref.double()))
        assert np.isfinite(err) and err <= tol, err


def test_static_scratch_allocates_nothing():
    """After a first call (which looks up the array's device address), calls
    at several r leave the device's free memory unchanged: nothing is
    allocated per call.  Every buffer is made before the first reading and
    the results are compared only after the last one."""
    w, h = _handle()
    rs = (8, 24, 40)
    G.prepare(h, max(rs), G.PREC_FP32)
    Ws = {r: torch.from_numpy(w.rhs(r)).to("cuda", torch.float32) for r in rs}
    Us = {r: [torch.full_like(Ws[r], float("nan")) for _ in range(2)] for r in rs}
    refs = {r: torch.empty_like(Ws[r]) for r in rs}
    for r in rs:
        G.evaluate(h, Ws[r], refs[r], G.PREC_FP32)
    G.evaluate_static(h, Ws[rs[0]], Us[rs[0]][0], G.PREC_FP32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(2):
        for r in rs:
            G.evaluate_static(h, Ws[r], Us[r][k], G.PREC_FP32)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for r in rs:
        for k in range(2):
            err = float(torch.linalg.norm((Us[r][k] - refs[r]).double()) / torch.linalg.norm(refs[r].double()))
            assert np.isfinite(err) and err <= FP32_TOL, (r, k, err)


def test_static_scratch_rejects_oversize_and_unprepared():
    w, h = _handle(1500)
    W = torch.zeros((w.n, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GofmmError) as e:  # not prepared yet
        G.evaluate_static(h, W, torch.empty_like(W), G.PREC_FP64)
    assert e.value.code == G.ERR_ARG
    G.prepare(h, 4096, G.PREC_FP64)
    big = torch.zeros((w.n, 4096), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GofmmError) as e:  # (N + 2 S) r * 8 bytes > 32 MiB
        G.evaluate_static(h, big, torch.empty_like(big), G.PREC_FP64)
    assert e.value.code == G.ERR_ARG and "scratch" in G.last_error()
