"""The C-ABI library on a machine without a GPU: it loads, exports every
entry point the header declares, compresses on host cores, reports errors
with the documented codes, and round-trips checkpoint files."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1707_00164_b300 as G
import workloads as wl
from common import assert_same_structure, both

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_entry_point():
    hdr = open(os.path.join(ROOT, "include", "gofmm.h")).read()
    names = set(re.findall(r"^\s*(?:[\w\*\s]+?)\b(gofmm_\w+)\s*\(", hdr, flags=re.M))
    names.discard("gofmm_block_fn")
    assert {"gofmm_compress", "gofmm_evaluate", "gofmm_free"} <= names
    lib = ctypes.CDLL(G.gofmm.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n


def _small():
    w = wl.scaled(wl.C1, 300)
    return w, w.matrix()


@pytest.mark.parametrize("over,code", [
    (dict(leaf_size=0), G.ERR_ARG), (dict(max_rank=0), G.ERR_ARG), (dict(tau=-1.0), G.ERR_ARG),
    (dict(kappa=0), G.ERR_ARG), (dict(distance=9), G.ERR_ARG), (dict(far_mode=5), G.ERR_ARG),
])
def test_bad_parameters_are_rejected(over, code):
    w, K = _small()
    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.gaussian(K.points, 0.3, 1e-3), G.default_params(**over))
    assert e.value.code == code


def test_callback_errors_and_nonfinite_entries():
    w, K = _small()

    def bad(I, J):
        raise RuntimeError("user failure")

    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.callback(w.n, bad), G.default_params(leaf_size=32))
    assert e.value.code == G.ERR_CALLBACK

    def nan(I, J):
        out = K(I, J)
        out[0, 0] = math.nan
        return out

    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.callback(w.n, nan), G.default_params(leaf_size=32))
    assert e.value.code == G.ERR_NONFINITE
    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.callback(w.n, K), G.default_params(cache_mode=G.CACHE_NONE))
    assert e.value.code == G.ERR_ARG


def test_export_import_roundtrip(tmp_path):
    w = wl.scaled(wl.C1, 700)
    h, st, K = both(w, leaf_size=32, callback=False)
    path = str(tmp_path / "s.bin")
    G.export(h, path)
    h2 = G.import_(path, G.Entries.gaussian(K.points, w.bandwidth, w.shift))
    assert_same_structure(h2, st)
    s1, s2 = G.structure(h), G.structure(h2)
    for node in s1["P"]:
        assert np.array_equal(s1["P"][node], s2["P"][node])
    bad = tmp_path / "junk.bin"
    bad.write_bytes(b"not a structure file at all")
    with pytest.raises(G.GofmmError) as e:
        G.import_(str(bad), G.Entries.gaussian(K.points, w.bandwidth, w.shift))
    assert e.value.code == G.ERR_IO
    with pytest.raises(G.GofmmError) as e:
        G.import_(path, G.Entries.gaussian(K.points[:100], w.bandwidth, w.shift))
    assert e.value.code == G.ERR_ARG


def test_stats_flop_count_matches_oracle():
    w = wl.scaled(wl.C1, 1024)
    h, st, K = both(w, leaf_size=32, budget=0.05, callback=False)
    s = G.stats(h)
    f = O.flop_count(st, 1)
    assert s["flops_n2s"] == f["n2s"] and s["flops_s2s"] == f["s2s"] and s["flops_l2l"] == f["l2l"]
    assert s["flops_s2n"] == f["s2n"]
    # only the T part of P counts: s (ncols - s) entries per node
    t_entries = sum(P.shape[0] * (P.shape[1] - P.shape[0]) for P in st.P.values())
    assert s["interp_t_entries"] == t_entries and s["flops_n2s"] == 2 * t_entries
    assert s["interp_entries"] == sum(P.size for P in st.P.values())
    assert s["skel_total"] == sum(v.size for v in st.skel.values())


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the no-GPU failure path")
def test_evaluate_without_a_gpu_fails_loudly():
    w, K = _small()
    h = G.compress(G.Entries.gaussian(K.points, 0.3, 1e-3), G.default_params(leaf_size=32))
    W = np.ones((w.n, 2))
    U = np.zeros_like(W)
    for fn in (G.evaluate_host, G.evaluate_host_async):
        with pytest.raises(G.GofmmError) as e:
            fn(h, W, U, G.PREC_FP64)
        assert e.value.code == G.ERR_CUDA
        assert not U.any()


def test_host_evaluation_argument_errors():
    """Checked before any device work (no GPU needed): overlapping W and U,
    mismatched dtype and precision, both host entry points alike."""
    w, K = _small()
    h = G.compress(G.Entries.gaussian(K.points, 0.3, 1e-3), G.default_params(leaf_size=32))
    W = np.ones((w.n, 2))
    for fn in (G.evaluate_host, G.evaluate_host_async):
        with pytest.raises(G.GofmmError) as e:
            fn(h, W, W, G.PREC_FP64)  # U aliases W
        assert e.value.code == G.ERR_ARG
        with pytest.raises(G.GofmmError) as e:
            fn(h, W, np.zeros_like(W), G.PREC_FP32)  # F64 data, FP32 precision
        assert e.value.code == G.ERR_UNSUPPORTED


def test_device_sampling_needs_a_generator_and_a_gpu():
    w, K = _small()
    with pytest.raises(G.GofmmError) as e:  # no GPU here: fails loudly, no host fallback
        G.compress(G.Entries.gaussian(K.points, 0.3, 1e-3), G.default_params(leaf_size=32, sample_device=1))
    assert e.value.code == G.ERR_CUDA
    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.callback(w.n, K), G.default_params(leaf_size=32, sample_device=1))
    assert e.value.code == G.ERR_ARG
    with pytest.raises(G.GofmmError) as e:
        G.compress(G.Entries.gaussian(K.points, 0.3, 1e-3), G.default_params(leaf_size=32, sample_device=2))
    assert e.value.code == G.ERR_ARG


def test_header_and_library_from_plain_c(tmp_path):
    """include/gofmm.h compiles as C99 and the library links and runs from C."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_from_c")
    lib = G.gofmm.LIB_PATH
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "abi_from_c.c"), lib, "-lm",
                           "-Wl,-rpath," + os.path.dirname(lib), "-o", exe])
    out = subprocess.run([exe, str(tmp_path / "c.bin")], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("c abi ok")
