"""Write tests/golden/<name>_rows.npz: sampled rows of K~W computed by the FP64
oracle alone, for a workload of `workloads` (default: the precision workload,
IMQ kernel on 4-D uniform points, N = 131072, m = 256, s = 512, tau = 1e-6,
r = 2048).

Stored: 100 seeded rows x the first COLS columns (default: all r) of the
oracle's K~W for the workload's seeded W, of its absolute-value evaluation
(Alg. 7 on |P|, |K|, |W|: the element-wise rounding-error scale), of the
exact K W and of the exact |K| |W| (the sum condition of each row), and the
oracle's eps2 on them.  The right-hand side is evaluated
in column blocks of 256 to bound the host memory.
Run:  python tests/golden/make_rows.py [workload-name] [cols]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
import workloads as wl  # noqa: E402

BLOCK = 256


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else wl.C3.name
    w = wl.WORKLOADS[name]
    cols = int(sys.argv[2]) if len(sys.argv) > 2 else w.r
    K = w.matrix()
    t0 = time.time()
    st = O.compress(K, w.n, O.Params(**w.params()))
    t1 = time.time()
    W = w.rhs(w.r)[:, :cols]
    rows = wl.sample_rows(w.n)
    U = np.empty((rows.size, cols))
    Ua = np.empty((rows.size, cols))
    for c0 in range(0, cols, BLOCK):
        Wb = W[:, c0:c0 + BLOCK]
        U[:, c0:c0 + BLOCK] = O.evaluate(st, K, Wb)[rows]
        Ua[:, c0:c0 + BLOCK] = O.evaluate_abs(st, K, Wb)[rows]
    t2 = time.time()
    exact = O.dense_rows(K, rows, W)
    kabs = O.dense_rows(O.AbsEntries(K), rows, np.abs(W))
    eps = O.eps2(U, exact)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_rows.npz")
    np.savez_compressed(out, rows=rows, cols=np.arange(cols), u_oracle=U, u_abs=Ua, u_exact=exact,
                        u_kabs=kabs, eps2=eps,
                        skel_total=sum(st.skel[h].size for h in st.skel),
                        far_pairs=sum(len(v) for v in st.far.values()))
    print(f"compress {t1 - t0:.1f}s evaluate {t2 - t1:.1f}s eps2 {eps:.4e} -> {out}")


if __name__ == "__main__":
    main()
