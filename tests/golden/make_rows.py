"""Write tests/golden/<name>_rows.npz: sampled rows of K~W computed by the FP64
oracle alone, for a workload of `workloads` (default: the precision workload,
IMQ kernel on 4-D uniform points, N = 131072, m = 256, s = 512, tau = 1e-6).

Stored: 100 seeded rows x the first COLS columns of the oracle's K~W for the
workload's seeded W (only those columns are evaluated), the same rows of the
exact K W, and the oracle's eps2 on them.
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


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else wl.C3.name
    cols = int(sys.argv[2]) if len(sys.argv) > 2 else 64
    w = wl.WORKLOADS[name]
    K = w.matrix()
    t0 = time.time()
    st = O.compress(K, w.n, O.Params(**w.params()))
    t1 = time.time()
    W = w.rhs(w.r)[:, :cols]
    U = O.evaluate(st, K, W)
    t2 = time.time()
    rows = wl.sample_rows(w.n)
    exact = O.dense_rows(K, rows, W)
    eps = O.eps2(U[rows], exact)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_rows.npz")
    np.savez_compressed(out, rows=rows, cols=np.arange(cols), u_oracle=U[rows], u_exact=exact, eps2=eps,
                        skel_total=sum(st.skel[h].size for h in st.skel),
                        far_pairs=sum(len(v) for v in st.far.values()))
    print(f"compress {t1 - t0:.1f}s evaluate {t2 - t1:.1f}s eps2 {eps:.4e} -> {out}")


if __name__ == "__main__":
    main()
