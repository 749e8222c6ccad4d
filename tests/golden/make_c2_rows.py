"""Write tests/golden/c2_rows.npz: sampled rows of K~W for the FP32
throughput workload (Gaussian h = 0.8, 6-D standard normal points, N = 65536,
m = 128, s = 256, tau = 1e-5, kappa = 32, budget 3 %, W = its seeded
N x 512 right-hand side), computed by the FP64 oracle alone.

Stored: 100 seeded rows x all 512 columns of the oracle's K~W, of its
absolute-value evaluation (Alg. 7 on |P|, |K|, |W|: the element-wise
rounding-error scale), of the exact K W and of the exact |K| |W| (the
sum condition of each row), and the oracle's eps2 on them.
The full-size GPU tests compare the library's evaluation at r = 512 against
these values, element by element.
Run:  python tests/golden/make_c2_rows.py   (about five minutes)
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
    w = wl.C2
    K = w.matrix()
    t0 = time.time()
    st = O.compress(K, w.n, O.Params(**w.params()))
    t1 = time.time()
    W = w.rhs(r=w.r)
    rows = wl.sample_rows(w.n)
    U = O.evaluate(st, K, W)[rows]
    t2 = time.time()
    Ua = O.evaluate_abs(st, K, W)[rows]
    exact = O.dense_rows(K, rows, W)
    kabs = O.dense_rows(O.AbsEntries(K), rows, np.abs(W))
    eps = O.eps2(U, exact)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_rows.npz")
    np.savez_compressed(out, rows=rows, cols=np.arange(w.r), u_oracle=U, u_abs=Ua,
                        u_exact=exact, u_kabs=kabs, eps2=eps,
                        skel_total=sum(st.skel[h].size for h in st.skel),
                        far_pairs=sum(len(v) for v in st.far.values()))
    print(f"compress {t1 - t0:.1f}s evaluate {t2 - t1:.1f}s eps2 {eps:.4e} -> {out}")


if __name__ == "__main__":
    main()
