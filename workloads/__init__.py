"""Seeded synthetic inputs for GOFMM evaluation: point clouds, kernel-matrix
entry routines and right-hand sides.

This module defines the *problem instances* only.  It holds none of the
method's arithmetic (no distances between Gram vectors, no trees, no
skeletons, no evaluation).  Both the FP64 oracle and the native library take
their inputs from here:

* the oracle receives an entry routine ``K(I, J)`` -- the only input the
  method requires (§1, problem statement: a routine that returns K_IJ for
  arbitrary row and column index sets);
* the native library receives either the same routine as a callback, or the
  points and kernel parameters for its own built-in generator.

Kernel families (the synthetic stand-ins for the paper's "kernel matrices in
six dimensions" class and its Gaussian-kernel learning workloads, §3):

* Gaussian:  K_ij = exp(-|x_i - x_j|^2 / (2 h^2)) + shift * [i == j]
* inverse multiquadric (IMQ):  K_ij = 1 / sqrt(1 + |x_i - x_j|^2 / l^2) + shift * [i == j]

Both are SPD for distinct points and shift > 0.  The squared distance is
accumulated coordinate by coordinate in index order so that every consumer
that follows the same recipe obtains bit-identical squared distances.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

GAUSSIAN = "gaussian"
IMQ = "imq"


@dataclasses.dataclass
class KernelMatrix:
    """An SPD kernel matrix given by points; callable as ``K(I, J)``.

    The points are private to the instance: a method that is handed this
    object sees only blocks of entries (``__call__``) and diagonal entries
    (``diag``).
    """

    kind: str
    points: np.ndarray  # (N, d) float64, row-major
    bandwidth: float    # h for Gaussian, l for IMQ
    shift: float        # added on the diagonal

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def dim(self) -> int:
        return int(self.points.shape[1])

    def sqdist(self, I: np.ndarray, J: np.ndarray) -> np.ndarray:
        X = self.points
        I = np.asarray(I, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        acc = np.zeros((I.size, J.size), dtype=np.float64)
        for k in range(X.shape[1]):
            diff = X[I, k][:, None] - X[J, k][None, :]
            acc += diff * diff
        return acc

    def _f(self, d2: np.ndarray) -> np.ndarray:
        h = self.bandwidth
        if self.kind == GAUSSIAN:
            return np.exp(-(d2 / (2.0 * h * h)))
        if self.kind == IMQ:
            return 1.0 / np.sqrt(1.0 + d2 / (h * h))
        raise ValueError(self.kind)

    def __call__(self, I, J) -> np.ndarray:
        I = np.asarray(I, dtype=np.int64).reshape(-1)
        J = np.asarray(J, dtype=np.int64).reshape(-1)
        out = self._f(self.sqdist(I, J))
        if self.shift != 0.0:
            eq = I[:, None] == J[None, :]
            out[eq] += self.shift
        return out

    def diag(self, I) -> np.ndarray:
        I = np.asarray(I, dtype=np.int64).reshape(-1)
        return self._f(np.zeros(I.size)) + self.shift

    def dense(self) -> np.ndarray:
        idx = np.arange(self.n)
        return self(idx, idx)

    def block_callback(self) -> Callable:
        """Entry routine in the C-ABI callback form: fills ``out`` (row-major
        nI x nJ, float64) with K(I, J) and returns 0."""

        def fn(I: np.ndarray, J: np.ndarray, out: np.ndarray) -> int:
            out[...] = self(I, J)
            return 0

        return fn


# --------------------------------------------------------------------------
# Workload definitions.  Each is fully determined by its seeds.
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    n: int
    dim: int
    dist: str            # "uniform" (unit cube) or "normal" (standard normal)
    kernel: str
    bandwidth: float
    shift: float
    leaf_size: int
    max_rank: int
    tau: float
    kappa: int
    budget: float
    r: int
    point_seed: int
    w_seed: int
    entries_via_callback: bool = False

    def points(self) -> np.ndarray:
        rng = np.random.Generator(np.random.PCG64(self.point_seed))
        if self.dist == "uniform":
            return rng.random((self.n, self.dim))
        if self.dist == "normal":
            return rng.standard_normal((self.n, self.dim))
        raise ValueError(self.dist)

    def matrix(self) -> KernelMatrix:
        return KernelMatrix(self.kernel, self.points(), self.bandwidth, self.shift)

    def rhs(self, r: Optional[int] = None, dtype=np.float64) -> np.ndarray:
        r = self.r if r is None else r
        rng = np.random.Generator(np.random.PCG64(self.w_seed))
        return rng.standard_normal((self.n, r)).astype(dtype)

    def params(self, **over) -> dict:
        p = dict(leaf_size=self.leaf_size, max_rank=self.max_rank, tau=self.tau,
                 kappa=self.kappa, budget=self.budget)
        p.update(over)
        return p


# Plain FP64 GOFMM at N = 4096 (entries only through a callback).
C1 = Workload("gaussian3d_n4096_fp64", 4096, 3, "uniform", GAUSSIAN, 0.3, 1e-3,
              leaf_size=64, max_rank=64, tau=1e-5, kappa=32, budget=0.03, r=16,
              point_seed=1, w_seed=2, entries_via_callback=True)

# FP32 GPU evaluate at N = 65536, r = 512 (the throughput workload).
C2 = Workload("gaussian6d_n65536_r512", 65536, 6, "normal", GAUSSIAN, 0.8, 1e-2,
              leaf_size=128, max_rank=256, tau=1e-5, kappa=32, budget=0.03, r=512,
              point_seed=3, w_seed=4)

# Precision study at N = 131072, r = 2048 (IMQ kernel).
C3 = Workload("imq4d_n131072_r2048", 131072, 4, "uniform", IMQ, 0.5, 1e-2,
              leaf_size=256, max_rank=512, tau=1e-6, kappa=32, budget=0.03, r=2048,
              point_seed=5, w_seed=6)

# A workload whose compression reaches an eps2 against the exact K W below
# 1e-4 at the throughput workload's N and r: the FP64 workload's 3-D Gaussian
# (h 0.3 on the unit cube) at N = 65536, m 128, s 256 (ranks stay below the
# cap: mean 80, max 240), tau 1e-9, r = 512; eps2 2.4e-5 (FP64 evaluation).
ACCURATE = Workload("gaussian3d_n65536_r512", 65536, 3, "uniform", GAUSSIAN, 0.3, 1e-3,
                    leaf_size=128, max_rank=256, tau=1e-9, kappa=32, budget=0.03, r=512,
                    point_seed=1, w_seed=2)

WORKLOADS = {w.name: w for w in (C1, C2, C3, ACCURATE)}


def scaled(w: Workload, n: int, r: Optional[int] = None, **over) -> Workload:
    """Same recipe at another size (tests use this for fast cases)."""
    d = dataclasses.asdict(w)
    d.update(n=n, name=f"{w.name}@n{n}")
    if r is not None:
        d["r"] = r
    d.update(over)
    return Workload(**d)


def batching_instances(count: int = 64, seed: int = 7):
    """Uneven instances for the batched form: N log-uniform in [2048, 65536],
    Gaussian with h ~ U[0.3, 1.0], d ~ U{2..8}, standard-normal points,
    shift 1e-2, tau 1e-5, max rank 256, leaf 256, r ~ U{16..256}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(2048), math.log(65536)))))
        h = float(rng.uniform(0.3, 1.0))
        d = int(rng.integers(2, 9))
        r = int(rng.integers(16, 257))
        out.append(Workload(f"batch{k}", n, d, "normal", GAUSSIAN, h, 1e-2,
                            leaf_size=256, max_rank=256, tau=1e-5, kappa=32,
                            budget=0.03, r=r, point_seed=1000 + k, w_seed=2000 + k))
    return out


def sample_rows(n: int, count: int = 100, seed: int = 11) -> np.ndarray:
    """Seeded row sample for the accuracy metric (§3: 100 sampled rows)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int64)


def serving_matrices(seed: int = 8):
    """Eight resident matrices for the serving workload: N in {16384, 32768,
    65536, 131072, 262144, 32768, 65536, 131072}, Gaussian (h 0.8) and
    inverse multiquadric (l 0.5) alternating, d ~ U{3..6}, standard-normal
    points, shift 1e-2, tau 1e-5, m 256, s 256, kappa 32, budget 3 %."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = [16384, 32768, 65536, 131072, 262144, 32768, 65536, 131072]
    out = []
    for k, n in enumerate(ns):
        d = int(rng.integers(3, 7))
        kern, bw = (GAUSSIAN, 0.8) if k % 2 == 0 else (IMQ, 0.5)
        out.append(Workload(f"serve{k}", n, d, "normal", kern, bw, 1e-2, leaf_size=256, max_rank=256,
                            tau=1e-5, kappa=32, budget=0.03, r=512, point_seed=3000 + k, w_seed=4000 + k))
    return out


def serving_requests(count: int = 2000, n_matrices: int = 8, seed: int = 9):
    """Seeded request stream: matrix uniform over the resident ones, r
    uniform in [1, 512], unit-rate exponential inter-arrival gaps (scale by
    the arrival rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mats = rng.integers(0, n_matrices, size=count)
    rs = rng.integers(1, 513, size=count)
    gaps = rng.exponential(1.0, size=count)
    return mats, rs, gaps


def hss_fmm_cases():
    """Fixed-rank HSS (budget 0) against FMM (budget 3 % and 10 %) on two
    synthetic kernels, r = 512 right-hand sides, tau = 0 (every node keeps
    min(s, its columns) skeletons): the 6-D Gaussian recipe of the throughput
    workload at N = 16384 (m 128) and the 3-D Gaussian of the FP64 workload
    at N = 4096 (m 64).  Returns [(label, workload)]."""
    out = []
    base = [(scaled(C2, 16384, r=512, leaf_size=128, tau=0.0, name="gaussian6d_n16384"),
             [(64, 0.0), (128, 0.0), (256, 0.0), (512, 0.0), (64, 0.03), (64, 0.10), (128, 0.03),
              (128, 0.10), (256, 0.03)]),
            (scaled(C1, 4096, r=512, leaf_size=64, tau=0.0, name="gaussian3d_n4096",
                    entries_via_callback=False),
             [(32, 0.0), (64, 0.0), (128, 0.0), (256, 0.0), (32, 0.03), (32, 0.10), (64, 0.03), (64, 0.10)])]
    for w, cfgs in base:
        for s, b in cfgs:
            label = f"{w.name} {'HSS' if b == 0 else 'FMM'} s{s} budget {b:.0%}"
            out.append((label, dataclasses.replace(w, max_rank=s, budget=b)))
    return out
