#!/usr/bin/env python
"""Throughput of the GOFMM evaluation U = K~ W on B300.

Workload (one "step" = one whole evaluation, Alg. 7: gather, N2S, S2S, S2N,
L2L, scatter): the Gaussian kernel matrix on 65536 seeded 6-D standard
normal points (h = 0.8, shift 1e-2), compressed with m = 128, s = 256,
tau = 1e-5, kappa = 32, budget 3 %, times a seeded FP32 N x 512 block W.
Compression runs once before timing (host FP64).

  python bench.py [--steps K] [--warmup W] [--precision fp32] [--impl native|reference]

One JSON line on stdout (rank 0).  With torchrun (N ranks, one GPU each) the
ranks evaluate independent right-hand-side blocks against the same
compressed matrix (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import pickle
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "GOFMM evaluate N·r/s & %roofline; serve p50/p99; vs plain FP32 at ε2≤1e-4"
UNIT = "N*r/s"
WORKLOAD = wl.C2
GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_rows.npz")
GOLDEN_C3 = os.path.join(ROOT, "tests", "golden", "imq4d_n131072_r2048_rows.npz")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic_tc_gemm.txt")
# B300: 148 SMs x 128 FP32 lanes x 2 flop (FMA) per clock
SMS, FP32_LANES = 148, 128
# tensor-core dense rate relative to BF16 (nominal: TF32 1.1 / BF16 2.25 PFLOP/s)
NOMINAL_RATIO = {"tf32": 1.1 / 2.25, "bf16": 1.0, "bf16x3": 1.0 / 3.0}
DTYPE_NAME = {"fp64": "f64", "fp32": "f32", "tf32": "tf32 (fp32 accumulate)", "bf16": "bf16 (fp32 accumulate)",
              "bf16x3": "bf16x3 split (hi*hi+hi*lo+lo*hi, fp32 accumulate)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="bf16x3",
                    help="headline mode: fp32 (CUDA cores) or tf32 / bf16 / bf16x3 (tensor cores)")
    ap.add_argument("--no-modes", action="store_true", help="skip timing the other precision modes")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched form")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision workload")
    ap.add_argument("--cache", default="blocks", choices=["blocks", "none"],
                    help="main workload with cached K blocks (default) or with every entry generated in the kernels")
    ap.add_argument("--no-generated", action="store_true",
                    help="skip the run without cached blocks (entries generated in the kernels)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default tensor-core configuration instead of autotuning it")
    ap.add_argument("--config", default="",
                    help="force the tensor-core configuration of the main workload, piece/schedule/order "
                         "(e.g. 128/staged/local); no autotuning")
    ap.add_argument("--no-study", action="store_true", help="skip the HSS-vs-FMM accuracy/time study")
    ap.add_argument("--n", type=int, default=0,
                    help="profiling only: the same recipe at another N (not a bench line)")
    ap.add_argument("--budget", type=float, default=0.0,
                    help="profiling only, with --n: another near-field budget (e.g. 0.06 at N = 32768 keeps "
                         "the 15 near leaves per leaf of N = 65536 at 3 %%)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks --
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.path = tempfile.mktemp(prefix="gofmm_clocks_", suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for rec in csv.reader(f):
                    if len(rec) >= 9:
                        rows.append([x.strip() for x in rec])
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ oracle --
def oracle_structure(w: wl.Workload):
    """The oracle's compression of workload w, cached in the temp directory
    under a hash of the oracle source and the workload (compression is not
    part of any timed number)."""
    import oracle as O
    src = open(os.path.join(ROOT, "oracle", "gofmm_oracle.py"), "rb").read()
    key = hashlib.sha256(src + repr(sorted(w.params().items())).encode() + w.name.encode()).hexdigest()[:16]
    path = os.path.join(tempfile.gettempdir(), f"gofmm_oracle_{w.name}_{key}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    st = O.compress(w.matrix(), w.n, O.Params(**w.params()))
    with open(path + ".tmp", "wb") as f:
        pickle.dump(st, f)
    os.replace(path + ".tmp", path)
    return st


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 0) for d in threadpool_info() if d.get("user_api") == "blas"]
        return int(max(n)) if n else os.cpu_count()
    except Exception:
        return os.cpu_count()


def cpu_baseline(w: wl.Workload, r_sample: int = 16):
    import oracle as O
    st = oracle_structure(w)
    K = w.matrix()
    W = w.rhs(w.r)[:, :r_sample]
    t0 = time.perf_counter()
    O.evaluate(st, K, W)
    t = time.perf_counter() - t0
    return {"value": w.n * r_sample / t, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": f"FP64 oracle evaluation (Alg. 7, numpy) of the whole N={w.n} matrix on "
                      f"{r_sample} of the {w.r} right-hand-side columns; oracle compression untimed",
            "seconds": round(t, 3)}


def reference_arm(args):
    """The oracle as it stands on the host cores.  One step = the rows of
    K~ W for 4 leaves (512 rows, all 512 columns), which includes the full
    upward pass; value = rows * r / seconds."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    w = WORKLOAD
    st = oracle_structure(w)
    K = w.matrix()
    W = w.rhs(w.r)
    nl = st.tree.n_leaves
    per_step = 4

    def step(i):
        leaves = [(i * per_step + k) * 37 % nl for k in range(per_step)]
        out = O.evaluate_leaves(st, K, W, leaves)
        return sum(v.shape[0] for v in out.values())

    for i in range(args.warmup):
        step(i)
    rows = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        rows += step(args.warmup + i)
    t = time.perf_counter() - t0
    value = rows * w.r / t
    sample = (f"FP64 oracle rows of K~W for {per_step} leaves per step ({per_step * w.leaf_size} of "
              f"{w.n} rows, all {w.r} columns, full upward pass each step); oracle compression untimed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(w, "fp64-oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def config_dict(w, precision, cache="blocks"):
    return {"workload": w.name, "N": w.n, "r": w.r, "dim": w.dim, "kernel": "gaussian",
            "h": w.bandwidth, "m": w.leaf_size, "s": w.max_rank, "tau": w.tau, "kappa": w.kappa,
            "budget": w.budget, "precision": precision, "cache": cache,
            "l2": ("inputs larger than L2: the cached K blocks (>= 4 GB in FP32) are read every step"
                   if cache == "blocks" else "no cached blocks: entries generated in the GEMM kernels; "
                   "W and the skeleton weights (>= 0.6 GB) are larger than L2")}


# ------------------------------------------------------------ multi-rank --
def shared_handle(G, entries, params, rank, world, barrier, path, device=0):
    """Rank 0 compresses and writes a checkpoint, the other ranks import it:
    every rank evaluates the same compressed matrix."""
    if world == 1:
        return G.compress(entries, params)
    h = None
    if rank == 0:
        h = G.compress(entries, params)
        G.export(h, path)
    barrier()
    if rank != 0:
        h = G.import_(path, entries, params.cache_mode, device)
    return h


def rank_rhs_seed(w, rank):
    """Every rank multiplies its own right-hand sides (weak scaling)."""
    return w.w_seed + rank


def whole_job_value(n, r, world, ms_per_rank, reduce_max):
    """Units of all ranks over the slowest rank's time: (value, max ms)."""
    ms_max = reduce_max(ms_per_rank)
    return n * r * world / (ms_max / 1e3), ms_max


# -------------------------------------------------------- batching/serving --
SCHED_NAMES = ["fused", "staged", "pair", "hybrid"]  # GOFMM_SCHED_*
ORDER_NAMES = ["critical", "local", "schedule", "ready", "levels"]  # GOFMM_ORDER_*


def compress_many(G, works, device):
    """Native host compression of several workloads (no GPU work)."""
    out = []
    for w in works:
        pts = w.points()
        ent = (G.Entries.gaussian(pts, w.bandwidth, w.shift) if w.kernel == wl.GAUSSIAN
               else G.Entries.imq(pts, w.bandwidth, w.shift))
        out.append(G.compress(ent, G.default_params(**w.params(), device=device)))
    return out


def batching_bench(G, torch, dev, works, handles, steps, warmup, tuning=True):
    """64 uneven instances (N log-uniform in [2048, 65536], r in {16..256})
    as one static batch, replayed as a CUDA graph: either one
    dependency-driven launch for every stage of all of them or one grouped
    launch per stage step (the batch autotuner's choice); compared with the
    same 64 evaluations issued one after another."""
    prec = G.PREC_BF16X3
    stream = torch.cuda.current_stream(dev)
    for w, h in zip(works, handles):
        G.prepare(h, w.r, prec)
    tune = G.autotune_batch(handles, [w.r for w in works], prec, None, stream) if tuning else None
    for h in handles:
        G.trim(h)
    Ws = [torch.from_numpy(w.rhs().astype(np.float32)).to(dev) for w in works]
    Us = [torch.empty_like(W) for W in Ws]
    B = G.Batch(handles, [w.r for w in works], prec)
    for _ in range(max(warmup, 2)):
        B.evaluate(Ws, Us, stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        B.evaluate(Ws, Us, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    if B.info()["error"]:
        raise RuntimeError("batched evaluation reported a kernel error")
    ms = a.elapsed_time(b) / steps
    # the same evaluations one by one (each replayed from its own graph)
    seq_ref = [torch.empty_like(W) for W in Ws]
    for _ in range(2):
        for h, W, U in zip(handles, Ws, seq_ref):
            G.evaluate(h, W, U, prec, stream)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(max(1, steps // 2)):
        for h, W, U in zip(handles, Ws, seq_ref):
            G.evaluate(h, W, U, prec, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = a.elapsed_time(b) / max(1, steps // 2)
    same = all(torch.equal(U, R) for U, R in zip(Us, seq_ref))
    nr = sum(w.n * w.r for w in works)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    peak = peaks.get("bf16_tflops", 1800.0) * NOMINAL_RATIO["bf16x3"]
    hbm = peaks.get("hbm_gbs", 6400.0)
    # roofline of the batch: each instance's algorithmic flops (T part of P)
    # and bytes (cached blocks and T entries once at 4 B, W read once,
    # skeleton weights and potentials written and read once, U written once)
    # against the split-BF16 tensor peak and the HBM bandwidth; the batch's
    # bound is the sum over instances of the larger of the two times
    flops = alg_bytes = bound_s = 0.0
    for w, h in zip(works, handles):
        st = G.stats(h)
        f = w.r * (st["flops_n2s"] + st["flops_s2s"] + st["flops_s2n"] + st["flops_l2l"])
        by = ((st["near_entries"] + st["far_entries"] + st["interp_t_entries"]) * 4 + w.n * w.r * 4
              + 4 * st["skel_total"] * w.r * 4 + w.n * w.r * 4)
        flops += f
        alg_bytes += by
        bound_s += max(f / (peak * 1e12), by / (hbm * 1e9))
    info = B.info()
    B.free()
    return {"workload": "64 Gaussian instances, N log-uniform [2048, 65536], d U{2..8}, h U[0.3, 1], "
                        "r U{16..256}, m 256, s 256, tau 1e-5; split BF16x3",
            "instances": len(works), "sum_N_r": nr, "ms_per_batch": ms, "value": nr / (ms / 1e3),
            "unit": UNIT, "launches_per_batch": info["launches"], "graph": True,
            "flops_per_batch": flops, "tflops": flops / (ms / 1e3) / 1e12,
            "frac_of_split_bf16_peak": flops / (ms / 1e3) / 1e12 / peak,
            "roofline": {"algorithmic_bytes": alg_bytes, "bound": "hbm" if alg_bytes / (hbm * 1e9) > flops / (peak * 1e12)
                         else "tensor", "tensor_ms": flops / (peak * 1e12) * 1e3,
                         "hbm_ms": alg_bytes / (hbm * 1e9) * 1e3, "bound_ms": bound_s * 1e3,
                         "frac_of_bound": bound_s * 1e3 / ms, "hbm_gbs": hbm, "split_bf16_tflops": peak,
                         "note": "per instance the larger of algorithmic flops / tensor peak and algorithmic bytes / "
                                 "HBM bandwidth, summed over the instances (of measured peaks)"},
            "sequential_ms": seq_ms, "sequential_value": nr / (seq_ms / 1e3),
            "bitwise_equal_to_sequential": bool(same),
            "autotune": None if tune is None else {
                "piece": tune["piece"], "schedule": SCHED_NAMES[tune["schedule"]],
                "candidates_ms": {f'{c["piece"]}/{SCHED_NAMES[c["schedule"]]}': round(c["ms"], 4)
                                  for c in tune["candidates"]}}}


def precision_bench(G, torch, dev, w, h, steps, tuning=True):
    """The precision workload (IMQ, 4-D uniform points, N = 131072, m 256,
    s 512, tau 1e-6, r = 2048): every mode timed, with eps2 against the FP64
    oracle rows of the same structure and against the exact K W rows."""
    g = np.load(GOLDEN_C3) if os.path.exists(GOLDEN_C3) else None
    W = torch.from_numpy(w.rhs(w.r).astype(np.float32)).to(dev)
    U = torch.empty_like(W)
    stream = torch.cuda.current_stream(dev)
    st = G.stats(h)
    flops = w.r * (st["flops_n2s"] + st["flops_s2s"] + st["flops_s2n"] + st["flops_l2l"])
    out = {"workload": f"{w.name}: IMQ l 0.5, 4-D uniform points, N {w.n}, m {w.leaf_size}, s {w.max_rank}, "
                       f"tau {w.tau}, r {w.r}", "flops_per_step": flops, "modes": {}}
    for name in ("fp32", "tf32", "bf16", "bf16x3"):
        pr = G.PRECISIONS[name]
        G.prepare(h, w.r, pr)
        tune = G.autotune(h, w.r, pr, None, stream) if name != "fp32" and tuning else None
        for _ in range(2):
            G.evaluate(h, W, U, pr, stream)
        G.synchronize(h, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nst = max(2, min(steps, 5))
        a.record(stream)
        for _ in range(nst):
            G.evaluate(h, W, U, pr, stream)
        b.record(stream)
        G.synchronize(h, stream)
        ms = a.elapsed_time(b) / nst
        ent = {"ms": ms, "value": w.n * w.r / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12}
        if tune is not None:
            ent["config"] = {k: tune[k] for k in ("piece", "schedule", "order")}
            ent["tune_ms"] = [round(c["ms"], 4) for c in tune["candidates"]]
        if g is not None:
            got = U[torch.from_numpy(g["rows"]).to(dev)][:, : g["u_oracle"].shape[1]].double().cpu().numpy()
            ent["eps2_vs_oracle_fp64"] = float(np.linalg.norm(got - g["u_oracle"]) / np.linalg.norm(g["u_oracle"]))
            ent["eps2_vs_exact_KW"] = float(np.linalg.norm(got - g["u_exact"]) / np.linalg.norm(g["u_exact"]))
        out["modes"][name] = ent
    return out


def serving_bench(G, torch, dev, works, handles, loads=(0.5, 0.8, 1.0), prec_name="bf16"):
    """Continuous batching over 8 resident matrices: seeded Poisson arrivals,
    matrix uniform, r uniform in [1, 512], tensor cores in `prec_name` (BF16
    as the serving workload states; split BF16x3 for eps2 <= 1e-4); admission
    by a workspace pool sized from free HBM.  Saturation throughput from a
    closed run (all requests at t = 0), then open-loop runs at fractions of
    it with p50/p99 latency (arrival to completion, host clock)."""
    import time as _t
    prec = G.PRECISIONS[prec_name]
    for h in handles:
        G.prepare(h, 512, prec)
        G.trim(h)  # keep only the tensor-core tiles resident
    Wfull = [torch.from_numpy(w.rhs(512).astype(np.float32)).to(dev) for w in works]
    free, _ = torch.cuda.mem_get_info(dev)
    reserve = 16 << 30
    pool = int(max(4 << 30, min((free - reserve) // 2, 64 << 30)))   # request workspaces
    out_budget = int(max(2 << 30, min((free - reserve) // 2, 64 << 30)))  # request outputs U
    eng = G.Engine(prec, pool, dev.index or 0)
    mats, rs, gaps = wl.serving_requests()
    stream = torch.cuda.current_stream(dev)
    units = np.array([works[m].n * int(r) for m, r in zip(mats, rs)], dtype=np.float64)

    def run(arrivals):
        pending = {}
        lat = np.zeros(len(mats))
        i = done = 0
        waiting = []          # arrived, output not yet allocated (admission by free HBM)
        inflight = []         # events of the steps the GPU may still be running
        used = 0
        t0 = _t.perf_counter()
        while done < len(mats):
            now = _t.perf_counter() - t0
            while i < len(mats) and arrivals[i] <= now:
                waiting.append(i)
                i += 1
            while waiting:
                k = waiting[0]
                m, r = int(mats[k]), int(rs[k])
                need = works[m].n * r * 4
                if used + need > out_budget and pending:
                    break
                U = torch.empty((works[m].n, r), dtype=torch.float32, device=dev)
                rid = eng.submit(handles[m], Wfull[m][:, :r], U)
                pending[rid] = (k, U, need)
                used += need
                waiting.pop(0)
            if pending:
                # at most two steps in flight: the host prepares step k + 1
                # while the GPU runs step k
                eng.step(stream)
                ev = torch.cuda.Event()
                ev.record(stream)
                inflight.append(ev)
                if len(inflight) > 2:
                    inflight.pop(0).synchronize()
                tnow = _t.perf_counter() - t0
                for rid in list(pending):
                    if eng.poll(rid) == G.Engine.DONE:
                        k, _U, need = pending.pop(rid)
                        used -= need
                        lat[k] = tnow - arrivals[k]
                        done += 1
            elif i < len(mats):
                _t.sleep(max(0.0, min(1e-3, arrivals[i] - now)))
        stream.synchronize()
        return lat, _t.perf_counter() - t0

    run(np.zeros(len(mats)))  # warm-up (graphs, caches, allocator)
    lat0, t_sat = run(np.zeros(len(mats)))
    sat_rate = len(mats) / t_sat
    out = {"workload": "8 resident matrices (N 16384..262144, Gaussian h 0.8 / IMQ l 0.5, d 3..6, m 256, "
                       f"s 256, tau 1e-5); 2000 seeded requests, matrix uniform, r U[1, 512]; {prec_name}",
           "pool_bytes": pool, "output_budget_bytes": out_budget, "saturation": {"requests_per_s": sat_rate, "value": units.sum() / t_sat,
                                               "unit": UNIT, "seconds": t_sat},
           "loads": {}}
    for ld in loads:
        arrivals = np.cumsum(gaps) / (ld * sat_rate)
        lat, tt = run(arrivals)
        out["loads"][f"{ld:.1f}x"] = {"rate_per_s": ld * sat_rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                                      "p99_ms": float(np.percentile(lat, 99) * 1e3),
                                      "value": units.sum() / tt, "unit": UNIT}
    st = eng.stats()
    out["engine"] = {"steps": st["steps"], "launches": st["launches"], "max_in_flight": st["max_active"]}
    eng.free()
    return out


def hss_fmm_study(G, torch, dev, steps=5):
    """Accuracy against time for fixed-rank HSS (budget 0, the paper's way to
    enforce HSS in §3) and FMM (budget 3 % and 10 %), as in §4 "Comparison
    between FMM and HSS" (Fig. 6): compression time on the host, evaluation
    time on the GPU in split BF16x3 (tensor cores, default launch
    configuration) and FP64 (CUDA cores), and eps2 of each against the exact
    K W on 100 seeded rows (FP64, from the workload's own entry routine)."""
    stream = torch.cuda.current_stream(dev)
    exact = {}
    cases = []
    for label, w in wl.hss_fmm_cases():
        K = w.matrix()
        rows = wl.sample_rows(w.n)
        Wn = w.rhs(w.r)
        if w.name not in exact:
            exact[w.name] = K(rows, np.arange(w.n)) @ Wn
        ref = exact[w.name]
        t0 = time.perf_counter()
        h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift),
                       G.default_params(**w.params(), device=dev.index or 0))
        st = G.stats(h)
        ent = {"case": label, "scheme": "HSS" if w.budget == 0 else "FMM", "N": w.n, "m": w.leaf_size,
               "s": w.max_rank, "budget": w.budget, "compress_s": round(time.perf_counter() - t0, 3),
               "mean_rank": round(st["mean_rank"], 1), "max_rank": st["max_rank"],
               "near_pairs": st["near_pairs"], "far_pairs": st["far_pairs"],
               "gflop_per_eval": w.r * (st["flops_n2s"] + st["flops_s2s"] + st["flops_s2n"] + st["flops_l2l"]) / 1e9}
        for name, dt in (("bf16x3", np.float32), ("fp64", np.float64)):
            pr = G.PRECISIONS[name]
            W = torch.from_numpy(Wn.astype(dt)).to(dev)
            U = torch.empty_like(W)
            G.prepare(h, w.r, pr)
            for _ in range(2):
                G.evaluate(h, W, U, pr, stream)
            G.synchronize(h, stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                G.evaluate(h, W, U, pr, stream)
            b.record(stream)
            G.synchronize(h, stream)
            got = U[torch.from_numpy(rows).to(dev)].double().cpu().numpy()
            ent[name] = {"eval_ms": round(a.elapsed_time(b) / steps, 4),
                         "eps2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
            del W, U
        G.free(h)
        cases.append(ent)
    return {"what": "fixed-rank HSS (budget 0) vs FMM (budget 3 %, 10 %), tau 0, r 512; eps2 against the exact "
                    "K W on 100 seeded rows; compression on the host, evaluation on the GPU",
            "cases": cases}


def accurate_bench(G, torch, dev, steps=10, tuning=True):
    """The evaluation at a configuration whose compression error is small:
    workloads.ACCURATE (3-D Gaussian, N = 65536, r = 512, ranks below the
    cap, tau 1e-9).  Split BF16x3 (autotuned) and FP64 timed; eps2 of each
    against the exact K W on 100 seeded rows (FP64, from the workload's own
    entry routine) and of BF16x3 against the FP64 evaluation (the precision
    error; the FP64 path matches the oracle to 1e-12 in the tests)."""
    w = wl.ACCURATE
    K = w.matrix()
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    h = G.compress(G.Entries.gaussian(K.points, w.bandwidth, w.shift),
                   G.default_params(**w.params(), device=dev.index or 0))
    comp = time.perf_counter() - t0
    st = G.stats(h)
    rows = wl.sample_rows(w.n)
    Wn = w.rhs(w.r)
    exact = K(rows, np.arange(w.n)) @ Wn
    flops = w.r * (st["flops_n2s"] + st["flops_s2s"] + st["flops_s2n"] + st["flops_l2l"])
    out = {"workload": f"{w.name}: Gaussian h {w.bandwidth} on {w.dim}-D uniform points, N {w.n}, m {w.leaf_size}, "
                       f"s {w.max_rank}, tau {w.tau}, budget {w.budget:.0%}, r {w.r}",
           "compress_s": round(comp, 2), "mean_rank": round(st["mean_rank"], 1), "max_rank": st["max_rank"],
           "flops_per_eval": flops, "modes": {}}
    got = {}
    for name, dt in (("fp64", np.float64), ("bf16x3", np.float32)):
        pr = G.PRECISIONS[name]
        W = torch.from_numpy(Wn.astype(dt)).to(dev)
        U = torch.empty_like(W)
        G.prepare(h, w.r, pr)
        tune = G.autotune(h, w.r, pr, None, stream) if name == "bf16x3" and tuning else None
        for _ in range(2):
            G.evaluate(h, W, U, pr, stream)
        G.synchronize(h, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            G.evaluate(h, W, U, pr, stream)
        b.record(stream)
        G.synchronize(h, stream)
        ms = a.elapsed_time(b) / steps
        got[name] = U[torch.from_numpy(rows).to(dev)].double().cpu().numpy()
        ent = {"ms": ms, "value": w.n * w.r / (ms / 1e3), "unit": UNIT, "tflops": flops / (ms / 1e3) / 1e12,
               "eps2_vs_exact_KW": float(np.linalg.norm(got[name] - exact) / np.linalg.norm(exact))}
        if tune is not None:
            ent["config"] = {k: tune[k] for k in ("piece", "schedule", "order")}
        out["modes"][name] = ent
        del W, U
    out["modes"]["bf16x3"]["eps2_vs_fp64_evaluation"] = float(
        np.linalg.norm(got["bf16x3"] - got["fp64"]) / np.linalg.norm(got["fp64"]))
    G.free(h)
    return out


# ------------------------------------------------------------------ native --
def native_arm(args):
    import torch

    import paper_1707_00164_b300 as G
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOAD if not args.n else wl.scaled(WORKLOAD, args.n, **({"budget": args.budget} if args.budget else {}))
    prec_name = args.precision
    # host-only compression of the batching and serving matrices, overlapped
    # with the throughput measurement below
    import threading
    extra = {}
    want_batch = rank == 0 and world == 1 and not args.no_batch and not args.n
    want_serve = rank == 0 and world == 1 and not args.no_serve and not args.n
    want_prec = rank == 0 and world == 1 and not args.no_precision and not args.n

    def _bg():
        try:
            if want_prec:
                extra["precision"] = (wl.C3, compress_many(G, [wl.C3], local)[0])
            if want_batch:
                bw = wl.batching_instances()
                extra["batch"] = (bw, compress_many(G, bw, local))
            if want_serve:
                sw = wl.serving_matrices()
                extra["serve"] = (sw, compress_many(G, sw, local))
        except Exception as e:  # reported in the JSON line
            extra["error"] = repr(e)[:300]

    bg = threading.Thread(target=_bg, daemon=True)
    bg.start()
    prec = G.PRECISIONS[prec_name]
    K = w.matrix()
    entries = G.Entries.gaussian(K.points, w.bandwidth, w.shift)
    params = G.default_params(**w.params(), device=local,
                              cache_mode=G.CACHE_NONE if args.cache == "none" else G.CACHE_BLOCKS)
    t0 = time.perf_counter()
    h = shared_handle(G, entries, params, rank, world,
                      (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None),
                      os.path.join(tempfile.gettempdir(), f"gofmm_bench_{w.name}.bin"), local)
    compress_s = time.perf_counter() - t0
    st = G.stats(h)
    r = w.r
    G.prepare(h, r, prec)
    Wn = wl.scaled(w, w.n, w_seed=rank_rhs_seed(w, rank)).rhs(r).astype(np.float32)
    W = torch.from_numpy(Wn).to(dev)
    U = torch.empty_like(W)
    stream = torch.cuda.current_stream(dev)
    # tensor-core launch configuration picked by the library's autotuner
    # (outside the timed region, like compression)
    tune = None
    if prec_name in ("tf32", "bf16", "bf16x3") and args.config:
        pc, sc, oc = args.config.split("/")
        G.set_tc_config(h, prec, int(pc), SCHED_NAMES.index(sc), ORDER_NAMES.index(oc))
        tune = dict(G.get_tc_config(h, prec), forced=True, candidates=[])
    elif prec_name in ("tf32", "bf16", "bf16x3") and not args.no_tune:
        tune = G.autotune(h, r, prec, None, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        G.evaluate(h, W, U, prec, stream)
    G.synchronize(h, stream)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            G.evaluate(h, W, U, prec, stream)
        e1.record(stream)
        G.synchronize(h, stream)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps

    def reduce_max(x):
        if world == 1:
            return x
        t = torch.tensor([x], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    value, ms_max = whole_job_value(w.n, r, world, ms, reduce_max)

    # CUDA-event timing on the evaluation's stream: the production path
    # (timing level 2: gather + the GEMM launch(es)) and a per-stage
    # breakdown (level 1: one launch per stage)
    def timed(level):
        G.set_timing(h, level)
        acc_t = {"gather": [], "upward": [], "s2s": [], "s2n": [], "leaf": [], "total": []}
        n_l = 0
        for _ in range(args.steps):
            G.evaluate(h, W, U, prec, stream)
            t = G.stage_times(h)
            n_l = t["launches"]
            for k in acc_t:
                acc_t[k].append(t[k])
        G.set_timing(h, 0)
        return {k: statistics.mean(v) for k, v in acc_t.items()}, n_l

    prod_ms, launches = timed(2)
    st_ms, _ = timed(1)

    # end to end through the C ABI with pinned host buffers: every step
    # copies its W in and its U out.  Asynchronous calls (the copies of one
    # step overlap the evaluation of the next; two result buffers
    # alternate), the clock stopped after the last step's U is on the host;
    # the synchronous call (each step waits for its U) reported beside it
    Wh = torch.from_numpy(Wn).pin_memory()
    Uhs = [torch.empty_like(Wh).pin_memory() for _ in range(2)]
    for k in range(2):
        G.evaluate_host_async(h, Wh.numpy(), Uhs[k].numpy(), prec, stream)
    G.synchronize(h, stream)
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        G.evaluate_host_async(h, Wh.numpy(), Uhs[i % 2].numpy(), prec, stream)
    G.synchronize(h, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        G.evaluate_host(h, Wh.numpy(), Uhs[0].numpy(), prec, stream)
    e2e_sync_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": w.n * r * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": Wn.nbytes,
           "d2h_bytes_per_step": Wn.nbytes}
    e2e_sync = {"value": w.n * r * world / e2e_sync_s, "unit": UNIT,
                "note": "gofmm_evaluate_host, each call waits for its U"}

    # accuracy against the oracle's rows (FP64 K~W, same structure) and the exact rows
    golden = np.load(GOLDEN) if (os.path.exists(GOLDEN) and w is WORKLOAD and rank == 0) else None

    def accuracy(pr):
        return accuracy_of(h, pr)

    def accuracy_of(hh, pr):
        if golden is None:
            return None
        G.evaluate(hh, W, U, pr, stream)
        G.synchronize(hh, stream)
        g = golden
        got = U[torch.from_numpy(g["rows"]).to(dev)][:, : g["u_oracle"].shape[1]].double().cpu().numpy()
        return {"eps2_vs_oracle_fp64": float(np.linalg.norm(got - g["u_oracle"]) / np.linalg.norm(g["u_oracle"])),
                "eps2_vs_exact_KW": float(np.linalg.norm(got - g["u_exact"]) / np.linalg.norm(g["u_exact"])),
                "rows": int(g["rows"].size), "cols": int(g["u_oracle"].shape[1])}

    acc = accuracy(prec)

    # every precision mode on the same matrix and W (context for the headline)
    modes = None
    if rank == 0 and not args.no_modes:
        modes = {}
        for name in ("fp32", "tf32", "bf16", "bf16x3"):
            pr = G.PRECISIONS[name]
            G.prepare(h, r, pr)
            for _ in range(3):
                G.evaluate(h, W, U, pr, stream)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            nst = max(3, min(args.steps, 10))
            a.record(stream)
            for _ in range(nst):
                G.evaluate(h, W, U, pr, stream)
            b.record(stream)
            G.synchronize(h, stream)
            mms = a.elapsed_time(b) / nst
            modes[name] = {"ms": mms, "value": w.n * r / (mms / 1e3), "accuracy": accuracy(pr)}

    # roofline of the grouped-GEMM kernel (all its launches in one evaluation)
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    # the dominant kernel: the grouped GEMM.  Tensor-core path: one
    # dependency-driven launch per evaluation doing N2S, S2S, S2N and L2L;
    # CUDA-core path: the S2S launch (the largest of its per-stage launches)
    flops_all = r * (st["flops_n2s"] + st["flops_s2s"] + st["flops_s2n"] + st["flops_l2l"])
    if prec_name in ("fp32", "fp64"):
        flops, launch_ms = r * st["flops_s2s"], st_ms["s2s"]
    else:  # every GEMM launch of the production path (one launch when fused)
        flops = flops_all
        launch_ms = prod_ms["upward"] + prod_ms["s2s"] + prod_ms["s2n"] + prod_ms["leaf"]
    achieved = flops / (launch_ms / 1e3) / 1e12
    gemm_ms = st_ms["upward"] + st_ms["s2s"] + st_ms["s2n"] + st_ms["leaf"]
    if prec_name in ("fp32", "fp64"):
        mhz = peaks.get("sm_max_mhz", 2032.0)
        per_lane = 2.0 if prec_name == "fp32" else 2.0 / 64.0
        peak = SMS * FP32_LANES * per_lane * mhz * 1e6 / 1e12
        bound, peak_src = "alu", f"derived: {SMS} SMs x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz"
    else:
        bf16 = peaks.get("bf16_tflops", 1800.0)
        peak = bf16 * NOMINAL_RATIO[prec_name]
        bound, peak_src = "tensor", (f"of measured bf16 burst ({bf16:.0f} TFLOP/s) x nominal ratio "
                                     f"{NOMINAL_RATIO[prec_name]:.3f} for {prec_name}")
    # DRAM bytes of the GEMM launches of one evaluation, per launch
    # configuration, from an ncu capture of the same kernel source (null
    # when the source, workload or precision differs)
    traffic = None
    tr = {}
    if os.path.exists(TRAFFIC_PATH):
        for line in open(TRAFFIC_PATH):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("#")[0].split("=", 1)
                tr[k.strip()] = v.strip()
        src = os.path.join(ROOT, "paper_1707_00164_b300", "csrc", tr.get("source", "-"))
        current = (tr.get("precision") == prec_name and os.path.exists(src) and tr.get("workload") == w.name
                   and args.cache == "blocks"
                   and hashlib.sha256(open(src, "rb").read()).hexdigest() == tr.get("sha256"))
        if current and tune is not None:
            cfg = (f"{tune['piece']}/{SCHED_NAMES[tune['schedule']]}/"
                   f"{ORDER_NAMES[tune['order']]}")
            traffic = float(tr[cfg]) if cfg in tr else None
    if prec_name in ("fp32", "fp64"):
        kdesc = "gemm_simt_kernel, S2S launch (every far pair of every level)"
    elif tune is None or tune["schedule"] == G.SCHED_FUSED:
        kdesc = (f"tc_gemm_kernel<{prec_name}>: one dependency-driven persistent launch per evaluation "
                 f"(all N2S, S2S, S2N and L2L tiles)")
    else:
        kname = "tc_gemm_pair_kernel" if tune["schedule"] == G.SCHED_PAIR else "tc_gemm_kernel"
        kdesc = f"{kname}<{prec_name}>: every launch of the staged schedule (N2S, S2S, S2N, L2L)"
    # algorithmic bytes of those launches: every cached block and the T part
    # of every interpolation matrix once (the identity part of P is a copy of
    # skeleton rows, counted with the right-hand sides), W read once,
    # skeleton weights and potentials written and read once each, U written
    # once (FP32)
    be = {"tf32": 4, "bf16": 2, "bf16x3": 4, "fp32": 4, "fp64": 8}[prec_name]
    alg_bytes = ((st["near_entries"] + st["far_entries"] + st["interp_t_entries"]) * be + w.n * r * be
                 + 4 * st["skel_total"] * r * be + w.n * r * 4)
    # per stage (one launch per stage, timing level 1): algorithmic flops and
    # bytes of the stage against the tensor (or ALU) and HBM peaks
    hbm = peaks.get("hbm_gbs", 6400.0)
    stage_work = {
        "upward": (r * st["flops_n2s"], st["interp_t_entries"] * be + w.n * r * be + st["skel_total"] * r * be),
        "s2s": (r * st["flops_s2s"], st["far_entries"] * be + 2 * st["skel_total"] * r * be),
        "s2n": (r * st["flops_s2n"], st["interp_t_entries"] * be + 2 * st["skel_total"] * r * be),
        "leaf": (r * st["flops_l2l"], st["near_entries"] * be + w.n * r * be + w.n * r * 4),
    }
    if st_ms["s2n"] < 0.01 * st_ms["s2s"]:
        # the tensor-core plan pulls each node's parent part into its S2S
        # task (no S2N launches): the S2N work is timed with S2S
        fs, bs = stage_work.pop("s2n")
        stage_work["s2s"] = (stage_work["s2s"][0] + fs, stage_work["s2s"][1] + bs)
    per_stage = {}
    for k, (fl, by) in stage_work.items():
        t = st_ms[k] / 1e3
        if t > 0:
            per_stage[k] = {"ms": round(st_ms[k], 4), "tflops": fl / t / 1e12, "frac_compute": fl / t / 1e12 / peak,
                            "gbs": by / t / 1e9, "frac_hbm": by / t / 1e9 / hbm}
    roofline = {"kernel": kdesc, "bound": bound, "algorithmic_bytes": alg_bytes, "per_stage": per_stage,
                "per_stage_note": ("one launch per stage (timing level 1); flops per stage from the structure; bytes "
                                   "= cached blocks / interpolation tiles of the stage once + right-hand sides read "
                                   "and written once; frac_compute against the peak above, frac_hbm against "
                                   f"{hbm:.0f} GB/s"),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": peak_src, "traffic": traffic, "flops_per_launch": flops,
                "launch_ms": launch_ms,
                "per_stage_breakdown_ms": {k: round(v, 4) for k, v in st_ms.items()},
                "per_stage_gemm_ms": gemm_ms}

    dense = None
    if rank == 0 and world == 1 and not args.no_dense:
        dense = dense_reference(torch, K, W, dev)

    bg.join()
    # the same matrix with no cached blocks (GOFMM_CACHE_NONE): every K block
    # generated inside the GEMM kernels, on the tensor cores (split BF16x3,
    # autotuned) and on the CUDA cores (plain FP32)
    generated = None
    if rank == 0 and world == 1 and not args.n and not args.no_generated:
        try:
            hg = G.compress(entries, G.default_params(**w.params(), device=local, cache_mode=G.CACHE_NONE))
            generated = {"cache": "none: block entries generated in the GEMM kernels"}
            for name in ("bf16x3", "fp32"):
                pr = G.PRECISIONS[name]
                G.prepare(hg, r, pr)
                tg = G.autotune(hg, r, pr, None, stream) if name != "fp32" else None
                for _ in range(2):
                    G.evaluate(hg, W, U, pr, stream)
                G.synchronize(hg, stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                nst = max(3, min(args.steps, 10))
                a.record(stream)
                for _ in range(nst):
                    G.evaluate(hg, W, U, pr, stream)
                b.record(stream)
                G.synchronize(hg, stream)
                gms = a.elapsed_time(b) / nst
                ent = {"ms": gms, "value": w.n * r / (gms / 1e3), "accuracy": accuracy_of(hg, pr)}
                if tg is not None:
                    ent["config"] = {k: tg[k] for k in ("piece", "schedule", "order")}
                # ALU / SFU roofline of the entry generation: every entry the
                # evaluation needs (near and far blocks, once) costs 3 d + 4
                # ALU operations (differences, squares and their sum, the
                # scale) and one SFU operation (exp or rsqrt); peaks from the
                # SM count, 128 FP32 lanes and 16 SFU lanes per SM, and the
                # SM clock sampled during the main run
                sgen = G.stats(hg)
                n_entries = sgen["near_entries"] + sgen["far_entries"]
                mhz = clk.summary().get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
                alu_ops = n_entries * (3 * w.dim + 4)
                alu_peak = SMS * FP32_LANES * mhz * 1e6
                sfu_peak = SMS * 16 * mhz * 1e6
                ent["generator_roofline"] = {
                    "bound": "alu", "entries_per_eval": n_entries, "ops_per_entry": 3 * w.dim + 4,
                    "achieved_gops": alu_ops / (gms / 1e3) / 1e9, "peak_gops": alu_peak / 1e9,
                    "frac": alu_ops / (gms / 1e3) / alu_peak,
                    "sfu_frac": n_entries / (gms / 1e3) / sfu_peak,
                    "alu_bound_ms": 1e3 * alu_ops / alu_peak,
                    "note": (f"derived peak: {SMS} SMs x {FP32_LANES} FP32 lanes x {mhz:.0f} MHz (one op per lane "
                             f"per clock); SFU {SMS} x 16 lanes; entries counted once (the kernel generates each "
                             f"block once per tile of r-tiles)")}
                generated[name] = ent
            G.free(hg)
        except Exception as e:
            generated = {"error": repr(e)[:300]}
    # compression of the throughput workload with the sampled blocks K_{I'a}
    # generated on the host and on the GPU (not part of any timed number)
    compression = None
    if rank == 0 and world == 1 and not args.n:
        compression = {}
        for mode in (0, 1):
            t0 = time.perf_counter()
            hc = G.compress(entries, G.default_params(**w.params(), device=local, sample_device=mode))
            compression["device_sampling_s" if mode else "host_sampling_s"] = round(time.perf_counter() - t0, 3)
            G.free(hc)
        compression["host_threads"] = os.cpu_count()
    batching = serving = precision = None
    if "precision" in extra:
        try:
            precision = precision_bench(G, torch, dev, *extra["precision"], steps=args.steps,
                                        tuning=not args.no_tune)
        except Exception as e:
            precision = {"error": repr(e)[:300]}
        extra.pop("precision")
    if "batch" in extra:
        try:
            batching = batching_bench(G, torch, dev, *extra["batch"], steps=max(3, min(args.steps, 10)),
                                      warmup=args.warmup, tuning=not args.no_tune)
        except Exception as e:
            batching = {"error": repr(e)[:300]}
        extra.pop("batch")
    if "serve" in extra:
        try:
            serving = serving_bench(G, torch, dev, *extra["serve"])
        except Exception as e:
            serving = {"error": repr(e)[:300]}
        try:  # the served form at eps2 <= 1e-4 against the FP64 oracle
            serving["bf16x3"] = serving_bench(G, torch, dev, *extra["serve"], prec_name="bf16x3")
        except Exception as e:
            serving["bf16x3"] = {"error": repr(e)[:300]}
        extra.pop("serve")
    if "error" in extra:
        batching = batching or {"error": extra["error"]}

    accurate = None
    if rank == 0 and world == 1 and not args.n and not args.no_study:
        try:
            accurate = accurate_bench(G, torch, dev, tuning=not args.no_tune)
        except Exception as e:
            accurate = {"error": repr(e)[:300]}
    study = None
    if rank == 0 and world == 1 and not args.n and not args.no_study:
        try:
            study = hss_fmm_study(G, torch, dev)
        except Exception as e:
            study = {"error": repr(e)[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAME[prec_name],
            "data": "synthetic: seeded 6-D standard-normal points, Gaussian kernel; seeded N(0,1) W",
            "config": config_dict(w, prec_name, args.cache), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(), "e2e": e2e, "e2e_sync": e2e_sync, "gpu_launches": launches * args.steps,
            "autotune": tune, "accuracy": acc, "modes": modes, "dense_cublas": dense, "precision_workload": precision, "batching": batching,
            "serving": serving, "hss_vs_fmm": study, "accurate_workload": accurate,
            "compress_seconds": round(compress_s, 2), "compression": compression, "generated_blocks": generated,
            "structure": {k: st[k] for k in ("depth", "mean_rank", "max_rank", "near_pairs", "far_pairs",
                                              "near_entries", "far_entries")},
        }))
    if world > 1:
        torch.distributed.destroy_process_group()


def dense_reference(torch, K, W, dev):
    """cuBLAS dense K W on the same GPU for context (K materialised in FP32,
    N^2 * 4 bytes; SGEMM with TF32 off, then with TF32 on)."""
    n = K.n
    try:
        X = torch.from_numpy(K.points).to(dev)
        Kd = torch.empty((n, n), dtype=torch.float32, device=dev)
        inv = 1.0 / (2 * K.bandwidth ** 2)
        for i0 in range(0, n, 4096):
            d2 = torch.cdist(X[i0:i0 + 4096], X).square_()
            Kd[i0:i0 + 4096] = torch.exp(-d2 * inv).float()
        Kd.diagonal().add_(K.shift)
        del X
        out = {}
        for name, tf32 in (("sgemm", False), ("tf32", True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            torch.matmul(Kd, W)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                torch.matmul(Kd, W)
            b.record()
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / 3
            out[name] = {"ms": ms, "value": n * W.shape[1] / (ms / 1e3)}
        torch.backends.cuda.matmul.allow_tf32 = False
        del Kd
        torch.cuda.empty_cache()
        return out
    except Exception as e:  # context only; never fails the bench
        return {"error": str(e)[:200]}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
