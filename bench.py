"""Benchmark: exact KRP leverage-score sampling at scale on one GB300.

Workload (sampler at scale): N=3 factors of 2^22 x 32 FP32, N(0,1) with 1% of
rows x100, leaf size F=32, J=2^16 samples per draw.  One step = one draw
preceded by a full-factor update of factor d mod 3 with fresh N(0,1) rows
(tree rebuild), the per-draw preparation (G, G⁺, eigendecompositions, E_k),
the batched descent with weights, and the fused gather of the sketched rows SA.
All inputs are seeded and synthetic; every buffer is larger than L2 (129 MB),
and every step streams a 512 MiB factor and its 277 MB tree, so no L2 flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|bf16x3|exact] [--no-cpu-baseline]
                  [--workload sampler|batch512|rank_sweep|sparse_als|accuracy] [--rank R]
                  [--ranks 25,50,100] [--nnz N] [--sweeps S] [--trials T]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
(independent draws, disjoint draw ids); value = samples of all ranks / max time.
The default workload is the headline line; batch512 (512 small least-squares
problems: per-problem launches vs one launch per phase vs graph replay) and
rank_sweep (N=4, 2^20 x R, U(-1,1), J=2^17, dense solve with 8 planted
right-hand sides) and sparse_als (STS-CP on a 2^22 x 2^22 x 2^14 Zipf tensor:
FP32, BF16x3, TF32x3 and graph-replayed sweeps) and accuracy (Sec. 4.2: distortion
and residual ratio for N in {3..9}, R in {16, 32, 64}) print their own lines.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FACT, I_ROWS, RANK, LEAF, J_DRAW = 3, 1 << 22, 32, 32, 1 << 16
# dram__bytes_read.sum + dram__bytes_write.sum of one krp_descent_fast<32> launch of this
# workload (one-pass ncu capture of the first timed draw); to be re-taken whenever that kernel changes.
DESCENT_DRAM_BYTES = 3_818_774_016 + 12_289_536
METRIC = "KRP leverage samples/s (one-factor update + prepare + draw + gather per step)"
UNIT = "samples/s"
WORKLOAD = "krp_sampler_N3_I2^22_R32_F32_J2^16_update_per_draw"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "tf32x3", "exact"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="sampler: skip the other precision forms")
    ap.add_argument("--sts-sweeps", type=int, default=12,
                    help="sampler: STS-CP sweeps per precision at R=25 for the metric's second half (0 skips)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--sts-seeds", type=int, default=3, help="sampler: STS-CP sampling seeds per precision")
    ap.add_argument("--workload", default="sampler",
                    choices=["sampler", "batch512", "rank_sweep", "sparse_als", "accuracy"],
                    help="sampler: the headline line; batch512: 512 small least-squares problems "
                         "(per-problem launches vs one launch per phase vs graph replay); "
                         "rank_sweep: N=4, I=2^20, U(-1,1), J=2^17 at --rank R")
    ap.add_argument("--rank", type=int, default=32)
    ap.add_argument("--descent", choices=["auto", "team", "node_major", "node_major_tc"], default="auto",
                    help="rank_sweep: descent form for 32 < R <= 128")
    ap.add_argument("--ranks", default="25,50,100", help="sparse_als: decomposition ranks")
    ap.add_argument("--nnz", type=int, default=200_000_000, help="sparse_als: nonzeros")
    ap.add_argument("--sweeps", type=int, default=20, help="sparse_als: ALS sweeps per configuration")
    ap.add_argument("--trials", type=int, default=5, help="accuracy: problems per (N, R)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)}


# ------------------------------------------------------------ CPU oracle ----
def oracle_tree_steps(Us64, fresh64, n_steps, n_samples, d_first=0):
    """The FP64 oracle as it stands, stepping like the GPU workload: per step
    the one-factor update (factor d mod 3 replaced by its fresh rows, FP64
    segment tree rebuilt: Alg. 3), the per-draw preparation (Grams, G⁺,
    eigendecompositions) and n_samples draws of Alg. 2/4 on the FP64 trees
    (krp_sample_tree: samples d0 .. d0 + n_samples - 1 of the step's draw).
    The trees of the factors not updated are built once, untimed.  Returns
    (total samples, total seconds, per-step seconds)."""
    from oracle import krp_oracle as O
    cur = list(Us64)
    trees = {k: O.TreeFP64(cur[k], LEAF) for k in range(N_FACT)}
    total, steps = 0, []
    for d in range(d_first, d_first + n_steps):
        k = d % N_FACT
        t0 = time.perf_counter()
        cur[k] = fresh64[k]
        trees[k] = O.TreeFP64(cur[k], LEAF)
        prep = O.SamplerPrep(cur, -1)
        d0 = (d * n_samples) % J_DRAW
        O.krp_sample_tree(cur, -1, n_samples, 1, d, F=LEAF, d0=d0, prep=prep, trees=trees)
        steps.append(time.perf_counter() - t0)
        total += n_samples
    return total, sum(steps), steps


def cores_used():
    try:
        import numpy.__config__  # noqa: F401
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count()
    return n


REF_SAMPLES_PER_STEP = 2048


def run_reference(args, rank):
    """Reference arm: the CPU oracle timed on this machine's host cores, every
    step the GPU workload's step with a bounded draw: a one-factor update
    (FP64 tree rebuild), the preparation, and 2048 samples of the draw drawn
    by Alg. 2/4 on the FP64 segment trees.  value = samples drawn / time."""
    if rank != 0:
        return
    from paper_2301_12584_gb300 import synth
    Us = synth.skewed_row_factors(N_FACT, I_ROWS, RANK, seed=0)
    Us64 = [U.astype(np.float64) for U in Us]
    del Us
    fresh64 = [synth.fresh_factor(I_ROWS, RANK, seed=1000 + d).astype(np.float64) for d in range(N_FACT)]
    oracle_tree_steps(Us64, fresh64, args.warmup, REF_SAMPLES_PER_STEP)
    n, secs, per = oracle_tree_steps(Us64, fresh64, args.steps, REF_SAMPLES_PER_STEP, d_first=args.warmup)
    v = n / secs
    sample = (f"oracle per step: one-factor update (FP64 tree rebuild), preparation, and {REF_SAMPLES_PER_STEP} "
              f"samples of the step's J=2^16 draw by the FP64 tree descent (N=3, I=2^22, R=32, F=32); "
              f"value = samples drawn / time")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores_used(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------- other workloads ----
def _events_ms(stream, fn, steps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for d in range(steps):
        fn(d)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_batch512(args):
    """512 independent dense KRP least-squares problems: N=3, I_j log-uniform in
    [256, 65536] per factor, R from {8, 16, 32}, N(0,1) factors, 4 right-hand
    sides planted with 1e-3 noise, J=4096 samples each.  One batch = rebuild
    every tree from its source + prepare + sample + planted rows + solve."""
    import torch
    from paper_2301_12584_gb300 import krpls, synth
    from paper_2301_12584_gb300.krpls import Batch, Sampler
    P, N, J, NRHS = 512, 3, 4096, 4
    rng = np.random.default_rng(4)
    shapes = []
    for _ in range(P):
        R = int(rng.choice([8, 16, 32]))
        shapes.append(([int(np.exp(rng.uniform(np.log(256), np.log(65536)))) for _ in range(N)], R))
    dev = torch.device("cuda", 0)
    krpls.lib()
    stream = torch.cuda.Stream(device=dev)
    sams, srcs, xt = [], [], []
    for p, (I, R) in enumerate(shapes):
        Us = synth.gaussian_factors(N, I, R, seed=10_000 + p)
        d = [torch.from_numpy(U).to(dev) for U in Us]
        s = Sampler(I, R, R, stream=stream)
        for k in range(N):
            s.set_factor(k, d[k])
        sams.append(s)
        srcs += d
        xt.append(synth.planted_solution(R, NRHS, seed=20_000 + p).ravel())
    torch.cuda.synchronize()
    X_true = torch.from_numpy(np.concatenate(xt).astype(np.float32)).to(dev)
    batch = Batch(sams, stream)
    batch.set_sources(srcs)
    off = batch.row_off
    idx = torch.zeros((P, N, J), dtype=torch.int32, device=dev)
    w = torch.zeros((P, J), device=dev)
    SA = torch.zeros(J * off[-1], device=dev)
    B = torch.zeros((P, J, NRHS), device=dev)
    X = torch.zeros(off[-1] * NRHS, device=dev)

    def batched(d):
        batch.build()
        batch.sample(J, 1, d, idx, w, SA)
        batch.planted_rows(J, idx, X_true, NRHS, 1e-3, 2, B)
        batch.solve_dense(J, SA, w, B, NRHS, X)

    SAp = [SA[J * off[p]: J * off[p + 1]] for p in range(P)]
    Xp = [X[off[p] * NRHS: off[p + 1] * NRHS] for p in range(P)]
    Xtp = [X_true[off[p] * NRHS: off[p + 1] * NRHS] for p in range(P)]

    def per_problem(d):
        for p in range(P):
            s = sams[p]
            for k in range(N):
                s.set_factor(k, srcs[p * N + k])
            s.sample(-1, J, 1, d, idx[p], w[p], None, SAp[p])
            s.planted_rows(-1, J, idx[p], Xtp[p], NRHS, 1e-3, 2, B[p])
            s.solve_dense(J, SAp[p], w[p], B[p], NRHS, Xp[p])

    steps, warm = max(args.steps, 1), max(args.warmup, 3)
    with torch.cuda.stream(stream):
        for d in range(warm):
            per_problem(d)
        ms_per = _events_ms(stream, per_problem, steps)
        X_single = X.clone()
        best = batch.autotune(J)
        for d in range(warm):
            batched(d)
        ms_batched = _events_ms(stream, batched, steps)
        n0 = krpls.launch_count()
        batched(0)
        launches = krpls.launch_count() - n0
        torch.cuda.synchronize()
        batch.capture_begin()
        batched(0)
        nodes = batch.capture_end()
        for _ in range(warm):
            batch.replay()
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.2)
        ms_graph = _events_ms(stream, lambda d: batch.replay(), steps)
        clk = clocks.stop()
    assert batch.sync_status() == 0, "device status"
    Xb = X.cpu().numpy()
    Xs = X_single.cpu().numpy()
    Xt = X_true.cpu().numpy()
    err_planted, diff_single = [], []
    for p in range(P):
        sl = slice(off[p] * NRHS, off[p + 1] * NRHS)
        err_planted.append(np.linalg.norm(Xb[sl] - Xt[sl]) / np.linalg.norm(Xt[sl]))
        diff_single.append(np.linalg.norm(Xb[sl] - Xs[sl]) / np.linalg.norm(Xs[sl]))
    print(json.dumps({
        "metric": "512 KRP least-squares problems: tree builds + prepare + sample + planted rows + solve",
        "value": ms_graph, "unit": "ms per batch", "higher_is_better": False, "n_gpus": 1, "steps": steps,
        "warmup": warm, "dtype": "f32", "data": "synthetic", "vs_baseline": None,
        "config": {"workload": "batch512_N3_I[256,65536]_R{8,16,32}_J4096_nrhs4", "P": P, "J": J,
                   "rows_total": int(sum(sum(I) for I, _ in shapes)), "l2": "factors 1.3 GB > L2"},
        "per_problem_ms": ms_per, "batched_ms": ms_batched, "graph_ms": ms_graph,
        "speedup_graph_vs_per_problem": ms_per / ms_graph,
        "autotune": {"descent_ctas_per_problem": best},
        "gpu_launches_per_batch": launches, "graph_nodes": nodes,
        "x_rel_err_vs_planted_median": float(np.median(err_planted)),
        "x_rel_diff_batched_vs_per_problem_max": float(np.max(diff_single)),
        "clocks": clk,
    }), flush=True)


def run_rank_sweep(args):
    """N=4 factors of 2^20 x R, U(-1,1), F=R; one step = prepare + draw J=2^17
    (with SA) + planted rows (8 right-hand sides, 1e-3 noise) + dense solve."""
    import torch
    from paper_2301_12584_gb300 import krpls, synth
    from paper_2301_12584_gb300.krpls import Sampler
    N, I, R, J, NRHS = 4, 1 << 20, int(args.rank), 1 << 17, 8
    dev = torch.device("cuda", 0)
    krpls.lib()
    stream = torch.cuda.Stream(device=dev)
    Us = synth.uniform_factors(N, I, R, seed=0)
    s = Sampler([I] * N, R, R, stream=stream)
    s.set_descent_form({"auto": 0, "team": 1, "node_major": 2, "node_major_tc": 3}[args.descent])
    for k in range(N):
        s.set_factor(k, torch.from_numpy(Us[k]).to(dev))
    Xt = synth.planted_solution(R, NRHS, seed=1)
    X_true = torch.from_numpy(Xt).to(dev)
    idx = torch.zeros((N, J), dtype=torch.int32, device=dev)
    w = torch.zeros(J, device=dev)
    SA = torch.zeros((J, R), device=dev)
    B = torch.zeros((J, NRHS), device=dev)
    X = torch.zeros((R, NRHS), device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    phase = []

    def step(d, timed=True):
        e = [ev() for _ in range(5)]
        e[0].record(stream)
        s.sample_prepare(-1)
        e[4].record(stream)
        s.sample_draw(-1, J, 1, d, idx, w, None, SA)
        e[1].record(stream)
        s.planted_rows(-1, J, idx, X_true, NRHS, 1e-3, 2, B)
        e[2].record(stream)
        s.solve_dense(J, SA, w, B, NRHS, X)
        e[3].record(stream)
        if timed:
            phase.append(e)

    steps, warm = max(args.steps, 1), max(args.warmup, 3)
    with torch.cuda.stream(stream):
        for d in range(warm):
            step(d, False)
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.2)
        ms = _events_ms(stream, lambda d: step(warm + d), steps)
        clk = clocks.stop()
    assert s.sync_status() == 0, s.last_error()
    sample_ms = statistics.mean(p[0].elapsed_time(p[1]) for p in phase)
    prep_ms = statistics.mean(p[0].elapsed_time(p[4]) for p in phase)
    draw_ms = statistics.mean(p[4].elapsed_time(p[1]) for p in phase)
    solve_ms = statistics.mean(p[2].elapsed_time(p[3]) for p in phase)
    # descent roofline by nominal path bytes: every sample reads its whole
    # root-to-leaf path of Z_k (4 Tp bytes a level) and one leaf block per factor
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    Tp = (R * (R + 1) // 2 + 7) // 8 * 8
    depth = (-(-I // R) - 1).bit_length()
    path_bytes = N * (4 * Tp * depth + 4 * R * R)
    achieved = path_bytes * J / (draw_ms / 1e3) / 1e9
    kernel = "krp_descent_fast" if R <= 32 else (
        ("krp_descent_nm<64>" if R <= 64 else "krp_descent_nm<128>") if args.descent == "node_major" else
        "nt_level<0..3> + nt_scan + nt_part (tensor-core node-major)" if args.descent == "node_major_tc" else
        ("krp_descent_team<64,2>" if R <= 64 else "krp_descent_team<128,8>"))
    roof = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "algorithmic_bytes_per_launch": path_bytes * J,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "note": "nominal bytes; the upper tree levels are L2 hits, so DRAM traffic is lower"}
    # errors of the last step against FP64 on the same sketch, and against the planted X
    from oracle import krp_oracle as O
    SA64 = SA.cpu().numpy().astype(np.float64)
    SB64 = w.cpu().numpy().astype(np.float64)[:, None] * B.cpu().numpy().astype(np.float64)
    Xo = O.lstsq(SA64, SB64)
    Xg = X.cpu().numpy()
    print(json.dumps({
        "metric": "KRP leverage samples/s, rank sweep (prepare + draw + planted rows + dense solve per step)",
        "value": J / (ms / 1e3), "unit": "samples/s", "higher_is_better": True, "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": ms, "dtype": "f32", "data": "synthetic", "vs_baseline": None,
        "config": {"workload": f"rank_sweep_N4_I2^20_R{R}_J2^17_nrhs8", "R": R, "descent": args.descent,
                   "l2": "inputs larger than L2"},
        "phases_ms": {"prepare_and_draw": sample_ms, "prepare": prep_ms, "draw": draw_ms, "solve": solve_ms},
        "roofline": roof,
        "x_rel_err_vs_fp64_same_sketch": float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)),
        "x_rel_err_vs_planted": float(np.linalg.norm(Xg - Xt) / np.linalg.norm(Xt)),
        "clocks": clk,
    }), flush=True)


SPARSE_DIMS = (1 << 22, 1 << 22, 1 << 14)


def sparse_setup(nnz, dev, stream):
    """The synthetic 2^22 x 2^22 x 2^14 Zipf(1.1) tensor with nnz nonzeros
    (rank-16 U(0,1) values x lognormal(0, 0.5) noise), its fiber index, and
    the initial factors' row scales.  Returns (tensor, scales, seconds)."""
    from paper_2301_12584_gb300 import synth
    from paper_2301_12584_gb300.krpls import SparseTensor
    dims = SPARSE_DIMS
    t0 = time.perf_counter()
    coords, vals = synth.sparse_zipf_tensor(dims, int(nnz), seed=0, device=dev)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    t = SparseTensor(dims, coords, vals, stream=stream)
    t_index = time.perf_counter() - t0
    # Row scale of the initial factors: N(0,1) rows times sqrt(nonzeros of that
    # index + 0.01) / mean.  Plain N(0,1) rows give every index the same
    # leverage, and at this density (2^44 possible (i_0, i_1) fibers for the
    # 2^14 mode) the first sketches would see almost no nonzeros.
    scales = []
    for k in range(3):
        cnt = np.bincount(coords[k], minlength=dims[k]).astype(np.float64) + 0.01
        scales.append(np.sqrt(cnt / cnt.mean()).astype(np.float32))
    return t, scales, {"generate": t_gen, "index": t_index}


def sparse_rank_runs(t, scales, R, S, modes, dev, stream, seeds=(1,)):
    """S STS-CP sweeps (Alg. 6, J = 2^16 per solve) at rank R from the same
    start for each mode in `modes` (fp32, bf16x3, exact: the sampler's
    precision; fp32_graph: FP32 with sweeps 2..S replayed from a CUDA graph),
    once per sampling seed in `seeds`.  Per mode: median sweep time of sweeps
    2..S (over all seeds) and the fit after each sweep (fit not timed).  Each
    sweep's fit is that of one random sketch, so precisions are compared by
    the mean fit of the second half of the sweeps averaged over the seeds,
    next to FP32's own spread over the seeds."""
    import torch
    from paper_2301_12584_gb300 import krpls, synth
    from paper_2301_12584_gb300.krpls import Sampler
    dims, J = SPARSE_DIMS, 1 << 16
    Us0 = synth.gaussian_factors(3, list(dims), R, seed=0)
    Ud = [torch.from_numpy(U * sc[:, None]).to(dev) for U, sc in zip(Us0, scales)]
    del Us0
    row = {"R": R}
    precs = {"fp32": krpls.KRP_PREC_FP32, "bf16x3": krpls.KRP_PREC_BF16X3, "tf32x3": krpls.KRP_PREC_TF32X3,
             "exact": krpls.KRP_PREC_EXACT, "fp32_graph": krpls.KRP_PREC_FP32}
    for mode in modes:
        times, per_seed, fits_first, status = [], [], None, 0
        for seed in seeds:
            s = Sampler(list(dims), R, 0, precs[mode], stream=stream)
            for k in range(3):
                s.set_factor(k, Ud[k])
            sigma = torch.zeros(R, device=dev)
            fits = []
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                for sw in range(S):
                    if mode == "fp32_graph" and sw == 1:
                        s.capture_begin()
                        s.cp_als_sweep(t, J, seed, 3 * sw, sigma)
                        s.capture_end()
                    torch.cuda.synchronize()
                    a.record(stream)
                    if mode == "fp32_graph" and sw >= 1:
                        s.replay()
                    else:
                        s.cp_als_sweep(t, J, seed, 3 * sw, sigma)
                    b.record(stream)
                    torch.cuda.synchronize()
                    if sw >= 1:
                        times.append(a.elapsed_time(b))
                    fits.append(s.cp_fit(t, sigma))
            status = status or s.sync_status()
            per_seed.append(statistics.mean(fits[S // 2:]))
            fits_first = fits_first or fits
            s.close()
        mean_fit = statistics.mean(per_seed)
        row[mode] = {"status": status, "sweep_ms_median_2_to_S": statistics.median(times),
                     "fit_last": fits_first[-1], "fit_mean_second_half": mean_fit,
                     "fit_mean_second_half_per_seed": [round(f, 7) for f in per_seed],
                     "seeds": list(seeds), "fits_first_seed": [round(f, 6) for f in fits_first]}
        if len(per_seed) > 1:
            row[mode]["seed_spread_rel"] = (max(per_seed) - min(per_seed)) / abs(mean_fit)
    base = row["fp32"]["fit_mean_second_half"] if "fp32" in row else None
    for mode in modes:
        if mode != "fp32" and base:
            row[mode]["mean_fit_rel_diff_vs_fp32"] = abs(row[mode]["fit_mean_second_half"] - base) / abs(base)
    del Ud
    torch.cuda.empty_cache()
    return row


def run_sparse_als(args):
    """STS-CP (Alg. 6) on a synthetic sparse 2^22 x 2^22 x 2^14 tensor with Zipf(1.1)
    coordinates and rank-16 U(0,1) values x lognormal(0, 0.5) noise; J = 2^16
    samples per least-squares solve; per rank: FP32 trees, BF16x3 and TF32x3 trees, exact
    decisions (R <= 32), and the FP32 sweep captured as a CUDA graph.  Reports
    the median sweep time of sweeps 2..S and the fit after each sweep (fit not
    timed)."""
    import torch
    from paper_2301_12584_gb300 import krpls
    dev = torch.device("cuda", 0)
    krpls.lib()
    stream = torch.cuda.Stream(device=dev)
    t, scales, setup_s = sparse_setup(args.nnz, dev, stream)
    ranks = [int(r) for r in str(args.ranks).split(",") if r]
    S = max(int(args.sweeps), 3)
    results = []
    for R in ranks:
        modes = (("fp32", "bf16x3", "tf32x3", "exact", "fp32_graph") if R <= 32
                 else ("fp32", "bf16x3", "tf32x3", "fp32_graph"))
        results.append(sparse_rank_runs(t, scales, R, S, modes, dev, stream))
    print(json.dumps({
        "metric": "STS-CP sweep time (median of sweeps 2..S), sparse 3-mode tensor",
        "value": results[0]["fp32"]["sweep_ms_median_2_to_S"], "unit": "ms per sweep",
        "higher_is_better": False, "n_gpus": 1, "steps": S, "dtype": "f32", "data": "synthetic",
        "vs_baseline": None,
        "config": {"workload": f"sparse_als_2^22x2^22x2^14_nnz{int(args.nnz)}_J2^16", "nnz": int(args.nnz),
                   "ranks": ranks, "sweeps": S,
                   "init": "N(0,1) rows x sqrt((nnz of the index + 0.01) / mean), seed 0"},
        "setup_s": setup_s,
        "results": results,
    }), flush=True)


def run_accuracy(args):
    """Sec. 4.2 least squares: A = U_1 ⊙ ... ⊙ U_N (I = 2^16, N(0,1) with 1% of
    entries x10), b = c_1 ⊗ ... ⊗ c_N (N(0,1)), J = 5000 leverage samples;
    distortion D = kappa(SQ) - 1 and eps = residual / optimal residual - 1
    (both evaluated without forming A or b) for N in {3, 5, 7, 9} and R in
    {16, 32, 64}.  Timed: build + sample + right-hand side + solve per problem."""
    import torch
    from oracle import krp_oracle as O
    from paper_2301_12584_gb300 import krpls, synth
    from paper_2301_12584_gb300.krpls import Sampler
    I, J = 1 << 16, 5000
    dev = torch.device("cuda", 0)
    krpls.lib()
    stream = torch.cuda.Stream(device=dev)
    rows = []
    for N in (3, 5, 7, 9):
        for R in (16, 32, 64):
            Ds, eps, ms = [], [], []
            for trial in range(max(1, int(args.trials))):
                seed = 1000 * N + 10 * R + trial
                Us = synth.skewed_entry_factors(N, I, R, seed=seed)
                rng = np.random.default_rng(seed + 7)
                cs = [rng.standard_normal(I).astype(np.float32) for _ in range(N)]
                Ud = [torch.from_numpy(U).to(dev) for U in Us]
                cd = [torch.from_numpy(c).to(dev) for c in cs]
                idx = torch.zeros((N, J), dtype=torch.int32, device=dev)
                w = torch.zeros(J, device=dev)
                SA = torch.zeros((J, R), device=dev)
                B = torch.zeros((J, 1), device=dev)
                X = torch.zeros((R, 1), device=dev)
                s = Sampler([I] * N, R, 0, stream=stream)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a.record(stream)
                    for k in range(N):
                        s.set_factor(k, Ud[k])
                    s.sample(-1, J, seed, 0, idx, w, None, SA)
                    s.kron_rows(-1, J, idx, cd, B)
                    s.solve_dense(J, SA, w, B, 1, X)
                    b.record(stream)
                torch.cuda.synchronize()
                assert s.sync_status() == 0, s.last_error()
                ms.append(a.elapsed_time(b))
                D, _ = s.sketch_distortion(-1, J, SA)
                Ds.append(D)
                U64 = [U.astype(np.float64) for U in Us]
                c64 = [c.astype(np.float64) for c in cs]
                res, G, Atb = O.kron_lstsq_residual(U64, -1, c64, X.cpu().numpy()[:, 0].astype(np.float64))
                res_opt, _, _ = O.kron_lstsq_residual(U64, -1, c64, np.linalg.solve(G, Atb))
                eps.append(res / res_opt - 1.0)
                s.close()
            rows.append({"N": N, "R": R, "D_mean": float(np.mean(Ds)), "eps_mean": float(np.mean(eps)),
                         "eps_max": float(np.max(eps)), "ms_per_problem_median": float(np.median(ms[1:] or ms))})
    print(json.dumps({
        "metric": "least-squares accuracy: distortion D and residual ratio eps (Sec. 4.2), I=2^16, J=5000",
        "value": float(np.mean([r["eps_mean"] for r in rows])), "unit": "mean eps", "higher_is_better": False,
        "n_gpus": 1, "steps": int(args.trials), "dtype": "f32", "data": "synthetic", "vs_baseline": None,
        "config": {"workload": "accuracy_I2^16_J5000_N{3,5,7,9}_R{16,32,64}", "trials": int(args.trials)},
        "results": rows,
    }), flush=True)


# ------------------------------------------------------------------ ours ----
def sampler_run(prec, Ud, Fd, dev, stream, warmup, steps, draws, dist=None, clocks_index=None):
    """The headline step (one-factor update from device rows, prepare, draw
    with fused gather) on a sampler of the given precision: `warmup` untimed
    steps, then `steps` timed with CUDA events on the sampler's stream
    (barrier + synchronize on both sides), with per-phase events."""
    import torch
    from paper_2301_12584_gb300 import krpls, replicas
    from paper_2301_12584_gb300.krpls import Sampler
    s = Sampler([I_ROWS] * N_FACT, RANK, LEAF, prec, stream=stream)
    for k in range(N_FACT):
        s.set_factor(k, Ud[k])
    J = J_DRAW
    idx = torch.zeros((N_FACT, J), dtype=torch.int32, device=dev)
    w = torch.zeros(J, dtype=torch.float32, device=dev)
    SA = torch.zeros((J, RANK), dtype=torch.float32, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    phases = []

    def step(d, timed):
        if timed:
            e = [ev() for _ in range(4)]
            e[0].record(stream)
        s.set_factor(d % N_FACT, Fd[d % N_FACT])
        if timed:
            e[1].record(stream)
        s.sample_prepare(-1)
        if timed:
            e[2].record(stream)
        s.sample_draw(-1, J, 1, draws[d], idx, w, None, SA)
        if timed:
            e[3].record(stream)
            phases.append(e)

    clk = None
    with torch.cuda.stream(stream):
        for d in range(warmup):
            step(d, False)
        torch.cuda.synchronize()
        assert s.sync_status() == 0, s.last_error()
        if dist:
            dist.barrier()
        clocks = ClockSampler(clocks_index) if clocks_index is not None else None
        if clocks:
            clocks.start()
            time.sleep(0.2)
        n0 = krpls.launch_count()
        t_start, t_end = ev(), ev()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t_start.record(stream)
        for d in range(warmup, warmup + steps):
            step(d, True)
        t_end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        n_launch = krpls.launch_count() - n0
        if clocks:
            clk = clocks.stop()
    assert s.sync_status() == 0, s.last_error()
    ms = replicas.max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
    out = {"ms": ms, "n_launch": n_launch, "clocks": clk,
           "phases_ms": {"update": statistics.mean(p[0].elapsed_time(p[1]) for p in phases),
                         "prepare": statistics.mean(p[1].elapsed_time(p[2]) for p in phases),
                         "draw": statistics.mean(p[2].elapsed_time(p[3]) for p in phases)},
           "exact_redecisions_per_row_stage": s.exact_count() / float(J * N_FACT * (warmup + steps))
           if prec == krpls.KRP_PREC_EXACT else None}
    return s, idx, w, SA, out


def main():
    args = parse()
    from paper_2301_12584_gb300 import replicas
    rank, local, world = replicas.rank_env()
    if args.workload != "sampler" and args.impl == "ours":
        if world > 1 and rank != 0:
            return
        {"batch512": run_batch512, "rank_sweep": run_rank_sweep, "sparse_als": run_sparse_als,
         "accuracy": run_accuracy}[args.workload](args)
        return
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank)
        return

    import torch
    from paper_2301_12584_gb300 import krpls, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    krpls.lib()
    precs = {"fp32": krpls.KRP_PREC_FP32, "bf16x3": krpls.KRP_PREC_BF16X3, "tf32x3": krpls.KRP_PREC_TF32X3,
             "exact": krpls.KRP_PREC_EXACT}

    # ---- inputs (seeded, synthetic): same generator as the tests
    Us = synth.skewed_row_factors(N_FACT, I_ROWS, RANK, seed=0)
    fresh = [synth.fresh_factor(I_ROWS, RANK, seed=1000 + d) for d in range(N_FACT)]
    stream = torch.cuda.Stream(device=dev)
    Ud = [torch.from_numpy(U).to(dev) for U in Us]
    Fd = [torch.from_numpy(U).to(dev) for U in fresh]
    Fh = [torch.from_numpy(U).pin_memory() for U in fresh]
    torch.cuda.synchronize()
    J = J_DRAW
    draws = replicas.draw_ids(rank, 0, args.warmup + args.steps)          # this rank's own Philox draw ids
    e2e_draws = replicas.draw_ids(rank, 500_000, max(args.e2e_steps, 0))

    s, idx, w, SA, head = sampler_run(precs[args.precision], Ud, Fd, dev, stream, args.warmup, args.steps, draws,
                                      dist, local)
    ms = head["ms"]
    value = replicas.whole_job_rate(J * args.steps, world, ms)
    drw = head["phases_ms"]["draw"]

    # ---- roofline of the descent kernel (one launch per draw)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    T = RANK * (RANK + 1) // 2
    Tp = (T + 7) // 8 * 8
    depth = (I_ROWS // LEAF - 1).bit_length()
    bytes_per_sample = N_FACT * (4 * T * depth + 4 * LEAF * RANK)     # nominal tree path + leaf block
    achieved = bytes_per_sample * J / (drw / 1e3) / 1e9
    roof = {"kernel": "krp_descent_fast<32>" + (", exact decisions" if args.precision == "exact" else ""),
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": DESCENT_DRAM_BYTES if args.precision == "fp32" else None,
            "traffic_frac": DESCENT_DRAM_BYTES / (drw / 1e3) / 1e9 / hbm if args.precision == "fp32" else None,
            "algorithmic_bytes_per_launch": bytes_per_sample * J,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "note": ("achieved/frac: nominal bytes (every sample reads its full root-to-leaf path); "
                     "traffic: ncu DRAM bytes per launch (upper levels are L2 hits); traffic_frac: that "
                     "traffic over the live launch time, against the same peak")}
    # tree rebuild (update): read the fresh rows once, write the sampler's copy and the tree
    # (and the low parts in the exact-decision mode), informational
    L = 1 << depth
    build_bytes = 2 * I_ROWS * RANK * 4 + L * Tp * 4 * (2 if args.precision == "exact" else 1)
    upd = head["phases_ms"]["update"]
    update_info = {"ms": upd, "bytes": build_bytes, "GBps": build_bytes / (upd / 1e3) / 1e9,
                   "frac": build_bytes / (upd / 1e3) / 1e9 / hbm,
                   "note": "read the fresh factor once, write the sampler's copy and the tree"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        idx_h = torch.zeros((N_FACT, J), dtype=torch.int32).pin_memory()
        w_h = torch.zeros(J, dtype=torch.float32).pin_memory()
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            for d in range(args.e2e_steps):
                k = d % N_FACT
                s.set_factor(k, Fh[k].data_ptr())               # H2D of the step's input from pinned host
                s.sample(-1, J, 1, e2e_draws[d], idx, w, None, SA)
                idx_h.copy_(idx, non_blocking=True)            # D2H of the step's result
                w_h.copy_(w, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
        e_ms = replicas.max_over_ranks(a.elapsed_time(b), dist, dev)
        e2e = {"value": replicas.whole_job_rate(J * args.e2e_steps, world, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": I_ROWS * RANK * 4, "d2h_bytes_per_step": J * (N_FACT * 4 + 4)}
    s.close()

    # ---- the other precision forms of the same step (rank 0 at N=1: extra keys)
    forms = {args.precision: {"value": value, "ms_per_step": ms / args.steps, "phases_ms": head["phases_ms"],
                              "exact_redecisions_per_row_stage": head["exact_redecisions_per_row_stage"]}}
    if world == 1 and not args.no_forms:
        for name in ("fp32", "bf16x3", "tf32x3", "exact"):
            if name == args.precision:
                continue
            sf, _, _, _, out = sampler_run(precs[name], Ud, Fd, dev, stream, args.warmup, args.steps, draws)
            sf.close()
            forms[name] = {"value": J * args.steps / (out["ms"] / 1e3), "ms_per_step": out["ms"] / args.steps,
                           "phases_ms": out["phases_ms"],
                           "exact_redecisions_per_row_stage": out["exact_redecisions_per_row_stage"]}
    del Ud, Fd
    torch.cuda.empty_cache()

    # ---- the metric's second half: STS-CP sweep time, mixed vs FP32 (rank 0 at N=1)
    sts = None
    if world == 1 and args.sts_sweeps > 0:
        t, scales, setup_s = sparse_setup(args.nnz, dev, stream)
        seeds = tuple(range(1, max(1, args.sts_seeds) + 1))
        row = sparse_rank_runs(t, scales, 25, max(3, args.sts_sweeps), ("fp32", "bf16x3", "tf32x3", "exact"), dev,
                               stream,
                               seeds)
        t.close()
        sts = {"workload": f"sts_cp_2^22x2^22x2^14_nnz{int(args.nnz)}_R25_J2^16", "unit": "ms per sweep",
               "sweeps": max(3, args.sts_sweeps), "seeds": list(seeds), "setup_s": setup_s,
               "fit_note": ("fit_mean_second_half: mean fit of sweeps S/2..S, averaged over the sampling seeds; "
                            "seed_spread_rel: (max - min) of the per-seed means over their mean"),
               **{m: {"sweep_ms_median_2_to_S": row[m]["sweep_ms_median_2_to_S"],
                      "fit_mean_second_half": row[m]["fit_mean_second_half"], "fit_last": row[m]["fit_last"],
                      "fit_mean_second_half_per_seed": row[m]["fit_mean_second_half_per_seed"],
                      "seed_spread_rel": row[m].get("seed_spread_rel"),
                      "mean_fit_rel_diff_vs_fp32": row[m].get("mean_fit_rel_diff_vs_fp32"),
                      "status": row[m]["status"]} for m in ("fp32", "bf16x3", "tf32x3", "exact")}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Us64 = [U.astype(np.float64) for U in Us]
        fresh64 = [U.astype(np.float64) for U in fresh]
        n, secs, _ = oracle_tree_steps(Us64, fresh64, 1, J_DRAW)
        cpu = {"value": n / secs, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
               "sample": ("one step of the workload by the FP64 oracle: one-factor update (FP64 segment-tree "
                          "rebuild, Alg. 3), preparation, and the full J=2^16 draw by the FP64 tree descent "
                          "(Alg. 2/4), no extrapolation"),
               "seconds": secs}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision, "N": N_FACT, "I": I_ROWS, "R": RANK,
                       "F": LEAF, "J": J, "l2": "inputs larger than L2 (no flush needed)",
                       "parallelism": f"replicas x{world}"},
            "phases_ms": head["phases_ms"],
            "update": update_info,
            "roofline": roof,
            "clocks": head["clocks"],
            "gpu_launches": head["n_launch"],
            "e2e": e2e,
            "cpu_baseline": cpu,
            "forms": forms,
            "sts_cp": sts,
        }), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
