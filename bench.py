#!/usr/bin/env python3
"""ProHD benchmark on GB300.

Workload: a pair of n = m = 2,000,000 point sets in D = 256 (A ~ N(0, S),
S = Q diag(1/i) Q^T; B the same law shifted by 0.1 sigma along a random unit
vector, 0.1% multivariate Student-t (nu = 3) points), synthetic and seeded.
A step is one full ProHD estimate (Algorithm 3) of that pair, resident in HBM:
directions (centroid axis + top-8 principal components), selection
(alpha = 0.01 per side on the centroid axis, alpha/8 per component),
gather, and the exact Hausdorff distance of the subsets on FP16 tensor-core
tiles with FP32 rescoring and an FP64 witness.

Reported beside the throughput: relative error of the estimate against the
exact Hausdorff distance of the full sets (same library, FP32-rescored, FP64
witness), the speedup over that exact computation, the BF16-tile variant,
an end-to-end number through prohd_estimate_host (host buffers, copies in the
timed region), the roofline of the dominant kernel, and the FP64 CPU oracle
timed on a bounded sample on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl prohd|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ProHD set-pairs/s at 2M×D256 + rel. err vs FP64 exact; speedup over GPU exact HD"
UNIT = "set-pairs/s"
N_POINTS = 2_000_000
DIM = 256
M_PCS = 8
ALPHA = 0.01
# DRAM bytes (read + write) per full-size launch from one ncu capture of the
# current kernel at 400k + 400k points: the reads (and the projection's key
# writes) grow with the points (x5 to 2M + 2M); the Gram's writes (its running
# sums reaching DRAM) are scaled x5 too, an upper estimate. None: no capture of
# the current kernel.
GRAM_TRAFFIC = (826.25e6 + 22.39e6) * 5
PROJ_TRAFFIC = (819.41e6 + 26.96e6) * 5
# the contraction's traffic per row of the two FP16 copies (100k + 100k capture)
HD_TRAFFIC_PER_ROW = (136.72e6 + 4.64e6) / 200_000
WORKLOAD = ("anisotropic Gaussian pair, n=m=2,000,000, D=256 (eigenvalues 1/i, random rotation); "
            "B shifted 0.1 sigma along a random unit vector with 0.1% Student-t (nu=3) points; "
            "ProHD with centroid axis + top-8 PCs, alpha=0.01 per side (alpha/8 per PC), FP16 tiles")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# ---------------------------------------------------------------- distributed

def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", self.gpu, "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if mx and s >= 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- data

def make_pair(seed: int, n: int):
    from paper_2511_18207_gb300 import workloads as W

    return W.anisotropic_pair(n, n, DIM, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=seed)


# ---------------------------------------------------------------- oracle sample

def oracle_sample(A, B, rows_cov: int = 200_000, rows_hd: int = 256) -> dict:
    """Times the FP64 oracle's ProHD on a bounded sample of the workload.

    Measured: the covariance accumulated over every k-th row, centroids and
    the power iteration, the full selection (projection and sort of every
    point), and the subset HD for the first `rows_hd` outer rows of each
    direction. The full-pair time is extrapolated from those measurements:
    covariance x N / rows used, subset HD x subset rows / rows_hd (both costs
    are linear in the rows); the other stages ran in full. Both the measured
    and the extrapolated seconds are returned, with the factors."""
    import numpy as np

    import oracle

    nA, nB = A.shape[0], B.shape[0]
    N = nA + nB
    sa = max(1, N // rows_cov)
    t0 = time.perf_counter()
    _, C = oracle.union_covariance(A[::sa], B[::sa])
    t_cov = time.perf_counter() - t0
    rows_used = A[::sa].shape[0] + B[::sa].shape[0]
    f_cov = N / rows_used
    t0 = time.perf_counter()
    u0 = oracle.centroid_axis(oracle.centroid(A), oracle.centroid(B))
    U, _, _ = oracle.power_iteration(C, M_PCS, seed=0)
    t_dir = time.perf_counter() - t0
    dirs = np.vstack([u0[None, :], U])
    t0 = time.perf_counter()
    ia = oracle.select(A, dirs, oracle.k_list(nA, 1 + M_PCS, ALPHA, ALPHA / M_PCS))
    ib = oracle.select(B, dirs, oracle.k_list(nB, 1 + M_PCS, ALPHA, ALPHA / M_PCS))
    t_sel = time.perf_counter() - t0
    As, Bs = A[ia], B[ib]
    ra, rb = min(rows_hd, As.shape[0]), min(rows_hd, Bs.shape[0])
    t0 = time.perf_counter()
    oracle.directed_hd(As, Bs, 0, ra)
    oracle.directed_hd(Bs, As, 0, rb)
    t_hd = time.perf_counter() - t0
    f_hd = (As.shape[0] + Bs.shape[0]) / (ra + rb)
    measured = {"covariance": t_cov, "centroids+power": t_dir, "selection": t_sel, "subset_hd": t_hd}
    extrap = {"covariance": t_cov * f_cov, "centroids+power": t_dir, "selection": t_sel, "subset_hd": t_hd * f_hd}
    total = sum(extrap.values())
    return {"seconds_per_pair": total, "sample_seconds": sum(measured.values()), "value": 1.0 / total,
            "cores": oracle.num_threads(), "extrapolated": True,
            "scale_factors": {"covariance": round(f_cov, 3), "subset_hd": round(f_hd, 3)},
            "stages_s_measured": {k: round(v, 4) for k, v in measured.items()},
            "stages_s_extrapolated": {k: round(v, 4) for k, v in extrap.items()},
            "sample": (f"measured: covariance over every {sa}-th row ({rows_used} of {N} rows), centroids, power "
                       f"iteration and selection on all {N} points, subset HD outer loop on {ra}+{rb} of "
                       f"{As.shape[0]}+{Bs.shape[0]} subset rows; the full pair's time is extrapolated with "
                       f"covariance x{f_cov:.1f} and subset HD x{f_hd:.1f}"),
            "nsel": [int(As.shape[0]), int(Bs.shape[0])]}


def oracle_full_runs() -> dict:
    """The FP64 oracle's ProHD run in full (no sampling, no extrapolation) on
    the two smaller workloads: 2,000 + 2,000 points in D = 16 (Gaussian with
    1% scaled outliers; m = 2, alpha = 0.02) with its exact HD too, and the
    200,000 + 200,000 point, D = 256 mixture pair (m = 8, alpha = 0.01).
    Wall seconds on the host cores."""
    import oracle
    from paper_2511_18207_gb300 import workloads as W

    out = {"cores": oracle.num_threads()}
    A, B = W.gaussian_outliers(2000, 2000, 16, seed=0)
    t0 = time.perf_counter()
    o = oracle.prohd(A, B, alpha=0.02, m=2, alpha_p=0.02, seed=0)
    t_p = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = oracle.hausdorff(A, B)
    t_h = time.perf_counter() - t0
    out["gaussian_2k_D16"] = {"prohd_s": t_p, "exact_hd_s": t_h, "H_hat": o["H_hat"], "H": h["H"]}
    A, B = W.mixture_pair(200_000, 256, 16, seed=1)
    t0 = time.perf_counter()
    o = oracle.prohd(A, B, alpha=0.01, m=8, seed=0)
    t_p = time.perf_counter() - t0
    out["mixture_200k_D256"] = {"prohd_s": t_p, "H_hat": o["H_hat"], "nsel": [int(o["idxA"].size),
                                                                              int(o["idxB"].size)],
                                "exact_hd": "not run: about 3e13 FP64 operations, beyond a bench run's minutes"}
    return out


def subsample_check(ctx, A, B, dev, n_sub: int = 20_000, seed: int = 11) -> dict:
    """GPU results against the FP64 oracle on a seeded 20,000-point subsample
    of each set of the 2M pair: the GPU's exact HD (FP16 tiles with FP32
    rescoring) and its ProHD estimate (plain and refined) against the
    oracle's brute-force FP64 exact HD and the oracle's own ProHD estimate."""
    import numpy as np
    import torch

    import oracle
    from paper_2511_18207_gb300 import prohd

    rng = np.random.default_rng(seed)
    ia = np.sort(rng.choice(A.shape[0], n_sub, replace=False))
    ib = np.sort(rng.choice(B.shape[0], n_sub, replace=False))
    As, Bs = np.ascontiguousarray(A[ia]), np.ascontiguousarray(B[ib])
    At, Bt = torch.from_numpy(As).to(dev), torch.from_numpy(Bs).to(dev)
    g_exact = prohd.decode_hd(ctx.hausdorff_exact(At, Bt, "fp16"))
    torch.cuda.synchronize()
    g_est = prohd.prohd_estimate_sync(At, Bt, m=M_PCS, alpha_c=ALPHA, precision="fp16")
    g_ref = prohd.prohd_estimate_sync(At, Bt, m=M_PCS, alpha_c=ALPHA, precision="fp16", refine=1)
    t0 = time.perf_counter()
    o_exact = oracle.hausdorff(As, Bs)
    t_exact = time.perf_counter() - t0
    o_est = oracle.prohd(As, Bs, alpha=ALPHA, m=M_PCS, seed=0)
    H = o_exact["H"]
    return {"n": n_sub, "H_fp64": H, "oracle_exact_hd_s": t_exact,
            "gpu_exact_rel_err": abs(g_exact["H"] - H) / H,
            "gpu_hhat_rel_err_vs_fp64_exact": abs(g_est["H"] - H) / H,
            "gpu_hhat_signed_vs_fp64_exact": (g_est["H"] - H) / H,
            "gpu_refined_rel_err_vs_fp64_exact": abs(g_ref["H"] - H) / H,
            "gpu_hhat_rel_diff_vs_oracle_hhat": abs(g_est["H"] - o_est["H_hat"]) / o_est["H_hat"],
            "note": "GPU directions come from tensor-core covariance partials, the oracle's from FP64 two-pass "
                    "sums, so the candidate sets (and H_hat) can differ slightly"}


# ---------------------------------------------------------------- GPU arm

def part_arm(args):
    """One of the secondary measurements alone (--workload batched|learned):
    a JSON line of its own, the sub-object's figures under the line's keys."""
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    peaks, peak_src = load_peaks()
    if args.workload == "batched":
        r = batched_arm(args, peaks, peak_src, dist, dev)
        line = {"metric": "batched ProHD set-pairs/s (512 uneven pairs)", "value": world * r["value"],
                "unit": "set-pairs/s", "n_gpus": world, "steps": r["steps"], "warmup": args.warmup,
                "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": {"workload": r["workload"]}, "batched": r}
    else:
        r = learned_arm(args, peaks, dev) if rank == 0 else None
        line = None if r is None else {
            "metric": "learned-direction training samples/s (batch 256, D = 128)", "value": r["samples_per_s"],
            "unit": "samples/s", "n_gpus": world, "steps": r["steps"], "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic", "config": {"workload": r["workload"]}, "learned": r}
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2511_18207_gb300 import prohd

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    peaks, peak_src = load_peaks()
    n = args.n

    A, B = make_pair(seed=args.seed + rank, n=n)
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    ctx = prohd.Context()
    st = torch.cuda.current_stream()

    def params(prec):
        return prohd.default_params(m=M_PCS, alpha_c=ALPHA, precision=prec)

    p16, pbf = params("fp16"), params("bf16")
    out = torch.empty(ctypes.sizeof(prohd.Result), dtype=torch.uint8, device=dev)
    ws_need = max(ctx.lib.prohd_estimate_workspace_size(n, n, DIM, ctypes.byref(p16)),
                  ctx.lib.prohd_estimate_workspace_size(n, n, DIM, ctypes.byref(pbf)))
    ws = ctx.workspace(ws_need)

    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_idx = visible[local] if local < len(visible) else str(local)
    clocks = ClockSampler(gpu_idx)
    clocks.start()

    def run_steps(p, k):
        for _ in range(k):
            ctx.prohd_estimate(At, Bt, params=p, out=out, ws=ws)

    # warm-up
    run_steps(p16, args.warmup)
    torch.cuda.synchronize()

    # phases: K eager steps with CUDA events around each phase on the same stream
    ctx.profile_read(reset=True)
    ctx.profile_enable(True)
    l0 = ctx.launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    run_steps(p16, args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    per_call = (ctx.launch_count() - l0) // args.steps
    ctx.profile_enable(False)
    phases = ctx.profile_read(reset=True)
    ms_eager = e0.elapsed_time(e1) / args.steps

    # timed region: the estimate captured once in a CUDA graph (every entry point
    # is capturable: no allocation, no synchronisation), K replays
    graph = None
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(st)
        with torch.cuda.stream(gs):
            run_steps(p16, 1)
        st.wait_stream(gs)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            ctx.prohd_estimate(At, Bt, params=p16, out=out, ws=ws)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
    except Exception as ex:  # eager steps keep the measurement going
        print(f"graph capture unavailable ({ex}); timing eager steps", file=sys.stderr)
        graph = None
    barrier(dist)
    torch.cuda.synchronize()
    e0.record(st)
    if graph is not None:
        for _ in range(args.steps):
            graph.replay()
    else:
        run_steps(p16, args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(dist)
    launches = per_call * args.steps
    t_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
    ms_step = t_ms / args.steps
    res16 = prohd.decode_result(out)

    # end to end through the C ABI with host buffers (H2D copies + D2H of the result),
    # right after the device-resident steps
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    hres = prohd.Result()
    hws_need = ctx.lib.prohd_estimate_host_workspace_size(n, n, DIM, ctypes.byref(p16))
    ws = ctx.workspace(hws_need)
    ctx.prohd_estimate_host(Ah, Bh, params=p16, out_host=hres, ws=ws)
    torch.cuda.synchronize()
    # this host's pinned copy rate now: the floor of the end-to-end time
    h2d_dst = torch.empty(2 * n * DIM, dtype=torch.float32, device=dev)
    h2d_ms = []
    for _ in range(3):
        e0.record(st)
        with torch.cuda.stream(st):
            h2d_dst[: n * DIM].copy_(Ah.view(-1), non_blocking=True)
            h2d_dst[n * DIM:].copy_(Bh.view(-1), non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        h2d_ms.append(e0.elapsed_time(e1))
    del h2d_dst
    h2d_gbs = 2 * n * DIM * 4 / min(h2d_ms) / 1e6
    e2e_steps = max(3, min(args.steps, 10))
    barrier(dist)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(e2e_steps):
        ctx.prohd_estimate_host(Ah, Bh, params=p16, out_host=hres, ws=ws)
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev) / e2e_steps
    ws = ctx.workspace(ws_need)

    # BF16 tiles
    run_steps(pbf, 1)
    torch.cuda.synchronize()
    e0.record(st)
    run_steps(pbf, args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms_bf = e0.elapsed_time(e1) / args.steps
    resbf = prohd.decode_result(out)

    # one-sided refinement max(h(A_sel, B), h(B_sel, A)) on the same pair:
    # the same candidate sets, each selected point's nearest neighbour
    # searched in the whole other set (never above H)
    refined = None
    if not args.no_refined:
        pr = prohd.default_params(m=M_PCS, alpha_c=ALPHA, precision="fp16", refine=1)
        rws = ctx.workspace(ctx.lib.prohd_estimate_workspace_size(n, n, DIM, ctypes.byref(pr)))
        ctx.prohd_estimate(At, Bt, params=pr, out=out, ws=rws)
        torch.cuda.synchronize()
        kr = max(1, min(args.steps, 3))
        ctx.profile_read(reset=True)
        ctx.profile_enable(True)
        e0.record(st)
        for _ in range(kr):
            ctx.prohd_estimate(At, Bt, params=pr, out=out, ws=rws)
        e1.record(st)
        torch.cuda.synchronize()
        ctx.profile_enable(False)
        rph = ctx.profile_read(reset=True)
        resr = prohd.decode_result(out)
        refined = {"ms_per_step": e0.elapsed_time(e1) / kr, "steps": kr, "H": resr["H"], "status": resr["status"],
                   "phases_ms_per_step": {k: round(v[0] / kr, 4) for k, v in rph.items() if v[1]}}
        # the two subset-vs-full-set distances take the row-pruned passes
        # (sampled lower bounds, a prefix contraction, the exact path on the
        # rows left), so there is no dense flop count to rate them by
        refined["note"] = "h(A_sel, B) and h(B_sel, A) through the row-pruned passes of hausdorff_exact_pruned"
        del rws
        ws = ctx.workspace(ws_need)

    # exact Hausdorff distance of the full sets (the comparison the metric names)
    exact = None
    if not args.no_exact:
        small = torch.randn(4096, DIM, device=dev)
        ctx.hausdorff_exact(small, small, "fp16")  # loads the kernels
        torch.cuda.synchronize()
        hout = torch.empty(ctypes.sizeof(prohd.HdResult), dtype=torch.uint8, device=dev)
        hws = ctx.workspace(ctx.lib.hausdorff_exact_workspace_size(n, n, DIM, 1))
        e0.record(st)
        ctx.hausdorff_exact(At, Bt, "fp16", out=hout, ws=hws)
        e1.record(st)
        torch.cuda.synchronize()
        exact = prohd.decode_hd(hout)
        exact["ms"] = e0.elapsed_time(e1)
        # the same exact distance with row pruning (a sampled lower bound, a
        # prefix contraction that drops rows certainly below it, the exact
        # path on the rest)
        pws = ctx.workspace(ctx.lib.hausdorff_exact_pruned_workspace_size(n, n, DIM, 1))
        pout = torch.empty(ctypes.sizeof(prohd.HdResult), dtype=torch.uint8, device=dev)
        e0.record(st)
        ctx.hausdorff_exact_pruned(At, Bt, "fp16", out=pout, ws=pws)
        e1.record(st)
        torch.cuda.synchronize()
        pr = prohd.decode_hd(pout)
        _, kept = ctx.hausdorff_exact_pruned(At, Bt, "fp16", out=pout, ws=pws, want_kept=True)
        exact["pruned"] = {"ms": e0.elapsed_time(e1), "H": pr["H"], "status": pr["status"], "rows_kept": kept,
                           "equals_dense": pr["H"] == exact["H"]}
        del pws
        ws = ctx.workspace(ws_need)
    clk = clocks.stop()


    # roofline of the dominant kernel
    nsa, nsb = res16["nsel_a"], res16["nsel_b"]
    cand = {}
    for name, (ms, cnt) in phases.items():
        if cnt:
            cand[name] = (ms / cnt, cnt)
    single = {k: v for k, v in cand.items() if k in ("gram", "hd_contract", "power", "project")}
    dom = max(single, key=lambda k: single[k][0]) if single else None
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # the library's rule for the pruned subset distance: FP16/BF16 tiles,
    # D <= 256, subset bounds (2 sum_d k_d) of at least 8,192 rows each and a
    # product of at least the context's threshold (default 1e9)
    kc, kp = prohd.k_of(ALPHA, n), prohd.k_of(ALPHA / M_PCS, n)
    bound = 2 * (kc + M_PCS * kp)
    subset_pruned = DIM <= 256 and bound >= 8192 and float(bound) * bound >= 1e9

    def roof_for(name):
        roof = None
        if name == "gram":
            t = cand["gram"][0] / 1e3
            # the method's work for the covariance (Algorithm 2): one read of both
            # sets and 2 N D^2 flops for the D x D Gram of the N = 2n points; the
            # roofline is the larger of the two bound times
            by = 2.0 * n * DIM * 4
            fl = 2.0 * (2 * n) * DIM * DIM
            if DIM <= 256 and DIM % 4 == 0:
                pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
                t_hbm, t_tc = by / (peaks["hbm_gbs"] * 1e9), fl / (pk * 1e12)
                # the tensor cores run two BF16 MMAs per point over the full
                # 256 x 256 product (a two-part split, X = sum h h^T + 2 m h^T)
                dp = 256 if DIM > 128 else 2 * ((DIM + 63) // 64) * 64
                issued = 2.0 * 2 * 256 * dp * (2 * n) / (2 if DIM <= 128 else 1)
                note = {"issued_tflops": issued / t / 1e12, "issued_frac_of_sustained_bf16": issued / t / 1e12 / pk,
                        "issued_work": "2 BF16 MMAs per point over the CTA pair's 256-row product"}
                if t_hbm >= t_tc:
                    roof = {"kernel": "gram_tc_kernel", "bound": "hbm", "achieved": by / t / 1e9,
                            "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": GRAM_TRAFFIC,
                            "peak_source": f"{peak_src} copy bandwidth",
                            "work": "one read of both sets (2 n D 4 bytes); 2 N D^2 flops take less time at the "
                                    "sustained BF16 peak", "tensor_view": {"achieved_tflops": fl / t / 1e12,
                                                                          "peak_tflops": pk,
                                                                          "frac": fl / t / 1e12 / pk},
                            "split_products": note}
                else:
                    roof = {"kernel": "gram_tc_kernel", "bound": "tensor", "achieved": fl / t / 1e12, "peak": pk,
                            "unit": "TFLOP/s", "traffic": GRAM_TRAFFIC, "peak_source": f"{peak_src} sustained BF16",
                            "work": "2 N D^2 flops", "split_products": note}
            else:
                roof = {"kernel": "gram_kernel", "bound": "alu", "achieved": fl / t / 1e12, "peak": fp32_peak,
                        "unit": "TFLOP/s", "traffic": None,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        elif name == "hd_contract":
            t = cand["hd_contract"][0] / 1e3
            fl = 2.0 * nsa * nsb * DIM
            if subset_pruned:
                # the pruned form runs four contractions whose sizes depend on
                # the rows kept (device counts): the plain product's work over
                # this time is an equivalent rate, not a fraction of the peak
                roof = {"kernel": "hd_tc_kernel (pruned subset distance)", "bound": "tensor", "achieved": None,
                        "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "traffic": None,
                        "dense_equivalent_tflops": fl / t / 1e12,
                        "note": "rows that cannot attain either directed maximum skip the full contraction; "
                                "the result equals the plain contraction's"}
            else:
                roof = {"kernel": "hd_tc_kernel", "bound": "tensor", "achieved": fl / t / 1e12,
                        "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "traffic": HD_TRAFFIC_PER_ROW * (nsa + nsb),
                        "peak_source": f"{peak_src} bf16 burst (fp16 has the same nominal rate)"}
        elif name == "project":
            t = cand["project"][0] / 1e3  # one launch projects both sets
            by = 2 * (n * DIM * 4.0 + (1 + M_PCS) * n * 4.0)
            roof = {"kernel": "proj_pair_tma_kernel", "bound": "hbm", "achieved": by / t / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": PROJ_TRAFFIC,
                    "peak_source": f"{peak_src} copy bandwidth",
                    "work": "one read of both sets and one write of the 1 + m keys per point"}
        elif name == "power":
            roof = {"kernel": "subspace_kernel", "bound": "latency", "achieved": None, "peak": None, "unit": None,
                    "traffic": None}
        if roof and roof.get("achieved") is not None:
            roof["frac"] = roof["achieved"] / roof["peak"]
        return roof

    roof = roof_for(dom)
    stage_roofs = {k: roof_for(k) for k in ("gram", "project", "hd_contract") if k in cand}

    batched = None
    if not args.no_batched:
        batched = batched_arm(args, peaks, peak_src, dist, dev)
    learned_res = None
    if not args.no_learned and rank == 0:
        learned_res = learned_arm(args, peaks, dev)

    cpu = None
    subsample = None
    if rank == 0 and world == 1 and not args.no_cpu:
        s = oracle_sample(A, B)
        cpu = {"value": s["value"], "unit": UNIT, "cores": s["cores"], "kind": "oracle", "sample": s["sample"],
               "extrapolated": True, "sample_seconds": s["sample_seconds"], "scale_factors": s["scale_factors"],
               "stages_s_measured": s["stages_s_measured"], "stages_s_extrapolated": s["stages_s_extrapolated"],
               "full_runs": oracle_full_runs()}
        subsample = subsample_check(ctx, A, B, dev)

    H = exact["H"] if exact else None
    line = {
        "metric": METRIC, "value": world * 1000.0 / ms_step, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_POINTS else WORKLOAD.replace("2,000,000", f"{n:,}"),
                   "n_a": n, "n_b": n, "D": DIM, "m": M_PCS, "alpha": ALPHA, "tiles": "fp16",
                   "parallelism": f"replicas x{world} (independent pairs per rank)",
                   "l2": "inputs (4.1 GB) larger than L2; no flush"},
        "H_hat": res16["H"], "H_exact": H, "rel_err_vs_exact": (abs(res16["H"] - H) / H) if H else None,
        "signed_err": ((res16["H"] - H) / H) if H else None,
        "exact_ms": exact["ms"] if exact else None,
        "exact_pruned": exact.get("pruned") if exact else None,
        "speedup_vs_gpu_exact": (exact["ms"] / ms_step) if exact else None,
        "speedup_vs_gpu_exact_pruned": (exact["pruned"]["ms"] / ms_step) if exact and exact.get("pruned") else None,
        "nsel": [nsa, nsb], "status": res16["status"], "exact_status": exact["status"] if exact else None,
        "rescored": [res16["n_rescored_a"], res16["n_rescored_b"]],
        "subset_hd": "pruned (equal to the plain contraction)" if subset_pruned else "plain contraction",
        "refined": (dict(refined, rel_err_vs_exact=(H - refined["H"]) / H if H else None) if refined else None),
        "bf16": {"value": world * 1000.0 / ms_bf, "ms_per_step": ms_bf, "H_hat": resbf["H"],
                 "rel_err_vs_exact": (abs(resbf["H"] - H) / H) if H else None,
                 "rel_err_lowp_before_rescoring": (abs(resbf["H_lowp"] - resbf["H"]) / resbf["H"])},
        "fp16_rel_err_lowp_before_rescoring": abs(res16["H_lowp"] - res16["H"]) / res16["H"],
        "phases_ms_per_step": {k: round(v[0] * v[1] / args.steps, 4) for k, v in cand.items()},
        "timing": ("CUDA-graph replays of one prohd_estimate" if graph is not None else "eager calls"),
        "eager_ms_per_step": ms_eager,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 2 * n * DIM * 4, "d2h_bytes_per_step": ctypes.sizeof(prohd.Result),
                "h2d_gbs_measured": h2d_gbs, "h2d_floor_ms": 2 * n * DIM * 4 / h2d_gbs / 1e6,
                "overlap": "each set copied in row ranges on the library's copy stream; the Gram reads each range "
                           "as it lands (sets of at least 131,072 rows)"},
        "gpu_launches": launches,
        "roofline": roof,
        "stage_rooflines": stage_roofs,
        "cpu_baseline": cpu,
        "fp64_subsample_20k": subsample,
        "clocks": clk,
        "batched": batched,
        "learned": learned_res,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched pairs

BATCH_WORKLOAD = ("512 independent pairs, set sizes log-uniform on [1e3, 1e5], D uniform on {64, 128, 256}, "
                  "each set a Gaussian mixture of K ~ U{4..32} components (means ~ N(0, 4I), variances ~ U[0.2, 2]); "
                  "ProHD with centroid axis + top-8 PCs, alpha = 0.01, FP16 subset tiles; one planned, graph-captured batch")


def batched_arm(args, peaks, peak_src, dist, dev):
    """512 uneven pairs in one planned batch (CUDA graph replay, autotuned
    item sizes). Returns the sub-object of the JSON line."""
    import numpy as np
    import torch
    from paper_2511_18207_gb300 import prohd, workloads as W

    pairs = W.batched_pairs_device(512, seed=args.seed + 7)
    torch.cuda.synchronize()
    npts = sum(a.shape[0] + b.shape[0] for a, b in pairs)
    nbytes = sum((a.numel() + b.numel()) * 4 for a, b in pairs)
    ctx = prohd.context()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = prohd.Batch(ctx, pairs, m=M_PCS, alpha_c=ALPHA, precision="fp16")
        tuned_ms = b.autotune(st)
        b.use_graph(True)
        for _ in range(args.warmup):
            b.run(st)
        st.synchronize()
        l0 = ctx.launch_count()
        steps = max(args.steps, 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        st.synchronize()
        e0.record(st)
        for _ in range(steps):
            b.run(st)
        e1.record(st)
        st.synchronize()
        ms = max_over_ranks(dist, e0.elapsed_time(e1), dev) / steps
        launches = (ctx.launch_count() - l0) // steps
        res = b.results()
        its = b.iterations()
        # stage times of one direct (profiled) run
        b.use_graph(False)
        ctx.profile_enable(True)
        ctx.profile_read(reset=True)
        for _ in range(3):
            b.run(st)
        st.synchronize()
        ph = ctx.profile_read(reset=True)
        ctx.profile_enable(False)
        b.use_graph(True)
        ref = None
        if not args.no_refined:
            # the same batch with params.refine = 1 (graph replay), and the
            # refinement's own phase time from one profiled direct run
            b1 = prohd.Batch(ctx, pairs, m=M_PCS, alpha_c=ALPHA, precision="fp16", refine=1)
            b1.set_tunables(**b.tunables())
            b1.use_graph(True)
            for _ in range(max(args.warmup, 2)):
                b1.run(st)
            st.synchronize()
            barrier(dist)
            e0.record(st)
            for _ in range(steps):
                b1.run(st)
            e1.record(st)
            st.synchronize()
            ms1 = max_over_ranks(dist, e0.elapsed_time(e1), dev) / steps
            res1 = b1.results()
            b1.use_graph(False)
            ctx.profile_enable(True)
            ctx.profile_read(reset=True)
            b1.run(st)
            st.synchronize()
            ph1 = ctx.profile_read(reset=True)
            ctx.profile_enable(False)
            ref = {"ms_per_batch": ms1, "value": 1000.0 * len(pairs) / ms1, "unit": "set-pairs/s",
                   "refine_ms": round(ph1.get("hd_rescore", (0.0, 0))[0], 4)}
            b1.close()
    phases = {k: round(v[0] / 3, 4) for k, v in ph.items() if v[1]}
    # per-pair error against the exact HD of the full sets (FP16 tiles, FP32
    # rescoring, FP64 witness: the FP32 path's result)
    rels, rels1, bad = [], [], 0
    for pi, ((A, B), r) in enumerate(zip(pairs, res)):
        ex = prohd.hausdorff_exact_sync(A, B, "fp16")
        if r["status"] != "OK" or ex["status"] != "OK":
            bad += 1
            continue
        rels.append((ex["H"] - r["H"]) / ex["H"])
        if ref is not None:
            # the one-sided refinement of the same pair, from the refined batch
            r1 = res1[pi]
            rels1.append((ex["H"] - r1["H"]) / ex["H"] if r1["status"] == "OK" else np.nan)
    rels = np.asarray(rels)
    rels1 = np.asarray(rels1)
    # roofline figures per stage (algorithmic work / stage time)
    gram_fl = 0.0
    gram_bytes = 0.0
    proj_bytes = 0.0
    hd_elems = 0.0
    for (A, B), r in zip(pairs, res):
        n, D = A.shape[0] + B.shape[0], A.shape[1]
        gram_fl += 2.0 * n * D * D
        gram_bytes += n * D * 4.0
        proj_bytes += n * D * 4.0 + (1 + M_PCS) * n * 4.0
        hd_elems += float(r["nsel_a"]) * float(r["nsel_b"]) * D
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    stages = {}
    if "gram" in phases:
        # the method's work: one read of every set, 2 N D^2 flops; the
        # larger of the two bound times decides the bound
        t = phases["gram"] / 1e3
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        if gram_bytes / (peaks["hbm_gbs"] * 1e9) >= gram_fl / (pk * 1e12):
            a = gram_bytes / t / 1e9
            stages["gram"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": a / peaks["hbm_gbs"], "work": "one read of every set (n D 4 bytes per set)"}
        else:
            a = gram_fl / t / 1e12
            stages["gram"] = {"bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                              "work": "2 N D^2 flops per pair"}
    if "project" in phases:
        a = proj_bytes / (phases["project"] / 1e3) / 1e9
        stages["project"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": a / peaks["hbm_gbs"], "work": "read n*D*4 + write nd*n*4 bytes per set"}
    if "hd_contract" in phases:
        # FP16 tiles on the tensor cores (2 flops per (a, b, k)), with the
        # prep, margins and FP32 rescoring of the candidates inside the phase
        a = 2.0 * hd_elems / (phases["hd_contract"] / 1e3) / 1e12
        pk = peaks["bf16_tflops"]
        stages["hd_contract"] = {"bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                                 "work": "2 flops per (a, b, k) of the candidate subsets (FP16 tiles); the phase "
                                         "also holds the copies, margins and rescoring"}
    if "power" in phases:
        stages["power"] = {"bound": "latency", "iterations_sum": int(its.sum()), "iterations_max": int(its.max()),
                           "iterations_mean": float(its.mean()),
                           "note": "one CTA per pair; the phase ends with the slowest pair of each D class"}
    dom = max(phases, key=phases.get) if phases else None
    return {
        "workload": BATCH_WORKLOAD, "pairs": len(pairs), "points": npts, "bytes": nbytes,
        "value": 1000.0 * len(pairs) / ms, "unit": "set-pairs/s", "ms_per_batch": ms, "steps": steps,
        "graph": True, "tunables": b.tunables(), "autotune_best_ms": tuned_ms, "gpu_launches": launches,
        "phases_ms": phases, "dominant_phase": dom, "stages": stages,
        "status_not_ok": bad,
        "rel_err_vs_exact": {"max_abs": float(np.abs(rels).max()) if rels.size else None,
                             "mean_abs": float(np.abs(rels).mean()) if rels.size else None,
                             "frac_exact": float((rels == 0).mean()) if rels.size else None,
                             "overestimates": int((rels < 0).sum()),
                             "note": "(H_exact - H_hat) / H_exact per pair; exact HD of the full sets on the GPU"},
        "refined_rel_err_vs_exact": ({"max": float(np.nanmax(rels1)), "mean": float(np.nanmean(rels1)),
                                      "min": float(np.nanmin(rels1)), "frac_exact": float((rels1 == 0).mean()),
                                      "not_ok": int(np.isnan(rels1).sum()),
                                      "note": "max(h(A_sel,B), h(B_sel,A)) per pair from the batch planned with "
                                              "refine = 1; never above H, so every entry is >= 0"}
                                     if rels1.size else None),
        "refined": ref,
        "l2": "inputs (13 GB) larger than L2; no flush",
    }


# ---------------------------------------------------------------- learned directions

LEARNED_WORKLOAD = ("learned directions: network 10D -> 256 -> 256 -> 4D (D = 128, BF16 tensor-core GEMMs, FP32 "
                    "accumulate, Adam), trained on generated anisotropic Student-t (nu = 3) mixture pairs "
                    "(n ~ U[5k, 20k]) labelled by exact-HD witnesses; held-out pairs of n = 100,000 against plain "
                    "ProHD at an equal candidate budget")


def learned_arm(args, peaks, dev):
    """Training throughput of the network and its held-out gain."""
    import torch
    from paper_2511_18207_gb300 import learned, prohd

    ctx = prohd.context()
    t0 = time.time()
    X, Y = learned.make_dataset(ctx, args.learned_pairs, D=128, seed=args.seed + 11)
    t_data = time.time() - t0
    net = prohd.Mlp(ctx, 128, seed=1)
    B = 256
    # warm-up, then the timed steps (CUDA events on the launching stream)
    learned.train(net, X, Y, steps=args.warmup, batch=B, lr=1e-3, seed=1)
    st = torch.cuda.current_stream()
    l0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    losses, _ = learned.train(net, X, Y, steps=args.learned_steps, batch=B, lr=1e-3, seed=2)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.learned_steps
    launches = (ctx.launch_count() - l0) // args.learned_steps
    s = net.nparam
    n_in, h, n_out = 1280, 256, 512
    fwd = 2.0 * B * (n_in * h + h * h + h * n_out)
    bwd = 2.0 * B * (n_in * h + 2 * h * h + 2 * h * n_out)  # weight gradients, and input gradients of layers 2-3
    fl = fwd + bwd
    ev = learned.evaluate(ctx, net, args.learned_eval, n=100_000, D=128, seed=args.seed + 12345)
    ev.pop("rows")
    return {
        "workload": LEARNED_WORKLOAD, "params": s, "train_pairs": args.learned_pairs, "data_prep_s": t_data,
        "batch": B, "steps": args.learned_steps, "ms_per_step": ms, "samples_per_s": 1000.0 * B / ms,
        "gpu_launches_per_step": launches, "loss_first20": float(losses[:20].mean()),
        "loss_last20": float(losses[-20:].mean()),
        "roofline": {"kernel": "mlp_gemm_bf16_kernel (whole train step)", "bound": "latency",
                     "achieved": fl / (ms / 1e3) / 1e12, "unit": "TFLOP/s",
                     "peak": peaks["bf16_tflops"], "frac": fl / (ms / 1e3) / 1e12 / peaks["bf16_tflops"],
                     "note": "GEMMs of 256 x <=1280 x <=512: the step is launch- and latency-bound, not tensor-bound"},
        "held_out": ev,
    }


# ---------------------------------------------------------------- reference arm

def reference_arm(args):
    """The FP64 oracle as the reference: each step is one bounded sample of
    the 2M pair (oracle_sample); ms_per_step is that step's measured time,
    and value is the full-pair throughput extrapolated from it by the stated
    factors (the full pair would take minutes per step on the host cores)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    A, B = make_pair(seed=args.seed, n=args.n)
    for _ in range(args.warmup):
        oracle_sample(A, B, rows_cov=50_000, rows_hd=32)
    t0 = time.perf_counter()
    sample_s = 0.0
    pair_s = 0.0
    last = None
    for _ in range(args.steps):
        t1 = time.perf_counter()
        last = oracle_sample(A, B)
        sample_s += time.perf_counter() - t1
        pair_s += last["seconds_per_pair"]
    wall = time.perf_counter() - t0
    value = args.steps / pair_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sample_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "extrapolated": True,
        "ms_per_full_pair_extrapolated": 1000.0 * pair_s / args.steps,
        "step_note": ("a step is one bounded sample of the pair, timed (ms_per_step); value is the full pair's "
                      "throughput extrapolated from it by scale_factors"),
        "scale_factors": last["scale_factors"],
        "config": {"workload": WORKLOAD if args.n == N_POINTS else WORKLOAD.replace("2,000,000", f"{args.n:,}"),
                   "n_a": args.n, "n_b": args.n, "D": DIM, "m": M_PCS, "alpha": ALPHA,
                   "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"], "extrapolated": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "stages_s_measured": last["stages_s_measured"], "stages_s_extrapolated": last["stages_s_extrapolated"],
        "wall_s": wall,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["prohd", "reference"], default="prohd")
    ap.add_argument("--n", type=int, default=N_POINTS, help="points per set (default: the 2M workload)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-pair batch measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-direction measurement")
    ap.add_argument("--no-refined", action="store_true", help="skip the one-sided refinement measurements")
    ap.add_argument("--learned-pairs", type=int, default=50_000)
    ap.add_argument("--learned-steps", type=int, default=4000)
    ap.add_argument("--learned-eval", type=int, default=32)
    ap.add_argument("--workload", choices=["pair", "batched", "learned"], default="pair",
                    help="pair: the 2M x 2M headline line (with the batch and learned objects); "
                         "batched / learned: only that measurement, on a line of its own")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload != "pair":
        part_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
