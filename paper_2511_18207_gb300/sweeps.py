"""Parameter sweeps of ProHD on random clouds (Evaluation – Datasets and Experimental Setup data: U[0,1]^D
against U[0,1]^D + 0.1), the synthetic halves of the paper's sensitivity and
scalability studies (Evaluation – Parameter Sensitivity and Scalability Analysis):

* ``alpha``: the selection fraction (Fig. 2's sweep, here on random clouds);
* ``dim``: D in {2, ..., 256} at 100k + 100k points (Fig. 3);
* ``ratio``: n_B / n_A in {0.125, 0.25, 0.5, 1} with n_A = 100k, D = 4 (Fig. 4);
* ``size``: n_A = n_B from 100k to 1M, D = 4 (Fig. 5);
* ``adaptive``: the adaptive alpha schedule of Conclusion and Future Work (doubling alpha on the
  refined estimate until it stabilises) at D = 4, 64, 256.

Every point runs through the library: the estimate of Algorithm 3
(``prohd_estimate``), its one-sided refinement (``refine = 1``) and the exact
Hausdorff distance of the full sets (``hausdorff_exact`` with FP16 tiles and FP32 rescoring, the ground
truth),
each timed with CUDA events on the launching stream after one warm-up call.
Errors are (H - estimate) / H per pair, averaged over seeds.

``python -m paper_2511_18207_gb300.sweeps [--which alpha,dim,ratio,size]
[--seeds 5]`` prints one JSON object per point and a markdown table.
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import prohd
from . import workloads as W

SWEEPS = {
    "alpha": [dict(n_a=100_000, n_b=100_000, D=4, alpha=a) for a in (0.0025, 0.005, 0.01, 0.02, 0.04, 0.08)]
    + [dict(n_a=100_000, n_b=100_000, D=64, alpha=a) for a in (0.0025, 0.005, 0.01, 0.02, 0.04, 0.08)],
    "dim": [dict(n_a=100_000, n_b=100_000, D=d, alpha=0.01) for d in (2, 4, 8, 16, 32, 64, 128, 256)],
    "ratio": [dict(n_a=100_000, n_b=int(100_000 * r), D=4, alpha=0.01) for r in (0.125, 0.25, 0.5, 1.0)],
    "size": [dict(n_a=n, n_b=n, D=4, alpha=0.01) for n in (100_000, 250_000, 500_000, 1_000_000)],
    # adaptive alpha (prohd_estimate_adaptive): alpha doubled from 0.25% up to
    # 16% until the refined estimate grows by at most rel_tol
    "adaptive": [dict(n_a=100_000, n_b=100_000, D=d, alpha=0.0025, alpha_max=0.16, rel_tol=t)
                 for d in (4, 64, 256) for t in (1e-3, 1e-2)],
}


def _timed(fn, torch):
    fn()  # warm-up (loads kernels, sizes the workspace)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    out = fn()
    e1.record(st)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def run_point(pt: dict, seeds: int, torch, power_max_iters: int | None = None) -> dict:
    """One sweep point averaged over ``seeds`` random-cloud pairs
    (``power_max_iters`` caps the direction stage's iterations)."""
    ctx = prohd.context()
    D = pt["D"]
    m = max(1, int(math.isqrt(D)))
    rows = []
    for s in range(seeds):
        A, B = W.random_clouds(pt["n_a"], pt["n_b"], D, seed=1000 * s + D)
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        p0 = prohd.default_params(m=m, alpha_c=pt["alpha"], precision="fp16", power_max_iters=power_max_iters)
        p1 = prohd.default_params(m=m, alpha_c=pt["alpha"], precision="fp16", refine=1,
                                  power_max_iters=power_max_iters)
        o0, t0 = _timed(lambda: ctx.prohd_estimate(At, Bt, params=p0), torch)
        r0 = prohd.decode_result(o0)
        o1, t1 = _timed(lambda: ctx.prohd_estimate(At, Bt, params=p1), torch)
        r1 = prohd.decode_result(o1)
        oe, te = _timed(lambda: ctx.hausdorff_exact(At, Bt, "fp16"), torch)
        ex = prohd.decode_hd(oe)
        if "OK" != r0["status"] or "OK" != r1["status"] or "OK" != ex["status"]:
            raise RuntimeError(f"status {r0['status']} / {r1['status']} / {ex['status']} at {pt}, seed {s}")
        H = ex["H"]
        rows.append(dict(err=(H - r0["H"]) / H, err1=(H - r1["H"]) / H, ms=t0, ms1=t1, ms_exact=te,
                         frac=(r0["nsel_a"] + r0["nsel_b"]) / (pt["n_a"] + pt["n_b"])))
        del At, Bt
    a = {k: np.array([r[k] for r in rows]) for k in rows[0]}
    return dict(pt, m=m, seeds=seeds, power_max_iters=power_max_iters,
                rel_err_mean_abs=float(np.abs(a["err"]).mean()), rel_err_mean_signed=float(a["err"].mean()),
                overestimates=int((a["err"] < 0).sum()),
                refined_rel_err_mean=float(a["err1"].mean()), refined_rel_err_max=float(a["err1"].max()),
                ms=float(np.median(a["ms"])), refined_ms=float(np.median(a["ms1"])),
                exact_ms=float(np.median(a["ms_exact"])), subset_frac=float(a["frac"].mean()))


def run_adaptive_point(pt: dict, seeds: int, torch, power_max_iters: int | None = None) -> dict:
    """One adaptive-alpha point averaged over ``seeds`` random-cloud pairs."""
    ctx = prohd.context()
    D = pt["D"]
    m = max(1, int(math.isqrt(D)))
    rows = []
    for s in range(seeds):
        A, B = W.random_clouds(pt["n_a"], pt["n_b"], D, seed=1000 * s + D)
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        p = prohd.default_params(m=m, alpha_c=pt["alpha"], precision="fp16", power_max_iters=power_max_iters)
        (o, sched), t = _timed(lambda: ctx.prohd_estimate_adaptive(At, Bt, pt["alpha_max"], pt["rel_tol"],
                                                                   params=p), torch)
        r = prohd.decode_result(o)
        ex = prohd.decode_hd(ctx.hausdorff_exact(At, Bt, "fp16"))
        if r["status"] != "OK" or ex["status"] != "OK":
            raise RuntimeError(f"status {r['status']} / {ex['status']} at {pt}, seed {s}")
        rows.append(dict(err=(ex["H"] - r["H"]) / ex["H"], ms=t, steps=sched["steps"], alpha=sched["alpha_c"],
                         frac=(r["nsel_a"] + r["nsel_b"]) / (pt["n_a"] + pt["n_b"]), reason=sched["reason"]))
        del At, Bt
    a = {k: np.array([r[k] for r in rows]) for k in rows[0] if k != "reason"}
    return dict(pt, m=m, seeds=seeds, rel_err_mean=float(a["err"].mean()), rel_err_max=float(a["err"].max()),
                ms=float(np.median(a["ms"])), steps_mean=float(a["steps"].mean()),
                alpha_final_mean=float(a["alpha"].mean()), subset_frac=float(a["frac"].mean()),
                reasons=sorted({r["reason"] for r in rows}))


def run(which, seeds: int = 5, log=None, power_max_iters: int | None = None) -> dict:
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("the sweeps run on the GPU")
    out = {}
    for name in which:
        res = []
        for pt in SWEEPS[name]:
            point = run_adaptive_point if name == "adaptive" else run_point
            r = point(pt, seeds, torch, power_max_iters)
            res.append(r)
            if log is not None:
                print(json.dumps(dict(sweep=name, **r)), file=log, flush=True)
        out[name] = res
    return out


def markdown(out: dict) -> str:
    lines = []
    for name, res in out.items():
        lines.append(f"### {name}\n")
        if name == "adaptive":
            lines.append("| n_A | n_B | D | alpha_0 | alpha_max | rel_tol | steps | final alpha | subset "
                         "| err (mean / max) | ms | stop |")
            lines.append("|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---|")
            for r in res:
                lines.append(f"| {r['n_a']:,} | {r['n_b']:,} | {r['D']} | {r['alpha']} | {r['alpha_max']} "
                             f"| {r['rel_tol']} | {r['steps_mean']:.1f} | {r['alpha_final_mean']:.4f} "
                             f"| {100 * r['subset_frac']:.2f}% | {100 * r['rel_err_mean']:.2f}% / "
                             f"{100 * r['rel_err_max']:.2f}% | {r['ms']:.2f} | {', '.join(r['reasons'])} |")
            lines.append("")
            continue
        lines.append("| n_A | n_B | D | alpha | subset | |err| Alg. 3 | above H | err refined (mean / max) "
                     "| ms Alg. 3 | ms refined | ms exact |")
        lines.append("|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|")
        for r in res:
            lines.append(f"| {r['n_a']:,} | {r['n_b']:,} | {r['D']} | {r['alpha']} | {100 * r['subset_frac']:.2f}% "
                         f"| {100 * r['rel_err_mean_abs']:.2f}% | {r['overestimates']}/{r['seeds']} "
                         f"| {100 * r['refined_rel_err_mean']:.2f}% / {100 * r['refined_rel_err_max']:.2f}% "
                         f"| {r['ms']:.2f} | {r['refined_ms']:.2f} | {r['exact_ms']:.1f} |")
        lines.append("")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--which", default="alpha,dim,ratio,size,adaptive")
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--json", default=None, help="write the results here as one JSON object")
    ap.add_argument("--power-max-iters", type=int, default=None, help="cap of the direction stage's iterations")
    args = ap.parse_args(argv)
    which = [w for w in args.which.split(",") if w]
    for w in which:
        if w not in SWEEPS:
            raise SystemExit(f"unknown sweep {w}; choose from {', '.join(SWEEPS)}")
    out = run(which, args.seeds, log=sys.stderr, power_max_iters=args.power_max_iters)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f)
    print(markdown(out))


if __name__ == "__main__":
    main()
