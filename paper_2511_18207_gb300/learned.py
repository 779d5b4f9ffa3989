"""Learned directions: training data, training loop and evaluation.

Host orchestration of library calls only (every arithmetic step of the
features, the network, its gradient and update, the selection and the
Hausdorff distances runs in the CUDA library):

* training pairs: anisotropic Student-t (nu = 3) mixtures on the device;
  features from ``prohd_features``; label = the unit witness direction
  (a* - b*)/||a* - b*|| of the exact HD (``hausdorff_exact``);
* training: Adam steps of ``prohd_mlp_train_step`` over shuffled minibatches;
* evaluation at an equal candidate budget: plain ProHD keeps k_p per
  component on 8 components; the learned form adds the network's 4
  directions and keeps k_p * 8/12 on all 12, so the candidate count before
  deduplication is the same; both against the exact HD of the full sets.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import prohd
from . import workloads as W


def _pair(seed: int, n_lo: int, n_hi: int, D: int, device: str):
    import torch

    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    na = int(torch.randint(n_lo, n_hi + 1, (1,), generator=g))
    nb = int(torch.randint(n_lo, n_hi + 1, (1,), generator=g))
    K = int(torch.randint(2, 9, (1,), generator=g))
    s = int(torch.randint(0, 2**31 - 1, (1,), generator=g))
    A = W.student_t_mixture_device(na, D, K, seed=2 * s, device=device)
    B = W.student_t_mixture_device(nb, D, K, seed=2 * s + 1, device=device)
    return A, B


def witness_label(ctx, A, B):
    """Unit witness direction of the exact HD (FP16 tiles, FP32 rescoring)."""
    r = prohd.decode_hd(ctx.hausdorff_exact(A, B, "fp16"))
    d = A[r["wit_a"]].double() - B[r["wit_b"]].double()
    n = float(d.norm())
    return (d / n if n > 0 else d).float(), r


def make_dataset(ctx, npairs: int, n_lo: int = 5000, n_hi: int = 20000, D: int = 128, seed: int = 0,
                 device: str = "cuda"):
    """(features [N, 10D], labels [N, D]) device tensors of npairs generated pairs."""
    import torch

    X = torch.empty((npairs, 10 * D), dtype=torch.float32, device=device)
    Y = torch.empty((npairs, D), dtype=torch.float32, device=device)
    for i in range(npairs):
        A, B = _pair(seed * 1_000_003 + i, n_lo, n_hi, D, device)
        ctx.prohd_features(A, B, feat=X[i])
        Y[i], _ = witness_label(ctx, A, B)
    torch.cuda.synchronize()
    return X, Y


def train(net, X, Y, steps: int, batch: int = 256, lr: float = 1e-3, precision: str = "bf16", seed: int = 0,
          log_every: int = 0):
    """Adam steps over seeded shuffled minibatches; returns the loss history
    (host floats, one per step) and the wall time of the steps."""
    import torch

    N = X.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    perm = torch.randperm(N, generator=g)
    pos = 0
    losses = torch.empty(steps, dtype=torch.float32, device=X.device)
    torch.cuda.synchronize()
    t0 = time.time()
    for s in range(steps):
        if pos + batch > N:
            perm = torch.randperm(N, generator=g)
            pos = 0
        idx = perm[pos:pos + batch].to(X.device)
        pos += batch
        net.train_step(X[idx], Y[idx], lr=lr, precision=precision, loss=losses[s:s + 1])
        if log_every and (s + 1) % log_every == 0:
            print(f"step {s + 1} loss {float(losses[s]):.4f}", flush=True)
    torch.cuda.synchronize()
    return losses.cpu().numpy(), time.time() - t0


def alignment(dirs, w) -> float:
    """max over directions of (u . w)^2."""
    d = dirs.double()
    d = d / d.norm(dim=1, keepdim=True)
    return float(((d @ w.double()) ** 2).max())


def evaluate(ctx, net, npairs: int, n: int = 100_000, D: int = 128, alpha: float = 0.01, seed: int = 12345,
             precision: str = "bf16", device: str = "cuda") -> dict:
    """Held-out pairs of n points per set: relative error of plain ProHD and
    of the learned form at an equal candidate budget, against the exact HD."""
    import torch

    m = 8
    ap = alpha / m
    rows = []
    for i in range(npairs):
        A, B = _pair(seed * 1_000_003 + i, n, n, D, device)
        feat, dirs, eig = ctx.prohd_features(A, B)
        w, ex = witness_label(ctx, A, B)
        H = ex["H"]
        nA, nB = A.shape[0], B.shape[0]
        kc = [prohd.k_of(alpha, nA), prohd.k_of(alpha, nB)]
        # plain: centroid axis + 8 components, alpha_p per component
        kpA, kpB = prohd.k_of(ap, nA), prohd.k_of(ap, nB)
        rp = prohd.decode_result(ctx.prohd_estimate_dirs(A, B, dirs, [kc[0]] + [kpA] * m, [kc[1]] + [kpB] * m,
                                                         precision="fp16"))
        # learned: + 4 network directions, alpha_p * 8/12 on all 12
        u = net.forward(feat[None, :], precision=precision, want64=True)[1][0]
        all_dirs = torch.cat([dirs, u], dim=0)
        kqA, kqB = prohd.k_of(ap * m / (m + 4), nA), prohd.k_of(ap * m / (m + 4), nB)
        rl = prohd.decode_result(ctx.prohd_estimate_dirs(A, B, all_dirs, [kc[0]] + [kqA] * (m + 4),
                                                         [kc[1]] + [kqB] * (m + 4), precision="fp16"))
        rows.append(dict(H=H, plain=rp["H"], learned=rl["H"], nsel_plain=rp["nsel_a"] + rp["nsel_b"],
                         nsel_learned=rl["nsel_a"] + rl["nsel_b"], align_plain=alignment(dirs[1:], w),
                         align_learned=alignment(u, w)))
    ep = np.array([abs(r["plain"] - r["H"]) / r["H"] for r in rows])
    el = np.array([abs(r["learned"] - r["H"]) / r["H"] for r in rows])
    return dict(pairs=npairs, n=n, D=D, alpha=alpha,
                rel_err_plain_mean=float(ep.mean()), rel_err_learned_mean=float(el.mean()),
                rel_err_plain_max=float(ep.max()), rel_err_learned_max=float(el.max()),
                learned_better=int((el < ep).sum()), learned_worse=int((el > ep).sum()),
                align_plain_mean=float(np.mean([r["align_plain"] for r in rows])),
                align_learned_mean=float(np.mean([r["align_learned"] for r in rows])),
                nsel_plain_mean=float(np.mean([r["nsel_plain"] for r in rows])),
                nsel_learned_mean=float(np.mean([r["nsel_learned"] for r in rows])),
                rows=rows)


def main():
    import argparse
    import json

    ap = argparse.ArgumentParser(description="train the learned-direction network and evaluate its gain")
    ap.add_argument("--pairs", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--eval-pairs", type=int, default=16)
    ap.add_argument("--eval-n", type=int, default=100_000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--precision", default="bf16")
    ap.add_argument("--checkpoint", default="")
    args = ap.parse_args()
    ctx = prohd.context()
    t0 = time.time()
    X, Y = make_dataset(ctx, args.pairs)
    t_data = time.time() - t0
    net = prohd.Mlp(ctx, 128, seed=1)
    losses, t_train = train(net, X, Y, args.steps, lr=args.lr, precision=args.precision, log_every=200)
    if args.checkpoint:
        net.save(args.checkpoint)
    ev = evaluate(ctx, net, args.eval_pairs, n=args.eval_n, precision=args.precision)
    ev.pop("rows")
    print(json.dumps(dict(data_s=t_data, train_s=t_train, loss_first=float(losses[:20].mean()),
                          loss_last=float(losses[-20:].mean()), eval=ev)))


if __name__ == "__main__":
    main()
