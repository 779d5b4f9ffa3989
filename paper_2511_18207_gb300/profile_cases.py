"""Small, fixed workloads for kernel profiling (``ncu``) of single kernels.

    python -m paper_2511_18207_gb300.profile_cases directions   # Gram + block iteration, 400k + 400k x 256
    python -m paper_2511_18207_gb300.profile_cases exact        # distance contraction, 100k x 100k x 256, FP16
    python -m paper_2511_18207_gb300.profile_cases pruned       # row-pruned exact distance, 2M x 2M x 256 (launch list)
    python -m paper_2511_18207_gb300.profile_cases estimate     # one ProHD estimate, 2M x 2M x 256 (launch list)
    python -m paper_2511_18207_gb300.profile_cases estimate_small  # one ProHD estimate, 400k x 400k x 256 (captures)
    python -m paper_2511_18207_gb300.profile_cases batch        # the 512-pair batch, one direct run (launch list)
    python -m paper_2511_18207_gb300.profile_cases batch_refined  # the same batch with refine = 1 (launch list)

Each case runs its call twice (the second launch is the one to capture, e.g.
``ncu --clock-control none -k regex:gram_tc_kernel -s 1 -c 1``), keeps the
device footprint to a few hundred MB (inputs larger than L2), and prints a
one-line result. Every capture must keep ``--clock-control none``: without it
ncu locks the GPU clocks, and a shared GPU's next user inherits the lock.
"""
from __future__ import annotations

import sys


def directions():
    import torch

    from . import prohd, workloads as W

    A, B = W.anisotropic_pair(400_000, 400_000, 256, seed=1)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c = prohd.context()
    for _ in range(2):
        d, e = c.prohd_directions(At, Bt, m=8)
    torch.cuda.synchronize()
    print("eigenvalues", e.cpu().numpy()[:4])


def exact():
    import torch

    from . import prohd, workloads as W

    A, B = W.mixture_pair(100_000, 256, 16, seed=3)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    r = None
    for _ in range(2):
        r = prohd.hausdorff_exact_sync(At, Bt, "fp16")
    print("H", r["H"], r["status"])


def pruned():
    # the benchmark's anisotropic pair; for a launch list (one-pass metric)
    # only: the inputs and workspace hold about 8 GB on the device
    import torch

    from . import prohd, workloads as W

    A, B = W.anisotropic_pair(2_000_000, 2_000_000, 256, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=0)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c = prohd.context()
    kept = None
    for _ in range(2):
        out, kept = c.hausdorff_exact_pruned(At, Bt, "fp16", want_kept=True)
    r = prohd.decode_hd(out)
    print("H", r["H"], r["status"], "rows kept", kept)


def estimate():
    # the benchmark's pair and estimate (m = 8, alpha = 0.01, FP16 tiles): two
    # calls, the second is the one to list (about 5.5 GB on the device)
    import torch

    from . import prohd, workloads as W

    A, B = W.anisotropic_pair(2_000_000, 2_000_000, 256, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=0)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    r = None
    for _ in range(2):
        r = prohd.prohd_estimate_sync(At, Bt, m=8, alpha_c=0.01, precision="fp16")
    print("H_hat", r["H"], r["status"], "|A_sel|", r["nsel_a"], "|B_sel|", r["nsel_b"])


def estimate_small():
    # the benchmark's law at 400k + 400k points (about 1.5 GB on the device),
    # for full captures of the selection and distance kernels
    import torch

    from . import prohd, workloads as W

    A, B = W.anisotropic_pair(400_000, 400_000, 256, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=0)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    r = None
    for _ in range(2):
        r = prohd.prohd_estimate_sync(At, Bt, m=8, alpha_c=0.01, precision="fp16")
    print("H_hat", r["H"], r["status"], "|A_sel|", r["nsel_a"], "|B_sel|", r["nsel_b"])


def _batch(refine: int):
    # the benchmark's 512 uneven pairs (13 GB drawn on the device, about 8 GB
    # of workspace, 16 GB with refine = 1) planned with the tuned item sizes and
    # run once without the graph: one launch per stage, for a launch list
    import torch

    from . import prohd, workloads as W

    pairs = W.batched_pairs_device(512, seed=7)
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = prohd.Batch(prohd.context(), pairs, m=8, alpha_c=0.01, precision="fp16", refine=refine)
        b.set_tunables(32768, 32768, 131072)
        b.use_graph(False)
        b.run(st)
        st.synchronize()
    res = b.results()
    print("pairs", len(res), "H sum", sum(r["H"] for r in res))


def batch():
    _batch(0)


def batch_refined():
    _batch(1)


CASES = {"directions": directions, "exact": exact, "pruned": pruned, "estimate": estimate,
         "estimate_small": estimate_small, "batch": batch, "batch_refined": batch_refined}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        sys.exit(f"usage: python -m paper_2511_18207_gb300.profile_cases {{{'|'.join(CASES)}}}")
    CASES[sys.argv[1]]()
