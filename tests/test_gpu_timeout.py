"""Bounded device waits: a limit that runs out is reported, and the context recovers.

Every wait on an mbarrier (the tensor-core kernels and the TMA-fed
projection) is bounded by params.wait_timeout_ns, read from %globaltimer. When a wait runs out the
kernel raises a CTA-wide abort flag, lets the copies it issued land (with a
limit of its own), completes its issued MMAs, frees its tensor memory and
returns; the result then carries PROHD_ETIMEOUT. A limit of 1 ns makes the
first wait that is not already satisfied run out (the first accumulator wait
of the contraction is never satisfied on entry), so the abort path runs for
certain. Nothing here faults or hangs a GPU: the failure is a limit the host
sets. The next call with the default limit, on the same context and stream,
must succeed and agree with the oracle."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _check_against_oracle(A, B, r, dirs, kA, kB):
    ia, ib = oracle.select(A, dirs, kA), oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(r["idxA"], ia)
    np.testing.assert_array_equal(r["idxB"], ib)
    sub = oracle.hausdorff(A[ia], B[ib])
    assert rel(r["H"], sub["H"]) <= 1e-5, (r["H"], sub["H"])


def test_contraction_timeout_is_reported_and_the_next_call_succeeds():
    torch = torch_cuda()
    A, B = W.mixture_pair(30_000, 64, 8, seed=11)
    m, alpha = 4, 0.02
    c = ctx()
    At, Bt = dev(A), dev(B)
    d, _ = c.prohd_directions(At, Bt, m=m)
    torch.cuda.synchronize()
    dirs = d.cpu().numpy()
    kA = oracle.k_list(A.shape[0], 1 + m, alpha, alpha / m)
    kB = oracle.k_list(B.shape[0], 1 + m, alpha, alpha / m)
    idxA = torch.empty(A.shape[0], dtype=torch.int32, device="cuda")
    idxB = torch.empty(B.shape[0], dtype=torch.int32, device="cuda")
    # selection onwards with the given directions: the projection's TMA
    # ring and the distance contraction have bounded waits
    short = prohd.default_params(m=m, alpha_c=alpha, precision="fp16", wait_timeout_ns=1)
    out = c.prohd_estimate_dirs(At, Bt, d, kA, kB, params=short, idxA=idxA, idxB=idxB)
    torch.cuda.synchronize()
    assert prohd.decode_result(out)["status"] == "ETIMEOUT"
    # default limit, same context and stream
    normal = prohd.default_params(m=m, alpha_c=alpha, precision="fp16")
    out = c.prohd_estimate_dirs(At, Bt, d, kA, kB, params=normal, idxA=idxA, idxB=idxB)
    torch.cuda.synchronize()
    r = prohd.decode_result(out)
    assert r["status"] == "OK", r
    r["idxA"] = idxA[: r["nsel_a"]].cpu().numpy()
    r["idxB"] = idxB[: r["nsel_b"]].cpu().numpy()
    _check_against_oracle(A, B, r, dirs, kA, kB)


def test_gram_and_contraction_timeout_in_a_full_estimate():
    # the full estimate: the tensor-core Gram (D = 64) and the contraction
    # both run with the 1 ns limit; the later stages run on whatever the
    # aborted Gram left (as after a non-finite input), and the status says so
    torch_cuda()
    A, B = W.mixture_pair(30_000, 64, 8, seed=12)
    m, alpha = 4, 0.02
    r = prohd.prohd_estimate_sync(dev(A), dev(B), m=m, alpha_c=alpha, precision="fp16", wait_timeout_ns=1)
    assert r["status"] == "ETIMEOUT", r["status"]
    r = prohd.prohd_estimate_sync(dev(A), dev(B), want_indices=True, want_dirs=True, m=m, alpha_c=alpha,
                                  precision="fp16")
    assert r["status"] == "OK", r
    kA = oracle.k_list(A.shape[0], 1 + m, alpha, alpha / m)
    kB = oracle.k_list(B.shape[0], 1 + m, alpha, alpha / m)
    _check_against_oracle(A, B, r, r["dirs"], kA, kB)
