"""hausdorff_exact_noalloc: the FP32 exact Hausdorff distance for callers that
cannot allocate device memory (for example code running under another
component's stream capture, or a plugin whose host framework owns the
allocator). It uses a fixed scratch array inside the library instead of a
workspace. Checked through the C ABI against hausdorff_exact (FP32) on two
calls in a row, so the second call also shows that the shared scratch left
behind by the first is reset. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2511_18207_gb300 import prohd

pytestmark = pytest.mark.gpu


def _run(lib, ctx, A, B, noalloc):
    import torch

    out = torch.empty(ctypes.sizeof(prohd.HdResult), dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pa, pb, po = (ctypes.c_void_p(t.data_ptr()) for t in (A, B, out))
    if noalloc:
        rc = lib.hausdorff_exact_noalloc(ctx.h, pa, A.shape[0], pb, B.shape[0], A.shape[1], po, st)
    else:
        need = lib.hausdorff_exact_workspace_size(A.shape[0], B.shape[0], A.shape[1], 0)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        rc = lib.hausdorff_exact(ctx.h, pa, A.shape[0], pb, B.shape[0], A.shape[1], 0, po,
                                 ctypes.c_void_p(ws.data_ptr()), need, st)
    assert rc == prohd.PROHD_OK, lib.prohd_last_error(ctx.h)
    torch.cuda.synchronize()
    return prohd.decode_hd(out)


def test_noalloc_matches_workspace_entry_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = prohd.load_library()
    ctx = prohd.Context()
    rng = np.random.default_rng(77)
    cases = [((3000, 48), (2500, 48), 0.0), ((1200, 48), (4000, 48), 0.7)]  # second call: other sizes and data
    for (sa, sb, shift) in cases:
        A = torch.from_numpy(rng.standard_normal(sa).astype(np.float32)).cuda()
        B = torch.from_numpy((rng.standard_normal(sb) + shift).astype(np.float32)).cuda()
        ref = _run(lib, ctx, A, B, noalloc=False)
        got = _run(lib, ctx, A, B, noalloc=True)
        assert got["status"] == "OK"
        for k in ("H", "h_ab", "h_ba"):
            assert abs(got[k] - ref[k]) <= 1e-5 * ref[k], (k, got[k], ref[k])


def test_noalloc_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = prohd.Context()
    A = torch.zeros((200_000, 4), device="cuda")
    with pytest.raises(prohd.ProHDError, match="2 MiB scratch"):
        ctx.hausdorff_exact_noalloc(A, A)
