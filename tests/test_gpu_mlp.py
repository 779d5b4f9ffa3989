"""The learned-direction network on the GPU against the FP64 oracle
(oracle/mlp.py), and the learned form of ProHD end to end.

Tolerances: the FP32 path accumulates K <= 10 D products per output in FP32
(relative error of a few 1e-7 times sqrt(K) on sums of mixed-sign terms);
its outputs, loss and gradients are held to 1e-5 of each tensor's largest
entry (1e-4 for the first layer's gradient, a sum over the batch of products
of two computed quantities). The BF16 path rounds every GEMM operand to 8
significant bits (relative 2^-8 per operand): it is held to an oracle that rounds
the same operands to BF16, and normwise to 3e-2 of the FP64 network."""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(D, B, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 10 * D)).astype(np.float32)
    Wl = rng.standard_normal((B, D))
    Wl /= np.linalg.norm(Wl, axis=1, keepdims=True)
    return X, Wl.astype(np.float32)


def _gpu_params(net):
    return omlp.unflatten(net.params.double().cpu().numpy(), net.D)


@pytest.mark.parametrize("D", [8, 64, 128])
def test_init_is_the_oracle_init(D):
    torch = torch_cuda()
    net = prohd.Mlp(ctx(), D, seed=7)
    torch.cuda.synchronize()
    P = omlp.init_params(D, 7)
    G = _gpu_params(net)
    for k in P:
        assert np.array_equal(G[k], P[k]), k
    # Adam moments start at zero
    assert float(net.state[net.nparam:].abs().max()) == 0.0


@pytest.mark.parametrize("D,B", [(8, 5), (64, 33), (128, 256)])
def test_fp32_forward_loss_gradient_match_oracle(D, B):
    torch = torch_cuda()
    net = prohd.Mlp(ctx(), D, seed=3)
    X, Wl = _problem(D, B, seed=D)
    Xt, Wt = dev(X), dev(Wl)
    u = net.forward(Xt, precision="fp32")
    loss, grad = net.loss_grad(Xt, Wt, precision="fp32")
    torch.cuda.synchronize()
    P = omlp.init_params(D, 3)
    f = omlp.forward(P, X.astype(np.float64), Wl.astype(np.float64))
    G = omlp.backward(P, f)
    np.testing.assert_allclose(u.cpu().numpy(), f["U"], rtol=0, atol=2e-5)
    assert abs(float(loss) - f["loss_mean"]) <= 1e-5
    Gg = omlp.unflatten(grad.double().cpu().numpy(), D)
    for k in G:
        tol = (1e-4 if k == "W1" else 1e-5) * max(np.abs(G[k]).max(), 1e-12)
        np.testing.assert_allclose(Gg[k], G[k], rtol=0, atol=tol, err_msg=k)


@pytest.mark.parametrize("D,B", [(8, 5), (64, 64), (128, 256)])
def test_bf16_gradient_matches_oracle(D, B):
    # against the oracle with every product operand rounded to BF16 (the same
    # ReLU decisions on the same rounded operands); what remains is FP32
    # against FP64 accumulation, about 1e-6 relative, and the operands whose
    # FP32 and FP64 values straddle a BF16 rounding boundary (about 2.5e-4 of
    # them, each then one BF16 unit, 2^-8, apart): measured 2.6e-4 normwise on
    # the outputs
    torch = torch_cuda()
    net = prohd.Mlp(ctx(), D, seed=4)
    X, Wl = _problem(D, B, seed=D + 1)
    u = net.forward(dev(X), precision="bf16")
    loss, grad = net.loss_grad(dev(X), dev(Wl), precision="bf16")
    torch.cuda.synchronize()
    P = omlp.init_params(D, 4)
    f = omlp.forward(P, X.astype(np.float64), Wl.astype(np.float64), bf16=True)
    G = omlp.backward(P, f)
    assert np.linalg.norm(u.cpu().numpy() - f["U"]) <= 2e-3 * np.linalg.norm(f["U"])
    assert abs(float(loss) - f["loss_mean"]) <= 1e-4
    # Gradients: a flipped operand upstream can move a near-zero
    # pre-activation across 0, and a flipped ReLU mask adds or removes a whole
    # term of a B-term weight-gradient sum (about 1/sqrt(B) of its column);
    # measured 3.8% normwise on W2 at B = 64. A wrong fragment layout or
    # stride would be O(1).
    Gg = omlp.unflatten(grad.double().cpu().numpy(), D)
    for k in G:
        assert np.linalg.norm(Gg[k] - G[k]) <= 5e-2 * np.linalg.norm(G[k]) + 1e-12, k
    # and the BF16 path stays near the FP64 network (operand rounding only)
    f64 = omlp.forward(P, X.astype(np.float64), Wl.astype(np.float64))
    assert np.linalg.norm(u.cpu().numpy() - f64["U"]) <= 3e-2 * np.linalg.norm(f64["U"])


def test_adam_steps_match_oracle():
    # the same seeded gradients on both sides (Adam's own arithmetic, FP32
    # against FP64), then a train step equals gradient + Adam on the GPU
    torch = torch_cuda()
    D = 16
    net = prohd.Mlp(ctx(), D, seed=5)
    P = omlp.init_params(D, 5)
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    rng = np.random.default_rng(11)
    for step in range(1, 4):
        G = {k: rng.standard_normal(v.shape) * 10.0 ** rng.uniform(-4, 0) for k, v in P.items()}
        gflat = omlp.flatten({k: G[k].astype(np.float32).astype(np.float64) for k in G}, D)
        net.adam(torch.from_numpy(gflat.astype(np.float32)).cuda(), lr=1e-2)
        omlp.adam_step(P, M, V, {k: G[k].astype(np.float32).astype(np.float64) for k in G}, lr=1e-2, step=step)
    torch.cuda.synchronize()
    Gp = _gpu_params(net)
    for k in P:
        np.testing.assert_allclose(Gp[k], P[k], rtol=0, atol=1e-6 * max(1.0, np.abs(P[k]).max()), err_msg=k)
    # train_step = loss_grad + Adam with the same step count
    X, Wl = _problem(D, 32, seed=3)
    a = prohd.Mlp(ctx(), D, seed=6)
    b = prohd.Mlp(ctx(), D, seed=6)
    a.train_step(dev(X), dev(Wl), lr=1e-3, precision="fp32")
    _, g = b.loss_grad(dev(X), dev(Wl), precision="fp32")
    b.adam(g, lr=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(a.state, b.state)


def test_training_reduces_the_loss_on_a_learnable_target():
    # label = direction of the centroid-difference block of the features: a
    # linear function of the input, reachable by the network
    torch = torch_cuda()
    D, N = 32, 2048
    rng = np.random.default_rng(0)
    X = rng.standard_normal((N, 10 * D)).astype(np.float32)
    Y = X[:, :D] / np.linalg.norm(X[:, :D], axis=1, keepdims=True)
    net = prohd.Mlp(ctx(), D, seed=0)
    from paper_2511_18207_gb300 import learned
    losses, _ = learned.train(net, dev(X), dev(Y), steps=300, batch=256, lr=2e-3, precision="bf16")
    assert losses[-20:].mean() < 0.5 * losses[:20].mean(), (losses[:20].mean(), losses[-20:].mean())


def test_checkpoint_resume_is_bit_identical(tmp_path):
    torch = torch_cuda()
    D = 32
    rng = np.random.default_rng(1)
    X = dev(rng.standard_normal((512, 10 * D)).astype(np.float32))
    Yn = rng.standard_normal((512, D))
    Y = dev((Yn / np.linalg.norm(Yn, axis=1, keepdims=True)).astype(np.float32))
    c = ctx()
    a = prohd.Mlp(c, D, seed=9)
    for i in range(5):
        a.train_step(X[i * 64:(i + 1) * 64], Y[i * 64:(i + 1) * 64], lr=1e-3)
    path = os.path.join(tmp_path, "net.ckpt")
    a.save(path, rng_state=b"sampler-state")
    for i in range(5, 8):
        a.train_step(X[i * 64:(i + 1) * 64], Y[i * 64:(i + 1) * 64], lr=1e-3)
    b, rs = prohd.Mlp.load(c, path)
    assert rs == b"sampler-state" and b.step == 5
    for i in range(5, 8):
        b.train_step(X[i * 64:(i + 1) * 64], Y[i * 64:(i + 1) * 64], lr=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(a.state, b.state)
    # a truncated file and a foreign one are rejected by prohd_mlp_load
    with open(path, "rb") as f:
        whole = f.read()
    with open(path, "wb") as f:
        f.write(whole[: len(whole) - 4])
    with pytest.raises(ValueError):
        prohd.Mlp.load(c, path)
    with open(path, "wb") as f:
        f.write(b"BADMAGIC" + whole[8:])
    with pytest.raises(ValueError):
        prohd.Mlp.load(c, path)


def test_features_match_oracle():
    torch = torch_cuda()
    A, B = W.anisotropic_pair(6000, 5000, 64, seed=2)
    feat, dirs, eig = ctx().prohd_features(dev(A), dev(B))
    torch.cuda.synchronize()
    f = omlp.features(A, B)
    g = feat.cpu().numpy().astype(np.float64)
    D = 64
    # centroid difference and variances: FP32-shifted sums, FP64 accumulation
    np.testing.assert_allclose(g[:D], f[:D], rtol=0, atol=1e-5 * np.abs(f[:D]).max())
    np.testing.assert_allclose(g[9 * D:], f[9 * D:], rtol=0, atol=1e-5 * np.abs(f[9 * D:]).max())
    # components: well separated (eigenvalues 1/i), compared up to the angle bound
    for l in range(8):
        a = g[(1 + l) * D:(2 + l) * D]
        b = f[(1 + l) * D:(2 + l) * D]
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b), l


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_estimate_with_given_directions(prec):
    torch = torch_cuda()
    A, B = W.mixture_pair(20_000, 64, 8, seed=3)
    rng = np.random.default_rng(4)
    dirs = rng.standard_normal((11, 64))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    kA = [200] + [25] * 10
    kB = [150] + [19] * 10
    c = ctx()
    idxA = torch.empty(A.shape[0], dtype=torch.int32, device="cuda")
    idxB = torch.empty(B.shape[0], dtype=torch.int32, device="cuda")
    out = c.prohd_estimate_dirs(dev(A), dev(B), torch.from_numpy(dirs).cuda(), kA, kB, precision=prec,
                                idxA=idxA, idxB=idxB)
    torch.cuda.synchronize()
    r = prohd.decode_result(out)
    assert r["status"] == "OK"
    ia = oracle.select(A, dirs, kA)
    ib = oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(idxA[: r["nsel_a"]].cpu().numpy(), ia)
    np.testing.assert_array_equal(idxB[: r["nsel_b"]].cpu().numpy(), ib)
    assert rel(r["H"], oracle.hausdorff(A[ia], B[ib])["H"]) <= 1e-5


def test_learned_form_end_to_end_and_gain():
    """Trains on generated pairs (Student-t mixtures, exact-HD witness
    labels), checks that the network learned its objective on the training
    pairs (its directions align with the witness directions better than the
    principal components do), and runs the learned form of ProHD on held-out
    pairs at an equal candidate budget, printing both forms' error against
    the exact HD (the gain is measured, not asserted: Algorithm 3's estimate
    is not monotone in the direction set)."""
    torch = torch_cuda()
    from paper_2511_18207_gb300 import learned
    c = ctx()
    D = 64
    X, Y = learned.make_dataset(c, 256, n_lo=2000, n_hi=4000, D=D, seed=1)
    net = prohd.Mlp(c, D, seed=1)
    losses, _ = learned.train(net, X, Y, steps=400, batch=128, lr=1e-3, precision="bf16")
    assert losses[-20:].mean() < losses[:20].mean()
    u = net.forward(X, precision="bf16")
    torch.cuda.synchronize()
    Xn, Yn, Un = X.double().cpu().numpy(), Y.double().cpu().numpy(), u.double().cpu().numpy()
    pcs = Xn[:, D:9 * D].reshape(-1, 8, D)
    pcs = pcs / np.maximum(np.linalg.norm(pcs, axis=2, keepdims=True), 1e-300)
    al_plain = (np.einsum("bld,bd->bl", pcs, Yn) ** 2).max(axis=1).mean()
    al_learned = (np.einsum("bjd,bd->bj", Un, Yn) ** 2).max(axis=1).mean()
    assert al_learned > al_plain, (al_learned, al_plain)
    ev = learned.evaluate(c, net, 6, n=8000, D=D, seed=77)
    print({k: v for k, v in ev.items() if k != "rows"})
    for r in ev["rows"]:
        assert r["learned"] > 0 and r["plain"] > 0 and r["H"] > 0
