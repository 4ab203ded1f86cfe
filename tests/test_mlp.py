"""GPU parity of the surrogate's tensor-core kernels against the fp64 CPU reference:
forward outputs and backpropagated gradients within bf16 tolerance, and AdamW training
that lowers the loss."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def ref_forward_bf16(theta, q):
    """fp64 forward with the bf16 rounding the kernels apply: bf16 weights, bf16 inputs
    to every layer, fp32-exact accumulation (kept in fp64 here)."""
    layers = omlp.unpack(theta)
    a = bf16_round(omlp.features(q))
    for li, (W, b) in enumerate(layers):
        z = a @ bf16_round(W).T + b
        if li < len(layers) - 1:
            a = bf16_round(np.maximum(z, 0.0))
        else:
            a = z
    return a


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _net(v, cap, theta):
    net = v.MLP(cap)
    net.set_params(theta.astype(np.float32))
    return net


@pytest.mark.parametrize("B", [128, 300, 1000])
def test_forward_matches_reference(B):
    v = lib()
    rng = np.random.default_rng(B)
    theta = omlp.init_params(7) + rng.normal(scale=0.02, size=omlp.n_params())
    theta = theta.astype(np.float32).astype(np.float64)
    q = rng.uniform(-np.pi, np.pi, size=(B, 7))
    net = _net(v, 1024, theta)
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    out = torch.zeros((B, 24), dtype=torch.float32, device="cuda")
    net.forward(qd, out)
    net.check()
    got = out.cpu().numpy().astype(np.float64)
    ref = ref_forward_bf16(theta, q.astype(np.float32).astype(np.float64))
    assert rel(got, ref) < 1e-2, rel(got, ref)
    ref64, _ = omlp.forward(theta, q)
    assert rel(got, ref64) < 5e-2
    net.close()


def test_gradients_match_reference():
    v = lib()
    B = 512
    rng = np.random.default_rng(1)
    theta = (omlp.init_params(3) + rng.normal(scale=0.02, size=omlp.n_params())).astype(np.float32).astype(np.float64)
    q = rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32).astype(np.float64)
    y = rng.uniform(0.0, 1.0, size=(B, 24)).astype(np.float32).astype(np.float64)
    mask = (rng.random((B, 24)) < 0.85).astype(np.float64)
    net = _net(v, B, theta)
    loss, g = net.grads(torch.from_numpy(q.astype(np.float32)).cuda(), torch.from_numpy(y.astype(np.float32)).cuda(),
                        torch.from_numpy(mask.astype(np.float32)).cuda())
    net.check()
    # reference: fp64 backprop on bf16-rounded weights (the kernels' operands)
    layers = omlp.unpack(theta)
    theta_r = np.concatenate([np.concatenate([bf16_round(W).ravel(), b]) for W, b in layers])
    lref, gref = omlp.loss_and_grad(theta_r, q, y, mask)
    assert abs(loss - lref) <= 2e-2 * lref
    p = 0
    for (i, o) in zip(omlp.SIZES[:-1], omlp.SIZES[1:]):
        gw, gb = g[p:p + o * i], g[p + o * i:p + o * i + o]
        rw, rb = gref[p:p + o * i], gref[p + o * i:p + o * i + o]
        assert rel(gw, rw) < 5e-2, (i, o, rel(gw, rw))
        assert rel(gb, rb) < 5e-2, (i, o, rel(gb, rb))
        p += o * i + o
    net.close()


def test_training_reduces_loss():
    v = lib()
    B = 2048
    rng = np.random.default_rng(5)
    net = _net(v, B, omlp.init_params(11))
    q = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)).cuda()
    # a smooth synthetic target in the range of sphere distances (metres)
    W = torch.from_numpy(rng.normal(size=(7, 24)).astype(np.float32)).cuda()
    y = 0.3 + 0.1 * torch.sin(q @ W)
    sums = torch.zeros(2, device="cuda")
    losses = []
    for it in range(300):
        net.train_step(q, y, None, lr=2e-3, wd=1e-4, loss_sums_dev=sums)
        if it % 50 == 0 or it == 299:
            s = sums.cpu().numpy()
            losses.append(s[0] / s[1])
    net.check()
    assert losses[-1] < 0.2 * losses[0], losses
    net.close()


@pytest.mark.parametrize("B", [128, 777, 65536])
def test_fused_forward_matches_layer_path(B):
    """The fused one-kernel forward and the per-layer GEMM forward round at the same
    points (bf16 features and activations); only fp32 accumulation order may differ."""
    v = lib()
    rng = np.random.default_rng(B + 1)
    theta = omlp.init_params(9) + rng.normal(scale=0.02, size=omlp.n_params())
    net = _net(v, B, theta)
    q = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)).cuda()
    a = torch.zeros((B, 24), device="cuda")
    b = torch.zeros((B, 24), device="cuda")
    net.forward(q, a)
    net.forward_layers(q, b)
    net.check()
    an, bn = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    assert rel(an, bn) < 2e-3, rel(an, bn)
    ref = ref_forward_bf16(theta.astype(np.float32).astype(np.float64), q.cpu().numpy().astype(np.float64))
    assert rel(an, ref) < 1e-2
    net.close()


@pytest.mark.parametrize("B", [1, 129, 300, 40000, 65536 + 77])
def test_fused_forward_ragged_batches(B):
    """Batches that leave a partial last tile, an odd number of tiles per CTA or fewer
    tiles than SMs: outputs match the per-layer path and rows past B stay untouched."""
    v = lib()
    rng = np.random.default_rng(100 + B)
    theta = omlp.init_params(4) + rng.normal(scale=0.02, size=omlp.n_params())
    net = _net(v, B, theta)
    q = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)).cuda()
    got = torch.full((B + 1, 24), 7.0, device="cuda")
    net.forward(q, got)
    net.check()
    assert bool((got[B] == 7.0).all())
    lay = torch.zeros((B, 24), device="cuda")
    net.forward_layers(q, lay)
    assert rel(got[:B].cpu().numpy().astype(np.float64), lay.cpu().numpy().astype(np.float64)) < 2e-3
    again = torch.zeros((B, 24), device="cuda")
    net.forward(q, again)
    assert torch.equal(again, got[:B])      # deterministic
    net.close()


def test_fused_forward_follows_training_updates():
    """After AdamW steps change the parameters on the device, the fused forward uses the
    new weights and biases (it agrees with the per-layer path that reads them directly)."""
    v = lib()
    B = 4096
    rng = np.random.default_rng(21)
    net = _net(v, B, omlp.init_params(12))
    q = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.uniform(0.1, 0.5, size=(B, 24)).astype(np.float32)).cuda()
    before = torch.zeros((B, 24), device="cuda")
    net.forward(q, before)
    for _ in range(20):
        net.train_step(q, y, None, lr=1e-2, wd=0.0)
    got = torch.zeros((B, 24), device="cuda")
    lay = torch.zeros((B, 24), device="cuda")
    net.forward(q, got)
    net.forward_layers(q, lay)
    net.check()
    assert not torch.equal(got, before)
    assert rel(got.cpu().numpy().astype(np.float64), lay.cpu().numpy().astype(np.float64)) < 2e-3
    net.close()


def test_checkpoint_round_trip_and_resume(tmp_path):
    """save() / load() carry the parameters, both AdamW moments and the step exactly; a
    network resumed from the file continues like the one that wrote it (the dW
    reductions use fp32 atomics, so the match is close, not bitwise)."""
    v = lib()
    B = 1024
    rng = np.random.default_rng(8)
    q = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)).cuda()
    W = torch.from_numpy(rng.normal(size=(7, 24)).astype(np.float32)).cuda()
    y = 0.3 + 0.1 * torch.sin(q @ W)
    a = _net(v, B, omlp.init_params(3))
    for _ in range(20):
        a.train_step(q, y, None, lr=2e-3, wd=1e-4)
    a.check()
    path = str(tmp_path / "mlp_state.npz")
    a.save(path)
    b = v.MLP(B)
    b.load(path)
    pa, m1a, m2a, sa = a.get_state()
    pb, m1b, m2b, sb = b.get_state()
    assert sa == sb == 20
    assert np.array_equal(pa, pb) and np.array_equal(m1a, m1b) and np.array_equal(m2a, m2b)
    assert np.abs(m1a).max() > 0 and np.abs(m2a).max() > 0
    for net in (a, b):
        for _ in range(10):
            net.train_step(q, y, None, lr=2e-3, wd=1e-4)
        net.check()
    pa, _, _, sa = a.get_state()
    pb, _, _, sb = b.get_state()
    assert sa == sb == 30
    # parameters whose gradient sums nearly cancel may take differently rounded AdamW
    # steps; the bulk agrees to fp32 rounding and the loss is the same
    assert float(np.quantile(np.abs(pa - pb), 0.999)) <= 1e-5
    la, _ = a.grads(q, y)
    lb, _ = b.grads(q, y)
    assert abs(la - lb) <= 1e-3 * la
    # a fresh network that only got the parameters restarts AdamW (step 0, zero moments)
    c = v.MLP(B)
    c.set_params(pa)
    _, m1c, m2c, sc = c.get_state()
    assert sc == 0 and not m1c.any() and not m2c.any()
    with pytest.raises(v.VedtError):
        c.set_state(pa, m1a, m2a, -1)
    for net in (a, b, c):
        net.close()
