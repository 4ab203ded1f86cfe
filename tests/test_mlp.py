"""GPU parity of the surrogate's tensor-core kernels against the fp64 CPU reference,
element by element (tests/mlp_bounds.py): bit-exact outputs, loss and gradients on
exact-grid networks, magnitude-scaled bounds on realistic ones; AdamW training that lowers
the loss; the fused forward against the per-layer path; checkpoints."""
import numpy as np
import pytest
import torch

import mlp_bounds as mb
from oracle import mlp as omlp
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _net(v, cap, theta):
    net = v.MLP(cap)
    net.set_params(np.asarray(theta, np.float32))
    return net


def _run_forward(v, theta, q, fused):
    B = q.shape[0]
    net = _net(v, B, theta)
    qd = torch.from_numpy(np.asarray(q, np.float32)).cuda()
    out = torch.zeros((B, 24), dtype=torch.float32, device="cuda")
    (net.forward if fused else net.forward_layers)(qd, out)
    net.check()
    net.close()
    return out.cpu().numpy()


def _run_grads(v, theta, q, y, mask):
    B = q.shape[0]
    net = _net(v, B, theta)
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    loss, g = net.grads(t(q), t(y), t(mask))
    net.check()
    net.close()
    return loss, g


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("B", [128, 300, 1000, 65536])
def test_forward_exact_grid_bitexact(B, fused):
    """On an exact-grid network every fp32 sum is exact in any order, so each of the B x 24
    outputs of the fused and of the per-layer forward equals the fp64 reference with the
    same bf16 rounding points bit for bit."""
    v = lib()
    th = mb.exact_network(B)
    q = mb.exact_inputs(B + 1, B)
    r = mb.reference(th, q)
    assert mb.exact_margin_forward(r) < 2.0 ** 23
    got = _run_forward(v, th, q, fused)
    bad = np.argwhere(got.astype(np.float64) != r["out"])
    assert bad.size == 0, (len(bad), bad[:5])


@pytest.mark.parametrize("B", [300, 512, 2048])
def test_gradients_exact_grid_bitexact(B):
    """Exact-grid network and targets: the loss and every dW / db entry of all five layers
    equal the fp64 backpropagation with the kernels' rounding points bit for bit (2048
    rows take two split-K chunks of 1024 added atomically)."""
    v = lib()
    th = mb.exact_network(B)
    q = mb.exact_inputs(B + 1, B)
    r = mb.reference(th, q)
    y, mask = mb.exact_targets(B + 2, r["out"])
    r = mb.reference(th, q, y, mask)
    assert mb.exact_margin_backward(r, mask.sum()) < 2.0 ** 23.5
    loss, g = _run_grads(v, th, q, y, mask)
    assert np.float32(loss) == np.float32(r["loss"])
    bad = np.flatnonzero(g.astype(np.float64) != r["flat"])
    assert bad.size == 0, (len(bad), bad[:5], g[bad[:5]], r["flat"][bad[:5]])


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("B", [128, 300, 1000, 65536])
def test_forward_realistic_elementwise(B, fused):
    """He-initialised network, uniform joint angles: every output within 2^-7 of its own
    dot product's magnitude sum of the same-rounding fp64 reference (mlp_bounds)."""
    v = lib()
    th, q, _, _ = mb.realistic_case(B, B)
    r = mb.reference(th, q)
    S = mb.magnitudes(r)
    got = _run_forward(v, th, q, fused)
    ok = mb.within(got, r["out"], S["out"], mb.TOL_FWD)
    assert ok.all(), (int((~ok).sum()), np.argwhere(~ok)[:5])
    # and close to the unrounded fp64 network (bf16 operands only)
    ref64, _ = omlp.forward(th.astype(np.float64), q.astype(np.float64))
    assert np.abs(got - ref64).max() <= 0.05 * np.abs(ref64).max()


@pytest.mark.parametrize("B", [512, 4096])
def test_gradients_realistic_elementwise(B):
    """Every dW / db entry checked against the same-rounding fp64 backpropagation: at
    least 99.9 % within 2^-7 of the entry's propagated magnitude sum and all within 2^-2
    (a ReLU whose pre-activation rounds to zero on one side switches a whole term); the
    loss within 2^-10."""
    v = lib()
    th, q, y, mask = mb.realistic_case(B + 3, B)
    r = mb.reference(th, q, y, mask)
    S = mb.magnitudes(r)
    loss, g = _run_grads(v, th, q, y, mask)
    frac, all_ok = mb.grads_ok(g, r, S)
    assert frac >= mb.GRAD_QUANTILE and all_ok, (frac, all_ok)
    assert abs(loss - r["loss"]) <= 2.0 ** -10 * r["loss"]


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


@pytest.mark.parametrize("B", [1, 129, 300, 40000, 65536 + 77])
def test_fused_forward_ragged_batches_exact(B):
    """Batches that leave a partial last tile, an odd number of tiles per CTA or fewer
    tiles than SMs, on exact-grid networks: both forwards bit-exact against the reference,
    rows past B untouched, repeated calls identical."""
    v = lib()
    th = mb.exact_network(100 + B)
    q = mb.exact_inputs(200 + B, B)
    r = mb.reference(th, q)
    net = _net(v, B, th)
    qd = torch.from_numpy(q).cuda()
    got = torch.full((B + 1, 24), 7.0, device="cuda")
    net.forward(qd, got)
    net.check()
    assert bool((got[B] == 7.0).all())
    assert np.array_equal(got[:B].cpu().numpy().astype(np.float64), r["out"])
    lay = torch.zeros((B, 24), device="cuda")
    net.forward_layers(qd, lay)
    assert np.array_equal(lay.cpu().numpy().astype(np.float64), r["out"])
    again = torch.zeros((B, 24), device="cuda")
    net.forward(qd, again)
    assert torch.equal(again, got[:B])      # deterministic
    net.close()


def test_fused_forward_follows_training_updates():
    """After AdamW steps change the parameters on the device, the fused forward uses the
    new weights and biases: it agrees element-wise with the per-layer path, which reads
    them directly (both within 2^-7 of the magnitude sums at the trained parameters)."""
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
    S = mb.magnitudes(mb.reference(net.get_params(), q.cpu().numpy()))["out"]
    g, l = got.cpu().numpy().astype(np.float64), lay.cpu().numpy().astype(np.float64)
    assert mb.within(g, l, S, 2 * mb.TOL_FWD).all()
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
