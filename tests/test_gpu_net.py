"""GPU parity of the warm-start network's kernels (csrc/net.cu, through the C
ABI) against the FP64 oracle of oracle/net.py.

Tolerances.  A convolution output is an FP32 tensor-core sum of K = 27 cin
products of BF16 operands (exact in FP32), rounded once to BF16: against the
FP64 sum of the same operands it differs by at most half a BF16 ulp
(2^-9 relative) plus the FP32 summation error, at most K 2^-24 times the sum of
the absolute products (K <= 432 < 2^9): |gpu - ref| <= 2^-8 |ref| + 2^-14 mag
with mag = conv(|x|, |W|) + |b| covers both with margin.  Weight gradients are
FP32 sums of up to 512 products per brick per block plus a fixed-order sum
over at most 304 blocks: |gpu - ref| <= 2^-12 mag with mag the same sum of
absolute products.  The whole network stores 20 BF16 tensors in a chain; a
rounding decision that flips between FP32 and FP64 accumulation changes an
element by one BF16 ulp (2^-8 relative), so the relative L2 differences stay
near 1e-3: the whole-network checks allow 2e-2.
"""
import numpy as np
import pytest
import torch

import oracle.net as O
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import problems as P

pytestmark = pytest.mark.gpu
dev = "cuda:0"


def bf(shape, seed, scale=1.0):
    """Random BF16 tensor (CPU) and its FP64 value."""
    t = (torch.as_tensor(np.random.default_rng(seed).standard_normal(shape)) * scale).to(torch.bfloat16)
    return t, t.to(torch.float64)


def relu_mask(t):
    return (t > 0).to(torch.float64)


@pytest.mark.parametrize("cin,cout", [(8, 8), (8, 16), (16, 8), (16, 16)])
@pytest.mark.parametrize("N,batch", [(5, 1), (12, 3), (16, 2)])
def test_conv_forward_and_adjoint(cin, cout, N, batch):
    seed = 100 * cin + cout + N
    x, x64 = bf((batch, N, N, N, cin), seed)
    W = torch.as_tensor(np.random.default_rng(seed + 1).standard_normal((cout, 27, cin)) * 0.2).float()
    b = torch.as_tensor(np.random.default_rng(seed + 2).standard_normal(cout) * 0.1).float()
    Wq = O.bf16(W.double())
    for relu in (False, True):
        got = B.conv3d_bf16(x.to(dev), W.to(dev), b.to(dev), relu=relu).cpu().double()
        ref = O.conv(x64, Wq, b.double())
        if relu:
            ref = ref.clamp_min(0.0)
        mag = O.conv(x64.abs(), Wq.abs(), b.double().abs())
        err = (got - ref).abs()
        assert bool((err <= 2.0 ** -8 * ref.abs() + 2.0 ** -14 * mag).all()), float(err.max())
    # backward-data with a ReLU mask: input has cout channels, output cin
    g, g64 = bf((batch, N, N, N, cout), seed + 3)
    m, m64 = bf((batch, N, N, N, cout), seed + 4)
    got = B.conv3d_bf16(g.to(dev), W.to(dev), mask=m.to(dev), adjoint=True).cpu().double()
    gz = g64 * relu_mask(m64)
    ref = O.conv_adjoint(gz, Wq, cin)
    mag = O.conv_adjoint(gz.abs(), Wq.abs(), cin)
    err = (got - ref).abs()
    assert bool((err <= 2.0 ** -8 * ref.abs() + 2.0 ** -14 * mag).all()), float(err.max())


@pytest.mark.parametrize("cin,cout", [(8, 8), (8, 16), (16, 8), (16, 16)])
@pytest.mark.parametrize("N,batch", [(5, 1), (12, 3), (24, 1)])
def test_conv_weight_gradient(cin, cout, N, batch):
    seed = 7 * cin + cout + N
    x, x64 = bf((batch, N, N, N, cin), seed)
    g, g64 = bf((batch, N, N, N, cout), seed + 1)
    a, a64 = bf((batch, N, N, N, cout), seed + 2)
    for act in (None, a):
        dw, db = B.conv3d_bf16_wgrad(x.to(dev), g.to(dev), None if act is None else act.to(dev))
        gz = g64 if act is None else g64 * relu_mask(a64)
        rdw, rdb = O.conv_wgrad(x64, gz)
        mdw, mdb = O.conv_wgrad(x64.abs(), gz.abs())
        assert bool(((dw.cpu().double() - rdw).abs() <= 2.0 ** -12 * mdw + 1e-30).all())
        assert bool(((db.cpu().double() - rdb).abs() <= 2.0 ** -12 * mdb + 1e-30).all())


def test_conv_rejects_bad_arguments():
    x = torch.zeros((1, 4, 4, 4, 8), dtype=torch.bfloat16, device=dev)
    W = torch.zeros((8, 27, 12), dtype=torch.float32, device=dev)     # cin 12 unsupported
    with pytest.raises(B.XamgError) as e:
        B.conv3d_bf16(x, W)
    assert e.value.code == B.ERR_INVALID_ARG
    W = torch.zeros((8, 27, 8), dtype=torch.float32, device=dev)
    with pytest.raises(B.XamgError):
        B.conv3d_bf16(x, W, bias=torch.zeros(8, device=dev), adjoint=True)  # no bias on the adjoint


def _net_problem(N, batch, seed=11):
    rng = np.random.default_rng(seed)
    inp = rng.standard_normal((batch, N ** 3, 2)).astype(np.float32)
    tgt = rng.standard_normal((batch, N ** 3)).astype(np.float32)
    p = P.net_init(seed)
    o = 0
    for ci, co, _ in O.LAYERS:
        o += co * 27 * ci
        p[o:o + co] = 0.05 * rng.standard_normal(co)
        o += co
    return inp, tgt, p


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N,batch", [(16, 2), (24, 1)])
def test_network_forward_loss_and_gradient(N, batch):
    inp, tgt, p = _net_problem(N, batch)
    net = B.Net(N, batch)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    di, dt = torch.as_tensor(inp).to(dev), torch.as_tensor(tgt).to(dev)
    out = torch.empty((batch, N ** 3), dtype=torch.float32, device=dev)
    net.forward(di, out)
    onet = O.Net(p.astype(np.float64), emulate=True)
    L_ref, dW_ref = onet.grads(inp, tgt, N)
    y_ref = onet.a["y"][..., 0].reshape(batch, -1).numpy()
    assert rel(out.cpu().numpy(), y_ref) < 2e-2
    L, g = net.loss_grad(di, dt)
    assert abs(L - L_ref) <= 2e-2 * L_ref
    gl = O.unflatten(g)
    for l, ((dW, db), (rW, rb)) in enumerate(zip(gl, dW_ref)):
        assert rel(dW.numpy(), rW.numpy()) < 2e-2, (l, rel(dW.numpy(), rW.numpy()))
        assert rel(db.numpy(), rb.numpy()) < 2e-2, (l, rel(db.numpy(), rb.numpy()))
    # unused weights get exactly zero gradient; repeated calls are bitwise equal
    assert float(gl[0][0][:, :, 2:].abs().max()) == 0.0 and float(gl[-1][0][1:].abs().max()) == 0.0
    L2, g2 = net.loss_grad(di, dt)
    assert L2 == L and np.array_equal(g2, g)


def test_train_step_is_adam_on_the_gradient_and_reduces_the_loss():
    N, batch = 16, 4
    inp, tgt, p = _net_problem(N, batch, seed=5)
    net = B.Net(N, batch)
    net.set_params(p)
    di, dt = torch.as_tensor(inp).to(dev), torch.as_tensor(tgt).to(dev)
    L0, g = net.loss_grad(di, dt)
    idx = torch.arange(batch, dtype=torch.int32, device=dev)
    lr, eps = 1e-3, 1e-8
    Ls = net.train_step(di, dt, idx, lr=lr, eps=eps)
    assert Ls == L0
    # first Adam step: w - lr g / (|g| + eps) (bias-corrected moments m = g, v = g^2)
    want = p - lr * g / (np.abs(g) + eps)
    assert np.allclose(net.get_params(), want, rtol=1e-5, atol=1e-7)
    losses = [net.train_step(di, dt, idx, lr=lr) for _ in range(30)]
    assert losses[-1] < 0.9 * L0
    # the index batch selects (and orders) the samples
    idx2 = torch.tensor([3, 1], dtype=torch.int32, device=dev)
    net2 = B.Net(N, 2)
    net2.set_params(p)
    la = net2.train_step(di, dt, idx2, lr=lr)
    net3 = B.Net(N, 2)
    net3.set_params(p)
    lc, _ = net3.loss_grad(di[[3, 1]].contiguous(), dt[[3, 1]].contiguous())
    assert la == lc


def test_predict_x0_normalises_columns():
    N, m = 16, 4
    n = N ** 3
    _, _, p = _net_problem(N, m)
    net = B.Net(N, m)
    net.set_params(p)
    rng = np.random.default_rng(2)
    Bh = rng.standard_normal((n, m)) * np.array([1.0, 3e-3, 0.0, 250.0])
    logk = rng.standard_normal(n).astype(np.float32)
    X0 = torch.empty((n, m), dtype=torch.float64, device=dev)
    scale = 0.37
    net.predict_x0(torch.as_tensor(Bh).to(dev), torch.as_tensor(logk).to(dev), X0, scale)
    torch.cuda.synchronize()
    X0 = X0.cpu().numpy()
    assert np.all(X0[:, 2] == 0.0)
    s = np.sqrt((Bh ** 2).mean(axis=0))
    for j in (0, 1, 3):
        inp = np.stack([Bh[:, j] / s[j], logk], axis=1)[None].astype(np.float32)
        y = O.Net(p.astype(np.float64), emulate=True).forward(inp, N).numpy()[0]
        assert rel(X0[:, j], y * s[j] * scale) < 2e-2
    # scale invariance: X0 of 2^k B is 2^k X0 (the normalisation divides it out)
    X1 = torch.empty((n, m), dtype=torch.float64, device=dev)
    net.predict_x0(torch.as_tensor(Bh * 8.0).to(dev), torch.as_tensor(logk).to(dev), X1, scale)
    torch.cuda.synchronize()
    assert np.array_equal(X1.cpu().numpy(), 8.0 * X0)


@pytest.mark.parametrize("kind", ["mse", "energy"])
def test_weighted_losses(kind):
    N, batch = 16, 2
    inp, tgt, p = _net_problem(N, batch, seed=3)
    w = np.array([0.5, 2.0], np.float32)
    net = B.Net(N, batch)
    net.set_params(p)
    di, dt = torch.as_tensor(inp).to(dev), torch.as_tensor(tgt).to(dev)
    code = B.LOSS_ENERGY if kind == "energy" else B.LOSS_MSE
    L, g = net.loss_grad(di, dt, loss=code, weight=torch.as_tensor(w).to(dev))
    L_ref, dW_ref = O.Net(p.astype(np.float64), emulate=True).grads(inp, tgt, N, kind, w)
    assert abs(L - L_ref) <= 2e-2 * L_ref
    for l, ((dW, db), (rW, rb)) in enumerate(zip(O.unflatten(g), dW_ref)):
        assert rel(dW.numpy(), rW.numpy()) < 2e-2, (l, rel(dW.numpy(), rW.numpy()))
        assert rel(db.numpy(), rb.numpy()) < 2e-2, (l, rel(db.numpy(), rb.numpy()))
    # a training step uses the weight of each selected sample row
    idx = torch.tensor([1, 0], dtype=torch.int32, device=dev)
    wt = torch.as_tensor(w).to(dev)
    la = net.train_step(di, dt, idx, lr=1e-3, loss=code, weight=wt)
    net2 = B.Net(N, batch)
    net2.set_params(p)
    lb, _ = net2.loss_grad(di[[1, 0]].contiguous(), dt[[1, 0]].contiguous(), loss=code,
                           weight=wt[[1, 0]].contiguous())
    assert la == lb
