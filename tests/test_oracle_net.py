"""Pins of the warm-start network's oracle (oracle/net.py) against the
definitions it restates: brute-force convolution sums, adjoint identities of
the convolution, pooling and upsampling, and central finite differences of
the whole FP64 network for the hand-written backward pass."""
import numpy as np
import pytest
import torch

import oracle.net as O
from paper_2103_07329_gb300 import problems as P

f64 = torch.float64


def rnd(shape, seed):
    return torch.as_tensor(np.random.default_rng(seed).standard_normal(shape))


def test_param_layout():
    assert O.param_count() == 62376
    assert [(ci, co) for ci, co, _ in O.LAYERS] == P.NET_LAYERS
    p = P.net_init(0)
    assert p.size == O.param_count() and p.dtype == np.float32
    layers = O.unflatten(p)
    assert float(layers[0][0][:, :, 2:].abs().max()) == 0.0      # unused input channels
    assert float(layers[-1][0][1:].abs().max()) == 0.0           # unused outputs
    assert all(float(b.abs().max()) == 0.0 for _, b in layers)


def test_conv_is_the_defining_sum():
    # out[v][co] = b[co] + sum_{t,ci} W[co][t][ci] x[v + off_t][ci], t = 9(dz+1)+3(dy+1)+(dx+1)
    N, ci, co = 3, 2, 3
    x = rnd((1, N, N, N, ci), 1)
    W = rnd((co, 27, ci), 2)
    b = rnd((co,), 3)
    ref = np.zeros((N, N, N, co))
    for z in range(N):
        for y in range(N):
            for xx in range(N):
                for c in range(co):
                    s = float(b[c])
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                zz, yy, x2 = z + dz, y + dy, xx + dx
                                if not (0 <= zz < N and 0 <= yy < N and 0 <= x2 < N):
                                    continue
                                t = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
                                for k in range(ci):
                                    s += float(W[c, t, k]) * float(x[0, zz, yy, x2, k])
                    ref[z, y, xx, c] = s
    got = O.conv(x, W, b)[0].numpy()
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_conv_adjoint_and_weight_gradient_identities():
    N, ci, co = 5, 8, 16
    x = rnd((2, N, N, N, ci), 4)
    W = rnd((co, 27, ci), 5)
    g = rnd((2, N, N, N, co), 6)
    lhs = float((O.conv(x, W) * g).sum())
    # <conv(x, W), g> = <x, conv_adjoint(g, W)>
    rhs = float((x * O.conv_adjoint(g, W, ci)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-10
    # the product is linear in W: <conv(x, W), g> = sum W * dW(x, g); db = sum of g
    dW, db = O.conv_wgrad(x, g)
    assert abs(lhs - float((W * dW).sum())) <= 1e-12 * abs(lhs) + 1e-10
    assert torch.allclose(db, g.sum(dim=(0, 1, 2, 3)), rtol=1e-14, atol=1e-12)
    # one entry by hand: tap (dz, dy, dx) = (1, 0, -1), channels (3, 5)
    t = 9 * 2 + 3 * 1 + 0
    s = 0.0
    for b_ in range(2):
        for z in range(N - 1):
            for y in range(N):
                for xx in range(1, N):
                    s += float(g[b_, z, y, xx, 3]) * float(x[b_, z + 1, y, xx - 1, 5])
    assert abs(float(dW[3, t, 5]) - s) <= 1e-12 * (1 + abs(s))


def test_pool_and_up_adjoints():
    x = rnd((2, 4, 4, 4, 8), 7)
    y = rnd((2, 2, 2, 2, 8), 8)
    assert abs(float((O.pool(x) * y).sum()) - float((x * O.up(y)).sum()) / 8) < 1e-12
    assert abs(float((O.up(y) * x).sum()) - float((y * O.up_adjoint(x)).sum())) < 1e-12
    # pooling averages the 2x2x2 children
    assert abs(float(O.pool(x)[1, 1, 0, 1, 3]) - float(x[1, 2:4, 0:2, 2:4, 3].mean())) < 1e-14


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    v = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9], dtype=f64)
    assert O.bf16(v).tolist() == [1.0, 1.0 + 2.0 ** -6, 1.0]


def _problem(N=8, batch=2, seed=11):
    rng = np.random.default_rng(seed)
    inp = rng.standard_normal((batch, N ** 3, 2))
    tgt = rng.standard_normal((batch, N ** 3))
    p = P.net_init(seed).astype(np.float64)
    # nonzero biases so that every term of the backward pass is exercised
    o = 0
    for ci, co, _ in O.LAYERS:
        o += co * 27 * ci
        p[o:o + co] = 0.05 * rng.standard_normal(co)
        o += co
    return inp, tgt, p


@pytest.mark.parametrize("kind", ["mse", "energy"])
def test_network_gradient_matches_finite_differences(kind):
    N = 8
    inp, tgt, p = _problem(N)
    net = O.Net(p, emulate=False)
    L0, dW = net.grads(inp, tgt, N, kind)
    g = O.flatten(dW)
    rng = np.random.default_rng(3)
    # entries from every layer's weights (used channels) and biases
    idx = []
    o = 0
    for l, (ci, co, _) in enumerate(O.LAYERS):
        ci_u = 2 if l == 0 else ci
        co_u = 1 if l == len(O.LAYERS) - 1 else co
        for _ in range(2):
            idx.append(o + (rng.integers(co_u) * 27 + rng.integers(27)) * ci + rng.integers(ci_u))
        o += co * 27 * ci
        idx.append(o + rng.integers(co_u))
        o += co
    h = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        Lp = O.Net(pp, emulate=False).loss(inp, tgt, N, kind)[0]
        Lm = O.Net(pm, emulate=False).loss(inp, tgt, N, kind)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, fd, g[i])
    # unused weights receive exactly zero gradient
    layers = O.unflatten(g)
    assert float(layers[0][0][:, :, 2:].abs().max()) == 0.0
    assert float(layers[-1][0][1:].abs().max()) == 0.0
    assert float(layers[-1][1][1:].abs().max()) == 0.0


def test_emulated_values_are_bf16():
    N = 8
    inp, tgt, p = _problem(N, batch=1)
    net = O.Net(p, emulate=True)
    L, dW = net.grads(inp, tgt, N)
    for k in ("x", "s0", "p1", "u2", "d0a"):
        a = net.a[k]
        assert torch.equal(a, O.bf16(a))
    # emulation changes values by BF16 rounding only: the FP64 loss is close
    L64 = O.Net(p, emulate=False).loss(inp, tgt, N)[0]
    assert not torch.equal(net.a["y"], O.bf16(net.a["y"]))   # the output is not rounded
    assert abs(L - L64) <= 2e-2 * L64


def test_energy_operator_is_the_diffusion_matrix():
    # the loss's stencil equals the matrix problems.diffusion7 assembles
    N = 8
    rng = np.random.default_rng(4)
    logk = rng.standard_normal(N ** 3)
    e = rng.standard_normal(N ** 3)
    A = P.diffusion7(N, np.exp(logk))
    import scipy.sparse as sp
    Ae = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)) @ e
    got = O.energy_apply(torch.as_tensor(e), torch.as_tensor(logk), N).numpy()
    assert np.allclose(got, Ae, rtol=1e-13, atol=1e-12)
    # e^T A e > 0 and the loss of the exact target is zero
    inp = np.stack([rng.standard_normal(N ** 3), logk], axis=1)[None]
    net = O.Net(np.zeros(O.param_count()), emulate=False)
    L, y, t, gy = net.loss(inp, np.zeros((1, N ** 3)), N, "energy")
    assert L == 0.0 and float(gy.abs().max()) == 0.0
    assert float(e @ Ae) > 0


def test_sample_weights_scale_each_sample():
    N = 8
    inp, tgt, p = _problem(N)
    net = O.Net(p, emulate=False)
    for kind in ("mse", "energy"):
        L1 = net.loss(inp, tgt, N, kind, weight=[1.0, 0.0])[0]
        L2 = net.loss(inp, tgt, N, kind, weight=[0.0, 1.0])[0]
        L = net.loss(inp, tgt, N, kind)[0]
        assert abs(L1 + L2 - L) <= 1e-12 * L
        L3 = net.loss(inp, tgt, N, kind, weight=[2.0, 0.5])[0]
        assert abs(L3 - (2 * L1 + 0.5 * L2)) <= 1e-12 * L3
