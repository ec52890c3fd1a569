"""Plain PyTorch-CPU (FP64) oracle of the warm-start network.

TEST INFRASTRUCTURE ONLY: the test-suite uses it to check the CUDA library's
network kernels; the library never imports it.

The network is the 3-D convolutional encoder-decoder that predicts the first
iterate X0 of the Krylov solve (the paper has no learned component; this is
the warm-started form the solver is measured with).  Layers, all 3x3x3
convolutions with zero padding, ReLU after all but the last:

  level 0 (edge N):   e0a 8->8, e0b 8->8            -> s0
  level 1 (N/2):      pool(s0), e1a 8->16, e1b 16->16 -> s1
  level 2 (N/4):      pool(s1), e2a, e2b 16->16      -> s2
  level 3 (N/8):      pool(s2), e3a, e3b 16->16
  level 2:            up(e3b) + s2, d2 16->16
  level 1:            up(d2) + s1, d1a 16->16, d1b 16->8
  level 0:            up(d1b) + s0, d0a 8->8, d0b 8->8 (linear); output = channel 0

pool = 2x2x2 average, up = nearest-neighbour upsampling by 2.  Tensors are
channels-last [batch, N, N, N, C] (z, y, x); weights W[cout][27][cin] with tap
t = 9 (dz+1) + 3 (dy+1) + (dx+1) of a cross-correlation
out[v][co] = b[co] + sum_{t,ci} W[co][t][ci] in[v + off_t][ci].

Every step is a library primitive (torch.nn.functional.conv3d, avg_pool3d and
the gradient routines torch.nn.grad.conv3d_input / conv3d_weight) or a plain
tensor expression, evaluated in FP64.  With ``emulate=True`` the values the
CUDA kernels store in BF16 (activations, activation gradients, weights as
tensor-core operands, the packed input) are rounded to BF16 at the same
points; everything else stays FP64.  The network output (channel 0 of the
last layer) is kept unrounded, as the kernels store it in FP32.  The backward
pass is written out layer by layer in reverse order (no autograd), so tests
can pin it against finite differences of the FP64 forward pass.

Two losses, for e_b = y_b - t_b and sample weights w_b:
  "mse":    sum_b w_b |e_b|^2 / (batch N^3)
  "energy": sum_b w_b e_b^T A_b e_b / batch, A_b the cell-centred diffusion
            operator of unit cells with log coefficient = input channel 1:
            (A e)_c = sum over the six faces of T_f (e_c - e_nb), T_f =
            2 k_c k_nb / (k_c + k_nb), and T_f e_c with T_f = 2 k_c on a
            boundary face.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (cin, cout, relu) per layer, in the order of the flat parameter vector
LAYERS = [(8, 8, 1), (8, 8, 1), (8, 16, 1), (16, 16, 1), (16, 16, 1), (16, 16, 1), (16, 16, 1),
          (16, 16, 1), (16, 16, 1), (16, 16, 1), (16, 8, 1), (8, 8, 1), (8, 8, 0)]
NAMES = ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "d2", "d1a", "d1b", "d0a", "d0b"]

f64 = torch.float64


def param_count() -> int:
    return sum(co * 27 * ci + co for ci, co, _ in LAYERS)


def unflatten(p):
    """Flat parameter vector -> list of (W [cout, 27, cin], b [cout]) FP64 tensors."""
    p = torch.as_tensor(np.asarray(p, dtype=np.float64))
    out, o = [], 0
    for ci, co, _ in LAYERS:
        W = p[o:o + co * 27 * ci].reshape(co, 27, ci)
        o += co * 27 * ci
        b = p[o:o + co]
        o += co
        out.append((W, b))
    assert o == p.numel()
    return out


def flatten(grads) -> np.ndarray:
    return np.concatenate([torch.cat([dW.reshape(-1), db.reshape(-1)]).numpy() for dW, db in grads])


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned in FP64."""
    return x.to(torch.bfloat16).to(f64)


def _w5(W):
    """[cout, 27, cin] -> conv3d weight [cout, cin, 3, 3, 3] (kz, ky, kx)."""
    co, _, ci = W.shape
    return W.permute(0, 2, 1).reshape(co, ci, 3, 3, 3)


def _cf(x):  # channels-last -> channels-first
    return x.permute(0, 4, 1, 2, 3)


def _cl(x):  # channels-first -> channels-last
    return x.permute(0, 2, 3, 4, 1).contiguous()


def conv(x, W, b=None):
    """out[v][co] = b[co] + sum_{t,ci} W[co][t][ci] x[v + off_t][ci], zero outside the grid."""
    return _cl(F.conv3d(_cf(x), _w5(W), b, padding=1))


def conv_adjoint(g, W, cin):
    """gin[v][ci] = sum_{t,co} W[co][t][ci] g[v - off_t][co]: the gradient of
    <conv(x, W), g> with respect to x."""
    B, N = g.shape[0], g.shape[1]
    return _cl(torch.nn.grad.conv3d_input((B, cin, N, N, N), _w5(W), _cf(g), padding=1))


def conv_wgrad(x, g):
    """(dW[co][t][ci] = sum_v g[v][co] x[v + off_t][ci], db[co] = sum_v g[v][co])."""
    ci, co = x.shape[-1], g.shape[-1]
    d5 = torch.nn.grad.conv3d_weight(_cf(x), (co, ci, 3, 3, 3), _cf(g), padding=1)
    return d5.reshape(co, ci, 27).permute(0, 2, 1).contiguous(), g.sum(dim=(0, 1, 2, 3))


def pool(x):
    return _cl(F.avg_pool3d(_cf(x), 2))


def up(x):
    return x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def up_adjoint(g):
    """Sum of the 8 children: the gradient of <up(x), g> with respect to x."""
    B, N, _, _, C = g.shape
    return g.reshape(B, N // 2, 2, N // 2, 2, N // 2, 2, C).sum(dim=(2, 4, 6))


def pack_input(inp, N):
    """[batch, N^3, 2] pairs -> channels-last [batch, N, N, N, 8] (channels 2..7 zero)."""
    inp = torch.as_tensor(np.asarray(inp, dtype=np.float64))
    B = inp.shape[0]
    x = torch.zeros(B, N, N, N, 8, dtype=f64)
    x[..., :2] = inp.reshape(B, N, N, N, 2)
    return x


def energy_apply(e, logk, N):
    """(A e) for one sample: e, logk flat [N^3] (x fastest), A as above."""
    e = e.reshape(N, N, N)
    k = torch.exp(logk.reshape(N, N, N))
    out = torch.zeros_like(e)
    for ax in range(3):
        # interior faces between cells i and i+1 along axis ax
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, N - 1)
        hi[ax] = slice(1, N)
        lo, hi = tuple(lo), tuple(hi)
        T = 2.0 * k[lo] * k[hi] / (k[lo] + k[hi])
        flux = T * (e[lo] - e[hi])
        out[lo] += flux
        out[hi] -= flux
        # the two boundary faces
        for end in (0, N - 1):
            sl = [slice(None)] * 3
            sl[ax] = slice(end, end + 1)
            sl = tuple(sl)
            out[sl] += 2.0 * k[sl] * e[sl]
    return out.reshape(-1)


class Net:
    """Forward and backward passes of the network for one parameter vector."""

    def __init__(self, params, emulate: bool = True):
        self.emulate = emulate
        self.layers = unflatten(params)
        R = bf16 if emulate else (lambda t: t)
        self.R = R
        self.Wq = [R(W) for W, _ in self.layers]  # tensor-core operands

    def _conv(self, l, x, store=True):
        _, b = self.layers[l]
        y = conv(x, self.Wq[l], b)
        if LAYERS[l][2]:
            y = torch.clamp_min(y, 0.0)
        return self.R(y) if store else y

    def forward(self, inp, N):
        R = self.R
        a = {}
        a["x"] = R(pack_input(inp, N))
        a["e0a"] = self._conv(0, a["x"])
        a["s0"] = self._conv(1, a["e0a"])
        a["p0"] = R(pool(a["s0"]))
        a["e1a"] = self._conv(2, a["p0"])
        a["s1"] = self._conv(3, a["e1a"])
        a["p1"] = R(pool(a["s1"]))
        a["e2a"] = self._conv(4, a["p1"])
        a["s2"] = self._conv(5, a["e2a"])
        a["p2"] = R(pool(a["s2"]))
        a["e3a"] = self._conv(6, a["p2"])
        a["e3b"] = self._conv(7, a["e3a"])
        a["u2"] = R(up(a["e3b"]) + a["s2"])
        a["d2"] = self._conv(8, a["u2"])
        a["u1"] = R(up(a["d2"]) + a["s1"])
        a["d1a"] = self._conv(9, a["u1"])
        a["d1b"] = self._conv(10, a["d1a"])
        a["u0"] = R(up(a["d1b"]) + a["s0"])
        a["d0a"] = self._conv(11, a["u0"])
        a["y"] = self._conv(12, a["d0a"], store=False)
        self.a = a
        return a["y"][..., 0].reshape(a["y"].shape[0], -1)

    def loss(self, inp, target, N, kind="mse", weight=None):
        """(L, y, t, dL/dy) for the batch."""
        y = self.forward(inp, N)
        t = torch.as_tensor(np.asarray(target, dtype=np.float64)).reshape(y.shape)
        Bn = y.shape[0]
        w = torch.ones(Bn, dtype=f64) if weight is None else torch.as_tensor(np.asarray(weight, np.float64))
        e = y - t
        if kind == "mse":
            L = float((w[:, None] * e * e).sum() / e.numel())
            gy = 2.0 * w[:, None] * e / e.numel()
        else:
            logk = torch.as_tensor(np.asarray(inp, dtype=np.float64))[..., 1]
            Ae = torch.stack([energy_apply(e[b], logk[b], N) for b in range(Bn)])
            L = float((w[:, None] * e * Ae).sum() / Bn)
            gy = 2.0 * w[:, None] * Ae / Bn
        return L, y, t, gy

    def grads(self, inp, target, N, kind="mse", weight=None):
        """(loss, [(dW, db)] per layer) by the backward pass in reverse layer order."""
        R = self.R
        L, y, t, g0 = self.loss(inp, target, N, kind, weight)
        a = self.a
        gy = torch.zeros_like(a["y"])
        gy[..., 0] = R(g0).reshape(a["y"].shape[:-1])
        g = {"y": gy}
        dW = [None] * len(LAYERS)
        ins = ["x", "e0a", "p0", "e1a", "p1", "e2a", "p2", "e3a", "u2", "u1", "d1a", "u0", "d0a"]
        outs = ["e0a", "s0", "e1a", "s1", "e2a", "s2", "e3a", "e3b", "d2", "d1a", "d1b", "d0a", "y"]

        def back(l, need_input_grad=True):
            ci, co, relu = LAYERS[l]
            go = g[outs[l]]
            gz = go * (a[outs[l]] > 0) if relu else go
            dW[l] = conv_wgrad(a[ins[l]], gz)
            if need_input_grad:
                g[ins[l]] = R(conv_adjoint(gz, self.Wq[l], ci))

        back(12)
        back(11)
        g["d1b"] = R(up_adjoint(g["u0"]))
        back(10)
        back(9)
        g["d2"] = R(up_adjoint(g["u1"]))
        back(8)
        g["e3b"] = R(up_adjoint(g["u2"]))
        back(7)
        back(6)
        g["s2"] = R(g["u2"] + up(g["p2"]) / 8.0)
        back(5)
        back(4)
        g["s1"] = R(g["u1"] + up(g["p1"]) / 8.0)
        back(3)
        back(2)
        g["s0"] = R(g["u0"] + up(g["p0"]) / 8.0)
        back(1)
        back(0, need_input_grad=False)
        return L, dW
