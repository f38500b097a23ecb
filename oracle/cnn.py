"""FP64 CPU oracle of the learned Newton update's convolutional network.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this module; the solver library never does, and it
shares no code with the GPU path.

The network has no counterpart in the paper (it is this library's addition
that feeds the Krylov solve of Sec. 3 an initial guess and a coarse space),
so this module is the plain definition of what the library states it
computes:

* conv3d: 3x3x3 cross-correlation with 'same' zero padding over an NDHWC
  volume [B, nz, ny, nx, C]; weights [27, Cout, Cin] with tap
  t = 9 (dz+1) + 3 (dy+1) + (dx+1) reading the input at (x+dx, y+dy, z+dz);
* its two adjoints (data gradient and weight/bias gradient);
* the network: input conv (16 -> 32, ReLU), 6 residual blocks
  (conv 32 -> 32 + ReLU; conv 32 -> 32 + block input, ReLU) and an output
  conv (32 -> 16, linear), parameters in one flat vector (per layer the
  weights [27, Cout, Cin] then the Cout biases);
* the masked mean squared error over the first `nout` output channels and
  its gradient by the chain rule;
* one Adam step (Kingma & Ba 2015, Algorithm 1, with bias correction).

Everything is numpy float64; one matmul per tap is the only library
primitive.  Pinned by tests/test_oracle_cnn_pins.py (Dirac kernels, scipy's
correlate, brute-force loops, adjoint identities, finite differences, the
closed-form first Adam step).
"""
from __future__ import annotations

import numpy as np

C_IN = 16
C_HID = 32
C_OUT = 16
N_BLOCKS = 6


def taps():
    """(t, dx, dy, dz) for the 27 taps in the library's order."""
    out = []
    for t in range(27):
        out.append((t, t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1))
    return out


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))


def _window(xp, dx, dy, dz, nz, ny, nx):
    """The padded volume's view holding x[v + (dx, dy, dz)] at each v."""
    return xp[:, 1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx, :]


def conv3d(x, w, b=None):
    """y[v][co] = b[co] + sum_t sum_ci x[v + off(t)][ci] w[t][co][ci]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, nz, ny, nx, cin = x.shape
    assert w.shape[0] == 27 and w.shape[2] == cin
    xp = _pad(x)
    y = np.zeros((B, nz, ny, nx, w.shape[1]))
    for t, dx, dy, dz in taps():
        y += _window(xp, dx, dy, dz, nz, ny, nx) @ w[t].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_backward_data(dy, w, shape):
    """dx[u][ci] = sum_t sum_co dy[u - off(t)][co] w[t][co][ci] (the adjoint
    of conv3d in x); `shape` is x's shape."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    B, nz, ny, nx, cin = shape
    dxp = np.zeros((B, nz + 2, ny + 2, nx + 2, cin))
    for t, dx, dyy, dz in taps():
        _window(dxp, dx, dyy, dz, nz, ny, nx)[...] += dy @ w[t]
    return dxp[:, 1:-1, 1:-1, 1:-1, :].copy()


def conv3d_backward_weights(x, dy):
    """(dw, db): dw[t][co][ci] = sum_v dy[v][co] x[v + off(t)][ci],
    db[co] = sum_v dy[v][co]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    B, nz, ny, nx, cin = x.shape
    cout = dy.shape[-1]
    xp = _pad(x)
    dw = np.zeros((27, cout, cin))
    d2 = dy.reshape(-1, cout)
    for t, dx, dyy, dz in taps():
        dw[t] = d2.T @ _window(xp, dx, dyy, dz, nz, ny, nx).reshape(-1, cin)
    return dw, d2.sum(axis=0)


def layer_shapes():
    """[(cin, cout, kind)] with kind in {'relu', 'relu_res', 'linear'}."""
    L = [(C_IN, C_HID, "relu")]
    for _ in range(N_BLOCKS):
        L += [(C_HID, C_HID, "relu"), (C_HID, C_HID, "relu_res")]
    L.append((C_HID, C_OUT, "linear"))
    return L


def param_count() -> int:
    return sum(27 * ci * co + co for ci, co, _ in layer_shapes())


def unpack(params):
    """Flat parameter vector -> [(w [27, cout, cin], b [cout])]."""
    params = np.asarray(params, np.float64)
    out, off = [], 0
    for ci, co, _ in layer_shapes():
        w = params[off:off + 27 * co * ci].reshape(27, co, ci)
        off += 27 * co * ci
        out.append((w, params[off:off + co]))
        off += co
    assert off == params.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def forward(params, x, act_round=None):
    """Network output [B, nz, ny, nx, 16] and the activations list
    (acts[0] = x, acts[l+1] = output of layer l).  `act_round`, if given, is
    applied to every stored hidden activation (to evaluate the same network
    with the activations held at a lower precision)."""
    rnd = act_round if act_round is not None else (lambda a: a)
    layers = unpack(params)
    acts = [np.asarray(x, np.float64)]
    for l, ((ci, co, kind), (w, b)) in enumerate(zip(layer_shapes(), layers)):
        y = conv3d(acts[-1], w, b)
        if kind == "relu_res":
            y = y + acts[l - 1]
        if kind != "linear":
            y = rnd(np.maximum(y, 0.0))
        acts.append(y)
    return acts[-1], acts


def mse(pred, target, mask=None, nout=1):
    """(1 / (B V)) sum_v mask_v sum_{k < nout} (pred[v][k] - target[v][k])^2;
    pred [B, nz, ny, nx, >= nout], target [..., >= nout]."""
    pred = np.asarray(pred, np.float64)[..., :nout]
    target = np.asarray(target, np.float64)[..., :nout]
    m = np.ones(pred.shape[:-1]) if mask is None else np.asarray(mask, np.float64).reshape(pred.shape[:-1])
    return float(np.sum(m[..., None] * (pred - target) ** 2) / m.size)


def loss_and_grad(params, x, target, mask=None, nout=1, act_round=None):
    """Loss and its gradient with respect to the flat parameters, by the
    chain rule through the layers in reverse order."""
    out, acts = forward(params, x, act_round)
    layers = unpack(params)
    shapes = layer_shapes()
    m = np.ones(out.shape[:-1]) if mask is None else np.asarray(mask, np.float64).reshape(out.shape[:-1])
    nvox = m.size
    loss = mse(out, target, mask, nout)
    g = np.zeros_like(out)
    g[..., :nout] = 2.0 * m[..., None] * (out[..., :nout] - np.asarray(target, np.float64)[..., :nout]) / nvox
    grads = [None] * len(layers)
    # g is d loss / d acts[l+1] on entry to layer l's step
    skip = None  # gradient reaching a block input through its skip connection
    for l in range(len(layers) - 1, -1, -1):
        ci, co, kind = shapes[l]
        w, _ = layers[l]
        if kind != "linear":
            g = g * (acts[l + 1] > 0)  # through the ReLU
        if kind == "relu_res":
            skip = g  # d loss / d block input via the addition
        dw, db = conv3d_backward_weights(acts[l], g)
        grads[l] = (dw, db)
        if l > 0:
            g = conv3d_backward_data(g, w, acts[l].shape)
            if kind == "relu" and shapes[l + 1][2] == "relu_res":
                g = g + skip  # layer l is a block's first conv: its input is the block input
                skip = None
    return loss, pack(grads)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (p, m, v) (new arrays)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
