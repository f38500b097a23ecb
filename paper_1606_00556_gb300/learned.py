"""Host loops of the learned Newton update: mini-batch training of the
network (bo_cnn_backward + bo_cnn_adam_step) and a solve that starts from
the network's prediction and uses it as a coarse space.  Every arithmetic
step runs in the library's kernels; this module only picks batches and
sequences the calls.  (No counterpart in the paper: an addition that feeds
the Krylov solve of Sec. 3.)"""
from __future__ import annotations

import numpy as np

from . import CNN, Preconditioner


def train(net: CNN, X, Y, steps: int, batch: int, lr: float = 1e-3, nout: int = 3, seed: int = 0,
          mask=None, log_every: int = 0, lr_final: float = None):
    """`steps` Adam steps on mini-batches of `batch` samples drawn without
    replacement per epoch from X [n, V, 16] (bf16, device) and Y [n, V, 4]
    (f32, device).  The learning rate decays linearly to `lr_final`
    (default lr / 10).  Returns the losses logged every `log_every` steps
    (each a synchronising read)."""
    import torch
    n = X.shape[0]
    if batch > net.max_batch or batch > n:
        raise ValueError("batch larger than the network's max_batch or the data set")
    rng = np.random.default_rng(seed)
    lr_final = lr / 10 if lr_final is None else lr_final
    order = rng.permutation(n)
    pos = 0
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
    yb = torch.empty((batch,) + tuple(Y.shape[1:]), dtype=Y.dtype, device=Y.device)
    losses = []
    for it in range(steps):
        if pos + batch > n:
            order = rng.permutation(n)
            pos = 0
        idx = torch.as_tensor(order[pos:pos + batch], device=X.device)
        pos += batch
        torch.index_select(X, 0, idx, out=xb)
        torch.index_select(Y, 0, idx, out=yb)
        want = log_every and (it % log_every == 0 or it == steps - 1)
        loss = net.backward(xb, yb, mask, nout=nout, want_loss=bool(want))
        if want:
            losses.append((it, loss))
        net.adam_step(lr + (lr_final - lr) * it / max(1, steps - 1))
    return losses


def learned_solve(P: Preconditioner, net: CNN, x_feat, b, x, scale, ncomp: int = 3, coarse_tile=None,
                  tol: float = 1e-8, restart: int = 30, maxit: int = 500, pred=None):
    """Solve A x = b from the network's predicted Newton update.

    x_feat: the system's features [1, V, 16] bf16; scale: per-component
    factors of the prediction (x0[3c+k] = scale[k] pred[c][k]); ncomp: how
    many components the guess sets (1: pressure only).  The guess is kept
    only where it lowers the residual (else the solve starts from zero).
    coarse_tile: if given, the predicted pressure update also spans a
    coarse space of that tile size inside CPR.  Returns the solve's info
    dict with 'guess_used'."""
    import torch
    V = x_feat.shape[1]
    if pred is None:
        pred = torch.empty(1, V, 4, dtype=torch.float32, device=b.device)
    net.forward(x_feat, pred)
    if coarse_tile is not None:
        P.learned_coarse_space(pred[0], scale[0], coarse_tile)
    used = P.learned_guess(b, pred[0], scale, ncomp, x)
    info = P.solve(b, x, tol=tol, restart=restart, maxit=maxit, x0_is_zero=not used, raise_on_error=False)
    info["guess_used"] = used
    if coarse_tile is not None:
        P.set_coarse_space(None)
    return info
