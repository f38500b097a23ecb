"""Pins of the FP64 network oracle (oracle/cnn.py) to facts outside itself:
Dirac kernels, scipy's n-dimensional correlation, brute-force loops, the
adjoint identities that define the two gradients, central finite
differences of the loss, and the closed form of Adam's first steps."""
import numpy as np
import pytest

from oracle import cnn as O

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_tap_order():
    t = O.taps()
    assert t[13][1:] == (0, 0, 0)
    assert t[0][1:] == (-1, -1, -1) and t[26][1:] == (1, 1, 1)
    assert t[14][1:] == (1, 0, 0) and t[16][1:] == (0, 1, 0) and t[22][1:] == (0, 0, 1)
    for (a, dx, dy, dz), (b, ex, ey, ez) in zip(t, reversed(t)):
        assert (dx, dy, dz) == (-ex, -ey, -ez)  # tap 26 - t is the mirror of t


def test_dirac_identity_and_shift():
    rng = np.random.default_rng(0)
    x = _rand(rng, 2, 3, 4, 5, 6)
    w = np.zeros((27, 6, 6))
    w[13] = np.eye(6)
    np.testing.assert_array_equal(O.conv3d(x, w), x)
    # a Dirac at tap (dx, dy, dz) = (1, 0, 0): y[x] = x[x + 1], zero at the last column
    w = np.zeros((27, 6, 6))
    w[14] = np.eye(6)
    y = O.conv3d(x, w)
    np.testing.assert_array_equal(y[:, :, :, :-1], x[:, :, :, 1:])
    np.testing.assert_array_equal(y[:, :, :, -1], 0.0)


def test_single_channel_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    vol = _rand(rng, 5, 6, 7)  # (z, y, x)
    k = _rand(rng, 3, 3, 3)    # indexed [dz+1, dy+1, dx+1]
    w = np.zeros((27, 1, 1))
    for t, dx, dy, dz in O.taps():
        w[t, 0, 0] = k[dz + 1, dy + 1, dx + 1]
    y = O.conv3d(vol[None, ..., None], w, np.array([0.25]))[0, ..., 0]
    ref = scipy_ndimage.correlate(vol, k, mode="constant", cval=0.0) + 0.25
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


def test_brute_force_small():
    rng = np.random.default_rng(2)
    B, nz, ny, nx, ci, co = 2, 2, 3, 4, 3, 2
    x = _rand(rng, B, nz, ny, nx, ci)
    w = _rand(rng, 27, co, ci)
    b = _rand(rng, co)
    ref = np.zeros((B, nz, ny, nx, co))
    for bb in range(B):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    for o in range(co):
                        s = b[o]
                        for kz in (-1, 0, 1):
                            for ky in (-1, 0, 1):
                                for kx in (-1, 0, 1):
                                    zz, yy, xq = z + kz, y + ky, xx + kx
                                    if 0 <= zz < nz and 0 <= yy < ny and 0 <= xq < nx:
                                        t = 9 * (kz + 1) + 3 * (ky + 1) + (kx + 1)
                                        for i in range(ci):
                                            s += x[bb, zz, yy, xq, i] * w[t, o, i]
                        ref[bb, z, y, xx, o] = s
    np.testing.assert_allclose(O.conv3d(x, w, b), ref, rtol=1e-13, atol=1e-13)


def test_backward_data_is_adjoint():
    rng = np.random.default_rng(3)
    x = _rand(rng, 2, 3, 4, 5, 4)
    w = _rand(rng, 27, 6, 4)
    dy = _rand(rng, 2, 3, 4, 5, 6)
    lhs = np.sum(O.conv3d(x, w) * dy)
    rhs = np.sum(x * O.conv3d_backward_data(dy, w, x.shape))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs) + 1e-11


def test_backward_weights_is_adjoint():
    rng = np.random.default_rng(4)
    x = _rand(rng, 2, 3, 4, 5, 4)
    w = _rand(rng, 27, 6, 4)
    b = _rand(rng, 6)
    dy = _rand(rng, 2, 3, 4, 5, 6)
    dw, db = O.conv3d_backward_weights(x, dy)
    # conv3d is linear in (w, b): <conv3d(x; w, b), dy> = <w, dw> + <b, db>
    lhs = np.sum(O.conv3d(x, w, b) * dy)
    rhs = np.sum(w * dw) + np.sum(b * db)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs) + 1e-11


def test_zero_second_conv_makes_block_pass_through():
    # a residual block whose second convolution is zero passes a nonnegative input through
    rng = np.random.default_rng(5)
    p = 0.1 * rng.standard_normal(O.param_count())
    layers = O.unpack(p.copy())
    for l in (2, 4, 6, 8, 10, 12):
        layers[l] = (np.zeros_like(layers[l][0]), np.zeros_like(layers[l][1]))
    x = _rand(rng, 1, 3, 4, 4, 16)
    out, acts = O.forward(O.pack(layers), x)
    np.testing.assert_allclose(acts[13], acts[1], rtol=0, atol=0)


def _network_case(seed, nout):
    rng = np.random.default_rng(seed)
    p = O.pack([(rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci)), 0.1 * rng.standard_normal(co))
                for ci, co, _ in O.layer_shapes()])
    x = rng.standard_normal((2, 3, 3, 4, 16))
    tgt = rng.standard_normal((2, 3, 3, 4, 4))
    mask = (rng.uniform(size=(2, 3, 3, 4)) > 0.3).astype(float)
    return p, x, tgt, mask


@pytest.mark.parametrize("nout", [1, 3])
def test_gradient_matches_finite_differences(nout):
    p, x, tgt, mask = _network_case(6, nout)
    loss, g = O.loss_and_grad(p, x, tgt, mask, nout)
    assert np.isclose(loss, O.mse(O.forward(p, x)[0], tgt, mask, nout))
    rng = np.random.default_rng(7)
    # sample weights of every layer (first, middle, last) plus biases
    offs = np.cumsum([0] + [27 * ci * co + co for ci, co, _ in O.layer_shapes()])
    idx = []
    for l in range(len(offs) - 1):
        idx += list(rng.integers(offs[l], offs[l + 1], 3))
        idx.append(offs[l + 1] - 1)  # a bias
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (O.mse(O.forward(p + e, x)[0], tgt, mask, nout) - O.mse(O.forward(p - e, x)[0], tgt, mask, nout)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(8)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr = 1e-3
    # with bias correction the first step is -lr g / (|g| + eps)
    p1, m, v = O.adam_step(p, g, m, v, 1, lr)
    np.testing.assert_allclose(p1 - p, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a constant gradient keeps m_hat = g and v_hat = g^2: the same step again
    p2, m, v = O.adam_step(p1, g, m, v, 2, lr)
    np.testing.assert_allclose(p2 - p1, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9)
