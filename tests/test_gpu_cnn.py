"""GPU parity of the learned-update network's kernels against the FP64
network oracle (oracle/cnn.py), through the C ABI.

Inputs are BF16 values (what the kernels read); the oracle evaluates the
same BF16 values in FP64.  Tolerances follow from the arithmetic:
* FP32 outputs (data gradient, the FP32 forward modes, weight gradients of
  BF16-representable dY): FP32 accumulation of K terms, error below
  1e-5 of sum |terms| (K <= 27 * 32 products, or B V products per weight);
* BF16 outputs: one rounding to BF16 (relative 2^-9) on top of that.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1606_00556_gb300 as bo  # noqa: E402
from oracle import cnn as O  # noqa: E402

DIMS = [(10, 7, 5), (24, 20, 12)]  # 350 voxels (3 blocks of 128, ragged tail); 5760 voxels


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bo.bo_set_conv_engine(0)  # the mma.sync kernels; the tcgen05 tests switch engines themselves
    return bo.Context(0)


def _bf16(rng, shape, scale=1.0):
    return (torch.from_numpy(rng.standard_normal(shape) * scale).float()).to(torch.bfloat16)


def _np(t):
    return t.double().cpu().numpy() if t.dtype == torch.bfloat16 else t.cpu().numpy().astype(np.float64)


def _vol(t, dims):
    nx, ny, nz = dims
    return t.reshape(t.shape[0], nz, ny, nx, -1)


COMBOS = [(16, 32, "relu"), (32, 32, "relu"), (32, 32, "relu_res"), (32, 16, "linear_out"), (32, 32, "f32"),
          (16, 32, "f32"), (32, 16, "f32")]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("cin,cout,mode", COMBOS)
def test_conv_forward(ctx, dims, cin, cout, mode):
    rng = np.random.default_rng(cin * 100 + cout + len(mode) + dims[0])
    nx, ny, nz = dims
    V, B = nx * ny * nz, 2
    x = _bf16(rng, (B, V, cin)).cuda()
    w = _bf16(rng, (27, cout, cin), np.sqrt(2.0 / (27 * cin))).cuda()
    bias = torch.from_numpy(rng.standard_normal(cout) * 0.1).float().cuda()
    res = _bf16(rng, (B, V, cout)).cuda() if mode == "relu_res" else None
    y = torch.zeros(B, V, cout, dtype=torch.bfloat16, device="cuda") if mode != "f32" else None
    yf = None
    if mode == "f32":
        yf = torch.zeros(B, V, cout, dtype=torch.float32, device="cuda")
    elif mode == "linear_out":
        yf = torch.zeros(B, V, 4, dtype=torch.float32, device="cuda")
    bo.bo_conv3d_forward(ctx, dims, x, w, bias, residual=res, relu=mode in ("relu", "relu_res"), y=y, yf=yf)
    torch.cuda.synchronize()
    X, W, bb = _vol(_np(x), dims), _np(w), _np(bias)
    ref = O.conv3d(X, W, bb)
    mag = O.conv3d(np.abs(X), np.abs(W), np.abs(bb))  # sum |terms|
    if res is not None:
        ref = ref + _vol(_np(res), dims)
        mag = mag + np.abs(_vol(_np(res), dims))
    if mode in ("relu", "relu_res"):
        ref = np.maximum(ref, 0.0)
    acc_tol = 1e-5 * mag + 1e-30
    if mode == "f32":
        got = _vol(_np(yf), dims)
        assert np.all(np.abs(got - ref) <= acc_tol), np.max(np.abs(got - ref) / acc_tol)
        return
    got = _vol(_np(y), dims)
    tol = acc_tol + 2.0 ** -8 * np.abs(ref)  # one BF16 rounding
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
    if mode == "linear_out":
        gf = _vol(_np(yf), dims)
        assert np.all(np.abs(gf - ref[..., :4]) <= acc_tol[..., :4])


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_conv_backward_data(ctx, dims, cin, cout):
    rng = np.random.default_rng(7 + cin + cout)
    nx, ny, nz = dims
    V, B = nx * ny * nz, 2
    dy = _bf16(rng, (B, V, cout)).cuda()
    w = _bf16(rng, (27, cout, cin), 0.1).cuda()
    dx = torch.full((B, V, cin), float("nan"), dtype=torch.float32, device="cuda")
    bo.bo_conv3d_backward_data(ctx, dims, dy, w, dx)
    DY, W = _vol(_np(dy), dims), _np(w)
    shape = (B, nz, ny, nx, cin)
    ref = O.conv3d_backward_data(DY, W, shape)
    mag = O.conv3d_backward_data(np.abs(DY), np.abs(W), shape)
    got = _vol(_np(dx), dims)
    assert np.all(np.abs(got - ref) <= 1e-5 * mag + 1e-30)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_conv_backward_weights(ctx, dims, cin, cout):
    rng = np.random.default_rng(11 + cin + cout)
    nx, ny, nz = dims
    V, B = nx * ny * nz, 2
    x = _bf16(rng, (B, V, cin)).cuda()
    dy = _bf16(rng, (B, V, cout)).float().cuda()  # BF16-representable: the kernel's rounding is exact
    dw = torch.full((27, cout, cin), float("nan"), dtype=torch.float32, device="cuda")
    db = torch.full((cout,), float("nan"), dtype=torch.float32, device="cuda")
    bo.bo_conv3d_backward_weights(ctx, dims, x, dy, dw, db)
    X, DY = _vol(_np(x), dims), _vol(_np(dy), dims)
    ref_w, ref_b = O.conv3d_backward_weights(X, DY)
    mag_w, mag_b = O.conv3d_backward_weights(np.abs(X), np.abs(DY))
    assert np.all(np.abs(_np(dw) - ref_w) <= 1e-5 * mag_w + 1e-30)
    assert np.all(np.abs(_np(db) - ref_b) <= 1e-6 * mag_b + 1e-30)


def test_conv_rejects_unsupported(ctx):
    x = torch.zeros(1, 8, 8, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(27, 8, 8, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(8, device="cuda")
    y = torch.zeros(1, 8, 8, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(bo.BoError):
        bo.bo_conv3d_forward(ctx, (2, 2, 2), x, w, b, relu=True, y=y)


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a)).float().to(torch.bfloat16).double().numpy()


def _net_case(seed, dims, B):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    V = nx * ny * nz
    x = torch.zeros(B, V, 16, dtype=torch.bfloat16)
    x[..., :6] = _bf16(rng, (B, V, 6))
    tgt = torch.from_numpy(rng.standard_normal((B, V, 4))).float()
    mask = torch.from_numpy((rng.uniform(size=(B, V)) > 0.2).astype(np.float32))
    return x, tgt, mask


def test_network_forward_and_gradient(ctx):
    dims, B = (12, 10, 6), 2
    nx, ny, nz = dims
    net = bo.CNN(ctx, nx, ny, nz, max_batch=B, seed=3)
    assert net.nparam == O.param_count()
    # larger residual branches than the default initialisation, so every layer matters
    rng = np.random.default_rng(4)
    p = O.pack([(rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci)), 0.05 * rng.standard_normal(co))
                for ci, co, _ in O.layer_shapes()]).astype(np.float32)
    net.set_params(p)
    np.testing.assert_array_equal(net.get_params(), p)
    x, tgt, mask = _net_case(5, dims, B)
    xg, tg, mg = x.cuda(), tgt.cuda(), mask.cuda()
    pred = torch.zeros(B, nx * ny * nz, 4, device="cuda")
    net.forward(xg, pred)
    loss = net.backward(xg, tg, mg, nout=3)
    g = net.get_grads()
    # the oracle evaluates the same BF16 weights with the hidden activations
    # rounded to BF16, as the kernels store them
    pb = O.pack([(_bf16_round(w), b) for w, b in O.unpack(p.astype(np.float64))])
    X = _vol(_np(x), dims)
    T = _vol(tgt.numpy().astype(np.float64), dims)
    M = mask.numpy().astype(np.float64).reshape(B, nz, ny, nx)
    out, _ = O.forward(pb, X, act_round=_bf16_round)
    ref_loss, ref_g = O.loss_and_grad(pb, X, T, M, 3, act_round=_bf16_round)
    got = _vol(pred.cpu().numpy().astype(np.float64), dims)
    scale = np.abs(out[..., :4]).max()
    # activations stored in BF16 on both sides: differences come from FP32
    # summation order flipping a BF16 rounding, then propagating
    assert np.max(np.abs(got - out[..., :4])) <= 2e-2 * scale
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    cos = np.dot(g, ref_g) / (np.linalg.norm(g) * np.linalg.norm(ref_g))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - ref_g) <= 5e-2 * np.linalg.norm(ref_g)
    # every layer's gradient, not just the largest
    offs = np.cumsum([0] + [27 * ci * co + co for ci, co, _ in O.layer_shapes()])
    for l in range(len(offs) - 1):
        a, r = g[offs[l]:offs[l + 1]], ref_g[offs[l]:offs[l + 1]]
        assert np.linalg.norm(a - r) <= 0.1 * np.linalg.norm(r), l
    net.close()


def test_training_reduces_loss(ctx):
    dims, B = (16, 16, 8), 2
    nx, ny, nz = dims
    net = bo.CNN(ctx, nx, ny, nz, max_batch=B, seed=1)
    x, _, _ = _net_case(9, dims, B)
    xf = x.float()
    # a smooth function of the inputs the network can fit
    tgt = torch.zeros(B, nx * ny * nz, 4)
    tgt[..., 0] = 0.5 * xf[..., 0] - 0.25 * xf[..., 1] * xf[..., 2].abs()
    xg, tg = x.cuda(), tgt.cuda()
    l0 = net.backward(xg, tg, None, nout=1)
    for _ in range(300):
        net.backward(xg, tg, None, nout=1, want_loss=False)
        net.adam_step(2e-3)
    l1 = net.backward(xg, tg, None, nout=1)
    assert np.isfinite(l1) and l1 < 0.1 * l0, (l0, l1)
    net.close()


def test_adam_step_matches_oracle(ctx):
    dims = (8, 6, 4)
    net = bo.CNN(ctx, *dims, max_batch=1, seed=2)
    x, tgt, _ = _net_case(10, dims, 1)
    p0 = net.get_params().astype(np.float64)
    net.backward(x.cuda(), tgt.cuda(), None, nout=1, want_loss=False)
    g = net.get_grads().astype(np.float64)
    net.adam_step(1e-3)
    p1 = net.get_params().astype(np.float64)
    ref, _, _ = O.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    np.testing.assert_allclose(p1, ref, rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------- tcgen05 engine
@pytest.fixture
def tc_engine():
    bo.bo_set_conv_engine(1)
    yield
    assert bo.bo_tc_status() == bo.BO_OK  # no tcgen05 CTA gave up on a barrier
    bo.bo_set_conv_engine(0)


@pytest.mark.parametrize("dims", DIMS + [(64, 64, 8), (16, 16, 3)])
@pytest.mark.parametrize("mode", ["relu", "relu_res", "f32"])
def test_tc_conv_forward(ctx, tc_engine, dims, mode):
    # the tcgen05 kernel against the oracle, with the same tolerances as the mma.sync kernel
    test_conv_forward(ctx, dims, 32, 32, mode)


@pytest.mark.parametrize("dims", DIMS + [(64, 64, 8)])
def test_tc_conv_backward_data(ctx, tc_engine, dims):
    test_conv_backward_data(ctx, dims, 32, 32)


def test_tc_conv_equals_mma_sync_to_accumulation_order(ctx):
    # both engines sum the same BF16 products in FP32: FP32 outputs agree to rounding
    rng = np.random.default_rng(3)
    dims = (24, 20, 12)
    nx, ny, nz = dims
    V, B = nx * ny * nz, 3
    x = _bf16(rng, (B, V, 32)).cuda()
    w = _bf16(rng, (27, 32, 32), 0.1).cuda()
    bias = torch.from_numpy(rng.standard_normal(32) * 0.1).float().cuda()
    out = []
    for eng in (0, 1):
        bo.bo_set_conv_engine(eng)
        yf = torch.full((B, V, 32), float("nan"), device="cuda")
        bo.bo_conv3d_forward(ctx, dims, x, w, bias, yf=yf)
        torch.cuda.synchronize()
        out.append(yf.cpu().numpy().astype(np.float64))
    bo.bo_set_conv_engine(0)
    assert bo.bo_tc_status() == bo.BO_OK
    mag = O.conv3d(np.abs(_vol(_np(x), dims)), np.abs(_np(w))).reshape(B, V, 32) + np.abs(_np(bias))
    assert np.all(np.abs(out[0] - out[1]) <= 2e-5 * mag + 1e-30)


def test_tc_network_gradient(ctx, tc_engine):
    test_network_forward_and_gradient(ctx)
