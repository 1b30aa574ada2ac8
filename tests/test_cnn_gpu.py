"""Residual CNN kernels against the FP64 reference (oracle/cnn.py).

BF16 storage with FP32 accumulation: convolution outputs are rounded to
bf16 (2^-9 relative), so forward / data-gradient parity is gated at 4e-3
relative L2; weight gradients stay FP32 and are gated at 1e-4.  The
reference is fed the same bf16 values (weights, activations) as float64.
"""
import numpy as np
import pytest
import torch

from oracle import cnn as R
from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import cnn as C

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a = torch.as_tensor(a, dtype=torch.float64).cpu()
    b = torch.as_tensor(b, dtype=torch.float64).cpu()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def rand_bf16(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16).to(DEV)


PAIRS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 32), (32, 16), (1, 16), (16, 1)]


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_conv3d_forward(cin, cout, n):
    x = rand_bf16((2, 4, n, n, cin), 1)
    w = rand_bf16((27, cout, cin), 2, scale=1.0 / np.sqrt(27 * cin))
    bias = torch.linspace(-0.1, 0.1, cout, device=DEV)
    for relu in (False, True):
        y = B.pyro_conv3d(x, w, bias, relu)
        ref = R.conv3d(x.double().cpu(), w.double().cpu(), bias.double().cpu(), relu)
        assert rel(y, ref) < 4e-3


@pytest.mark.parametrize("cout", [16, 32, 1])
@pytest.mark.parametrize("shape", [(1, 3, 4, 128), (2, 2, 3, 256)])
def test_conv3d_forward_wide_row(shape, cout):
    """Rows of 128 voxels or more and 16 input channels take the kernel that
    stages nine input lines per 128-voxel output row (every z, y and x edge
    of the zero padding is in these shapes), one output channel included."""
    x = rand_bf16((*shape, 16), 3)
    w = rand_bf16((27, cout, 16), 4, scale=0.05)
    bias = torch.linspace(-0.1, 0.1, cout, device=DEV)
    for relu in (False, True):
        y = B.pyro_conv3d(x, w, bias, relu)
        assert rel(y, R.conv3d(x.double().cpu(), w.double().cpu(), bias.double().cpu(), relu)) < 4e-3


@pytest.mark.parametrize("cin,cout", [(16, 16), (1, 16), (16, 1)])
def test_conv3d_data_gradient_wide_row(cin, cout):
    """The data gradient through the flipped weights on 128-voxel rows."""
    x = rand_bf16((1, 3, 4, 128, cin), 8)
    w = rand_bf16((27, cout, cin), 9, scale=0.05)
    dy = rand_bf16((1, 3, 4, 128, cout), 10)
    dx = B.pyro_conv3d(dy, B.pyro_conv3d_flip_weights(w), None, False)
    xr = x.double().cpu().permute(0, 4, 1, 2, 3)
    ref = torch.nn.grad.conv3d_input(xr.shape, R.to_kernel(w.double().cpu()),
                                     dy.double().cpu().permute(0, 4, 1, 2, 3), padding=1)
    assert rel(dx, ref.permute(0, 2, 3, 4, 1)) < 4e-3


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (32, 64), (64, 64), (16, 1)])
def test_conv3d_data_gradient_by_flipped_weights(cin, cout):
    x = rand_bf16((2, 4, 16, 16, cin), 5)
    w = rand_bf16((27, cout, cin), 6, scale=0.05)
    dy = rand_bf16((2, 4, 16, 16, cout), 7)
    dx = B.pyro_conv3d(dy, B.pyro_conv3d_flip_weights(w), None, False)
    xr = x.double().cpu().permute(0, 4, 1, 2, 3)
    ref = torch.nn.grad.conv3d_input(xr.shape, R.to_kernel(w.double().cpu()),
                                     dy.double().cpu().permute(0, 4, 1, 2, 3), padding=1)
    assert rel(dx, ref.permute(0, 2, 3, 4, 1)) < 4e-3


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (16, 64), (32, 16), (32, 32), (32, 64), (64, 16), (64, 32),
                                      (64, 64), (1, 16), (16, 1)])
def test_conv3d_weight_gradient(cin, cout):
    x = rand_bf16((2, 4, 32, 32, cin), 8)
    dy = rand_bf16((2, 4, 32, 32, cout), 9)
    dw = B.pyro_conv3d_wgrad(x, dy)
    ref = R.conv3d_wgrad(x.double().cpu(), dy.double().cpu())
    assert rel(dw, ref) < 1e-4


@pytest.mark.parametrize("shape", [(1, 8, 8, 8), (1, 4, 4, 128), (3, 8, 16, 64), (2, 3, 6, 64)])
@pytest.mark.parametrize("cin,cout", [(16, 32), (64, 16)])
def test_conv3d_weight_gradient_shapes(shape, cin, cout):
    """The tensor-core weight gradient over 64-voxel chunks: a volume of
    eight chunks, rows wider than a chunk, a batch of three, and depth and
    height that are not powers of two (the division path)."""
    x = rand_bf16((*shape, cin), 20)
    dy = rand_bf16((*shape, cout), 21)
    dw = B.pyro_conv3d_wgrad(x, dy)
    ref = R.conv3d_wgrad(x.double().cpu(), dy.double().cpu())
    assert rel(dw, ref) < 1e-4


def test_elementwise_ops():
    x = rand_bf16((2, 8, 8, 16, 16), 10)
    p = torch.empty((2, 4, 4, 8, 16), device=DEV, dtype=torch.bfloat16)
    B.pyro_cnn_op(B.CNN_AVGPOOL2, x, p, dims=(8, 8, 16, 16))
    assert rel(p, R.avgpool2(x.double().cpu())) < 4e-3
    skip = rand_bf16((2, 8, 8, 16, 16), 11)
    u = torch.empty_like(x)
    B.pyro_cnn_op(B.CNN_UPSAMPLE2, p, u, b=skip, dims=(4, 4, 8, 16))
    assert rel(u, R.upsample2(p.double().cpu(), skip.double().cpu())) < 4e-3
    # the backward ops are the transposes of the forward ones
    g = rand_bf16((2, 4, 4, 8, 16), 12)
    gx = torch.empty_like(x)
    B.pyro_cnn_op(B.CNN_AVGPOOL2_BWD, g, gx, dims=(8, 8, 16, 16))
    lhs = float((p.double() * g.double()).sum())
    rhs = float((x.double() * gx.double()).sum())
    assert abs(lhs - rhs) < 1e-2 * abs(lhs) + 1e-3
    gu = rand_bf16((2, 8, 8, 16, 16), 13)
    gp = torch.empty_like(p)
    B.pyro_cnn_op(B.CNN_UPSAMPLE2_BWD, gu, gp, dims=(4, 4, 8, 16))
    ref = gu.double().cpu().reshape(2, 4, 2, 4, 2, 8, 2, 16).sum(dim=(2, 4, 6))
    assert rel(gp, ref) < 4e-3
    r = rand_bf16((2, 8, 8, 16, 16), 14)
    act = rand_bf16((2, 8, 8, 16, 16), 15)
    expect = r.double().cpu() * (act.double().cpu() > 0)
    B.pyro_cnn_op(B.CNN_RELU_BWD, act, r)
    assert torch.equal(r.double().cpu(), expect)
    db = B.pyro_cnn_bias_grad(gu)
    assert rel(db, gu.double().cpu().sum(dim=(0, 1, 2, 3))) < 1e-5


def test_elementwise_vector_and_scalar_kernels_agree():
    """Pooling and upsampling run 8 channels per thread on 16-byte aligned
    tensors and one element per thread otherwise: the same bits either way
    (an output 4 elements into a buffer is 8-byte aligned only)."""
    x = rand_bf16((2, 8, 8, 16, 16), 20)
    skip = rand_bf16((2, 8, 8, 16, 16), 21)
    def pair(shape):
        buf = torch.empty(int(np.prod(shape)) + 4, device=DEV, dtype=torch.bfloat16)
        return torch.empty(shape, device=DEV, dtype=torch.bfloat16), buf[4:].view(shape)
    pa, pu = pair((2, 4, 4, 8, 16))
    B.pyro_cnn_op(B.CNN_AVGPOOL2, x, pa, dims=(8, 8, 16, 16))
    B.pyro_cnn_op(B.CNN_AVGPOOL2, x, pu, dims=(8, 8, 16, 16))
    assert torch.equal(pa, pu)
    ua, uu = pair((2, 8, 8, 16, 16))
    B.pyro_cnn_op(B.CNN_UPSAMPLE2, pa, ua, b=skip, dims=(4, 4, 8, 16))
    B.pyro_cnn_op(B.CNN_UPSAMPLE2, pa, uu, b=skip, dims=(4, 4, 8, 16))
    assert torch.equal(ua, uu)
    ga, gu = pair((2, 4, 4, 8, 16))
    B.pyro_cnn_op(B.CNN_UPSAMPLE2_BWD, skip, ga, dims=(4, 4, 8, 16))
    B.pyro_cnn_op(B.CNN_UPSAMPLE2_BWD, skip, gu, dims=(4, 4, 8, 16))
    assert torch.equal(ga, gu)
    da, du = pair((2, 8, 8, 16, 16))
    B.pyro_cnn_op(B.CNN_AVGPOOL2_BWD, pa, da, dims=(8, 8, 16, 16))
    B.pyro_cnn_op(B.CNN_AVGPOOL2_BWD, pa, du, dims=(8, 8, 16, 16))
    assert torch.equal(da, du)


def reference_params(net):
    return {n: (p.w16.double().cpu(), p.b.double().cpu()) for n, p in net.params.items()}


def test_network_forward_matches_reference():
    net = C.ResidualCNN(DEV, seed=3)
    # the last layer is initialised small; scale it up so the branch matters
    p = net.params["c11"]
    p.w.mul_(10.0)
    B.pyro_cnn_op(B.CNN_F32_TO_BF16, p.w, p.w16)
    g = torch.Generator().manual_seed(4)
    x = torch.randn((2, 64, 64, 64), generator=g).to(DEV)
    out = net.forward(x)
    ref = R.network(x.double().cpu(), reference_params(net))
    branch = out.double().cpu() - x.double().cpu()
    assert rel(branch, ref - x.double().cpu()) < 3e-2
    assert net.n_params() > 400_000
    with pytest.raises(ValueError):
        net.forward(torch.zeros((1, 32, 32, 32), device=DEV))


def test_network_gradients_match_reference():
    """Weight gradients of the MSE through the whole network vs float64
    autograd of the reference (same bf16 weights); bf16 activations and
    gradients inside the network bound the agreement to a few percent."""
    net = C.ResidualCNN(DEV, seed=5)
    p = net.params["c11"]
    p.w.mul_(10.0)
    B.pyro_cnn_op(B.CNN_F32_TO_BF16, p.w, p.w16)
    g = torch.Generator().manual_seed(6)
    x = torch.randn((1, 64, 64, 64), generator=g).to(DEV)
    t = torch.randn((1, 64, 64, 64), generator=g).to(DEV)
    out, acts = net.forward(x, keep=True)
    dout = torch.empty((*out.shape, 1), device=DEV, dtype=torch.bfloat16)
    loss = B.pyro_cnn_mse(out, t, dout)
    grads = net.backward(acts, dout)
    params = {n: (w.clone().requires_grad_(True), b.clone().requires_grad_(True))
              for n, (w, b) in reference_params(net).items()}
    ref_out = R.network(x.double().cpu(), params)
    ref_loss = ((ref_out - t.double().cpu()) ** 2).mean()
    ref_loss.backward()
    assert abs(loss.item() - ref_loss.item()) < 1e-2 * ref_loss.item()
    for n in ("c0", "c5", "c8", "c11"):
        gw = grads[n][0].double().cpu().ravel()
        rw = params[n][0].grad.ravel()
        cos = float(gw @ rw / (gw.norm() * rw.norm()))
        assert cos > 0.99, (n, cos)
        assert rel(gw, rw) < 0.1, n


def test_training_lowers_the_loss():
    """Denoising a smooth volume: 40 Adam steps lower the MSE."""
    net = C.ResidualCNN(DEV, seed=7)
    g = torch.Generator().manual_seed(8)
    clean = torch.nn.functional.avg_pool3d(torch.randn((2, 1, 64, 64, 64), generator=g), 5, 1, 2)[:, 0].to(DEV)
    noisy = clean + 0.05 * torch.randn((2, 64, 64, 64), generator=g).to(DEV)
    losses = [net.train_step(noisy, clean, lr=1e-3) for _ in range(40)]
    assert losses[-1] < 0.7 * losses[0]
