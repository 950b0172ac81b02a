"""The learned warm start's network (BF16 tensor-core kernels, FP32
accumulation; both convolution paths: tcgen05 with the accumulator in tensor
memory, and WMMA mma.sync) against the FP64 oracle U-Net with the same
parameters.

The oracle emulates the GPU's BF16 storage of weights and activations in the
forward pass, so the forward output agrees to ~FP32 accumulation-order noise
plus rare BF16 rounding flips (relative L2 of the network's correction
<= 1e-2); the backward pass keeps BF16 activation gradients on the GPU and
FP64 in the oracle, so parameter gradients are compared per layer at
relative L2 <= 5e-2 (a wrong tap, transpose or skip connection gives O(1)).
"""
import numpy as np
import pytest

from oracle import unet as ounet
from paper_2202_08627_gb300 import inputs
from tests.problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


LEVELS, BASE, B, H, W = 3, 32, 2, 16, 24


def _net_and_params(path=1):
    from paper_2202_08627_gb300 import ei
    net = ei.UNet(levels=LEVELS, base=BASE, batch=B, height=H, width=W, seed=3)
    net.set_tensor_path(path)
    flat = net.get_params().astype(np.float64)
    p = ounet.unpack(flat, LEVELS, BASE)
    p["head.W"] = 0.2 * inputs.uniform_noise(p["head.W"].shape, 20)   # make the head matter
    p["head.b"] = 0.05 * inputs.uniform_noise(3, 21)
    for name, _, co in ounet.layout(LEVELS, BASE):
        p[name + ".b"] = 0.05 * inputs.uniform_noise(co, 22 + len(name))
    flat = ounet.pack(p, LEVELS, BASE)
    net.set_params(flat.astype(np.float32))
    return net, ounet.unpack(net.get_params().astype(np.float64), LEVELS, BASE)


def test_params_round_trip():
    net, _ = _net_and_params()
    a = net.get_params()
    net.set_params(a)
    np.testing.assert_array_equal(net.get_params(), a)


def test_training_checkpoint_resumes_bit_identically():
    """Parameters + Adam moments + step restored into a fresh network: the
    next training steps give bit-identical parameters."""
    from paper_2202_08627_gb300 import ei
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    xs = [torch.rand(B, H, W, 3, device="cuda", generator=g) for _ in range(5)]
    ts = [torch.rand(B, H, W, 3, device="cuda", generator=g) for _ in range(5)]
    a, _ = _net_and_params()
    for k in range(3):
        a.train_step(xs[k], ts[k], 1e-3)
    params = a.get_params()
    m, v, step = a.get_optimizer()
    assert step == 3 and np.any(m != 0) and np.any(v != 0)
    b = ei.UNet(levels=LEVELS, base=BASE, batch=B, height=H, width=W, seed=99)
    b.set_params(params)
    b.set_optimizer(m, v, step)
    for k in range(3, 5):
        a.train_step(xs[k], ts[k], 1e-3)
        b.train_step(xs[k], ts[k], 1e-3)
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    ma, va, sa = a.get_optimizer()
    mb, vb, sb = b.get_optimizer()
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(va, vb)
    assert sa == sb == 5


@pytest.mark.parametrize("path", [1, 0])
def test_forward_matches_oracle(path):
    net, p = _net_and_params(path)
    x = inputs.uniform_noise((B, H, W, 3), 30, 0.0, 1.0)
    y = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    ref = ounet.forward(x.astype(np.float32).astype(np.float64), p, LEVELS, bf16=True)
    assert rel_l2(y - x, ref - x) <= 1e-2, rel_l2(y - x, ref - x)


@pytest.mark.parametrize("path", [1, 0])
def test_gradients_match_oracle(path):
    net, p = _net_and_params(path)
    x = inputs.uniform_noise((B, H, W, 3), 31, 0.0, 1.0).astype(np.float32)
    t = inputs.uniform_noise((B, H, W, 3), 32, 0.0, 1.0).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    loss = net.train_step(xd, td, lr=1e-12)
    gy = 2.0 * (y - t) / y.size
    assert abs(loss - np.mean((y - t) ** 2)) <= 1e-5 * loss
    g = net.get_grads().astype(np.float64)
    ref = ounet.pack(ounet.backward(x.astype(np.float64), p, LEVELS, gy, bf16=True), LEVELS, BASE)
    off = 0
    blocks = [(name + ".W", 9 * ci * co) for name, ci, co in ounet.layout(LEVELS, BASE)]
    sizes = []
    for (name, ci, co) in ounet.layout(LEVELS, BASE):
        sizes += [(name + ".W", 9 * ci * co), (name + ".b", co)]
    sizes += [("head.W", BASE * 3), ("head.b", 3)]
    for name, n in sizes:
        e = rel_l2(g[off:off + n], ref[off:off + n])
        assert e <= 5e-2, (name, e)
        off += n
    assert off == g.size and blocks


def test_training_reduces_the_loss():
    from paper_2202_08627_gb300 import ei
    net = ei.UNet(levels=LEVELS, base=BASE, batch=B, height=H, width=W, seed=4)
    x = torch.from_numpy(inputs.uniform_noise((B, H, W, 3), 40, 0.0, 1.0).astype(np.float32)).cuda()
    # target: a smooth, learnable function of the input
    t = 0.5 * x + 0.2 * torch.roll(x, 1, dims=1)
    first = net.train_step(x, t, lr=2e-3)
    for _ in range(200):
        last = net.train_step(x, t, lr=2e-3)
    assert last < 0.1 * first, (first, last)


def test_tensor_paths_agree():
    """tcgen05 and WMMA convolutions differ only in FP32 summation order (and
    the BF16 rounding that follows), on a batch whose last tile is ragged."""
    x = torch.from_numpy(inputs.uniform_noise((B, H, W, 3), 40, 0.0, 1.0).astype(np.float32)).cuda()
    outs = []
    for path in (1, 0):
        net, _ = _net_and_params(path)
        outs.append(net.forward(x).cpu().numpy().astype(np.float64))
    xn = x.cpu().numpy()
    assert rel_l2(outs[0] - xn, outs[1] - xn) <= 1e-2
