"""Pins for the oracle's U-Net (the checker of the learned warm start).

Anchors: the convolution against explicit loops; the backward passes of the
convolution, pooling and upsampling by their adjoint identities; the whole
network's parameter gradient against central finite differences (FP64);
BF16 rounding on values whose nearest BF16 is known.
"""
import numpy as np

from oracle import unet
from paper_2202_08627_gb300 import inputs


def test_conv3_matches_loops():
    x = inputs.uniform_noise((2, 4, 5, 3), 1)
    W = inputs.uniform_noise((9, 3, 4), 2)
    b = inputs.uniform_noise(4, 3)
    y = unet.conv3(x, W, b)
    ref = np.zeros((2, 4, 5, 4))
    for bb in range(2):
        for i in range(4):
            for j in range(5):
                for t in range(9):
                    ii, jj = i + t // 3 - 1, j + t % 3 - 1
                    if 0 <= ii < 4 and 0 <= jj < 5:
                        ref[bb, i, j] += x[bb, ii, jj] @ W[t]
                ref[bb, i, j] += b
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13)


def test_conv3_backward_adjoint_identities():
    x = inputs.uniform_noise((2, 6, 4, 5), 4)
    W = inputs.uniform_noise((9, 5, 3), 5)
    gy = inputs.uniform_noise((2, 6, 4, 3), 6)
    gx, gW, gb = unet.conv3_backward(x, W, gy)
    y0 = unet.conv3(x, W, np.zeros(3))
    assert abs(np.vdot(y0, gy) - np.vdot(x, gx)) <= 1e-12 * abs(np.vdot(y0, gy))
    assert abs(np.vdot(y0, gy) - np.vdot(W, gW)) <= 1e-12 * abs(np.vdot(y0, gy))
    np.testing.assert_allclose(gb, gy.sum(axis=(0, 1, 2)), rtol=1e-14)


def test_pool_and_upsample_adjoints():
    x = inputs.uniform_noise((2, 4, 6, 3), 7)
    y = inputs.uniform_noise((2, 2, 3, 3), 8)
    assert abs(np.vdot(unet.pool2(x), y) - np.vdot(x, unet.pool2_backward(y))) < 1e-12
    z = inputs.uniform_noise((2, 4, 6, 3), 9)
    assert abs(np.vdot(unet.up2(y), z) - np.vdot(y, unet.up2_backward(z))) < 1e-12


def test_network_gradient_finite_differences():
    levels, base = 2, 32
    n = sum(9 * ci * co + co for _, ci, co in unet.layout(levels, base)) + base * 3 + 3
    flat = 0.3 * inputs.uniform_noise(n, 10)
    params = unet.unpack(flat, levels, base)
    x = inputs.uniform_noise((1, 4, 4, 3), 11)
    gy = inputs.uniform_noise((1, 4, 4, 3), 12)
    g = unet.pack(unet.backward(x, params, levels, gy), levels, base)
    rng = np.random.Generator(np.random.PCG64(13))
    h = 1e-6
    for idx in rng.choice(n, size=25, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[idx] += h
        fm[idx] -= h
        Lp = np.vdot(unet.forward(x, unet.unpack(fp, levels, base), levels), gy)
        Lm = np.vdot(unet.forward(x, unet.unpack(fm, levels, base), levels), gy)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1.0 + 2 ** -9, 3.0e-5])
    got = unet.bf16_round(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    np.testing.assert_array_equal(got[:5], [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0])
    assert abs(got[5] - 3.0e-5) <= 3.0e-5 * 2 ** -8
