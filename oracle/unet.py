"""FP64 NumPy U-Net for checking the library's learned warm start.

TEST INFRASTRUCTURE (see the package docstring).  Same topology and
parameter order as the library's network (include/ei.h): per encoder level
two 3x3 conv + ReLU with 2x2 average pooling between levels; per decoder
level (L-2 .. 0) nearest 2x upsampling, 3x3 conv + ReLU, 3x3 conv + ReLU over
the concatenation [upsampled path, skip], 3x3 conv + ReLU; a 1x1 head;
output = input + head.  Tensors are NHWC; conv weights [tap][c_in][c_out]
with tap = 3 dy + dx for the offset (dy - 1, dx - 1); the input is padded to
32 channels with zeros.

With bf16=True the forward pass rounds, like the GPU, the weights and every
stored activation to BF16 (round to nearest even) — the arithmetic in
between stays FP64.
"""
from __future__ import annotations

import numpy as np

IN_CHANNELS = 32


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3x3 convolution with zero padding: y[p] = sum_tap x[p + off(tap)] @ W[tap] + b."""
    B, H, Wd, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[2]))
    for t in range(9):
        a, c = divmod(t, 3)
        y += xp[:, a:a + H, c:c + Wd, :] @ W[t]
    return y + b


def conv3_backward(x: np.ndarray, W: np.ndarray, gy: np.ndarray):
    """(gx, gW, gb) of conv3."""
    B, H, Wd, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for t in range(9):
        a, c = divmod(t, 3)
        gW[t] = np.einsum("bhwi,bhwo->io", xp[:, a:a + H, c:c + Wd, :], gy)
        gxp[:, a:a + H, c:c + Wd, :] += gy @ W[t].T
    return gxp[:, 1:1 + H, 1:1 + Wd, :], gW, gy.sum(axis=(0, 1, 2))


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(gy):
    B, H, W, C = gy.shape
    return gy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def layout(levels: int, base: int):
    """[(name, c_in, c_out)] of the convs in creation order."""
    ch = [base << l for l in range(levels)]
    convs = []
    for l in range(levels):
        convs.append(("enc1_%d" % l, IN_CHANNELS if l == 0 else ch[l - 1], ch[l]))
        convs.append(("enc2_%d" % l, ch[l], ch[l]))
    for d in range(levels - 2, -1, -1):
        convs.append(("dup_%d" % d, ch[d + 1], ch[d]))
        convs.append(("da_%d" % d, 2 * ch[d], ch[d]))
        convs.append(("db_%d" % d, ch[d], ch[d]))
    return convs


def unpack(flat: np.ndarray, levels: int, base: int):
    """Split the flat parameter vector (export order) into a dict."""
    p, off = {}, 0
    for name, ci, co in layout(levels, base):
        n = 9 * ci * co
        p[name + ".W"] = flat[off:off + n].reshape(9, ci, co)
        off += n
        p[name + ".b"] = flat[off:off + co]
        off += co
    p["head.W"] = flat[off:off + base * 3].reshape(base, 3)
    off += base * 3
    p["head.b"] = flat[off:off + 3]
    off += 3
    assert off == flat.size
    return p


def pack(grads: dict, levels: int, base: int) -> np.ndarray:
    out = []
    for name, ci, co in layout(levels, base):
        out.append(grads[name + ".W"].ravel())
        out.append(grads[name + ".b"].ravel())
    out.append(grads["head.W"].ravel())
    out.append(grads["head.b"].ravel())
    return np.concatenate(out)


def forward(x: np.ndarray, params: dict, levels: int, bf16: bool = False, cache: dict | None = None):
    """y = x + head(net(x)); x, y [B][H][W][3]."""
    rnd = bf16_round if bf16 else (lambda a: a)
    P = {k: (rnd(v) if k.endswith(".W") and not k.startswith("head") else v) for k, v in params.items()}
    c = {} if cache is None else cache
    B, H, W, _ = x.shape
    xin = np.zeros((B, H, W, IN_CHANNELS))
    xin[..., :3] = x
    xin = rnd(xin)
    c["in"] = xin

    def conv_relu(name, inp):
        return rnd(np.maximum(conv3(inp, P[name + ".W"], P[name + ".b"]), 0.0))

    src = xin
    for l in range(levels):
        c["src%d" % l] = src
        c["e1_%d" % l] = conv_relu("enc1_%d" % l, src)
        c["e2_%d" % l] = conv_relu("enc2_%d" % l, c["e1_%d" % l])
        if l < levels - 1:
            src = rnd(pool2(c["e2_%d" % l]))
    cur = c["e2_%d" % (levels - 1)]
    for d in range(levels - 2, -1, -1):
        c["u%d" % d] = up2(cur)
        c["dup%d" % d] = conv_relu("dup_%d" % d, c["u%d" % d])
        c["cat%d" % d] = np.concatenate([c["dup%d" % d], c["e2_%d" % d]], axis=-1)
        c["da%d" % d] = conv_relu("da_%d" % d, c["cat%d" % d])
        c["db%d" % d] = conv_relu("db_%d" % d, c["da%d" % d])
        cur = c["db%d" % d]
    c["top"] = cur
    return x + cur @ P["head.W"] + P["head.b"]


def backward(x: np.ndarray, params: dict, levels: int, gy: np.ndarray, bf16: bool = False):
    """Gradients of sum(gy * y) with respect to every parameter (dict)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    P = {k: (rnd(v) if k.endswith(".W") and not k.startswith("head") else v) for k, v in params.items()}
    c = {}
    forward(x, params, levels, bf16, c)
    g = {}
    g["head.W"] = np.einsum("bhwc,bhwk->ck", c["top"], gy)
    g["head.b"] = gy.sum(axis=(0, 1, 2))
    gcur = gy @ P["head.W"].T

    def conv_back(name, inp, out, gout):
        gout = gout * (out > 0)
        gx, g[name + ".W"], g[name + ".b"] = conv3_backward(inp, P[name + ".W"], gout)
        return gx

    ge2 = {}
    for d in range(0, levels - 1):
        gda = conv_back("db_%d" % d, c["da%d" % d], c["db%d" % d], gcur)
        gcat = conv_back("da_%d" % d, c["cat%d" % d], c["da%d" % d], gda)
        cd = c["dup%d" % d].shape[-1]
        gdup, ge2[d] = gcat[..., :cd], gcat[..., cd:]
        gu = conv_back("dup_%d" % d, c["u%d" % d], c["dup%d" % d], gdup)
        gcur = up2_backward(gu)
    ge2[levels - 1] = gcur
    for l in range(levels - 1, -1, -1):
        ge1 = conv_back("enc2_%d" % l, c["e1_%d" % l], c["e2_%d" % l], ge2[l])
        gsrc = conv_back("enc1_%d" % l, c["src%d" % l], c["e1_%d" % l], ge1)
        if l > 0:
            ge2[l - 1] = ge2[l - 1] + pool2_backward(gsrc)
    return g
