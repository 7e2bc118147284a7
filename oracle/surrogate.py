"""CPU oracle of the learned surrogate network (test infrastructure only).

A convolutional encoder-decoder that maps a density grid to a displacement
field.  Plain numpy, FP64, with the tensors that the GPU keeps in bfloat16
(inputs, weights, every layer's stored output, every layer's output
gradient) rounded to bfloat16 at the same points, so that the GPU's forward
and backward passes can be compared with it element by element.

Architecture (``levels`` L, base width ``c0``; widths c_l = c0 * 2^l):

    encoder, l = 0 .. L-1:   h = relu(conv(x)); h = relu(conv(h)); skip_l = h;
                             x = avgpool2(h) (not after the last level)
    decoder, l = L-2 .. 0:   u = relu(conv(upsample2(x)));  x = relu(conv(u + skip_l))
    head:                    out = conv(x)   (2 channels, no activation)
                             [+ skip * skip_field, a fixed skip of an input field]

conv is a 3x3 cross-correlation with zero padding and a bias; tensors are
[batch, height, width, channels]; weights are [out, 3, 3, in].  The loss is
0.5 * mean((out - target)^2).

Pins (tests/test_oracle_surrogate.py): conv against scipy's 2-D correlation,
the backward pass against central finite differences of the forward pass,
pool / upsample adjointness.
"""

from __future__ import annotations

import numpy as np

__all__ = ["bf16", "layer_shapes", "init_params", "forward", "backward", "conv3x3", "conv3x3_backward",
           "avgpool2", "avgpool2_backward", "upsample2", "upsample2_backward", "mse_loss"]


def bf16(a, enable: bool = True):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    a = np.asarray(a, dtype=np.float64)
    if not enable:
        return a
    f = a.astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def layer_shapes(levels: int, c0: int, c_in: int = 1, c_out: int = 2):
    """Ordered (name, c_out, c_in) of every conv layer."""
    ch = [c0 * (2 ** l) for l in range(levels)]
    shapes = []
    cin = c_in
    for l in range(levels):
        shapes.append((f"enc{l}a", ch[l], cin))
        shapes.append((f"enc{l}b", ch[l], ch[l]))
        cin = ch[l]
    for l in range(levels - 2, -1, -1):
        shapes.append((f"dec{l}up", ch[l], ch[l + 1]))
        shapes.append((f"dec{l}c", ch[l], ch[l]))
    shapes.append(("head", c_out, ch[0]))
    return shapes


def init_params(levels: int, c0: int, seed: int = 0, c_in: int = 1, c_out: int = 2):
    """He-normal weights, small biases (float64)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, co, ci in layer_shapes(levels, c0, c_in, c_out):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if name == "head" else 1.0)
        P[name + ".w"] = rng.normal(0.0, std, size=(co, 3, 3, ci))
        P[name + ".b"] = rng.normal(0.0, 0.01, size=(co,))
    return P


def conv3x3(x, w, b):
    """out[n, i, j, o] = b[o] + sum_{dy, dx, c} x[n, i + dy - 1, j + dx - 1, c] w[o, dy, dx, c]."""
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, W, w.shape[0]))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("bhwc,oc->bhwo", xp[:, dy:dy + H, dx:dx + W, :], w[:, dy, dx, :])
    return out + b


def conv3x3_backward(x, w, dout):
    """Gradients of conv3x3 with respect to x, w and b."""
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            dw[:, dy, dx, :] = np.einsum("bhwo,bhwc->oc", dout, xp[:, dy:dy + H, dx:dx + W, :])
            dxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("bhwo,oc->bhwc", dout, w[:, dy, dx, :])
    db = dout.sum(axis=(0, 1, 2))
    return dxp[:, 1:-1, 1:-1, :], dw, db


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dout):
    return np.repeat(np.repeat(dout, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dout):
    B, H, W, C = dout.shape
    return dout.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse_loss(out, target):
    d = out - target
    return 0.5 * float(np.mean(d * d)), d / d.size


def forward(P, x, levels: int, round_bf16: bool = True, skip: float = 0.0, skip_field=None):
    """Forward pass; returns (output float64, cache for backward).  With
    skip_field ([batch, H, W, 2], not rounded), skip * skip_field is added to
    the output (it holds no parameters, so backward is unchanged)."""
    r = lambda a: bf16(a, round_bf16)  # noqa: E731
    W = {k: (r(v) if k.endswith(".w") else v) for k, v in P.items()}
    cache = {"x": r(x)}
    h = cache["x"]
    skips = []
    for l in range(levels):
        za = conv3x3(h, W[f"enc{l}a.w"], W[f"enc{l}a.b"])
        ya = r(np.maximum(za, 0.0))
        zb = conv3x3(ya, W[f"enc{l}b.w"], W[f"enc{l}b.b"])
        yb = r(np.maximum(zb, 0.0))
        cache[f"enc{l}a.in"], cache[f"enc{l}a.out"] = h, ya
        cache[f"enc{l}b.in"], cache[f"enc{l}b.out"] = ya, yb
        skips.append(yb)
        h = r(avgpool2(yb)) if l < levels - 1 else yb
    for l in range(levels - 2, -1, -1):
        u = upsample2(h)
        zu = conv3x3(u, W[f"dec{l}up.w"], W[f"dec{l}up.b"])
        yu = r(np.maximum(zu, 0.0))
        s = r(yu + skips[l])
        zc = conv3x3(s, W[f"dec{l}c.w"], W[f"dec{l}c.b"])
        yc = r(np.maximum(zc, 0.0))
        cache[f"dec{l}up.in"], cache[f"dec{l}up.out"] = u, yu
        cache[f"dec{l}c.in"], cache[f"dec{l}c.out"] = s, yc
        h = yc
    out = conv3x3(h, W["head.w"], W["head.b"])
    if skip_field is not None and skip != 0.0:
        out = out + skip * np.asarray(skip_field, dtype=np.float64)
    cache["head.in"] = h
    cache["W"] = W
    return out, cache


def backward(cache, dout, levels: int, round_bf16: bool = True):
    """Gradients of all parameters given d(loss)/d(out)."""
    r = lambda a: bf16(a, round_bf16)  # noqa: E731
    W = cache["W"]
    G = {}
    g = r(dout)
    dh, G["head.w"], G["head.b"] = conv3x3_backward(cache["head.in"], W["head.w"], g)
    dskip = {}
    # the decoder ran l = L-2 .. 0, so its gradients flow back l = 0 .. L-2
    for l in range(0, levels - 1):
        dz = r(dh * (cache[f"dec{l}c.out"] > 0))
        ds, G[f"dec{l}c.w"], G[f"dec{l}c.b"] = conv3x3_backward(cache[f"dec{l}c.in"], W[f"dec{l}c.w"], dz)
        dskip[l] = ds
        dzu = r(ds * (cache[f"dec{l}up.out"] > 0))
        du, G[f"dec{l}up.w"], G[f"dec{l}up.b"] = conv3x3_backward(cache[f"dec{l}up.in"], W[f"dec{l}up.w"], dzu)
        dh = upsample2_backward(du)
    for l in range(levels - 1, -1, -1):
        dyb = dh + dskip.get(l, 0.0)
        dz = r(dyb * (cache[f"enc{l}b.out"] > 0))
        dya, G[f"enc{l}b.w"], G[f"enc{l}b.b"] = conv3x3_backward(cache[f"enc{l}b.in"], W[f"enc{l}b.w"], dz)
        dz = r(dya * (cache[f"enc{l}a.out"] > 0))
        dx, G[f"enc{l}a.w"], G[f"enc{l}a.b"] = conv3x3_backward(cache[f"enc{l}a.in"], W[f"enc{l}a.w"], dz)
        if l > 0:
            dh = avgpool2_backward(dx)
    return G
