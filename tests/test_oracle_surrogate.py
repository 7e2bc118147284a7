"""Pins of the surrogate-network oracle: convolution against scipy's 2-D
correlation, the backward pass against central finite differences of the
forward pass (FP64, no bfloat16 rounding), adjointness of pooling and
upsampling, and the bfloat16 rounding rule."""

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import surrogate as S


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 0.0, 3.14159265], dtype=np.float64)
    r = S.bf16(x)
    assert r[0] == 1.0 and r[3] == -2.5 and r[4] == 0.0
    assert r[1] == 1.0                       # tie -> even
    assert r[2] == 1.0 + 2**-7               # above half -> up
    assert abs(r[5] - 3.140625) < 1e-12      # 8 significant bits
    assert np.all(np.abs(S.bf16(np.random.default_rng(0).normal(size=1000)) -
                         np.random.default_rng(0).normal(size=1000)) <=
                  2**-8 * np.abs(np.random.default_rng(0).normal(size=1000)))


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 9, 7, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    out = S.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.max(np.abs(out[n, :, :, o] - ref)) < 1e-12


def test_pool_upsample_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 4, 6, 3))
    y = rng.normal(size=(2, 8, 12, 3))
    assert abs(np.sum(S.upsample2(x) * y) - np.sum(x * S.upsample2_backward(y))) < 1e-10
    z = rng.normal(size=(2, 8, 12, 3))
    assert abs(np.sum(S.avgpool2(z) * x) - np.sum(z * S.avgpool2_backward(x))) < 1e-10


@pytest.mark.parametrize("levels,c_in,skip", [(2, 1, 0.0), (3, 1, 0.0), (2, 3, 2.5)])
def test_backward_matches_finite_differences(levels, c_in, skip):
    # with three input channels (density and a field) and the output skip
    # skip * field, which holds no parameters: the same gradients must hold
    rng = np.random.default_rng(3 + levels)
    P = S.init_params(levels, 4, seed=levels, c_in=c_in)
    H = 8
    x = rng.random((2, H, H, c_in))
    f = x[..., 1:3] if c_in == 3 else None
    t = rng.normal(size=(2, H, H, 2))

    def loss(PP):
        out, _ = S.forward(PP, x, levels, round_bf16=False, skip=skip, skip_field=f)
        return S.mse_loss(out, t)[0]

    out, cache = S.forward(P, x, levels, round_bf16=False, skip=skip, skip_field=f)
    _, dout = S.mse_loss(out, t)
    G = S.backward(cache, dout, levels, round_bf16=False)
    eps = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            orig = flat[idx]
            flat[idx] = orig + eps
            lp = loss(P)
            flat[idx] = orig - eps
            lm = loss(P)
            flat[idx] = orig
            fd = (lp - lm) / (2 * eps)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)
