"""Pins of the CPU reference of the correction network (oracle/net_oracle.py):
the convolution against a direct loop over the definition, and every gradient
against central finite differences."""
import numpy as np
import pytest

from oracle import net_oracle as no


def direct_conv(x, w, b):
    C, H, W = x.shape
    O = w.shape[0]
    y = np.zeros((O, H, W))
    for o in range(O):
        for i in range(H):
            for j in range(W):
                s = b[o]
                for c in range(C):
                    for u in range(3):
                        for v in range(3):
                            ii, jj = i + u - 1, j + v - 1
                            if 0 <= ii < H and 0 <= jj < W:
                                s += w[o, c, u, v] * x[c, ii, jj]
                y[o, i, j] = s
    return y


def test_conv_matches_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 7))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    assert np.max(np.abs(no.conv3x3(x, w, b) - direct_conv(x, w, b))) < 1e-12


def _loss(p, x, t):
    out, _ = no.forward(x, p)
    return no.mse(out, t)[0]


@pytest.mark.parametrize("name", ["w1", "b1", "w2", "b2", "w3", "b3"])
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(1)
    p = no.init_params(3, c_hidden=6, scale=1.0)
    p["w3"] *= 10
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, size=p[k].shape)
    x = rng.normal(size=(3, 6, 5))
    t = rng.normal(size=(3, 6, 5))
    out, cache = no.forward(x, p)
    _, g = no.mse(out, t)
    grads = no.backward(g, cache)
    flat = p[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
    h = 1e-6
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp = _loss(p, x, t)
        flat[i] = old - h
        lm = _loss(p, x, t)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        assert abs(grads[name].reshape(-1)[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, i)


def test_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = rng.normal(size=(4, 3, 3, 3))
    x = rng.normal(size=(3, 5, 4))
    gy = rng.normal(size=(4, 5, 4))
    gx = no.conv3x3_input_grad(gy, w)
    h = 1e-6
    for c, i, j in [(0, 0, 0), (1, 2, 3), (2, 4, 1), (0, 3, 2)]:
        xp = x.copy(); xp[c, i, j] += h
        xm = x.copy(); xm[c, i, j] -= h
        fd = (np.sum(gy * no.conv3x3(xp, w, np.zeros(4))) -
              np.sum(gy * no.conv3x3(xm, w, np.zeros(4)))) / (2 * h)
        assert abs(gx[c, i, j] - fd) < 1e-6


def test_bf16_rounding():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert no.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert no.bf16(np.array([1.0 + 3 * 2 ** -9]))[0] == 1.0 + 2 ** -7
    assert no.bf16(np.array([-2.5]))[0] == -2.5
