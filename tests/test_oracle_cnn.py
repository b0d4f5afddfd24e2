"""Pins of the oracle's learned-warm-start network (CPU only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.nn.functional as Fnn  # noqa: E402

from oracle import oracle as orc  # noqa: E402

SHAPES = [(4, 32), (32, 32), (32, 4)]


def split(p):
    out, k = [], 0
    for ci, co in SHAPES:
        w = p[k:k + co * ci * 27].reshape(co, ci, 27); k += co * ci * 27
        b = p[k:k + co]; k += co
        out.append((w, b))
    return out


def torch_net(p, x, ncell, per):
    """Independent FP64 evaluation with torch.conv3d (circular / zero padding)."""
    nx, ny, nz = ncell
    h = torch.tensor(x.reshape(1, 4, nz, ny, nx))
    layers = split(p)
    for li, (w, b) in enumerate(layers):
        # pad order for F.pad: (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi)
        for ax, lo_idx in ((0, 0), (1, 2), (2, 4)):  # physical x, y, z
            pad = [0] * 6
            pad[lo_idx] = pad[lo_idx + 1] = 1
            h = Fnn.pad(h, pad, mode="circular" if per[ax] else "constant")
        wt = torch.tensor(w.reshape(w.shape[0], w.shape[1], 3, 3, 3))
        h = Fnn.conv3d(h, wt, torch.tensor(b))
        if li < 2:
            h = torch.relu(h)
    return h.numpy().reshape(4, -1)


def rand_params(seed, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, orc.cnn_num_params())


@pytest.mark.parametrize("per", [(1, 1, 0), (0, 0, 0), (1, 1, 1)])
def test_forward_matches_independent_conv(per):
    ncell = (5, 6, 4)
    rng = np.random.default_rng(1)
    x = rng.normal(0, 1, (4, np.prod(ncell)))
    p = rand_params(2)
    y = orc.cnn_forward(p, x, ncell, per)
    ref = torch_net(p, x, ncell, per)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_identity_network():
    p = np.zeros(orc.cnn_num_params())
    k = 0
    for ci, co in SHAPES:
        w = np.zeros((co, ci, 27))
        for c in range(min(4, ci, co)):
            w[c, c, 13] = 1.0
        p[k:k + co * ci * 27] = w.ravel(); k += co * ci * 27 + co
    x = np.random.default_rng(3).random((4, 3 * 4 * 5))
    assert np.array_equal(orc.cnn_forward(p, x, (3, 4, 5), (1, 1, 0)), x)


def test_translation_equivariance_periodic():
    ncell = (6, 5, 4)
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, (4, 4, 5, 6))
    p = rand_params(5)
    y = orc.cnn_forward(p, x, ncell, (1, 1, 1)).reshape(4, 4, 5, 6)
    xs = np.roll(x, (1, 2, 3), axis=(1, 2, 3))
    ys = orc.cnn_forward(p, xs, ncell, (1, 1, 1)).reshape(4, 4, 5, 6)
    assert np.allclose(np.roll(y, (1, 2, 3), axis=(1, 2, 3)), ys, rtol=0, atol=1e-13)


def test_gradient_finite_difference():
    ncell = (3, 4, 3)
    per = (1, 0, 1)
    rng = np.random.default_rng(6)
    x = rng.normal(0, 1, (4, np.prod(ncell)))
    t = rng.normal(0, 1, (4, np.prod(ncell)))
    p = rand_params(7, 0.3)
    loss, g = orc.cnn_loss_grad(p, x, t, ncell, per)
    y = orc.cnn_forward(p, x, ncell, per)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14 * loss
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for k in idx:
        pp = p.copy(); pp[k] += h
        pm = p.copy(); pm[k] -= h
        fd = (orc.cnn_loss_grad(pp, x, t, ncell, per)[0] - orc.cnn_loss_grad(pm, x, t, ncell, per)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1e-3, abs(g[k])) + 1e-9, k


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5]); g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    orc.adam(p, g, m, v, 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    expect = np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p, expect, rtol=0, atol=1e-15)


def test_bf16_rounding_is_nearest_even():
    # identity network on inputs that need rounding: the stored input is rounded
    p = np.zeros(orc.cnn_num_params())
    k = 0
    for ci, co in SHAPES:
        w = np.zeros((co, ci, 27))
        for c in range(min(4, ci, co)):
            w[c, c, 13] = 1.0
        p[k:k + co * ci * 27] = w.ravel(); k += co * ci * 27 + co
    vals = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -9, 3.0])
    x = np.tile(vals[:, None], (1, 1))
    y = orc.cnn_forward(p, np.repeat(x, 1, axis=1), (1, 1, 1), (0, 0, 0), round_bf16=True)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 and goes to the even 1.0
    assert np.array_equal(y[:, 0], [1.0, 1.0078125, 1.0, 3.0])
