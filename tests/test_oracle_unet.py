"""Pins for the FP64 network oracle (oracle/unet.py): independent library convolution,
finite differences, adjoint identities, bfloat16 rounding cases, AdamW's first step."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv3_matches_torch_conv3d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 6, 5, 7, 3))
    w = rng.standard_normal((27, 3, 4))
    b = rng.standard_normal(4)
    y = U.conv3(x, w, b)
    wt = np.zeros((4, 3, 3, 3, 3))
    for t, (dz, dy, dx) in enumerate(U.TAPS):
        wt[:, :, dz + 1, dy + 1, dx + 1] = w[t].T
    ref = torch.nn.functional.conv3d(torch.from_numpy(x).permute(0, 4, 1, 2, 3), torch.from_numpy(wt),
                                     torch.from_numpy(b), padding=1).permute(0, 2, 3, 4, 1).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 6, 8, 3))
    yc = rng.standard_normal((2, 2, 3, 4, 3))
    assert np.sum(U.pool2(x) * yc) == pytest.approx(np.sum(x * U.pool2_backward(yc, None)), rel=1e-12)
    xc = rng.standard_normal((2, 2, 3, 4, 3))
    yf = rng.standard_normal((2, 4, 6, 8, 3))
    assert np.sum(U.up2(xc) * yf) == pytest.approx(np.sum(xc * U.up2_backward(yf)), rel=1e-12)


def test_conv3_backward_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 5, 3, 2))
    w = rng.standard_normal((27, 2, 3))
    g = rng.standard_normal((1, 4, 5, 3, 3))
    gx, gw, gb = U.conv3_backward(x, w, g)
    # <conv(x), g> is linear in x and in w: its gradients are gx and gw
    lhs = np.sum(U.conv3(x, w, np.zeros(3)) * g)
    assert lhs == pytest.approx(np.sum(x * gx), rel=1e-12)
    assert lhs == pytest.approx(np.sum(w * gw), rel=1e-12)


def test_network_gradient_matches_finite_differences():
    cin, cout, ch = 3, 2, (2, 3, 2, 2)
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(U.n_params(cin, cout, ch)) * 0.4
    x = rng.standard_normal((1, 8, 8, 8, cin))
    t = rng.standard_normal((1, 8, 8, 8, cout))
    mask = (rng.random((1, 8, 8, 8)) > 0.4).astype(float)
    L, g = U.loss_and_grad(theta, x, t, mask, cin, cout, ch)
    assert L == pytest.approx(U.loss(U.forward(theta, x, cin, cout, ch), t, mask), rel=1e-14)
    h = 1e-6
    for i in rng.choice(theta.size, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (U.loss(U.forward(tp, x, cin, cout, ch), t, mask) - U.loss(U.forward(tm, x, cin, cout, ch), t, mask)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-4, abs=1e-9), i


def test_bf16_rounding_ties_to_even():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -9, -2.5, 3.14159265])
    got = U.bf16_round(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0                    # halfway, mantissa of 1.0 is even
    assert got[2] == 1 + 2 ** -6            # halfway, rounds to the even neighbour above
    assert got[3] == 1.0
    assert got[4] == -2.5
    assert got[5] == 3.140625               # 8 significant bits


def test_adamw_first_step_is_sign_descent():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = U.adamw(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(new, theta - 0.01 * np.sign(g), rtol=1e-9)
    new2, _, _ = U.adamw(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12, wd=0.1)
    np.testing.assert_allclose(new2, theta - 0.01 * (np.sign(g) + 0.1 * theta), rtol=1e-9)
