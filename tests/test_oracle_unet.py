"""Pins of the U-Net oracle (learned pressure guess) against definitions that
do not share its code: brute-force loops, scipy's N-d correlation, adjoint
identities and central finite differences of the loss."""
import numpy as np
import pytest
import scipy.signal

from oracle import unet


def _brute_conv(X, W, b):
    nz, ny, nx, cin = X.shape
    cout = W.shape[1]
    Y = np.zeros((nz, ny, nx, cout))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for co in range(cout):
                    s = b[co]
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                kk, jj, ii = k + dz, j + dy, i + dx
                                if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx:
                                    t = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
                                    for ci in range(cin):
                                        s += X[kk, jj, ii, ci] * W[t, co, ci]
                    Y[k, j, i, co] = s
    return Y


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 5, 2))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(unet.conv3(X, W, b), _brute_conv(X, W, b), rtol=1e-12, atol=1e-12)


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((6, 5, 7, 3))
    W = rng.standard_normal((27, 4, 3))
    Y = unet.conv3(X, W)
    for co in range(4):
        ref = np.zeros(X.shape[:3])
        for ci in range(3):
            # kernel K[dz+1, dy+1, dx+1] = W[t, co, ci]
            K = W[:, co, ci].reshape(3, 3, 3)
            ref += scipy.signal.correlate(X[..., ci], K, mode="same", method="direct")
        np.testing.assert_allclose(Y[..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv_back_is_the_adjoint():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 6, 2, 3))
    W = rng.standard_normal((27, 5, 3))
    dY = rng.standard_normal((4, 6, 2, 5))
    dX, dW, db = unet.conv3_back(X, W, dY)
    # <conv(X), dY> = <X, dX>  (linear in X)  and  = <W, dW>  (linear in W)
    lhs = np.sum(unet.conv3(X, W) * dY)
    assert np.isclose(lhs, np.sum(X * dX), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * dW), rtol=1e-12)
    np.testing.assert_allclose(db, dY.sum(axis=(0, 1, 2)), rtol=1e-12)


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4, 6, 8, 3))
    Y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(unet.pool(X) * Y), np.sum(X * unet.up(Y) / 8.0), rtol=1e-12)
    assert np.isclose(np.sum(unet.up(Y) * X), np.sum(Y * unet.up_adjoint(X)), rtol=1e-12)
    # the mean of a constant block is the constant; upsampling then pooling is the identity
    np.testing.assert_allclose(unet.pool(unet.up(Y)), Y, rtol=1e-15)


def test_layout_counts():
    wo, bo, hw, hb, n = unet.layout()
    assert n == sum(27 * ci * co + co for _, ci, co in unet.CONVS) + 17
    assert hb == n - 1 and hw == n - 17
    # decoder inputs are [upsampled coarser output, skip of the same level]
    for q in range(3):
        lev = 2 - q
        low = unet.CONVS[7 + 2 * q][2]
        skip = unet.CONVS[2 * lev + 1][2]
        assert unet.CONVS[8 + 2 * q][1] == low + skip


def test_bf16_rounding():
    # exactly representable values stay, halfway cases go to even
    assert unet.bf16(np.array([1.0]))[0] == 1.0
    one_ulp = 2.0 ** -7
    assert unet.bf16(np.array([1.0 + one_ulp / 2]))[0] == 1.0          # tie -> even (1.0)
    assert unet.bf16(np.array([1.0 + 1.5 * one_ulp]))[0] == 1.0 + 2 * one_ulp   # tie -> even
    assert unet.bf16(np.array([1.0 + 0.6 * one_ulp]))[0] == 1.0 + one_ulp
    x = np.random.default_rng(5).standard_normal(1000)
    assert np.max(np.abs(unet.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_loss_is_mean_free():
    rng = np.random.default_rng(6)
    p = unet.init_params(0)
    planes = rng.standard_normal((4, 8, 8, 8))
    t = rng.standard_normal((8, 8, 8))
    l1, _, _ = unet.loss_and_grad(p, planes, t)
    l2, _, _ = unet.loss_and_grad(p, planes, t + 3.7)
    assert np.isclose(l1, l2, rtol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 8, 8)])
def test_gradient_matches_finite_differences(shape):
    rng = np.random.default_rng(7)
    p = unet.init_params(1)
    wo, bo, hw, hb, n = unet.layout()
    # nonzero biases so that their gradients are exercised
    for c, (_, _, co) in enumerate(unet.CONVS):
        p[bo[c]:bo[c] + co] = 0.05 * rng.standard_normal(co)
    nz, ny, nx = shape
    planes = rng.standard_normal((4, nz, ny, nx))
    t = rng.standard_normal(shape)
    _, g, _ = unet.loss_and_grad(p, planes, t)
    # per layer: the weight and the bias of largest gradient, one random weight
    idx = [hw + 3, hb]
    for c, (_, ci, co) in enumerate(unet.CONVS):
        nw = 27 * ci * co
        idx.append(wo[c] + int(np.argmax(np.abs(g[wo[c]:wo[c] + nw]))))
        idx.append(wo[c] + int(rng.integers(nw)))
        idx.append(bo[c] + int(np.argmax(np.abs(g[bo[c]:bo[c] + co]))))
    h = 1e-6
    nonzero = 0
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (unet.loss_and_grad(pp, planes, t)[0] - unet.loss_and_grad(pm, planes, t)[0]) / (2 * h)
        # central differences: O(h^2) truncation + O(eps_64 L / h) round-off
        assert abs(fd - g[k]) <= 1e-5 * abs(fd) + 3e-10, (k, fd, g[k])
        nonzero += abs(fd) > 1e-8
    assert nonzero >= 2 * len(unet.CONVS)



def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_planted_mistakes_exceed_the_device_tolerances(monkeypatch):
    """Plausible mistakes (mirrored taps, a dropped skip gradient, an
    upsampling adjoint that averages instead of sums) move the output or a
    layer's gradient by far more than the device parity tolerances (5e-3 on
    the output, 0.2 on a layer's gradient)."""
    rng = np.random.default_rng(8)
    nx, ny, nz = 24, 16, 8
    p = unet.init_params(5)
    wo, bo, hw, hb, n = unet.layout()
    for c, (_, _, co) in enumerate(unet.CONVS):
        p[bo[c]:bo[c] + co] = 0.05 * rng.standard_normal(co)
    planes = rng.standard_normal((4, nz, ny, nx))
    t = rng.standard_normal((nz, ny, nx))
    _, g0, o0 = unet.loss_and_grad(p, planes, t, emulate=True)

    def worst_layer(g):
        return max(_rel(g[wo[c]:wo[c] + 27 * ci * co], g0[wo[c]:wo[c] + 27 * ci * co])
                   for c, (_, ci, co) in enumerate(unet.CONVS))

    shift, back, up_adj = unet._shift, unet.conv3_back, unet.up_adjoint
    with monkeypatch.context() as m:     # kernel taps mirrored
        m.setattr(unet, "_shift", lambda Xp, tap, s: shift(Xp, 26 - tap, s))
        _, g1, o1 = unet.loss_and_grad(p, planes, t, emulate=True)

    def drop_skip(X, W, dY):             # decoder input gradient without its skip part
        dX, dW, db = back(X, W, dY)
        if (W.shape[2], W.shape[1]) in ((112, 48), (80, 32), (48, 16)):
            dX = dX.copy()
            dX[..., -W.shape[1]:] = 0.0
        return dX, dW, db
    with monkeypatch.context() as m:
        m.setattr(unet, "conv3_back", drop_skip)
        _, g2, _ = unet.loss_and_grad(p, planes, t, emulate=True)
    with monkeypatch.context() as m:     # upsampling adjoint averaging instead of summing
        m.setattr(unet, "up_adjoint", lambda dY: up_adj(dY) / 8.0)
        _, g3, _ = unet.loss_and_grad(p, planes, t, emulate=True)
    print(f"\nmirrored taps: output {_rel(o1, o0):.2f}, layer {worst_layer(g1):.2f}; "
          f"dropped skip gradient {worst_layer(g2):.2f}; averaging adjoint {worst_layer(g3):.2f}")
    assert _rel(o1, o0) > 0.1
    assert min(worst_layer(g1), worst_layer(g2), worst_layer(g3)) > 0.3
