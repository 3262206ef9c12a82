"""Pins of the FP64 U-Net oracle against facts that do not come from the oracle itself:
brute-force loops on tiny inputs, an FFT circular cross-correlation, adjoint identities
<A x, y> = <x, A* y>, central finite differences of the loss, Adam's closed-form first
step and the translation equivariance of the network."""
import numpy as np
import pytest

import oracle.unet as U

rng = np.random.default_rng(7)


def rand_params(scale=0.3):
    n = U.unpack(np.zeros(10_000_000))["_n"]
    P = {}
    for i, (ci, co) in enumerate(U.CONV_IO):
        P[f"cW{i}"] = rng.normal(0, scale / np.sqrt(9 * ci), (9, ci, co))
        P[f"cb{i}"] = rng.normal(0, 0.1, co)
    for j, (ci, co) in enumerate(U.UP_IO):
        P[f"uW{j}"] = rng.normal(0, scale / np.sqrt(ci), (4, co, ci))
        P[f"ub{j}"] = rng.normal(0, 0.1, co)
    P["hW"] = rng.normal(0, 0.3, (4, U.BASE))
    P["hb"] = rng.normal(0, 0.1, 4)
    return P, n


def test_pack_unpack_roundtrip():
    P, n = rand_params()
    theta = U.pack(P, n)
    Q = U.unpack(theta)
    for k in P:
        np.testing.assert_array_equal(P[k], Q[k])
    # 9*sum(Cin*Cout) = 1,753,344 conv weights + 1,408 conv biases + 172,032 transposed-conv
    # weights + 224 biases + 132 head = 1,927,140, plus 5,888 zero rows padding 9 Cin to Kp.
    assert n == 1_933_028


def test_conv3_brute_force():
    x = rng.normal(size=(2, 4, 5, 3))
    W = rng.normal(size=(9, 3, 2))
    b = rng.normal(size=2)
    z = U.conv3(x, W, b)
    B, H, Wd, C = x.shape
    for bb in range(B):
        for y in range(H):
            for xx in range(Wd):
                for co in range(2):
                    s = b[co]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            tap = (dy + 1) * 3 + (dx + 1)
                            s += sum(W[tap, ci, co] * x[bb, (y + dy) % H, (xx + dx) % Wd, ci] for ci in range(C))
                    assert abs(z[bb, y, xx, co] - s) < 1e-12


def test_conv3_against_fft_cross_correlation():
    x = rng.normal(size=(1, 16, 8, 3))
    W = rng.normal(size=(9, 3, 4))
    z = U.conv3(x, W, np.zeros(4))
    H, Wd = 16, 8
    for co in range(4):
        acc = np.zeros((H, Wd))
        for ci in range(3):
            k = np.zeros((H, Wd))
            for tap in range(9):
                dy, dx = tap // 3 - 1, tap % 3 - 1
                k[dy % H, dx % Wd] = W[tap, ci, co]
            acc += np.real(np.fft.ifft2(np.fft.fft2(x[0, :, :, ci]) * np.conj(np.fft.fft2(k))))
        np.testing.assert_allclose(z[0, :, :, co], acc, atol=1e-12)


def test_pool_and_tconv_brute_force():
    x = rng.normal(size=(2, 4, 6, 3))
    p = U.pool2(x)
    for b in range(2):
        for i in range(2):
            for j in range(3):
                np.testing.assert_allclose(p[b, i, j], x[b, 2 * i:2 * i + 2, 2 * j:2 * j + 2].mean(axis=(0, 1)))
    W = rng.normal(size=(4, 5, 3))
    bias = rng.normal(size=5)
    y = U.tconv2(x, W, bias)
    for b in range(2):
        for Y in range(8):
            for X in range(12):
                s = (Y % 2) * 2 + (X % 2)
                np.testing.assert_allclose(y[b, Y, X], W[s] @ x[b, Y // 2, X // 2] + bias, atol=1e-12)


def test_adjoint_identities():
    x = rng.normal(size=(2, 8, 4, 3))
    W = rng.normal(size=(9, 3, 5))
    yz = rng.normal(size=(2, 8, 4, 5))
    lhs = np.sum(U.conv3(x, W, np.zeros(5)) * yz)
    assert abs(lhs - np.sum(x * U.conv3_bwd_input(yz, W))) < 1e-9 * abs(lhs) + 1e-9
    dW, db = U.conv3_bwd_weight(x, yz)
    assert abs(lhs - np.sum(W * dW)) < 1e-9 * abs(lhs) + 1e-9
    np.testing.assert_allclose(db, yz.sum(axis=(0, 1, 2)))
    Wu = rng.normal(size=(4, 5, 3))
    yu = rng.normal(size=(2, 16, 8, 5))
    lhs = np.sum(U.tconv2(x, Wu, np.zeros(5)) * yu)
    dx, dWu, dbu = U.tconv2_bwd(x, yu, Wu)
    assert abs(lhs - np.sum(x * dx)) < 1e-9 * abs(lhs) + 1e-9
    assert abs(lhs - np.sum(Wu * dWu)) < 1e-9 * abs(lhs) + 1e-9
    yp = rng.normal(size=(2, 4, 2, 3))
    assert abs(np.sum(U.pool2(x) * yp) - np.sum(x * U.pool2_bwd(yp))) < 1e-12


def test_silu_grad_matches_difference_quotient():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(U.silu_grad(z), (U.silu(z + h) - U.silu(z - h)) / (2 * h), atol=1e-8)


def _fields(B, H, W):
    x = np.stack([0.1 + 0.05 * rng.random(B * H * W), 0.01 * rng.normal(size=B * H * W),
                  0.01 * rng.normal(size=B * H * W), 0.008 + 0.001 * rng.random(B * H * W)])
    y = x + 0.01 * rng.normal(size=x.shape) * np.array([[0.05], [0.01], [0.01], [0.001]])
    return x, y


NORM = (np.array([0.12, 0.0, 0.0, 0.0085]), np.array([0.05, 0.01, 0.01, 0.001]),
        np.array([0.002, 0.001, 0.001, 0.0001]))


def test_loss_gradient_against_finite_differences():
    B, H, W = 1, 16, 16
    P, n = rand_params(scale=1.0)
    x, y = _fields(B, H, W)
    loss, G, _ = U.loss_and_grad(P, x, y, B, H, W, NORM)
    keys = [k for k in P if not k.startswith("_")]
    checked = 0
    for k in keys:
        idxs = [tuple(rng.integers(0, s) for s in P[k].shape) for _ in range(2)]
        for idx in idxs:
            h = 1e-6 * max(1.0, abs(P[k][idx]))
            old = P[k][idx]
            P[k][idx] = old + h
            lp = U.loss_and_grad(P, x, y, B, H, W, NORM)[0]
            P[k][idx] = old - h
            lm = U.loss_and_grad(P, x, y, B, H, W, NORM)[0]
            P[k][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[k][idx]) <= 1e-5 * abs(G[k][idx]) + 1e-9 * loss, (k, idx, fd, G[k][idx])
            checked += 1
    assert checked == 2 * len(keys)


def _unrolled_loss(P, x0, targets, B, H, W):
    xs = np.asarray(x0, dtype=np.float64)
    out_scale = NORM[2][:, None]
    loss = 0.0
    for yj in targets:
        xs = U.predict(P, xs, B, H, W, NORM)
        r = (xs - yj) / out_scale
        loss += float((r * r).mean()) / len(targets)
    return loss


def test_unrolled_single_window_is_the_window_loss():
    B, H, W = 2, 16, 16
    P, _ = rand_params()
    x, y = _fields(B, H, W)
    l1, G1, _ = U.loss_and_grad(P, x, y, B, H, W, NORM)
    lu, Gu, _ = U.unrolled_loss_and_grad(P, x, [y], B, H, W, NORM)
    assert abs(lu - l1) <= 1e-12 * l1
    for k in G1:
        np.testing.assert_allclose(Gu[k], G1[k], rtol=1e-10, atol=1e-14 * np.abs(G1[k]).max())


def test_unrolled_gradient_against_finite_differences():
    """Three windows chained through the network: the gradient in the parameters (one
    entry of every tensor) and in the start fields (three entries) against central
    differences of the unrolled loss, evaluated with predict() alone."""
    B, H, W = 1, 16, 16
    P, _ = rand_params(scale=1.0)
    x, _ = _fields(B, H, W)
    targets = [x + 0.01 * (j + 1) * rng.normal(size=x.shape) * np.array([[0.05], [0.01], [0.01], [0.001]])
               for j in range(3)]
    loss, G, Gx = U.unrolled_loss_and_grad(P, x, targets, B, H, W, NORM)
    assert abs(loss - _unrolled_loss(P, x, targets, B, H, W)) <= 1e-12 * loss
    keys = [k for k in P if not k.startswith("_")]
    for k in keys:
        idx = tuple(rng.integers(0, s) for s in P[k].shape)
        h = 1e-6 * max(1.0, abs(P[k][idx]))
        old = P[k][idx]
        P[k][idx] = old + h
        lp = _unrolled_loss(P, x, targets, B, H, W)
        P[k][idx] = old - h
        lm = _unrolled_loss(P, x, targets, B, H, W)
        P[k][idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[k][idx]) <= 1e-5 * abs(G[k][idx]) + 1e-9 * loss, (k, idx, fd, G[k][idx])
    for c, m in ((0, 5), (2, 77), (3, 200)):
        h = 1e-7 * max(abs(x[c, m]), NORM[1][c])
        xp, xm = x.copy(), x.copy()
        xp[c, m] += h
        xm[c, m] -= h
        fd = (_unrolled_loss(P, xp, targets, B, H, W) - _unrolled_loss(P, xm, targets, B, H, W)) / (2 * h)
        assert abs(fd - Gx[c, m]) <= 1e-5 * abs(Gx[c, m]) + 1e-7 * loss / NORM[1][c], (c, m, fd, Gx[c, m])


def test_translation_equivariance():
    B, H, W = 1, 32, 32
    P, _ = rand_params()
    x, _ = _fields(B, H, W)
    o1, _ = U.forward(P, x, B, H, W, NORM)
    xs = U.nhwc_to_fields(np.roll(U.fields_to_nhwc(x, B, H, W), shift=(8, 16), axis=(1, 2)))
    o2, _ = U.forward(P, xs, B, H, W, NORM)
    np.testing.assert_allclose(np.roll(o1, shift=(8, 16), axis=(1, 2)), o2, atol=1e-12)


def test_zero_weights_give_head_bias():
    B, H, W = 1, 16, 16
    P, _ = rand_params()
    for k in list(P):
        if k.startswith(("cW", "uW")) or k == "hW":
            P[k] = np.zeros_like(P[k])
    x, _ = _fields(B, H, W)
    o, _ = U.forward(P, x, B, H, W, NORM)
    np.testing.assert_allclose(o, np.broadcast_to(P["hb"], o.shape), atol=0)


def test_adam_first_step_closed_form():
    w = rng.normal(size=100)
    g = rng.normal(size=100)
    w1, m, v = U.adam_step(w, g, np.zeros(100), np.zeros(100), 1, lr=1e-3)
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
