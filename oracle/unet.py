"""FP64 CPU oracle of the learned surrogate (test infrastructure only).

A plain NumPy restatement of the U-Net that ``include/evsur.h`` specifies, with
hand-written adjoints: periodic 3x3 convolutions with bias and SiLU, 2x2
average pooling, 2x2 stride-2 transposed convolutions, skip concatenation, a
1x1 head and the mean-squared loss on the normalised increment.  Tensors are
NHWC float64 arrays [batch][y][x][channel].  Only tests, the package's smoke
check and the benchmark's CPU baseline use this module; it shares no code with
the CUDA path.

Pins (tests/test_oracle_unet.py): the 3x3 convolution against an FFT circular
cross-correlation; pooling against a block mean; the transposed convolution and
every backward routine against adjoint identities and central finite
differences of the loss; Adam's first step against its closed form; the whole
network's translation equivariance by multiples of 8 pixels.
"""
from __future__ import annotations

import numpy as np

# Architecture (same tables as the header): 3x3 convolutions in execution order,
# transposed convolutions u2 u1 u0, head width.
CONV_IO = ((8, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256),
           (256, 128), (128, 128), (128, 64), (64, 64), (64, 32), (32, 32))
UP_IO = ((256, 128), (128, 64), (64, 32))
BASE = 32
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]   # tap = (dy+1)*3 + (dx+1)


def kp_of(cin):
    return -(-9 * cin // 64) * 64


def unpack(theta):
    """Canonical parameter vector -> dict of arrays.

    conv i: 'cW{i}' [9][Cin][Cout] (tap, ci, co), 'cb{i}' [Cout];
    up j:   'uW{j}' [4][Cout][Cin] (child s = 2 di + dj, co, ci), 'ub{j}' [Cout];
    head:   'hW' [4][BASE], 'hb' [4]."""
    theta = np.asarray(theta, dtype=np.float64)
    P, off = {}, 0
    for i, (ci, co) in enumerate(CONV_IO):
        kp = kp_of(ci)
        w = theta[off:off + kp * co].reshape(kp, co)
        P[f"cW{i}"] = w[:9 * ci].reshape(9, ci, co)
        off += kp * co
        P[f"cb{i}"] = theta[off:off + co]
        off += co
    for j, (ci, co) in enumerate(UP_IO):
        P[f"uW{j}"] = theta[off:off + 4 * co * ci].reshape(4, co, ci)
        off += 4 * co * ci
        P[f"ub{j}"] = theta[off:off + co]
        off += co
    P["hW"] = theta[off:off + 4 * BASE].reshape(4, BASE)
    off += 4 * BASE
    P["hb"] = theta[off:off + 4]
    off += 4
    P["_n"] = off
    return P


def pack(P, n):
    """Inverse of unpack (padded rows zero)."""
    theta, off = np.zeros(n), 0
    for i, (ci, co) in enumerate(CONV_IO):
        kp = kp_of(ci)
        w = np.zeros((kp, co))
        w[:9 * ci] = P[f"cW{i}"].reshape(9 * ci, co)
        theta[off:off + kp * co] = w.ravel()
        off += kp * co
        theta[off:off + co] = P[f"cb{i}"]
        off += co
    for j, (ci, co) in enumerate(UP_IO):
        theta[off:off + 4 * co * ci] = P[f"uW{j}"].ravel()
        off += 4 * co * ci
        theta[off:off + co] = P[f"ub{j}"]
        off += co
    theta[off:off + 4 * BASE] = P["hW"].ravel()
    off += 4 * BASE
    theta[off:off + 4] = P["hb"]
    return theta


# ---------------------------------------------------------------------------
# Layers and their adjoints
# ---------------------------------------------------------------------------

def shift(x, dy, dx):
    """s[b, y, x] = x[b, (y + dy) mod H, (x + dx) mod W]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3(x, W, b):
    """z[b,y,x,co] = b[co] + sum_{tap,ci} W[tap,ci,co] x[b, y+dy, x+dx, ci] (periodic)."""
    z = np.zeros(x.shape[:3] + (W.shape[2],))
    for t, (dy, dx) in enumerate(TAPS):
        z += shift(x, dy, dx) @ W[t]
    return z + b


def conv3_bwd_input(dz, W):
    """Adjoint of conv3 in x: dx[p] = sum_tap W[tap] dz[p - s_tap]."""
    dx = np.zeros(dz.shape[:3] + (W.shape[1],))
    for t, (dy, dx_) in enumerate(TAPS):
        dx += shift(dz, -dy, -dx_) @ W[t].T
    return dx


def conv3_bwd_weight(x, dz):
    """dW[tap, ci, co] = sum_p x[p + s_tap, ci] dz[p, co]; db[co] = sum_p dz[p, co]."""
    C = x.shape[3]
    dW = np.zeros((9, C, dz.shape[3]))
    for t, (dy, dx) in enumerate(TAPS):
        dW[t] = shift(x, dy, dx).reshape(-1, C).T @ dz.reshape(-1, dz.shape[3])
    return dW, dz.reshape(-1, dz.shape[3]).sum(0)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def pool2(x):
    """2x2 average pooling."""
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_bwd(dy):
    """Adjoint of pool2: every child receives a quarter."""
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2)


def tconv2(x, W, b):
    """y[b, 2i+di, 2j+dj, co] = b[co] + sum_ci W[2di+dj, co, ci] x[b, i, j, ci]."""
    B, h, w, _ = x.shape
    co = W.shape[1]
    y = np.zeros((B, 2 * h, 2 * w, co))
    for s in range(4):
        di, dj = divmod(s, 2)
        y[:, di::2, dj::2, :] = x @ W[s].T + b
    return y


def tconv2_bwd(x, dy, W):
    """Adjoints of tconv2: dx, dW, db."""
    dx = np.zeros(x.shape)
    dW = np.zeros(W.shape)
    C = x.shape[3]
    for s in range(4):
        di, dj = divmod(s, 2)
        g = dy[:, di::2, dj::2, :]
        dx += g @ W[s]
        dW[s] = g.reshape(-1, g.shape[3]).T @ x.reshape(-1, C)
    return dx, dW, dy.reshape(-1, dy.shape[3]).sum(0)


# ---------------------------------------------------------------------------
# The network
# ---------------------------------------------------------------------------

def fields_to_nhwc(F, B, H, W):
    """Planar fields [4][B*H*W] -> [B][H][W][4]."""
    return np.asarray(F, dtype=np.float64).reshape(4, B, H, W).transpose(1, 2, 3, 0)


def nhwc_to_fields(X):
    return X.transpose(3, 0, 1, 2).reshape(4, -1)


def forward(P, x_fields, B, H, W, norm):
    """Network output o [B][H][W][4] and the cache for backward.
    norm = (in_mean[4], in_scale[4], out_scale[4])."""
    mean, scale, _ = (np.asarray(v, dtype=np.float64) for v in norm)
    x = fields_to_nhwc(x_fields, B, H, W)
    xin = np.zeros((B, H, W, 8))
    xin[..., :4] = (x - mean) / scale
    c = {"xin": xin}

    def conv(i, inp):
        z = conv3(inp, P[f"cW{i}"], P[f"cb{i}"])
        c[f"in{i}"], c[f"z{i}"] = inp, z
        return silu(z)

    y00 = conv(0, xin)
    y01 = conv(1, y00)
    y10 = conv(2, pool2(y01))
    y11 = conv(3, y10)
    y20 = conv(4, pool2(y11))
    y21 = conv(5, y20)
    y30 = conv(6, pool2(y21))
    y31 = conv(7, y30)
    c["u0in"] = y31
    cat2 = np.concatenate([y21, tconv2(y31, P["uW0"], P["ub0"])], axis=3)
    y22 = conv(8, cat2)
    y23 = conv(9, y22)
    c["u1in"] = y23
    cat1 = np.concatenate([y11, tconv2(y23, P["uW1"], P["ub1"])], axis=3)
    y12 = conv(10, cat1)
    y13 = conv(11, y12)
    c["u2in"] = y13
    cat0 = np.concatenate([y01, tconv2(y13, P["uW2"], P["ub2"])], axis=3)
    y02 = conv(12, cat0)
    y03 = conv(13, y02)
    c["y03"] = y03
    o = y03 @ P["hW"].T + P["hb"]
    return o, c


def loss_and_grad(P, x_fields, y_fields, B, H, W, norm):
    """Loss = mean over pixels and channels of (o - (y - x)/out_scale)^2, and
    its gradient as a dict shaped like P."""
    out_scale = np.asarray(norm[2], dtype=np.float64)
    o, c = forward(P, x_fields, B, H, W, norm)
    x = fields_to_nhwc(x_fields, B, H, W)
    y = fields_to_nhwc(y_fields, B, H, W)
    r = o - (y - x) / out_scale
    n = r.size
    loss = float((r * r).sum() / n)
    G, _ = backward(P, c, 2.0 * r / n)
    return loss, G, o


def backward(P, c, do, need_dxin=False):
    """Gradients of the parameters given do = dL/do [B][H][W][4] and the cache of
    forward; with need_dxin also dL/dxin, the gradient in the normalised input
    [B][H][W][8] (channels 4..7 are the zero padding)."""
    G = {"hW": do.reshape(-1, 4).T @ c["y03"].reshape(-1, BASE), "hb": do.reshape(-1, 4).sum(0)}
    dy = do @ P["hW"]

    def conv_b(i, dy_, need_dx=True):
        dz = dy_ * silu_grad(c[f"z{i}"])
        G[f"cW{i}"], G[f"cb{i}"] = conv3_bwd_weight(c[f"in{i}"], dz)
        return conv3_bwd_input(dz, P[f"cW{i}"]) if need_dx else None

    def up_b(j, inp, dcat_up):
        dx, G[f"uW{j}"], G[f"ub{j}"] = tconv2_bwd(inp, dcat_up, P[f"uW{j}"])
        return dx

    d02 = conv_b(13, dy)
    dcat0 = conv_b(12, d02)
    d13 = up_b(2, c["u2in"], dcat0[..., 32:])
    d12 = conv_b(11, d13)
    dcat1 = conv_b(10, d12)
    d23 = up_b(1, c["u1in"], dcat1[..., 64:])
    d22 = conv_b(9, d23)
    dcat2 = conv_b(8, d22)
    d31 = up_b(0, c["u0in"], dcat2[..., 128:])
    d30 = conv_b(7, d31)
    dp2 = conv_b(6, d30)
    d21 = dcat2[..., :128] + pool2_bwd(dp2)
    d20 = conv_b(5, d21)
    dp1 = conv_b(4, d20)
    d11 = dcat1[..., :64] + pool2_bwd(dp1)
    d10 = conv_b(3, d11)
    dp0 = conv_b(2, d10)
    d01 = dcat0[..., :32] + pool2_bwd(dp0)
    d00 = conv_b(1, d01)
    dxin = conv_b(0, d00, need_dx=need_dxin)
    return G, dxin


def unrolled_loss_and_grad(P, x0_fields, targets, B, H, W, norm):
    """Training loss of k windows applied to the network's own predictions:
    x'_0 = x_0, x'_{j+1} = x'_j + out_scale * o(x'_j), and
    L = (1/k) sum_{j=1..k} mean over pixels and channels of ((x'_j - y_j)/out_scale)^2
    for targets y_1..y_k (planar [k][4][B*H*W]); k = 1 is loss_and_grad.  Returns
    (L, gradient dict shaped like P, dL/dx_0 planar [4][B*H*W]).  Backpropagation
    through the chain: dL/dx'_j = (its loss term) + dL/dx'_{j+1} (the identity path)
    + the network path, whose input gradient is dL/dxin / in_scale."""
    _, in_scale, out_scale = (np.asarray(v, dtype=np.float64) for v in norm)
    k = len(targets)
    xs = [np.asarray(x0_fields, dtype=np.float64)]
    for _ in range(k):
        xs.append(predict(P, xs[-1], B, H, W, norm))
    n = 4 * B * H * W
    loss = 0.0
    Gx = np.zeros((4, B * H * W))                     # dL/dx'_j, planar
    Gsum = None
    for j in range(k, 0, -1):
        r = (xs[j] - np.asarray(targets[j - 1], dtype=np.float64)) / out_scale[:, None]
        loss += float((r * r).sum()) / (n * k)
        Gx = Gx + 2.0 * r / out_scale[:, None] / (n * k)
        _, c = forward(P, xs[j - 1], B, H, W, norm)
        do = fields_to_nhwc(Gx * out_scale[:, None], B, H, W)      # x'_j = x'_{j-1} + out_scale o
        G, dxin = backward(P, c, do, need_dxin=True)
        Gsum = G if Gsum is None else {key: Gsum[key] + G[key] for key in G}
        Gx = Gx + nhwc_to_fields(dxin[..., :4]) / in_scale[:, None]
    return loss, Gsum, Gx


def predict(P, x_fields, B, H, W, norm):
    """Next-state fields x + out_scale * o, planar [4][B*H*W]."""
    o, _ = forward(P, x_fields, B, H, W, norm)
    return np.asarray(x_fields, dtype=np.float64) + nhwc_to_fields(o) * np.asarray(norm[2])[:, None]


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (returns new w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
