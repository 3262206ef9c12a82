"""Surrogate kernels against the FP64 U-Net oracle.

GEMM primitives: every operand kind (dense, implicit 3x3 gather, up-adjoint gather and
their MN-major forms for weight gradients) and every epilogue is compared with the
oracle's layer routines on BF16-exact inputs, at sizes spanning several CTA tiles with
ragged M and K tails.  FP32 outputs: |C - C_ref| <= 2e-6 sum_k |A||B| (FP32 accumulation
of K products, each exact in FP32, has relative error below K * 2^-24 of that sum; the
bound is a few times the expected random-walk value for K <= 2304).  BF16 outputs: one
more rounding, 2^-8 relative.

Whole network: loss, increments and every parameter gradient of the GPU path against
the oracle run with the same BF16-rounded weights.  Activations are BF16 on the GPU, so
each layer adds a relative error of about 2^-9; through the 20 layers of the forward
and the 40 of the backward pass that accumulates (as a random walk) to about 1-2 % --
tolerances: loss 2e-2, relative L2 of each gradient tensor 6e-2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.unet as U
import paper_2508_00577_gb300 as ev
from paper_2508_00577_gb300 import inputs
from paper_2508_00577_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

dev = "cuda"
gen = np.random.default_rng(11)


def bf(a):
    """BF16 device tensor and the exactly representable FP64 copy."""
    t = torch.tensor(np.asarray(a, dtype=np.float32), device=dev).to(torch.bfloat16).contiguous()
    return t, t.float().cpu().numpy().astype(np.float64)


def bf16_round(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def op(t, kind, ld, c0=0, C=0, rows=0, H=0, W=0):
    return S.sur_operand(t.data_ptr(), kind, ld, c0, C, rows, H, W)


def run(args):
    st = torch.zeros(2, dtype=torch.int32, device=dev)
    S.sur_gemm(args, st.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st[0]) == 0


def gemm(a, b, M, N, K, epi=S.SUR_EPI_F32, out=None, ldo=0, co0=0, bias=None, y=None, ldy=0, cy0=0, splits=1,
         shuf=0):
    g = S.sur_gemm_args()
    g.a, g.b, g.M, g.N, g.K, g.splits, g.epi = a, b, M, N, K, splits, epi
    g.bias = bias.data_ptr() if bias is not None else None
    g.out = out.data_ptr() if out is not None else None
    g.ldo, g.co0 = ldo, co0
    g.y = y.data_ptr() if y is not None else None
    g.ldy, g.cy0 = ldy, cy0
    g.shuf_cout = shuf
    run(g)


def close(c, ref, absref, tol=2e-6):
    err = np.abs(c - ref)
    assert np.all(err <= tol * absref + 1e-30), float((err / (absref + 1e-30)).max())


def padded(x):
    """Halo-padded NHWC copy (periodic halo of one pixel)."""
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)), mode="wrap")


def interior(a):
    return a[:, 1:-1, 1:-1, :]


@pytest.fixture(params=[True, False], ids=["tma", "cpasync"])
def tma(request):
    S.sur_set_tma(request.param)
    yield request.param
    S.sur_set_tma(True)


def test_dense_ragged():
    M, N, K = 300, 96, 200
    A, Ad = bf(gen.normal(size=(M, K)))
    B, Bd = bf(gen.normal(size=(N, K)))
    out = torch.full((M, N), float("nan"), device=dev)
    gemm(op(A, S.SUR_OP_DENSE, K, rows=M), op(B, S.SUR_OP_DENSE, K, rows=N), M, N, K, out=out, ldo=N)
    close(out.cpu().numpy(), Ad @ Bd.T, np.abs(Ad) @ np.abs(Bd).T)


@pytest.mark.parametrize("Cin,Cout,c0,ld,H,W", [(32, 64, 0, 32, 16, 32), (8, 32, 8, 16, 16, 32),
                                                 (256, 128, 0, 256, 16, 32), (64, 32, 0, 64, 256, 256),
                                                 (128, 64, 0, 128, 4, 8)])
def test_conv3_gather(Cin, Cout, c0, ld, H, W, tma):
    Bn = 2 if H * W < 65536 else 1
    x = bf16_round(gen.normal(size=(Bn, H, W, ld)))
    X, _ = bf(padded(x))
    Wt, Wd = bf(gen.normal(size=(9, Cin, Cout)) / np.sqrt(9 * Cin))
    kp = U.kp_of(Cin)
    Wb = torch.zeros(Cout, kp, dtype=torch.bfloat16, device=dev)
    Wb[:, :9 * Cin] = Wt.reshape(9 * Cin, Cout).t()
    M = Bn * H * W
    out = torch.full((Bn, H + 2, W + 2, Cout), float("nan"), device=dev)
    gemm(op(X, S.SUR_OP_CONV3, ld, c0, Cin, M, H, W), op(Wb, S.SUR_OP_DENSE, kp, rows=Cout), M, Cout, kp,
         out=out, ldo=Cout)
    xs = x[..., c0:c0 + Cin]
    ref = U.conv3(xs, Wd, np.zeros(Cout))
    absref = U.conv3(np.abs(xs), np.abs(Wd), np.zeros(Cout))
    close(interior(out.cpu().numpy()), ref, absref)


def test_conv_epilogue_bias_silu_halo(tma):
    Bn, H, W, Cin, Cout = 1, 32, 16, 32, 32
    x = bf16_round(gen.normal(size=(Bn, H, W, Cin)))
    X, _ = bf(padded(x))
    Wt, Wd = bf(gen.normal(size=(9, Cin, Cout)) / np.sqrt(9 * Cin))
    bias = torch.tensor(gen.normal(size=Cout), dtype=torch.float32, device=dev)
    kp = U.kp_of(Cin)
    Wb = torch.zeros(Cout, kp, dtype=torch.bfloat16, device=dev)
    Wb[:, :9 * Cin] = Wt.reshape(9 * Cin, Cout).t()
    M = Bn * H * W
    Z = torch.zeros(Bn, H + 2, W + 2, Cout, dtype=torch.bfloat16, device=dev)
    Y = torch.full((Bn, H + 2, W + 2, 2 * Cout), 7.0, dtype=torch.bfloat16, device=dev)
    gemm(op(X, S.SUR_OP_CONV3, Cin, 0, Cin, M, H, W), op(Wb, S.SUR_OP_DENSE, kp, rows=Cout), M, Cout, kp,
         epi=S.SUR_EPI_CONV, out=Z, ldo=Cout, bias=bias, y=Y, ldy=2 * Cout, cy0=0)
    z = U.conv3(x, Wd, bias.cpu().numpy().astype(np.float64))
    zg = interior(Z.float().cpu().numpy())
    assert np.all(np.abs(zg - z) <= 2 ** -8 * np.abs(z) + 1e-5)
    yg = Y.float().cpu().numpy()
    yi = interior(yg)[..., :Cout]
    assert np.all(np.abs(yi - U.silu(z)) <= 2 ** -7 * np.abs(U.silu(z)) + 1e-4)
    # The halo holds the periodic copies of the written channels; the others are untouched.
    np.testing.assert_array_equal(yg[..., :Cout], padded(yi))
    assert np.all(yg[..., Cout:] == 7.0)


def test_tconv_forward_shuffle_epilogue(tma):
    Bn, h, w, Cin, Cout = 2, 8, 16, 64, 32
    x = bf16_round(gen.normal(size=(Bn, h, w, Cin)))
    X, _ = bf(padded(x))
    Wu, Wud = bf(gen.normal(size=(4, Cout, Cin)) / np.sqrt(Cin))
    bias = torch.tensor(gen.normal(size=Cout), dtype=torch.float32, device=dev)
    Mc = Bn * h * w
    cat = torch.full((Bn, 2 * h + 2, 2 * w + 2, 2 * Cout), 3.0, dtype=torch.bfloat16, device=dev)
    gemm(op(X, S.SUR_OP_PIX, Cin, 0, Cin, Mc, h, w), op(Wu.reshape(4 * Cout, Cin), S.SUR_OP_DENSE, Cin, rows=4 * Cout),
         Mc, 4 * Cout, Cin, epi=S.SUR_EPI_SHUF, bias=bias, y=cat, ldy=2 * Cout, cy0=Cout, shuf=Cout)
    ref = U.tconv2(x, Wud, bias.cpu().numpy().astype(np.float64))
    cg = cat.float().cpu().numpy()
    ci = interior(cg)[..., Cout:]
    assert np.all(np.abs(ci - ref) <= 2 ** -8 * np.abs(ref) + 1e-5)
    np.testing.assert_array_equal(cg[..., Cout:], padded(ci))
    assert np.all(cg[..., :Cout] == 3.0)


def test_up_adjoint_gather():
    Bn, h, w, Cin, Cout = 2, 8, 16, 64, 32
    dcat, dcatd = bf(gen.normal(size=(Bn, 2 * h + 2, 2 * w + 2, 2 * Cout)))
    Wu, Wud = bf(gen.normal(size=(4, Cout, Cin)))
    WuT = Wu.reshape(4 * Cout, Cin).t().contiguous()
    Mc = Bn * h * w
    out = torch.full((Bn, h + 2, w + 2, Cin), float("nan"), device=dev)
    gemm(op(dcat, S.SUR_OP_UPADJ, 2 * Cout, Cout, Cout, Mc, h, w), op(WuT, S.SUR_OP_DENSE, 4 * Cout, rows=Cin),
         Mc, Cin, 4 * Cout, out=out, ldo=Cin)
    dy = interior(dcatd)[..., Cout:]
    ref = U.tconv2_bwd(np.zeros((Bn, h, w, Cin)), dy, Wud)[0]
    absref = U.tconv2_bwd(np.zeros((Bn, h, w, Cin)), np.abs(dy), np.abs(Wud))[0]
    close(interior(out.cpu().numpy()), ref, absref)


@pytest.mark.parametrize("Cin,Cout,splits,H,W", [(64, 32, 4, 16, 32), (8, 32, 3, 16, 32), (128, 256, 2, 16, 32),
                                                 (32, 64, 2, 4, 64), (64, 128, 3, 16, 8), (32, 32, 1, 8, 128)])
def test_conv_weight_gradient_mn_major_split_k(Cin, Cout, splits, H, W):
    """Weight gradient of a 3x3 convolution (TCONV3 x TPIX, pixels along K, split-K FP32
    atomics) against the oracle; the shapes cover one- to eight-row pixel boxes and
    8-, 32- and 64-channel operand atoms."""
    Bn = 2
    x = bf16_round(gen.normal(size=(Bn, H, W, Cin)))
    X, _ = bf(padded(x))
    dZ, dZd = bf(gen.normal(size=(Bn, H + 2, W + 2, Cout)))
    kp = U.kp_of(Cin)
    M = Bn * H * W
    out = torch.zeros(kp, Cout, device=dev)
    gemm(op(X, S.SUR_OP_TCONV3, Cin, 0, Cin, 9 * Cin, H, W), op(dZ, S.SUR_OP_TPIX, Cout, 0, 0, Cout, H, W),
         kp, Cout, M, epi=S.SUR_EPI_F32_ATOMIC, out=out, ldo=Cout, splits=splits)
    dz = interior(dZd)
    ref = U.conv3_bwd_weight(x, dz)[0].reshape(9 * Cin, Cout)
    absref = U.conv3_bwd_weight(np.abs(x), np.abs(dz))[0].reshape(9 * Cin, Cout)
    g = out.cpu().numpy()
    close(g[:9 * Cin], ref, absref)
    assert np.all(g[9 * Cin:] == 0)


def test_tconv_weight_gradient_mn_major():
    Bn, h, w, Cin, Cout = 2, 8, 16, 64, 32
    X, Xd = bf(gen.normal(size=(Bn, h + 2, w + 2, Cin)))
    dcat, dcatd = bf(gen.normal(size=(Bn, 2 * h + 2, 2 * w + 2, 2 * Cout)))
    Mc = Bn * h * w
    out = torch.zeros(4 * Cout, Cin, device=dev)
    gemm(op(dcat, S.SUR_OP_TUP, 2 * Cout, Cout, Cout, 4 * Cout, h, w), op(X, S.SUR_OP_TPIX, Cin, 0, 0, Cin, h, w),
         4 * Cout, Cin, Mc, epi=S.SUR_EPI_F32_ATOMIC, out=out, ldo=Cin, splits=2)
    dy = interior(dcatd)[..., Cout:]
    xi = interior(Xd)
    ref = U.tconv2_bwd(xi, dy, np.zeros((4, Cout, Cin)))[1].reshape(4 * Cout, Cin)
    absref = U.tconv2_bwd(np.abs(xi), np.abs(dy), np.zeros((4, Cout, Cin)))[1].reshape(4 * Cout, Cin)
    close(out.cpu().numpy(), ref, absref)


def test_bf16_epilogue_with_column_offset():
    M, N, K = 256, 64, 128
    A, Ad = bf(gen.normal(size=(M, K)))
    B, Bd = bf(gen.normal(size=(N, K)))
    out = torch.full((M, 2 * N), 5.0, dtype=torch.bfloat16, device=dev)
    gemm(op(A, S.SUR_OP_DENSE, K, rows=M), op(B, S.SUR_OP_DENSE, K, rows=N), M, N, K, epi=S.SUR_EPI_BF16,
         out=out, ldo=2 * N, co0=N)
    ref = Ad @ Bd.T
    o = out.float().cpu().numpy()
    assert np.all(np.abs(o[:, N:] - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * (np.abs(Ad) @ np.abs(Bd).T))
    assert np.all(o[:, :N] == 5.0)


def test_invalid_gemm_rejected_on_host():
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device=dev)
    out = torch.zeros(128, 48, device=dev)
    g = S.sur_gemm_args()
    g.a = op(A, S.SUR_OP_DENSE, 64, rows=128)
    g.b = op(A, S.SUR_OP_DENSE, 64, rows=48)
    g.M, g.N, g.K, g.splits, g.epi = 128, 48, 64, 1, S.SUR_EPI_F32   # N not a multiple of 32
    g.out, g.ldo = out.data_ptr(), 48
    st = torch.zeros(2, dtype=torch.int32, device=dev)
    with pytest.raises(S.SurError) as e:
        S.sur_gemm(g, st.data_ptr(), 0)
    assert e.value.code == S.SUR_EINVAL


# ---------------------------------------------------------------------------
# The network
# ---------------------------------------------------------------------------

NORM = (np.array([0.12, 0.0, 0.0, 0.0085]), np.array([0.05, 0.01, 0.01, 0.001]),
        np.array([0.002, 0.001, 0.001, 0.0001]))


def smooth_fields(Bn, H, W, seed):
    r = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    out = []
    for _ in range(Bn):
        k = r.integers(1, 3, size=(4, 2))
        ph = r.random((4, 2)) * 2 * np.pi
        f = [np.sin(2 * np.pi * k[c, 0] * yy / H + ph[c, 0]) * np.cos(2 * np.pi * k[c, 1] * xx / W + ph[c, 1])
             for c in range(4)]
        out.append(np.stack(f))
    base = np.stack(out, 1).reshape(4, -1)
    x = NORM[0][:, None] + NORM[1][:, None] * base
    y = x + NORM[2][:, None] * np.roll(base, 1, axis=1) * 0.5
    return x, y


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_network_forward_backward_against_oracle(tma):
    Bn, H, W = 2, 16, 32
    x, y = smooth_fields(Bn, H, W, 3)
    with S.Surrogate(H, W, seed=5) as m:
        m.set_norm(*NORM)
        # Give the head full-size weights so that every layer's gradient is exercised.
        theta = m.params()
        layout, n = S.param_layout()
        off = dict((nm, (o, s)) for nm, o, s in layout)
        o, s = off["head.w"]
        theta[o:o + 4 * S.BASE] *= 10.0
        m.set_params(theta)
        dx = torch.tensor(x, dtype=torch.float32, device=dev).contiguous()
        dy = torch.tensor(y, dtype=torch.float32, device=dev).contiguous()
        torch.cuda.synchronize()
        loss = m.forward_backward(dx.data_ptr(), dy.data_ptr(), Bn)
        g_gpu = m.grads().astype(np.float64)
        pred = torch.empty_like(dx)
        m.infer(dx.data_ptr(), pred.data_ptr(), Bn)
        torch.cuda.synchronize()
        pred = pred.cpu().numpy().astype(np.float64)
    # The GPU computes with BF16 copies of the weights (FP32 biases and head).
    theta_b = theta.astype(np.float64).copy()
    for nm, o, shp in layout:
        if nm.endswith(".w") and not nm.startswith("head"):
            sz = int(np.prod(shp))
            theta_b[o:o + sz] = bf16_round(theta_b[o:o + sz])
    P = U.unpack(theta_b)
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    loss_o, G, _ = U.loss_and_grad(P, x32, y32, Bn, H, W, NORM)
    assert abs(loss - loss_o) <= 2e-2 * loss_o, (loss, loss_o)
    g_orc = U.pack(G, n)
    report = []
    for nm, o, shp in layout:
        sz = int(np.prod(shp))
        a, b = g_gpu[o:o + sz], g_orc[o:o + sz]
        assert np.all(np.isfinite(a)), nm
        e = rel_l2(a, b)
        report.append((nm, e))
        assert e <= 6e-2, (nm, e)
    print("\nworst gradient tensors (relative L2 vs FP64 oracle):",
          sorted(report, key=lambda t: -t[1])[:5])
    ref = U.predict(P, x32, Bn, H, W, NORM)
    inc_err = rel_l2(pred - x32, ref - x32)
    print("increment relative L2 vs oracle:", inc_err)
    assert inc_err <= 2e-2


@pytest.mark.parametrize("k", [1, 3])
def test_unrolled_forward_backward_against_oracle(k):
    """k windows chained through the network (sur_forward_backward_unrolled): loss and every
    gradient tensor against the oracle's unrolled_loss_and_grad with the same BF16-rounded
    weights (tolerances of the single-window test); k = 1 also against the window loss."""
    Bn, H, W = 2, 16, 32
    x, _ = smooth_fields(Bn, H, W, 4)
    base = (x - NORM[0][:, None]) / NORM[1][:, None]
    targets = np.stack([x + (j + 1) * 0.5 * NORM[2][:, None] * np.roll(base, j + 1, axis=1) for j in range(k)])
    with S.Surrogate(H, W, seed=6) as m:
        m.set_norm(*NORM)
        theta = m.params()
        layout, n = S.param_layout()
        off = dict((nm, (o, s)) for nm, o, s in layout)
        o, s = off["head.w"]
        theta[o:o + 4 * S.BASE] *= 10.0
        m.set_params(theta)
        dx = torch.tensor(x, dtype=torch.float32, device=dev).contiguous()
        dt = torch.tensor(targets.reshape(k * 4, -1), dtype=torch.float32, device=dev).contiguous()
        torch.cuda.synchronize()
        loss = m.forward_backward_unrolled(dx.data_ptr(), dt.data_ptr(), k, Bn)
        g_gpu = m.grads().astype(np.float64)
        if k == 1:
            loss1 = m.forward_backward(dx.data_ptr(), dt.data_ptr(), Bn)
            g1 = m.grads().astype(np.float64)
            assert abs(loss - loss1) <= 1e-4 * loss1
            assert rel_l2(g_gpu, g1) <= 1e-3
    theta_b = theta.astype(np.float64).copy()
    for nm, o, shp in layout:
        if nm.endswith(".w") and not nm.startswith("head"):
            sz = int(np.prod(shp))
            theta_b[o:o + sz] = bf16_round(theta_b[o:o + sz])
    P = U.unpack(theta_b)
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = targets.astype(np.float32).astype(np.float64)
    loss_o, G, _ = U.unrolled_loss_and_grad(P, x32, list(t32), Bn, H, W, NORM)
    assert abs(loss - loss_o) <= 2e-2 * loss_o, (loss, loss_o)
    g_orc = U.pack(G, n)
    report = []
    for nm, o, shp in layout:
        sz = int(np.prod(shp))
        a, b = g_gpu[o:o + sz], g_orc[o:o + sz]
        assert np.all(np.isfinite(a)), nm
        e = rel_l2(a, b)
        report.append((nm, e))
        assert e <= 6e-2, (nm, e)
    print(f"\nk = {k}: loss {loss:.5e} (oracle {loss_o:.5e}); worst gradient tensors:",
          sorted(report, key=lambda t: -t[1])[:3])


def test_training_reduces_loss():
    Bn, H, W = 4, 32, 32
    x, y = smooth_fields(Bn, H, W, 9)
    dx = torch.tensor(x, dtype=torch.float32, device=dev).contiguous()
    dy = torch.tensor(y, dtype=torch.float32, device=dev).contiguous()
    torch.cuda.synchronize()
    with S.Surrogate(H, W, seed=1) as m:
        m.set_norm(*NORM)
        l0 = m.train_step(dx.data_ptr(), dy.data_ptr(), Bn, 1e-3)
        for _ in range(300):
            m.train_step(dx.data_ptr(), dy.data_ptr(), Bn, 1e-3, want_loss=False)
        l1 = m.forward_backward(dx.data_ptr(), dy.data_ptr(), Bn)
    print(f"\nloss {l0:.4e} -> {l1:.4e} after 300 Adam steps")
    assert l1 < 0.05 * l0


def droplet_batch(Bn, n, seed):
    """Bn droplet-pair domains of n x n (planar FP64 fields [4][Bn*n*n]) and the reduced temperatures."""
    import oracle.eos as E
    _, Tc = E.critical_point(E.CS, 0.1, 4.0)
    r = np.random.default_rng(seed)
    rho, ux, uy, T = [], [], [], []
    for b in range(Bn):
        tr = 0.75 + 0.1 * r.random()
        rv, rl = E.maxwell(E.CS, 0.1, 4.0, tr * Tc)
        r1, r2 = 6 + 4 * r.random(), 6 + 4 * r.random()
        f = inputs.two_droplets(n, n, r1, r2, 3.0, rv, rl, tr * Tc)
        rho.append(f[0])
        ux.append(f[1][0])
        uy.append(f[1][1])
        T.append(f[2])
    return np.stack([np.concatenate(v) for v in (rho, ux, uy, T)])


def test_rollout_fallback_paths():
    """Zero thresholds: every window falls back, and the rollout is exactly a plain
    lattice Boltzmann run of windows*steps from the equilibrium of the start fields;
    infinite thresholds: the rollout equals repeated inference."""
    Bn, n, windows, steps = 2, 64, 3, 10
    F0 = droplet_batch(Bn, n, 4)
    N = Bn * n * n
    p = ev.lbm_params.make(nx=n, ny=n, nz=Bn, eos=ev.LBM_EOS_CS, a=0.1, b=4.0, kappa=0.116, tau=0.3,
                           precision=ev.LBM_FP32)
    rho_mid = float(0.5 * (F0[0].max() + F0[0].min()))
    with S.Surrogate(n, n, seed=2) as m, ev.Lattice(p, F0[0], F0[1:3], F0[3]) as lb, \
            ev.Lattice(p, F0[0], F0[1:3], F0[3]) as lb2:
        m.set_norm(*NORM)
        d = torch.tensor(F0, dtype=torch.float32, device=dev).contiguous()
        torch.cuda.synchronize()
        nfb, used = m.rollout(lb.ctx, d.data_ptr(), Bn, windows, steps, rho_mid, 0.0, 0.0)
        assert nfb == windows and used.tolist() == [1] * windows
        e = torch.empty_like(d)
        ep = e.data_ptr()
        ev.lbm_step(lb2.ctx, windows * steps)
        ev.lbm_moments_device(lb2.ctx, ep, ep + 4 * N, ep + 12 * N)
        ev.lbm_sync(lb2.ctx)
        torch.cuda.synchronize()
        assert torch.equal(d, e)
        d2 = torch.tensor(F0, dtype=torch.float32, device=dev).contiguous()
        torch.cuda.synchronize()
        nfb, used = m.rollout(lb.ctx, d2.data_ptr(), Bn, windows, steps, rho_mid, 1e30, 1e30)
        assert nfb == 0 and used.tolist() == [0] * windows
        e2 = torch.tensor(F0, dtype=torch.float32, device=dev).contiguous()
        tmp = torch.empty_like(e2)
        for _ in range(windows):
            m.infer(e2.data_ptr(), tmp.data_ptr(), Bn)
            torch.cuda.synchronize()
            e2.copy_(tmp)
        torch.cuda.synchronize()
        assert torch.equal(d2, e2)


def test_rollout_interface_indicator():
    """The interface-position indicator counts, per domain, the nodes whose phase (rho
    above / below rho_mid) differs between the proposal and the current fields: a window
    is accepted at a threshold of the largest count and falls back just below it (the
    count taken here on the host from the same proposal)."""
    Bn, n, steps = 2, 64, 10
    F0 = droplet_batch(Bn, n, 5)
    Mb = n * n
    p = ev.lbm_params.make(nx=n, ny=n, nz=Bn, eos=ev.LBM_EOS_CS, a=0.1, b=4.0, kappa=0.116, tau=0.3,
                           precision=ev.LBM_FP32)
    rho_mid = float(0.5 * (F0[0].max() + F0[0].min()))
    with S.Surrogate(n, n, seed=9) as m, ev.Lattice(p, F0[0], F0[1:3], F0[3]) as lb:
        m.set_norm(NORM[0], NORM[1], NORM[2] * 4.0)         # larger increments than the default scale
        d = torch.tensor(F0, dtype=torch.float32, device=dev).contiguous()
        prop = torch.empty_like(d)
        m.infer(d.data_ptr(), prop.data_ptr(), Bn)
        torch.cuda.synchronize()
        a = (d[0].cpu().numpy() > rho_mid).reshape(Bn, Mb)
        b = (prop[0].cpu().numpy() > rho_mid).reshape(Bn, Mb)
        fmax = int((a != b).sum(axis=1).max())
        for shift, want_fallbacks in (((fmax + 0.25) / Mb, 0), ((fmax - 0.5) / Mb, 1)):
            dd = d.clone()
            torch.cuda.synchronize()
            nfb, used = m.rollout(lb.ctx, dd.data_ptr(), Bn, 1, steps, rho_mid, 1e30, 1e30, False, shift)
            assert nfb == want_fallbacks, (fmax, shift, nfb)
            if want_fallbacks == 0:
                assert torch.equal(dd, prop)
    print(f"\nlargest phase-flip count of the proposal: {fmax} of {Mb} nodes")
