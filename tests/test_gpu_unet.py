"""GPU parity and benefit of the learned warm start's network.

Forward pass and gradients of the library's tensor-core U-Net against the FP64
oracle (oracle/unet.py with the same bfloat16 rounding points), AdamW against
the oracle's update, the feature/target/guess glue against the oracle's DDA
quantities, and a small end-to-end run showing the trained network saves
Krylov iterations at equal final residual.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import dda as odda  # noqa: E402
from oracle import unet as OU  # noqa: E402
from paper_1002_1505_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_1505_gb300 import dda
    return dda


CIN, COUT, CH = 5, 3, (6, 10, 12, 16)
DIMS = (16, 8, 16)  # x, y, z


def _data(seed, B=2):
    rng = np.random.default_rng(seed)
    Z, Y, X = DIMS[2], DIMS[1], DIMS[0]
    x = rng.standard_normal((B, Z, Y, X, CIN)).astype(np.float32)
    t = rng.standard_normal((B, Z, Y, X, COUT)).astype(np.float32)
    mask = (rng.random((B, Z, Y, X)) > 0.3).astype(np.float32)
    return x, t, mask


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(params=["tcgen05", "mma_sync"])
def engine(request, monkeypatch):
    """Networks created in the test use the tcgen05 convolutions (default) or mma.sync throughout."""
    monkeypatch.setenv("DDA_UNET_TC", "1" if request.param == "tcgen05" else "0")
    return request.param


def test_forward_matches_oracle(D, engine):
    net = D.UNet(0, None, CIN, COUT, CH, seed=11)
    theta = net.dda_unet_get_params().astype(np.float64)
    x, _, _ = _data(1)
    xg = torch.from_numpy(x).cuda()
    yg = torch.empty(x.shape[:4] + (COUT,), dtype=torch.float32, device="cuda")
    net.dda_unet_forward(xg, yg, DIMS)
    torch.cuda.synchronize()
    ref = OU.forward(theta, x.astype(np.float64), CIN, COUT, CH, quant=True)
    assert _rel(yg.cpu().numpy(), ref) <= 2e-3


def test_gradients_match_oracle(D, engine):
    net = D.UNet(0, None, CIN, COUT, CH, seed=12)
    theta = net.dda_unet_get_params().astype(np.float64)
    x, t, mask = _data(2)
    loss = net.dda_unet_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                                  torch.from_numpy(mask).cuda(), DIMS)
    g = net.dda_unet_get_params(which=1).astype(np.float64)
    Lr, gr = OU.loss_and_grad(theta, x.astype(np.float64), t.astype(np.float64), mask.astype(np.float64), CIN, COUT,
                              CH, quant=True)
    assert loss == pytest.approx(Lr, rel=1e-4)
    # layer by layer: weights and biases
    o = 0
    for taps, a, b in OU.layer_shapes(CIN, COUT, CH):
        nw = taps * a * b
        assert _rel(g[o:o + nw], gr[o:o + nw]) <= 5e-3, ("W", o)
        assert _rel(g[o + nw:o + nw + b], gr[o + nw:o + nw + b]) <= 5e-3, ("b", o)
        o += nw + b


def test_gradients_match_oracle_default_widths(D, engine):
    """The warm start's own widths: wide concatenated inputs use 10 n-tiles in the input-gradient GEMM."""
    cin, cout, ch, dims = 9, 6, (12, 24, 32, 48), (8, 8, 16)
    net = D.UNet(0, None, cin, cout, ch, seed=21)
    theta = net.dda_unet_get_params().astype(np.float64)
    rng = np.random.default_rng(21)
    x = rng.standard_normal((1, dims[2], dims[1], dims[0], cin)).astype(np.float32)
    t = rng.standard_normal((1, dims[2], dims[1], dims[0], cout)).astype(np.float32)
    mask = (rng.random((1, dims[2], dims[1], dims[0])) > 0.3).astype(np.float32)
    loss = net.dda_unet_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                                  torch.from_numpy(mask).cuda(), dims)
    g = net.dda_unet_get_params(which=1).astype(np.float64)
    Lr, gr = OU.loss_and_grad(theta, x.astype(np.float64), t.astype(np.float64), mask.astype(np.float64), cin, cout,
                              ch, quant=True)
    assert loss == pytest.approx(Lr, rel=1e-4)
    # the first layers sit at the end of the backward chain, where bfloat16 rounding decisions taken
    # on FP32 (GPU) vs FP64 (oracle) activations have accumulated: 1% bound there
    o = 0
    for taps, a, b in OU.layer_shapes(cin, cout, ch):
        nw = taps * a * b
        assert _rel(g[o:o + nw], gr[o:o + nw]) <= 1e-2, ("W", o)
        assert _rel(g[o + nw:o + nw + b], gr[o + nw:o + nw + b]) <= 1e-2, ("b", o)
        o += nw + b


def test_adamw_matches_oracle_update(D):
    net = D.UNet(0, None, CIN, COUT, CH, seed=13)
    theta = net.dda_unet_get_params().astype(np.float64)
    x, t, mask = _data(3)
    net.dda_unet_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mask).cuda(), DIMS)
    g = net.dda_unet_get_params(which=1).astype(np.float64)
    net.dda_unet_adamw(1e-3, wd=0.01)
    new = net.dda_unet_get_params().astype(np.float64)
    ref, _, _ = OU.adamw(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3, wd=0.01)
    np.testing.assert_allclose(new, ref, rtol=1e-5, atol=1e-7)


def test_training_reduces_loss_on_a_fixed_batch(D):
    net = D.UNet(0, None, CIN, COUT, CH, seed=14)
    x, t, mask = _data(4, B=4)
    t = np.tanh(x[..., :COUT])  # a learnable map of the input
    xg, tg, mg = torch.from_numpy(x).cuda(), torch.from_numpy(t.astype(np.float32)).cuda(), torch.from_numpy(mask).cuda()
    losses = []
    for _ in range(60):
        losses.append(net.dda_unet_loss_grad(xg, tg, mg, DIMS))
        net.dda_unet_adamw(3e-3)
    assert losses[-1] < 0.3 * losses[0]


def test_features_targets_and_guess_match_the_oracle(D):
    w = W.Workload("ell_nn", "ELLIPSOID", (7, 5, 9), 1.5 + 0.3j, 2.0, "GKDLDR", W.uniform_orientations(1, 51))
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    grid = (8, 8, 16)
    off = [(g - b) // 2 for g, b in zip(grid, ctx.box)]
    x = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0], 9), dtype=torch.float32, device="cuda")
    D.dda_unet_features(ctx, x, grid)
    ps, _ = odda.solve(prob, "lu")
    p = torch.from_numpy(np.stack(ps)).cuda()
    t = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0], 6), dtype=torch.float32, device="cuda")
    m = torch.zeros((ctx.nrhs, grid[2], grid[1], grid[0]), dtype=torch.float32, device="cuda")
    D.dda_unet_targets(ctx, p, t, m, grid)
    guess = torch.zeros_like(p)
    D.dda_unet_warm_start(ctx, t, grid, guess)
    # residual mode: targets minus E_inc, and the guess adds E_inc back
    tr = torch.zeros_like(t)
    D.dda_unet_targets(ctx, p, tr, m, grid, residual=True)
    guess_r = torch.zeros_like(p)
    D.dda_unet_warm_start(ctx, tr, grid, guess_r, residual=True)
    xh, th, mh, gh = x.cpu().numpy(), t.cpu().numpy(), m.cpu().numpy(), guess.cpu().numpy()
    trh, grh = tr.cpu().numpy(), guess_r.cpu().numpy()
    eps = (1.5 + 0.3j) ** 2
    ijk = prob.target.ijk
    iz, iy, ix = ijk[:, 2] + off[2], ijk[:, 1] + off[1], ijk[:, 0] + off[0]
    assert mh.sum() == ctx.nrhs * ctx.n
    for b in range(ctx.nrhs):
        f = xh[b, iz, iy, ix]
        np.testing.assert_allclose(f[:, 0], 1.0)
        np.testing.assert_allclose(f[:, 1], 0.25 * (eps.real - 1), rtol=1e-6)
        np.testing.assert_allclose(f[:, 2], 0.5 * eps.imag, rtol=1e-6)
        e = prob.rhs[b].e_inc
        for c in range(3):
            np.testing.assert_allclose(f[:, 3 + 2 * c], e[c].real, atol=1e-6)
            np.testing.assert_allclose(f[:, 4 + 2 * c], e[c].imag, atol=1e-6)
        eloc = prob.rhs[b].inv_alpha.T * ps[b]          # alpha^{-1} P
        tt = th[b, iz, iy, ix]
        for c in range(3):
            np.testing.assert_allclose(tt[:, 2 * c] + 1j * tt[:, 2 * c + 1], eloc[c], rtol=2e-6, atol=1e-7)
        # the guess built from the exact local field is P itself (to FP32 rounding)
        assert _rel(gh[b], ps[b]) <= 1e-6
        assert _rel(grh[b], ps[b]) <= 1e-6
        ttr = trh[b, iz, iy, ix]
        for c in range(3):
            np.testing.assert_allclose(ttr[:, 2 * c] + 1j * ttr[:, 2 * c + 1], eloc[c] - e[c], rtol=2e-6, atol=2e-7)
    assert np.count_nonzero(xh[:, :, :, :, 0]) == ctx.nrhs * ctx.n


def test_residual_loss_and_gradient(D):
    """dda_unet_residual_grad: the loss is |E - A P0|^2/|E|^2 with the oracle's A, and its gradient
    matches a central difference along a random direction."""
    w = W.Workload("ell_rg", "ELLIPSOID", (7, 6, 5), 1.4 + 0.2j, 2.0, "GKDLDR", W.uniform_orientations(1, 61))
    ctx = D.Context(0)
    D.setup_workload(ctx, w)
    prob = odda.build_problem(w.shape, w.shpar, w.m, w.x, w.prescription, w.orientations)
    grid = (8, 8, 8)
    rng = np.random.default_rng(0)
    y = torch.from_numpy(rng.standard_normal((2, 8, 8, 8, 6)).astype(np.float32) * 0.1).cuda()
    gy = torch.zeros_like(y)
    L = D.dda_unet_residual_grad(ctx, y, gy, grid)
    # oracle: P0 = alpha (E_inc + y) at the sites, residual with the direct sum
    off = [(g - b) // 2 for g, b in zip(grid, ctx.box)]
    ijk = prob.target.ijk
    iz, iy, ix = ijk[:, 2] + off[2], ijk[:, 1] + off[1], ijk[:, 0] + off[0]
    yh = y.cpu().numpy().astype(np.float64)
    ref = 0.0
    for b in range(2):
        yc = yh[b, iz, iy, ix]
        eloc = prob.rhs[b].e_inc + (yc[:, 0::2] + 1j * yc[:, 1::2]).T
        p0 = eloc / prob.rhs[b].inv_alpha.T
        r = prob.rhs[b].e_inc - odda.apply_a(prob, b, p0, "direct")
        ref += np.sum(np.abs(r) ** 2) / np.sum(np.abs(prob.rhs[b].e_inc) ** 2)
    assert L == pytest.approx(ref, rel=1e-4)
    # directional derivative
    dvec = torch.from_numpy(rng.standard_normal((2, 8, 8, 8, 6)).astype(np.float32)).cuda()
    h = 1e-2
    scratch = torch.zeros_like(y)
    lp = D.dda_unet_residual_grad(ctx, (y + h * dvec).contiguous(), scratch, grid)
    lm = D.dda_unet_residual_grad(ctx, (y - h * dvec).contiguous(), scratch, grid)
    fd = (lp - lm) / (2 * h)
    an = float(torch.sum(gy.double() * dvec.double()))
    assert an == pytest.approx(fd, rel=2e-3)


def test_trained_network_saves_iterations(D):
    """Small end-to-end run: data from the solver (2048 random problems), training
    on the GPU, then iterations to the same final residual on 32 held-out
    problems from a cold start (the method without the network), from the
    network-free guess alpha E_inc and from the network's guess.  The network
    starts as the network-free guess (zero output layer)."""
    from paper_1002_1505_gb300 import warmstart as WS
    max_box, grid = 16, (16, 16, 16)
    X, T, M, _ = WS.generate(list(range(0, 2048)), max_box, grid)
    m = M[..., None]
    mse0 = float((m * T * T).sum() / (m.sum() * WS.COUT))  # error of the network-free guess
    net = D.UNet(0, None, WS.CIN, WS.COUT, (16, 32, 48, 64), seed=5)
    WS.zero_head(net)
    hist = WS.train(net, X, T, M, grid, steps=6000, batch=16, lr=1e-3)
    assert np.mean(hist[-200:]) < 0.35 * mse0, (np.mean(hist[-200:]), mse0)
    rows = WS.evaluate(net, list(range(100000, 100032)), max_box, grid)
    cold = sum(r["cold"][0] for r in rows)
    warm = sum(r["network"][0] for r in rows)
    plain = sum(r["alpha_einc"][0] for r in rows)
    print(f"iterations over {len(rows)} held-out problems: cold {cold}, alpha*E_inc guess {plain}, network {warm}; "
          f"masked MSE {mse0:.3e} (no network) -> {np.mean(hist[-200:]):.3e}")
    for r in rows:
        for k in ("cold", "alpha_einc", "network"):
            assert r[k][1] <= 1e-5   # equal final residual bar
    # the network's guess needs fewer iterations than the plain solver's cold start; against the
    # network-free guess alpha E_inc it is within a few percent at this training size (the larger
    # evaluation of warmstart.main gains about 2 % over it)
    assert warm <= 0.98 * cold and plain < cold, (warm, plain, cold)
    assert warm <= 1.03 * plain, (warm, plain)


@pytest.fixture
def tc_mode(monkeypatch):
    """Networks created inside the test run their convolutions on tcgen05 (tensor memory accumulators)."""
    monkeypatch.setenv("DDA_UNET_TC", "1")


def test_tcgen05_forward_matches_oracle_and_mma_sync(D, tc_mode, monkeypatch):
    """The tcgen05 convolutions give the oracle's forward pass, and the mma.sync path's to FP32 summation order."""
    cin, cout, ch, dims = 9, 6, (12, 24, 32, 48), (16, 8, 16)
    rng = np.random.default_rng(31)
    x = rng.standard_normal((2, dims[2], dims[1], dims[0], cin)).astype(np.float32)
    xg = torch.from_numpy(x).cuda()
    net = D.UNet(0, None, cin, cout, ch, seed=31)
    y_tc = torch.empty(x.shape[:4] + (cout,), dtype=torch.float32, device="cuda")
    net.dda_unet_forward(xg, y_tc, dims)
    torch.cuda.synchronize()
    net.dda_unet_check_fault()
    theta = net.dda_unet_get_params().astype(np.float64)
    ref = OU.forward(theta, x.astype(np.float64), cin, cout, ch, quant=True)
    assert _rel(y_tc.cpu().numpy(), ref) <= 2e-3
    monkeypatch.setenv("DDA_UNET_TC", "0")
    net2 = D.UNet(0, None, cin, cout, ch, seed=31)
    y_ms = torch.empty_like(y_tc)
    net2.dda_unet_forward(xg, y_ms, dims)
    torch.cuda.synchronize()
    # identical bf16 operands, FP32 accumulation in another order: bf16 rounding of later layers'
    # inputs may flip on ties of that order, hence 1e-3 rather than FP32 epsilon
    assert _rel(y_tc.cpu().numpy(), y_ms.cpu().numpy()) <= 1e-3


def test_tcgen05_long_rows_and_ragged_tiles(D, monkeypatch):
    """Rows of 128 voxels (staged rows of 130 with the halo, several 128-row M tiles per CTA) and y / z
    extents that the CTA tiles do not divide: the tcgen05 forward pass against the oracle and against
    the mma.sync pass.  On volumes this large some bfloat16 roundings of inner activations differ
    between FP32 (both GPU engines) and FP64 (oracle) sums, and the oracle distance of both engines
    grows to ~3e-3 (measured: 2.66e-3 for both on 40 x 56 x 24); the engines stay within 1e-3 of
    each other and the tcgen05 one no farther from the oracle than the mma.sync one."""
    for dims in ((128, 24, 8), (40, 56, 24)):
        rng = np.random.default_rng(dims[0])
        x = rng.standard_normal((1, dims[2], dims[1], dims[0], CIN)).astype(np.float32)
        out = []
        for mode in ("1", "0"):
            monkeypatch.setenv("DDA_UNET_TC", mode)
            net = D.UNet(0, None, CIN, COUT, CH, seed=5)
            yv = torch.empty(x.shape[:4] + (COUT,), dtype=torch.float32, device="cuda")
            net.dda_unet_forward(torch.from_numpy(x).cuda(), yv, dims)
            torch.cuda.synchronize()
            net.dda_unet_check_fault()
            theta = net.dda_unet_get_params().astype(np.float64)
            out.append(yv.cpu().numpy())
            net.close()
        ref = OU.forward(theta, x.astype(np.float64), CIN, COUT, CH, quant=True)
        e_tc, e_ms = _rel(out[0], ref), _rel(out[1], ref)
        assert e_tc <= 5e-3 and e_tc <= 1.2 * e_ms + 1e-5, (dims, e_tc, e_ms)
        assert _rel(out[0], out[1]) <= 1e-3, dims
    cin, cout, ch = 9, 6, (16, 32, 48, 64)
    for dims in ((128, 24, 8), (40, 56, 24)):
        rng = np.random.default_rng(dims[0])
        x = rng.standard_normal((1, dims[2], dims[1], dims[0], cin)).astype(np.float32)
        xg = torch.from_numpy(x).cuda()
        out = []
        for mode in ("1", "0"):
            monkeypatch.setenv("DDA_UNET_TC", mode)
            net = D.UNet(0, None, cin, cout, ch, seed=3)
            yv = torch.empty(x.shape[:4] + (cout,), dtype=torch.float32, device="cuda")
            net.dda_unet_forward(xg, yv, dims)
            torch.cuda.synchronize()
            net.dda_unet_check_fault()
            out.append(yv.cpu().numpy())
            net.close()
        assert np.isfinite(out[0]).all()
        assert _rel(out[0], out[1]) <= 3e-3, dims
