"""Tensor-core kernels of the learned guess vs the FP64 reference (oracle/unet_ref.py),
called through the C ABI (include/isis_unet.h).

Per-kernel checks feed both sides the same BF16 values, so only the FP32
accumulation order differs.  The whole-network gradient is checked by
direction (cosine) because the GPU keeps activations in BF16."""
import numpy as np
import pytest
import torch

import oracle
from oracle import unet_ref as U

pytestmark = pytest.mark.gpu


def _bf(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).cuda()


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _planar(X):
    """[V, C] -> the library's channel-planar order: element (v, c) at ((c / 8) V + v) 8 + c % 8."""
    V, C = X.shape
    return np.ascontiguousarray(X.reshape(V, C // 8, 8).transpose(1, 0, 2).reshape(-1))


def _unplanar(x, C):
    x = np.asarray(x).reshape(C // 8, -1, 8)
    return x.transpose(1, 0, 2).reshape(-1, C)


def _rows(t, C, idx):
    """Rows idx ([V, C] view) of a channel-planar device tensor, FP64 on the host."""
    return _np(t.view(C // 8, -1, 8)[:, torch.from_numpy(idx).cuda(), :]).transpose(1, 0, 2).reshape(len(idx), C)


@pytest.fixture(scope="module")
def lib(cuda_lib):
    from paper_1307_6748_gb300 import unet
    return unet._lib()


def _p(t):
    import ctypes
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    import ctypes
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("c1,up,c2,cout", [(16, 0, 0, 16), (32, 1, 16, 32), (64, 0, 0, 64), (64, 1, 64, 64),
                                           (32, 1, 16, 16)])
def test_conv_forward(lib, c1, up, c2, cout):
    lg = 3
    n = 1 << lg
    g = np.random.Generator(np.random.PCG64(c1 + cout + up))
    n1 = n >> up
    s1 = _bf(_planar(g.standard_normal((n1 ** 3, c1))))
    s2 = _bf(_planar(g.standard_normal((n ** 3, c2)))) if c2 else None
    W = _bf(g.standard_normal((27, cout, c1 + c2)) * 0.1)
    b = torch.from_numpy(g.standard_normal(cout).astype(np.float32)).cuda()
    out = torch.empty(n ** 3 * cout, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.isis_unet_conv3_fwd(_p(s1), c1, lg - up, _p(s2), c2, lg, _p(W), _p(b), cout, 1, _p(out), _p(err),
                                   _s()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    X1 = _unplanar(_np(s1), c1).reshape(n1, n1, n1, c1)
    if up:
        X1 = U.up(X1)
    X = X1 if not c2 else np.concatenate([X1, _unplanar(_np(s2), c2).reshape(n, n, n, c2)], axis=-1)
    ref = U.relu(U.conv3_fwd(X, _np(W), b.cpu().numpy().astype(np.float64))).reshape(-1, cout)
    got = _unplanar(_np(out), cout)
    assert np.abs(got - ref).max() <= 2 ** -7 * np.abs(ref).max() + 1e-6


@pytest.mark.parametrize("cout,cin", [(16, 16), (32, 96), (64, 128), (16, 48)])
def test_conv_input_gradient(lib, cout, cin):
    lg = 3
    n = 1 << lg
    g = np.random.Generator(np.random.PCG64(cout * 7 + cin))
    dz = _bf(_planar(g.standard_normal((n ** 3, cout))))
    W = _bf(g.standard_normal((27, cout, cin)) * 0.1)
    Wt = torch.empty_like(W)
    assert lib.isis_unet_transpose_w(_p(W), cout, cin, _p(Wt), _s()) == 0
    din = torch.empty(n ** 3 * cin, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.isis_unet_conv3_dgrad(_p(dz), cout, lg, _p(Wt), cin, _p(din), _p(err), _s()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = U.conv3_dgrad(_unplanar(_np(dz), cout).reshape(n, n, n, cout), _np(W)).reshape(-1, cin)
    got = _unplanar(din.cpu().numpy(), cin)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("c1,up,c2,cout", [(16, 0, 0, 16), (32, 1, 16, 32), (64, 1, 64, 64), (16, 0, 0, 32)])
def test_conv_weight_gradient(lib, c1, up, c2, cout):
    lg = 4
    n = 1 << lg
    g = np.random.Generator(np.random.PCG64(3 * c1 + cout + up))
    n1 = n >> up
    s1 = _bf(_planar(g.standard_normal((n1 ** 3, c1))))
    s2 = _bf(_planar(g.standard_normal((n ** 3, c2)))) if c2 else None
    dz = _bf(_planar(g.standard_normal((n ** 3, cout))))
    dw = torch.zeros(27 * cout * (c1 + c2), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.isis_unet_conv3_wgrad(_p(s1), c1, lg - up, _p(s2), c2, lg, _p(dz), cout, _p(dw), _p(err), _s()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    X1 = _unplanar(_np(s1), c1).reshape(n1, n1, n1, c1)
    if up:
        X1 = U.up(X1)
    X = X1 if not c2 else np.concatenate([X1, _unplanar(_np(s2), c2).reshape(n, n, n, c2)], axis=-1)
    ref = U.conv3_wgrad(X, _unplanar(_np(dz), cout).reshape(n, n, n, cout))
    got = dw.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_network_gradient_direction(cuda_lib):
    """Gradient of one training step of the GPU net vs the FP64 reference on the same parameters."""
    from paper_1307_6748_gb300 import synth, unet
    lg, n = 5, 32
    net = unet.UNet(seed=3)  # 32^3: the lowest level is 4^3
    P = {k: v.astype(np.float64) for k, v in net.state().items() if k not in ("mu", "sd", "scale")}
    eta = synth.lognormal_eta(n, float(n), 1.5, 9).cuda()
    target = (0.05 * synth.gaussian_field(n, float(n), 1.0, 10)).float().cuda().reshape(-1)
    net.features(eta, 1.0, lg)
    X0 = _unplanar(_np(net.acts(lg)[1]["x0"]), 16).reshape(n, n, n, 16)
    _, grads, _ = U.loss_and_grads(P, X0, target.cpu().numpy().astype(np.float64).reshape(n, n, n) / net.scale)
    net.train_step(eta, 1.0, target, lg, lr=0.0)  # lr 0: gradients only
    torch.cuda.synchronize()
    assert int(net.err.item()) == 0
    for k, ref in grads.items():
        got = net.view(net.G, k).cpu().numpy().astype(np.float64)
        ref = ref.reshape(-1)
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300)
        assert cos >= 0.98, (k, cos)
        assert abs(np.linalg.norm(got) / np.linalg.norm(ref) - 1) <= 0.1, k


def _sampled_conv_ref(s1, c1, up, s2, c2, lg, W, b, vs):
    """FP64 reference of the convolution at the voxels vs only (neighbours gathered on the device)."""
    n = 1 << lg
    i, j, k = vs // (n * n), (vs // n) % n, vs % n
    ref = np.zeros((len(vs), W.shape[1]))
    for t, (di, dj, dk) in enumerate(U.TAPS):
        ii, jj, kk = (i + di) % n, (j + dj) % n, (k + dk) % n
        if up:
            nc = n // 2
            u1 = ((ii // 2) * nc + jj // 2) * nc + kk // 2
        else:
            u1 = (ii * n + jj) * n + kk
        X = _rows(s1, c1, u1)
        if c2:
            u2 = (ii * n + jj) * n + kk
            X = np.concatenate([X, _rows(s2, c2, u2)], axis=1)
        ref += X @ W[t].T
    return U.relu(ref + b)


@pytest.mark.parametrize("lg,c1,up,c2,cout", [(5, 16, 0, 0, 32), (5, 64, 1, 64, 64), (6, 32, 1, 16, 16),
                                              (6, 64, 0, 0, 64), (7, 64, 1, 32, 32), (7, 16, 0, 0, 16),
                                              (8, 32, 1, 16, 16), (8, 16, 0, 0, 32), (9, 16, 0, 0, 16)])
def test_line_conv_forward(lib, lg, c1, up, c2, cout):
    """The line kernel (grids of 32..512 cells, packed weights): every voxel of a plane at each
    end, rows at the j wrap, the k wrap and random voxels, against the FP64 reference."""
    n = 1 << lg
    gen = torch.Generator(device="cuda").manual_seed(lg * 1000 + c1 + c2 + cout + up)
    n1 = n >> up
    s1 = torch.randn(n1 ** 3 * c1, generator=gen, device="cuda").to(torch.bfloat16)
    s2 = torch.randn(n ** 3 * c2, generator=gen, device="cuda").to(torch.bfloat16) if c2 else None
    W = (0.1 * torch.randn(27 * cout * (c1 + c2), generator=gen, device="cuda")).to(torch.bfloat16)
    b = torch.randn(cout, generator=gen, device="cuda")
    out = torch.empty(n ** 3 * cout, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Wl = torch.empty_like(W)
    assert lib.isis_unet_line_ok(c1, lg - up, c2, lg, cout) == 1
    assert lib.isis_unet_pack_w(_p(W), cout, c1 + c2, _p(Wl), _s()) == 0
    assert lib.isis_unet_line_fwd(_p(s1), c1, lg - up, _p(s2), c2, lg, _p(Wl), _p(b), cout, 1, _p(out), _p(err),
                                  _s()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    rng = np.random.Generator(np.random.PCG64(lg))
    plane0 = np.arange(n * n)
    planeL = (n - 1) * n * n + np.arange(n * n)
    if n > 64:
        plane0, planeL = plane0[rng.choice(n * n, 2048, replace=False)], planeL[rng.choice(n * n, 2048, replace=False)]
    vs = np.unique(np.concatenate([plane0, planeL, rng.integers(0, n ** 3, 4096),
                                   (n // 2) * n * n + (n - 1) * n + np.arange(n),   # last row of a plane (j wrap)
                                   (np.arange(n) * n + 3) * n + n - 1]))            # k = n - 1 (k wrap)
    Wn = _np(W).reshape(27, cout, c1 + c2)
    ref = _sampled_conv_ref(s1, c1, up, s2, c2, lg, Wn, b.cpu().numpy().astype(np.float64), vs)
    got = _rows(out, cout, vs)
    assert np.abs(got - ref).max() <= 2 ** -7 * np.abs(ref).max() + 1e-6


@pytest.mark.parametrize("lg", [3, 5, 7])
def test_stem_equals_conv_of_features(lib, lg):
    """First layer from the two features vs the FP64 convolution of the 16-channel features."""
    from paper_1307_6748_gb300 import synth
    n = 1 << lg
    eta = synth.lognormal_eta(n, float(n), 1.5, 11).cuda()
    x16 = torch.empty(n ** 3 * 16, dtype=torch.bfloat16, device="cuda")
    f2 = torch.empty(n ** 3 * 2, dtype=torch.bfloat16, device="cuda")
    assert lib.isis_unet_input(_p(eta), lg, -1.125, 1 / 1.5, 0.7, _p(x16), _p(f2), _s()) == 0
    g = np.random.Generator(np.random.PCG64(lg))
    W = _bf(g.standard_normal((27, 16, 16)) * 0.2)
    b = torch.from_numpy(g.standard_normal(16).astype(np.float32)).cuda()
    out = torch.empty(n ** 3 * 16, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.isis_unet_stem_fwd(_p(f2), lg, _p(W), 16, _p(b), _p(out), _p(err), _s()) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    X = _unplanar(_np(x16), 16)
    assert np.all(X[:, 2:] == 0) and np.array_equal(X[:, :2], _np(f2).reshape(-1, 2))
    if lg <= 5:
        ref = U.relu(U.conv3_fwd(X.reshape(n, n, n, 16), _np(W), b.cpu().numpy().astype(np.float64))).reshape(-1, 16)
        got = _unplanar(_np(out), 16)
    else:
        vs = np.random.Generator(np.random.PCG64(1)).integers(0, n ** 3, 8192)
        ref = _sampled_conv_ref(x16, 16, 0, None, 0, lg, _np(W), b.cpu().numpy().astype(np.float64), vs)
        got = _rows(out, 16, vs)
    assert np.abs(got - ref).max() <= 2 ** -7 * np.abs(ref).max() + 1e-6


WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "paper_1307_6748_gb300", "weights",
                                     "unet_symmetron.npz")


def _sym_solve(eta, a, phi, tol, init):
    from paper_1307_6748_gb300 import isis
    N = eta.shape[0]
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=3, n_coarsest=2, init=init)
    return isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(a_ssb=0.5), isis.Grid(N, float(N)), a, eta, phi,
                                  tol=tol, opts=opts)


def test_trained_guess_gain(cuda_lib):
    """What the trained net gains on held-out densities (seeds outside the training range), at
    the training cell size: a guess an order of magnitude closer to the converged field and
    fewer V-cycles to 1e-8, with the same converged answer."""
    from paper_1307_6748_gb300 import isis, synth, unet
    net = unet.UNet.load(WEIGHTS)
    assert unet.UNet.meta(WEIGHTS)["h"] == 1.0
    N = 128
    ref, phi_bg, phi_net = (torch.empty((N,) * 3, dtype=torch.float64, device="cuda") for _ in range(3))
    rms = lambda x: float(torch.sqrt(torch.mean(x * x)))
    total = {"bg": 0, "net": 0}
    for seed in (9100, 9101):
        eta = synth.lognormal_eta(N, float(N), 1.5, seed, device="cuda")
        for a in (0.8, 1.0):
            _sym_solve(eta, a, ref, 1e-10, isis.ISIS_INIT_BACKGROUND)
            bg = oracle.background_field(oracle.SYMMETRON, a, a_ssb=0.5)
            net.guess(eta, a, 0.5, phi_net)
            e_bg, e_net = rms(ref - bg), rms(ref - phi_net)
            assert e_net <= 0.2 * e_bg, (seed, a, e_net, e_bg)
            i_bg = _sym_solve(eta, a, phi_bg, 1e-8, isis.ISIS_INIT_BACKGROUND)
            i_net = _sym_solve(eta, a, phi_net, 1e-8, isis.ISIS_INIT_INPUT)
            assert i_net.cycles <= i_bg.cycles, (seed, a, i_net.cycles, i_bg.cycles)
            total["bg"] += i_bg.cycles
            total["net"] += i_net.cycles
            assert rms(phi_net - phi_bg) <= 1e-7 * rms(ref)
    assert total["net"] < total["bg"], total
    assert int(net.err.item()) == 0


def test_pooled_guess(cuda_lib):
    """On a grid twice as fine as the training cell size the net runs on the 8-cell means and
    its output is prolongated; the guess is still much closer than the background."""
    from paper_1307_6748_gb300 import isis, synth, unet
    net = unet.UNet.load(WEIGHTS)
    N, box = 128, 64.0  # h = 0.5 Mpc/h
    eta = synth.lognormal_eta(N, box, 1.5, 9200, device="cuda")
    ref, phi = (torch.empty((N,) * 3, dtype=torch.float64, device="cuda") for _ in range(2))
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=3, n_coarsest=2, init=isis.ISIS_INIT_BACKGROUND)
    isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(a_ssb=0.5), isis.Grid(N, box), 1.0, eta, ref, tol=1e-10,
                           opts=opts)
    net.guess(eta, 1.0, 0.5, phi, pooled=True)
    rms = lambda x: float(torch.sqrt(torch.mean(x * x)))
    assert rms(ref - phi) <= 0.5 * rms(ref - oracle.background_field(oracle.SYMMETRON, 1.0, a_ssb=0.5))
    assert int(net.err.item()) == 0


def test_training_reduces_loss(cuda_lib):
    """Adam steps of the library's own forward/backward kernels on solver-generated pairs."""
    from paper_1307_6748_gb300 import isis, synth, unet
    N, lg = 32, 5
    pairs = []
    for seed in range(6):
        eta = synth.lognormal_eta(N, float(N), 1.5, 500 + seed, device="cuda")
        a = 0.8 if seed % 2 == 0 else 1.0
        phi = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
        _sym_solve(eta, a, phi, 1e-8, isis.ISIS_INIT_BACKGROUND)
        pairs.append((eta, a, (phi - oracle.background_field(oracle.SYMMETRON, a, a_ssb=0.5)).float().reshape(-1)))
    net = unet.UNet(seed=1, mu=-1.125, sd=1.5)
    losses = []
    for step in range(60):
        eta, a, t = pairs[step % len(pairs)]
        losses.append(float(net.train_step(eta, a, t, lg, lr=1e-3).item()))
    assert int(net.err.item()) == 0
    assert np.mean(losses[-10:]) < 0.6 * np.mean(losses[:10]), losses
