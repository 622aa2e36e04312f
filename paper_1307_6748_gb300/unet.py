"""Learned initial guess for the symmetron FAS solve: a small 3-D U-Net whose
forward pass, backward pass and Adam step all run in the library's kernels
(include/isis_unet.h; tensor-core convolutions).  PyTorch only allocates
device memory.  The paper has no learned component: the net proposes the
initial guess and the multigrid solver always finishes the solve.

Network (4 levels, channels 16-32-64-64, skip connections by concatenation):
    e0 = relu(conv(x0))            grid n        16
    e1 = relu(conv(pool(e0)))      n/2           32
    e2 = relu(conv(pool(e1)))      n/4           64
    e3 = relu(conv(pool(e2)))      n/8           64
    d2 = relu(conv([up(e3), e2]))  n/4           64
    d1 = relu(conv([up(d2), e1]))  n/2           32
    d0 = relu(conv([up(d1), e0]))  n             16
    p  = head . d0 + b                           1
Input features: (ln eta - mu)/sd and (a - 0.9)/0.1.  Target: p ~ (chi - chi_bg(a)) / scale.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import isis

LAYERS = [("e0", (16,), 16), ("e1", (16,), 32), ("e2", (32,), 64), ("e3", (64,), 64),
          ("d2", (64, 64), 64), ("d1", (64, 32), 32), ("d0", (32, 16), 16)]
HEAD = 17  # 16 weights + bias

_bound = False


def _lib():
    global _bound
    lib = isis.load()
    if _bound:
        return lib
    vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
    sig = {
        "isis_unet_conv3_fwd": [vp, i, i, vp, i, i, vp, vp, i, i, vp, vp, vp],
        "isis_unet_conv3_dgrad": [vp, i, i, vp, i, vp, vp, vp],
        "isis_unet_conv3_wgrad": [vp, i, i, vp, i, i, vp, i, vp, vp, vp],
        "isis_unet_input": [vp, i, f, f, f, vp, vp, vp],
        "isis_unet_stem_fwd": [vp, i, vp, i, vp, vp, vp, vp],
        "isis_unet_pack_w": [vp, i, i, vp, vp],
        "isis_unet_line_ok": [i, i, i, i, i],
        "isis_unet_line_fwd": [vp, i, i, vp, i, i, vp, vp, i, i, vp, vp, vp],
        "isis_unet_pool_fwd": [vp, i, i, vp, vp],
        "isis_unet_pool_bwd": [vp, i, i, vp, vp],
        "isis_unet_relu_bwd": [vp, vp, ctypes.c_int64, vp, vp],
        "isis_unet_split_bwd": [vp, i, i, i, i, vp, vp, vp],
        "isis_unet_head": [vp, i, i, vp, vp, f, vp, vp, vp, vp, vp],
        "isis_unet_bias_grad": [vp, i, i, vp, vp],
        "isis_unet_adam": [vp, vp, vp, vp, ctypes.c_int64, f, f, f, f, i, vp, vp],
        "isis_unet_transpose_w": [vp, i, i, vp, vp],
        "isis_unet_to_bf16": [vp, ctypes.c_int64, vp, vp],
        "isis_unet_guess": [vp, i, d, d, vp, vp],
        "isis_unet_input_pooled": [vp, i, f, f, f, vp, vp],
        "isis_unet_guess_fine": [vp, i, d, d, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _bound = True
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ck(st, what):
    if st != 0:
        raise isis.IsisError(st, f"{what}: {isis.strerror(st)}")


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class UNet:
    """Parameters live in flat FP32 buffers (master copy, gradient, Adam
    moments) with a BF16 copy, per-tap transposes (input gradient) and
    per-stage packings (line convolution) for the convolutions.  Activations
    are channel-planar (include/isis_unet.h)."""

    def __init__(self, device="cuda", seed: int = 0, mu: float = -1.125, sd: float = 1.5, scale: float = 0.1):
        self.dev = torch.device(device)
        self.mu, self.sd, self.scale = mu, sd, scale
        rng = np.random.Generator(np.random.PCG64(seed))
        segs, off = {}, 0
        for name, pieces, cout in LAYERS:
            cin = sum(pieces)
            segs[name + ".W"] = (off, (27, cout, cin))
            off += _pad(27 * cout * cin)
            segs[name + ".b"] = (off, (cout,))
            off += _pad(cout)
        segs["head"] = (off, (HEAD,))
        off += _pad(HEAD)
        self.segs, self.n = segs, off
        host = np.zeros(off, dtype=np.float32)
        for name, pieces, cout in LAYERS:
            cin = sum(pieces)
            o, shp = segs[name + ".W"]
            host[o:o + 27 * cout * cin] = (rng.standard_normal(27 * cout * cin) * math.sqrt(2.0 / (27 * cin)))
        o, _ = segs["head"]
        host[o:o + 16] = rng.standard_normal(16) * 0.1
        f32 = dict(device=self.dev, dtype=torch.float32)
        self.P = torch.from_numpy(host).to(self.dev)
        self.G = torch.zeros(off, **f32)
        self.M1 = torch.zeros(off, **f32)
        self.M2 = torch.zeros(off, **f32)
        self.Pb = torch.empty(off, device=self.dev, dtype=torch.bfloat16)
        self.Wt = {name: torch.empty(27 * cout * sum(pieces), device=self.dev, dtype=torch.bfloat16)
                   for name, pieces, cout in LAYERS}
        self.Wl = {name: torch.empty(27 * cout * sum(pieces), device=self.dev, dtype=torch.bfloat16)
                   for name, pieces, cout in LAYERS}
        self.err = torch.zeros(1, device=self.dev, dtype=torch.int32)
        self.loss = torch.zeros(1, device=self.dev, dtype=torch.float64)
        self.step = 0
        self._acts = {}
        self._refresh()

    # -- parameter views --------------------------------------------------
    def view(self, buf, key):
        o, shp = self.segs[key]
        return buf[o:o + int(np.prod(shp))]

    def _refresh(self):
        """BF16 copy of the parameters, then the per-tap transposes and the line-kernel packing."""
        lib, s = _lib(), _s()
        _ck(lib.isis_unet_to_bf16(_p(self.P), self.n, _p(self.Pb), s), "to_bf16")
        self._derived()

    def _derived(self):
        lib, s = _lib(), _s()
        for name, pieces, cout in LAYERS:
            w = _p(self.view(self.Pb, name + ".W"))
            _ck(lib.isis_unet_transpose_w(w, cout, sum(pieces), _p(self.Wt[name]), s), "transpose_w")
            _ck(lib.isis_unet_pack_w(w, cout, sum(pieces), _p(self.Wl[name]), s), "pack_w")

    def state(self) -> dict:
        host = self.P.cpu().numpy()
        out = {"mu": self.mu, "sd": self.sd, "scale": self.scale}
        for k, (o, shp) in self.segs.items():
            out[k] = host[o:o + int(np.prod(shp))].reshape(shp).copy()
        return out

    def save(self, path: str, **meta):
        """Parameters and input/output scalings, plus metadata (model, training cell size h, ...)."""
        np.savez_compressed(path, **self.state(), **{"meta_" + k: v for k, v in meta.items()})

    @staticmethod
    def meta(path: str) -> dict:
        z = np.load(path)
        return {k[5:]: z[k].item() for k in z.files if k.startswith("meta_")}

    @classmethod
    def load(cls, path: str, device="cuda"):
        z = np.load(path)
        net = cls(device, mu=float(z["mu"]), sd=float(z["sd"]), scale=float(z["scale"]))
        host = net.P.cpu().numpy()
        for k, (o, shp) in net.segs.items():
            host[o:o + int(np.prod(shp))] = z[k].reshape(-1)
        net.P.copy_(torch.from_numpy(host))
        net._refresh()
        return net

    # -- activations ------------------------------------------------------
    def acts(self, lg: int):
        if lg in self._acts:
            return self._acts[lg]
        V = [1 << (3 * (lg - l)) for l in range(4)]
        bf = dict(device=self.dev, dtype=torch.bfloat16)
        f32 = dict(device=self.dev, dtype=torch.float32)
        A = {"x0": torch.empty(V[0] * 16, **bf), "f2": torch.empty(V[0] * 2, **bf), "e0": torch.empty(V[0] * 16, **bf),
             "p0": torch.empty(V[1] * 16, **bf), "e1": torch.empty(V[1] * 32, **bf),
             "p1": torch.empty(V[2] * 32, **bf), "e2": torch.empty(V[2] * 64, **bf),
             "p2": torch.empty(V[3] * 64, **bf), "e3": torch.empty(V[3] * 64, **bf),
             "d2": torch.empty(V[2] * 64, **bf), "d1": torch.empty(V[1] * 32, **bf),
             "d0": torch.empty(V[0] * 16, **bf), "pred": torch.empty(V[0], **f32)}
        self._acts[lg] = (V, A)
        return self._acts[lg]

    def grads_bufs(self, lg: int):
        key = ("g", lg)
        if key in self._acts:
            return self._acts[key]
        V = [1 << (3 * (lg - l)) for l in range(4)]
        bf = dict(device=self.dev, dtype=torch.bfloat16)
        f32 = dict(device=self.dev, dtype=torch.float32)
        B = {"dz": torch.empty(V[0] * 64, **bf), "dx": torch.empty(V[0] * 48, **f32),
             "dd0": torch.empty(V[0] * 16, **f32), "de0": torch.empty(V[0] * 16, **f32),
             "dd1": torch.empty(V[1] * 32, **f32), "de1": torch.empty(V[1] * 32, **f32),
             "dd2": torch.empty(V[2] * 64, **f32), "de2": torch.empty(V[2] * 64, **f32),
             "de3": torch.empty(V[3] * 64, **f32), "dp": torch.empty(V[1] * 16, **f32)}
        self._acts[key] = B
        return B

    # -- forward ----------------------------------------------------------
    def features(self, eta: torch.Tensor, a: float, lg: int, x16: bool = True):
        """The two input features (f2) and, for training, their 16-channel form (x0)."""
        V, A = self.acts(lg)
        _ck(_lib().isis_unet_input(_p(eta), lg, self.mu, 1.0 / self.sd, (a - 0.9) / 0.1,
                                   _p(A["x0"]) if x16 else None, _p(A["f2"]), _s()), "unet_input")

    def forward(self, lg: int, pred=True):
        """Forward pass on the features already in acts(lg)['f2']."""
        lib, s = _lib(), _s()
        V, A = self.acts(lg)
        P, Pb, err = self.P, self.Pb, self.err

        def conv(name, s1, c1, lg1, s2, c2, lgo, out, cout):
            b = _p(self.view(P, name + ".b"))
            if lib.isis_unet_line_ok(c1, lg1, c2, lgo, cout):
                _ck(lib.isis_unet_line_fwd(_p(s1), c1, lg1, _p(s2), c2, lgo, _p(self.Wl[name]), b, cout, 1, _p(out),
                                           _p(err), s), name)
            else:
                _ck(lib.isis_unet_conv3_fwd(_p(s1), c1, lg1, _p(s2), c2, lgo, _p(self.view(Pb, name + ".W")), b, cout,
                                            1, _p(out), _p(err), s), name)

        def pool(x, C, lgc, y):
            _ck(lib.isis_unet_pool_fwd(_p(x), C, lgc, _p(y), s), "pool")

        _ck(lib.isis_unet_stem_fwd(_p(A["f2"]), lg, _p(self.view(Pb, "e0.W")), 16, _p(self.view(P, "e0.b")),
                                   _p(A["e0"]), _p(err), s), "e0")
        pool(A["e0"], 16, lg - 1, A["p0"])
        conv("e1", A["p0"], 16, lg - 1, None, 0, lg - 1, A["e1"], 32)
        pool(A["e1"], 32, lg - 2, A["p1"])
        conv("e2", A["p1"], 32, lg - 2, None, 0, lg - 2, A["e2"], 64)
        pool(A["e2"], 64, lg - 3, A["p2"])
        conv("e3", A["p2"], 64, lg - 3, None, 0, lg - 3, A["e3"], 64)
        conv("d2", A["e3"], 64, lg - 3, A["e2"], 64, lg - 2, A["d2"], 64)
        conv("d1", A["d2"], 64, lg - 2, A["e1"], 32, lg - 1, A["d1"], 32)
        conv("d0", A["d1"], 32, lg - 1, A["e0"], 16, lg, A["d0"], 16)
        if pred:
            _ck(lib.isis_unet_head(_p(A["d0"]), 16, lg, _p(self.view(P, "head")), None, 0.0, _p(A["pred"]), None,
                                   None, None, s), "head")
        return A["pred"]

    # -- training ---------------------------------------------------------
    def train_step(self, eta: torch.Tensor, a: float, target: torch.Tensor, lg: int, lr: float = 1e-3):
        """One Adam step on the squared error of p against target/scale; returns the loss tensor (device)."""
        lib, s = _lib(), _s()
        self.features(eta, a, lg)
        self.forward(lg, pred=False)
        V, A = self.acts(lg)
        B = self.grads_bufs(lg)
        P, Pb, G, err = self.P, self.Pb, self.G, self.err
        G.zero_()
        self.loss.zero_()
        _ck(lib.isis_unet_head(_p(A["d0"]), 16, lg, _p(self.view(P, "head")), _p(target), 1.0 / self.scale,
                               _p(A["pred"]), _p(B["dd0"]), _p(self.view(G, "head")), _p(self.loss), s), "head")

        def layer(name, dY, Y, cout, s1, c1, lg1, s2, c2, lgo, din):
            n = (1 << (3 * lgo)) * cout
            dz = B["dz"][:n]
            _ck(lib.isis_unet_relu_bwd(_p(dY), _p(Y), n, _p(dz), s), "relu_bwd")
            _ck(lib.isis_unet_conv3_wgrad(_p(s1), c1, lg1, _p(s2), c2, lgo, _p(dz), cout,
                                          _p(self.view(G, name + ".W")), _p(err), s), name + " wgrad")
            _ck(lib.isis_unet_bias_grad(_p(dz), cout, lgo, _p(self.view(G, name + ".b")), s), "bias_grad")
            if din is not None:
                _ck(lib.isis_unet_conv3_dgrad(_p(dz), cout, lgo, _p(self.Wt[name]), c1 + c2, _p(din), _p(err), s),
                    name + " dgrad")

        dx = B["dx"]
        # decoder
        B["de0"].zero_()
        layer("d0", B["dd0"], A["d0"], 16, A["d1"], 32, lg - 1, A["e0"], 16, lg, dx)
        _ck(lib.isis_unet_split_bwd(_p(dx), 32, 16, lg, 1, _p(B["dd1"]), _p(B["de0"]), s), "split")
        B["de1"].zero_()
        layer("d1", B["dd1"], A["d1"], 32, A["d2"], 64, lg - 2, A["e1"], 32, lg - 1, dx)
        _ck(lib.isis_unet_split_bwd(_p(dx), 64, 32, lg - 1, 1, _p(B["dd2"]), _p(B["de1"]), s), "split")
        B["de2"].zero_()
        layer("d2", B["dd2"], A["d2"], 64, A["e3"], 64, lg - 3, A["e2"], 64, lg - 2, dx)
        _ck(lib.isis_unet_split_bwd(_p(dx), 64, 64, lg - 2, 1, _p(B["de3"]), _p(B["de2"]), s), "split")
        # encoder
        dp = B["dp"]
        layer("e3", B["de3"], A["e3"], 64, A["p2"], 64, lg - 3, None, 0, lg - 3, dp)
        _ck(lib.isis_unet_pool_bwd(_p(dp), 64, lg - 3, _p(B["de2"]), s), "pool_bwd")
        layer("e2", B["de2"], A["e2"], 64, A["p1"], 32, lg - 2, None, 0, lg - 2, dp)
        _ck(lib.isis_unet_pool_bwd(_p(dp), 32, lg - 2, _p(B["de1"]), s), "pool_bwd")
        layer("e1", B["de1"], A["e1"], 32, A["p0"], 16, lg - 1, None, 0, lg - 1, dp)
        _ck(lib.isis_unet_pool_bwd(_p(dp), 16, lg - 1, _p(B["de0"]), s), "pool_bwd")
        layer("e0", B["de0"], A["e0"], 16, A["x0"], 16, lg, None, 0, lg, None)
        # Adam, then the BF16 copies
        self.step += 1
        _ck(lib.isis_unet_adam(_p(P), _p(G), _p(self.M1), _p(self.M2), self.n, lr, 0.9, 0.999, 1e-8, self.step,
                               _p(Pb), s), "adam")
        self._derived()
        return self.loss

    # -- the guess ----------------------------------------------------------
    def guess(self, eta: torch.Tensor, a: float, a_ssb: float, phi: torch.Tensor, pooled: bool = False):
        """phi = chi_bg(a) + scale * net(eta, a): FP64 initial guess for isis_scalar_solve.

        pooled: eta's grid is twice as fine as the net's training cell size; the net runs on the
        8-cell means and its output is prolongated (trilinear) to eta's grid."""
        N = eta.shape[0]
        lg = int(round(math.log2(N))) - (1 if pooled else 0)
        lib = _lib()
        if pooled:
            V, A = self.acts(lg)
            _ck(lib.isis_unet_input_pooled(_p(eta), lg, self.mu, 1.0 / self.sd, (a - 0.9) / 0.1, _p(A["f2"]), _s()),
                "input_pooled")
        else:
            self.features(eta, a, lg, x16=False)
        pred = self.forward(lg)
        bg = isis.isis_background_field(isis.ISIS_SYMMETRON, isis.Params(a_ssb=a_ssb), a)
        if pooled:
            _ck(lib.isis_unet_guess_fine(_p(pred), lg, bg, self.scale, _p(phi), _s()), "guess_fine")
        else:
            _ck(lib.isis_unet_guess(_p(pred), lg, bg, self.scale, _p(phi), _s()), "guess")
        return phi


def _pad(n: int) -> int:
    return (n + 15) // 16 * 16
