"""Learned warm start for lid-driven cavities.

A small U-Net (about 1M parameters, BF16 weights and activations, FP32
accumulation and master weights) maps the flow parameters (Re, Pe, lid speed)
and the node coordinates to the steady fields (u_x, u_y, phi, omega, and the
density rho for a consistent pressure).  The prediction only initialises the
populations -- equilibrium plus the Chapman-Enskog non-equilibrium part implied
by the predicted gradients -- and the lattice Boltzmann method then runs to the
residual tolerance exactly as from a cold start, so the method, not the
network, decides the final state.  Training data are steady solutions the method itself
produces (batched runs to the tolerance).

Every arithmetic step runs in libddflb's kernels (tensor-core GEMM, im2col,
pooling, ...): this module sequences the calls and owns the buffers (allocated
with PyTorch).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import ddflb as D

CIN, COUT = 16, 8            # padded input / output channels (5 and 5 used)
LEAKY = 1
GEMM_PATH = 0       # GEMM kernel the library uses by default (0 tcgen05, 1 mma.sync)


def specs(c: int, cin: int = CIN, cout: int = COUT):
    """(name, input channels, output channels) of the U-Net's convolutions."""
    return [("e1a", cin, c), ("e1b", c, c), ("e2a", c, 2 * c), ("e2b", 2 * c, 2 * c),
            ("e3a", 2 * c, 4 * c), ("e3b", 4 * c, 4 * c), ("b1", 4 * c, 4 * c),
            ("b2", 4 * c, 4 * c), ("d3a", 8 * c, 4 * c), ("d3b", 4 * c, 2 * c),
            ("d2a", 4 * c, 2 * c), ("d2b", 2 * c, c), ("d1a", 2 * c, c), ("d1b", c, c),
            ("head", c, cout)]


def _ck(status):
    D._check(status)


@dataclass
class _V:
    """A channel slice of an NHWC buffer."""
    t: object      # torch tensor [B, H, W, cs]
    off: int       # first channel
    C: int         # channels in the slice

    @property
    def cs(self):
        return self.t.shape[-1]

    @property
    def ptr(self):
        return self.t.data_ptr() + self.off * self.t.element_size()


class UNet:
    def __init__(self, c=32, batch=16, H=128, W=128, device="cuda", seed=0, stream=None,
                 implicit=True):
        import torch
        assert H % 8 == 0 and W % 8 == 0
        self.torch = torch
        # 3x3 convolutions with >= 64 input channels as implicit GEMMs (no
        # patch matrix); the others through im2col + GEMM
        self.implicit = implicit
        self.c, self.B, self.H, self.W = c, batch, H, W
        self.dev = torch.device(device)
        self.lib = D.load()
        self.stream = stream or torch.cuda.current_stream(self.dev)
        self.s = self.stream.cuda_stream
        self.specs = specs(c)
        self.numel = 0
        gen = torch.Generator().manual_seed(seed)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.p = {}
        for name, ci, co in self.specs:
            k = ci if name == "head" else 9 * ci
            std = math.sqrt((1.0 if name == "head" else 2.0) / k)
            w = (torch.randn(co, k, generator=gen, dtype=torch.float64) * std).float().to(self.dev)
            b = torch.zeros(co, **f32) if name == "head" else \
                (0.01 * torch.randn(co, generator=gen, dtype=torch.float64)).float().to(self.dev)
            self.p[name] = {
                "w": w, "b": b, "wb": w.to(torch.bfloat16), "gw": torch.zeros_like(w),
                "gb": torch.zeros_like(b), "mw": torch.zeros_like(w), "vw": torch.zeros_like(w),
                "mb": torch.zeros_like(b), "vb": torch.zeros_like(b),
                "wT": torch.empty(k, co, dtype=torch.bfloat16, device=self.dev), "ci": ci, "co": co}
            self.numel += w.numel() + b.numel()
        self.t = 0
        self._alloc()

    # ------------------------------------------------------------------ buffers
    def _alloc(self):
        torch, B, c = self.torch, self.B, self.c
        H, W = self.H, self.W
        L = [(H, W), (H // 2, W // 2), (H // 4, W // 4), (H // 8, W // 8)]
        self.L = L
        bf = lambda lv, ch: torch.zeros(B, *L[lv], ch, dtype=torch.bfloat16, device=self.dev)
        f32 = lambda lv, ch: torch.zeros(B, *L[lv], ch, dtype=torch.float32, device=self.dev)
        A = self.a = {}
        A["x"] = bf(0, CIN)
        for name, lv, ch in [("e1a", 0, c), ("cat1", 0, 2 * c), ("p1", 1, c), ("e2a", 1, 2 * c),
                             ("cat2", 1, 4 * c), ("p2", 2, 2 * c), ("e3a", 2, 4 * c),
                             ("cat3", 2, 8 * c), ("p3", 3, 4 * c), ("b1", 3, 4 * c),
                             ("b2", 3, 4 * c), ("d3a", 2, 4 * c), ("d3b", 2, 2 * c),
                             ("d2a", 1, 2 * c), ("d2b", 1, c), ("d1a", 0, c), ("d1b", 0, c)]:
            A[name] = bf(lv, ch)
        G = self.g = {k: f32(lv, v.shape[-1]) for k, v in A.items() if k != "x"
                      for lv in [next(i for i, s in enumerate(L) if s == tuple(v.shape[1:3]))]}
        self.out = f32(0, COUT)
        self.gout = f32(0, COUT)
        V = lambda d, n, off=0, C=None: _V(d[n], off, C if C is not None else d[n].shape[-1] - off)
        # conv layer wiring: (name, level, input view, output view, grad-in view, grad-out view)
        self.layers = [
            ("e1a", 0, V(A, "x"), V(A, "e1a"), None, V(G, "e1a")),
            ("e1b", 0, V(A, "e1a"), V(A, "cat1", c), V(G, "e1a"), V(G, "cat1", c)),
            ("e2a", 1, V(A, "p1"), V(A, "e2a"), V(G, "p1"), V(G, "e2a")),
            ("e2b", 1, V(A, "e2a"), V(A, "cat2", 2 * c), V(G, "e2a"), V(G, "cat2", 2 * c)),
            ("e3a", 2, V(A, "p2"), V(A, "e3a"), V(G, "p2"), V(G, "e3a")),
            ("e3b", 2, V(A, "e3a"), V(A, "cat3", 4 * c), V(G, "e3a"), V(G, "cat3", 4 * c)),
            ("b1", 3, V(A, "p3"), V(A, "b1"), V(G, "p3"), V(G, "b1")),
            ("b2", 3, V(A, "b1"), V(A, "b2"), V(G, "b1"), V(G, "b2")),
            ("d3a", 2, V(A, "cat3"), V(A, "d3a"), V(G, "cat3"), V(G, "d3a")),
            ("d3b", 2, V(A, "d3a"), V(A, "d3b"), V(G, "d3a"), V(G, "d3b")),
            ("d2a", 1, V(A, "cat2"), V(A, "d2a"), V(G, "cat2"), V(G, "d2a")),
            ("d2b", 1, V(A, "d2a"), V(A, "d2b"), V(G, "d2a"), V(G, "d2b")),
            ("d1a", 0, V(A, "cat1"), V(A, "d1a"), V(G, "cat1"), V(G, "d1a")),
            ("d1b", 0, V(A, "d1a"), V(A, "d1b"), V(G, "d1a"), V(G, "d1b")),
        ]
        P0 = B * H * W
        kmax = max(9 * ci for n, ci, co in self.specs if n != "head")
        ci_of = {n: ci for n, ci, _ in self.specs}
        need = max(B * L[lv][0] * L[lv][1] * 9 * ci_of[n] for n, lv, *_ in self.layers)
        self.col = torch.empty(need, dtype=torch.bfloat16, device=self.dev)
        self.colT = torch.empty(need, dtype=torch.bfloat16, device=self.dev)
        self.dcol = torch.empty(need, dtype=torch.float32, device=self.dev)
        comax = max(co for _, _, co in self.specs)
        self.gbf = torch.empty(P0 * comax, dtype=torch.bfloat16, device=self.dev)
        self.gbT = torch.empty(P0 * comax, dtype=torch.bfloat16, device=self.dev)
        self.xT = torch.empty(P0 * c, dtype=torch.bfloat16, device=self.dev)
        self.splits_max = 48
        self.partial = torch.empty(self.splits_max * comax * kmax, dtype=torch.float32,
                                   device=self.dev)
        self.mse_part = torch.empty(256, dtype=torch.float64, device=self.dev)
        self.mse_loss = torch.empty(1, dtype=torch.float64, device=self.dev)

    # ------------------------------------------------------------------ primitives
    def _gemm(self, A, B, M, N, K, lda, ldb, Cf=0, ldc=0, Cb=0, ldcb=0, bias=0, act=0, acc=0,
              splits=1):
        _ck(self.lib.ddflb_nn_gemm(A, B, M, N, K, lda, ldb, Cf or None, ldc, Cb or None, ldcb,
                                   bias or None, act, acc, splits,
                                   self.partial.data_ptr() if splits > 1 else None, self.s))

    def _splits(self, M, N, K):
        tiles = ((M + 127) // 128) * ((N + 127) // 128)
        s = max(1, min(self.splits_max, 304 // max(tiles, 1), K // 2048))
        return s

    def _implicit_ok(self, C, H, W):
        """ddflb_nn_conv3x3 takes this layer (C a multiple of 64; 128-pixel
        tiles that are whole boxes of rows and images); else im2col + GEMM."""
        if not self.implicit or C % 64 or (self.B * H * W) % 128:
            return False
        bw = min(W, 128)
        bh = min(H, 128 // bw)
        bb = 128 // (bw * bh)
        return (128 % bw == 0 and (W < 128 or W % 128 == 0) and H % bh == 0
                and bw * bh * bb == 128 and self.B % bb == 0)

    def _conv_fwd(self, name, lv, vin, vout):
        p = self.p[name]
        H, W = self.L[lv]
        P, ci, co = self.B * H * W, p["ci"], p["co"]
        assert vin.C == ci and vout.C == co
        if self._implicit_ok(ci, H, W):
            # implicit GEMM: the taps are read from the activation, no patch matrix
            _ck(self.lib.ddflb_nn_conv3x3(vin.ptr, self.B, H, W, ci, vin.cs, p["wb"].data_ptr(),
                                          co, None, 0, vout.ptr, vout.cs, p["b"].data_ptr(),
                                          LEAKY, 0, self.s))
            return
        _ck(self.lib.ddflb_nn_im2col(vin.ptr, self.B, H, W, ci, vin.cs, self.col.data_ptr(), 0,
                                     self.s))
        self._gemm(self.col.data_ptr(), p["wb"].data_ptr(), P, co, 9 * ci, 9 * ci, 9 * ci,
                   Cb=vout.ptr, ldcb=vout.cs, bias=p["b"].data_ptr(), act=LEAKY)

    def _conv_bwd(self, name, lv, vin, vout, gin, gout):
        p = self.p[name]
        H, W = self.L[lv]
        P, ci, co = self.B * H * W, p["ci"], p["co"]
        gbf, gbT = self.gbf.data_ptr(), self.gbT.data_ptr()
        # through the activation (derivative read from the stored output)
        _ck(self.lib.ddflb_nn_act_bwd(gout.ptr, vout.ptr, P, co, gout.cs, vout.cs, LEAKY, gbf, co,
                                      self.s))
        _ck(self.lib.ddflb_nn_bias_grad(gout.ptr, P, co, gout.cs, p["gb"].data_ptr(), self.s))
        # dW [co][9ci] = g^T . im2col(x)
        _ck(self.lib.ddflb_nn_transpose(gbf, P, co, co, gbT, self.s))
        _ck(self.lib.ddflb_nn_im2col(vin.ptr, self.B, H, W, ci, vin.cs, self.colT.data_ptr(), 1,
                                     self.s))
        self._gemm(gbT, self.colT.data_ptr(), co, 9 * ci, P, P, P, Cf=p["gw"].data_ptr(),
                   ldc=9 * ci, splits=self._splits(co, 9 * ci, P))
        if gin is None:
            return
        if self._implicit_ok(co, H, W):
            # dX = conv3x3(g, W with the taps mirrored and the channels swapped)
            _ck(self.lib.ddflb_nn_conv3x3_flip(p["wb"].data_ptr(), co, ci, p["wT"].data_ptr(),
                                               self.s))
            _ck(self.lib.ddflb_nn_conv3x3(gbf, self.B, H, W, co, co, p["wT"].data_ptr(), ci,
                                          gin.ptr, gin.cs, None, 0, None, 0, 0, self.s))
            return
        # dX = col2im(g . W)
        _ck(self.lib.ddflb_nn_transpose(p["wb"].data_ptr(), co, 9 * ci, 9 * ci,
                                        p["wT"].data_ptr(), self.s))
        self._gemm(gbf, p["wT"].data_ptr(), P, 9 * ci, co, co, co, Cf=self.dcol.data_ptr(),
                   ldc=9 * ci)
        _ck(self.lib.ddflb_nn_col2im(self.dcol.data_ptr(), self.B, H, W, ci, gin.ptr, gin.cs,
                                     self.s))

    def _pool(self, src, lv, dst):
        H, W = self.L[lv]
        _ck(self.lib.ddflb_nn_pool(src.ptr, self.B, H, W, src.C, src.cs, dst.ptr, dst.cs, self.s))

    def _up(self, src, lv, dst):
        H, W = self.L[lv]  # source (coarse) level
        _ck(self.lib.ddflb_nn_upsample(src.ptr, self.B, H, W, src.C, src.cs, dst.ptr, dst.cs,
                                       self.s))

    # ------------------------------------------------------------------ network
    def forward(self, x=None):
        """x: BF16 [B, H, W, 16] (copied into the input buffer if given).
        Returns the FP32 output [B, H, W, 8]."""
        if x is not None:
            self.a["x"].copy_(x)
        A, c, Ly = self.a, self.c, {n: (lv, vi, vo) for n, lv, vi, vo, _, _ in self.layers}
        cv = lambda n: self._conv_fwd(n, *Ly[n])
        cv("e1a"); cv("e1b")
        self._pool(_V(A["cat1"], c, c), 0, _V(A["p1"], 0, c))
        cv("e2a"); cv("e2b")
        self._pool(_V(A["cat2"], 2 * c, 2 * c), 1, _V(A["p2"], 0, 2 * c))
        cv("e3a"); cv("e3b")
        self._pool(_V(A["cat3"], 4 * c, 4 * c), 2, _V(A["p3"], 0, 4 * c))
        cv("b1"); cv("b2")
        self._up(_V(A["b2"], 0, 4 * c), 3, _V(A["cat3"], 0, 4 * c))
        cv("d3a"); cv("d3b")
        self._up(_V(A["d3b"], 0, 2 * c), 2, _V(A["cat2"], 0, 2 * c))
        cv("d2a"); cv("d2b")
        self._up(_V(A["d2b"], 0, c), 1, _V(A["cat1"], 0, c))
        cv("d1a"); cv("d1b")
        p = self.p["head"]
        P = self.B * self.H * self.W
        self._gemm(A["d1b"].data_ptr(), p["wb"].data_ptr(), P, COUT, c, c, c,
                   Cf=self.out.data_ptr(), ldc=COUT, bias=p["b"].data_ptr(), act=0)
        return self.out

    def backward(self, target):
        """MSE loss against target (FP32 [B, H, W, 8]); fills every gradient.
        Returns the loss as a device scalar (FP64)."""
        G, A, c = self.g, self.a, self.c
        n = self.out.numel()
        _ck(self.lib.ddflb_nn_mse(self.out.data_ptr(), target.data_ptr(), n,
                                  self.gout.data_ptr(), self.mse_part.data_ptr(),
                                  self.mse_loss.data_ptr(), self.s))
        P = self.B * self.H * self.W
        p = self.p["head"]
        gbf, gbT = self.gbf.data_ptr(), self.gbT.data_ptr()
        _ck(self.lib.ddflb_nn_cast_bf16(self.gout.data_ptr(), P, COUT, COUT, gbf, COUT, self.s))
        _ck(self.lib.ddflb_nn_bias_grad(self.gout.data_ptr(), P, COUT, COUT, p["gb"].data_ptr(),
                                        self.s))
        _ck(self.lib.ddflb_nn_transpose(gbf, P, COUT, COUT, gbT, self.s))
        _ck(self.lib.ddflb_nn_transpose(A["d1b"].data_ptr(), P, c, c, self.xT.data_ptr(), self.s))
        self._gemm(gbT, self.xT.data_ptr(), COUT, c, P, P, P, Cf=p["gw"].data_ptr(), ldc=c,
                   splits=self._splits(COUT, c, P))
        _ck(self.lib.ddflb_nn_transpose(p["wb"].data_ptr(), COUT, c, c, p["wT"].data_ptr(), self.s))
        self._gemm(gbf, p["wT"].data_ptr(), P, c, COUT, COUT, COUT, Cf=G["d1b"].data_ptr(), ldc=c)
        Ly = {n: (lv, vi, vo, gi, go) for n, lv, vi, vo, gi, go in self.layers}
        cb = lambda n: self._conv_bwd(n, *Ly[n])
        cb("d1b"); cb("d1a")
        H1, W1 = self.L[1]
        up_b = lambda g_src, lv, dst: _ck(self.lib.ddflb_nn_upsample_bwd(
            g_src.ptr, self.B, *self.L[lv], g_src.C, g_src.cs, dst.ptr, dst.cs, self.s))
        pool_b = lambda g_src, lv, dst: _ck(self.lib.ddflb_nn_pool_bwd(
            g_src.ptr, self.B, *self.L[lv], g_src.C, g_src.cs, dst.ptr, dst.cs, 1, self.s))
        up_b(_V(G["cat1"], 0, c), 1, _V(G["d2b"], 0, c))
        cb("d2b"); cb("d2a")
        up_b(_V(G["cat2"], 0, 2 * c), 2, _V(G["d3b"], 0, 2 * c))
        cb("d3b"); cb("d3a")
        up_b(_V(G["cat3"], 0, 4 * c), 3, _V(G["b2"], 0, 4 * c))
        cb("b2"); cb("b1")
        pool_b(_V(G["p3"], 0, 4 * c), 2, _V(G["cat3"], 4 * c, 4 * c))
        cb("e3b"); cb("e3a")
        pool_b(_V(G["p2"], 0, 2 * c), 1, _V(G["cat2"], 2 * c, 2 * c))
        cb("e2b"); cb("e2a")
        pool_b(_V(G["p1"], 0, c), 0, _V(G["cat1"], c, c))
        cb("e1b"); cb("e1a")
        return self.mse_loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
        self.t += 1
        for name, _, _ in self.specs:
            p = self.p[name]
            _ck(self.lib.ddflb_nn_adam(p["w"].data_ptr(), p["gw"].data_ptr(), p["mw"].data_ptr(),
                                       p["vw"].data_ptr(), p["wb"].data_ptr(), p["w"].numel(), lr,
                                       beta1, beta2, eps, self.t, wd, self.s))
            _ck(self.lib.ddflb_nn_adam(p["b"].data_ptr(), p["gb"].data_ptr(), p["mb"].data_ptr(),
                                       p["vb"].data_ptr(), None, p["b"].numel(), lr, beta1, beta2,
                                       eps, self.t, 0.0, self.s))

    # ------------------------------------------------------------------ exchange
    def get_params(self):
        """FP32 master weights as numpy, in the oracle's layout (W[Co][3][3][Ci])."""
        out = {}
        for name, ci, co in self.specs:
            p = self.p[name]
            w = p["w"].double().cpu().numpy()
            out[name] = (w if name == "head" else w.reshape(co, 3, 3, ci),
                         p["b"].double().cpu().numpy())
        return out

    def grads(self):
        out = {}
        for name, ci, co in self.specs:
            p = self.p[name]
            g = p["gw"].double().cpu().numpy()
            out[name] = (g if name == "head" else g.reshape(co, 3, 3, ci),
                         p["gb"].double().cpu().numpy())
        return out


# ---------------------------------------------------------------------- data
RE_RANGE, PE_RANGE, U_RANGE = (100.0, 3200.0), (50.0, 3200.0), (0.05, 0.1)


def draws(n: int, seed: int):
    """Seeded cavity parameters: Re log-uniform [100, 3200], Pe log-uniform
    [50, 3200], lid speed uniform [0.05, 0.1]."""
    r = np.random.default_rng(seed)
    lg = lambda lo, hi: np.exp(r.uniform(math.log(lo), math.log(hi), n))
    return [dict(re=float(a), pe=float(b), u=float(c))
            for a, b, c in zip(lg(*RE_RANGE), lg(*PE_RANGE), r.uniform(*U_RANGE, n))]


def cavity_config(d, n, check=1000):
    """Lattice parameters of one cavity: nu = U L / Re, D = U L / Pe, L = n."""
    w = D.relaxation_rate(d["u"] * n / d["re"])
    wg = D.relaxation_rate(d["u"] * n / d["pe"])
    return D.Config(nx=n, ny=n, bc="cavity", u_lid=d["u"], phi_lid=1.0, phi_wall=0.0,
                    omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                    omega_g=(0, wg, wg, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2), check_every=check)


def run_to_steady(cfgs, starts, tol=1e-8, chunk=2000, max_steps=2_000_000, device="cuda",
                  scalar_residual=True):
    """Advance cavities (one batch) until every residual -- velocity and, by
    default, scalar: the vorticity depends on both lattices -- is below tol or
    the step cap; starts[i] = (rho, ux, uy, phi, grads).  Returns the batch and
    its stats."""
    b = D.Batch(cfgs, device=device).set_run(tol=tol, steps_per_launch=chunk,
                                             scalar_residual=scalar_residual)
    b.autotune(trial_steps=4, cache=True)
    for i, s in enumerate(starts):
        b.init(i, *s)
    done = 0
    while done < max_steps:
        b.step(chunk * 10)
        done += chunk * 10
        st = b.stats()
        if (st["flags"] != 0).all():
            break
    return b, b.stats()


def input_planes(d, n, xp=np):
    """Network input: normalised log Re, log Pe, lid speed and coordinates,
    zero-padded to 16 channels ([n, n, 16])."""
    lr = (math.log(d["re"]) - 0.5 * sum(map(math.log, RE_RANGE))) / (0.5 * math.log(RE_RANGE[1] / RE_RANGE[0]))
    lp = (math.log(d["pe"]) - 0.5 * sum(map(math.log, PE_RANGE))) / (0.5 * math.log(PE_RANGE[1] / PE_RANGE[0]))
    lu = (d["u"] - 0.075) / 0.025
    x = np.zeros((n, n, CIN), np.float32)
    g = (np.arange(n) + 0.5) / n * 2 - 1
    x[..., 0], x[..., 1], x[..., 2] = lr, lp, lu
    x[..., 3] = g[None, :]
    x[..., 4] = g[:, None]
    return x


OMEGA_SCALE = 20.0  # omega L / U spans a few tens in the cavity interior


def targets(fields, d, n):
    """Network target from steady fields: (ux/U, uy/U, phi, omega n / (U s),
    (rho - 1) / U^2), zero-padded to 8 channels."""
    U = d["u"]
    t = np.zeros((n, n, COUT), np.float32)
    t[..., 0] = fields["ux"] / U
    t[..., 1] = fields["uy"] / U
    t[..., 2] = fields["phi"]
    om = np.nan_to_num(fields["omega"], nan=0.0)
    t[..., 3] = np.clip(om * n / U / OMEGA_SCALE, -5, 5)
    t[..., 4] = (fields["rho"] - 1.0) / (U * U)
    return t


def steady_fields(b, i):
    f = b.fields(i, names=("rho", "ux", "uy", "phi", "omega"))
    return {k: v.double().cpu().numpy() for k, v in f.items()}


def _grad_tensors(net):
    return [t for name, _, _ in net.specs for t in (net.p[name]["gw"], net.p[name]["gb"])]


def _min_over_ranks(v: int, world: int, device) -> int:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return int(t.item())


def train(net, X, T, epochs, lr=1e-3, seed=0, log=None, world=1, rank=0):
    """Adam on minibatches of (inputs X [N,n,n,16] BF16, targets T [N,n,n,8]
    FP32), both on the device.  Data parallel over `world` ranks: each rank
    holds its own part of the training set, computes the gradient of its
    minibatch and the ranks average the gradients before every Adam step, so
    their weights stay identical (one step = a global batch of world x B).
    Returns the loss history (per epoch, this rank's last minibatch)."""
    from .distributed import average_gradients
    torch = net.torch
    g = torch.Generator().manual_seed(seed * 1000 + rank)
    hist = []
    N = X.shape[0]
    # every rank takes the same number of steps (the collectives stay in step)
    steps_per_epoch = max(1, _min_over_ranks(N // net.B, world, X.device))
    total = epochs * steps_per_epoch
    grads = _grad_tensors(net)
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g)
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = perm[s * net.B:(s + 1) * net.B].to(X.device)
            if idx.numel() < net.B:  # a rank with fewer samples than a batch repeats them
                idx = idx.repeat((net.B + idx.numel() - 1) // idx.numel())[:net.B]
            net.forward(X.index_select(0, idx))
            loss = net.backward(T.index_select(0, idx).contiguous())
            average_gradients(grads, world)
            # cosine decay of the learning rate
            net.adam(lr=lr * 0.5 * (1 + math.cos(math.pi * k / total)))
            acc += float(loss.item()) if s == steps_per_epoch - 1 else 0.0
            k += 1
        hist.append(acc)
        if log:
            log(ep, acc)
    return hist


def predict(net, X):
    """Network output for every sample of X (padded up to a whole batch)."""
    torch = net.torch
    outs = []
    for s in range(0, X.shape[0], net.B):
        xb = X[s:s + net.B]
        if xb.shape[0] < net.B:
            xb = torch.cat([xb, xb[:1].expand(net.B - xb.shape[0], *xb.shape[1:])])
        outs.append(net.forward(xb).clone())
    return torch.cat(outs)[:X.shape[0]]


def _rest(n):
    return (np.ones((n, n), np.float32), np.zeros((n, n), np.float32),
            np.zeros((n, n), np.float32), np.zeros((n, n), np.float32), None)


def warm_fields(pred_k, d):
    """Device init fields of one cavity from its prediction [n, n, 8]
    (ddflb_warm_fields: rescale, central differences, S_xy / omega split)."""
    return D.warm_fields(pred_k.contiguous(), d["u"], OMEGA_SCALE, 0.0, 1.0)


def _inputs(ds, n, device):
    import torch
    return torch.from_numpy(np.stack([input_planes(d, n) for d in ds])).to(torch.bfloat16).to(device)


def _steady_data(ds, n, starts, tol, max_steps, device):
    """Run the cavities `ds` from `starts` to the tolerance in one batch; the
    converged ones become training pairs (input planes, targets)."""
    b, st = run_to_steady([cavity_config(d, n) for d in ds], starts, tol=tol,
                          max_steps=max_steps, device=device)
    ok = [i for i in range(len(ds)) if st["flags"][i] == D.INST_CONVERGED]
    X = np.stack([input_planes(ds[i], n) for i in ok]) if ok else np.zeros((0, n, n, CIN), np.float32)
    T = np.stack([targets(steady_fields(b, i), ds[i], n) for i in ok]) if ok else np.zeros((0, n, n, COUT), np.float32)
    steps = [int(st["steps_to_tol"][i]) for i in ok]
    del b
    return X, T, steps


def _omega_err(f, ref):
    a, r = f["omega"], ref["omega"]
    m = np.isfinite(a) & np.isfinite(r)
    return float(np.linalg.norm((a - r)[m]) / np.linalg.norm(r[m]))


def experiment(n=128, n_train=512, n_test=64, epochs=60, batch=16, c=32, seed=1, tol=1e-8,
               max_steps=2_000_000, device="cuda", log=print, boot=0, boot_epochs=None,
               ref_tol=1e-10, ref_factor=4, world=None, rank=None):
    """The learned warm start, end to end, data parallel over the ranks of an
    initialised process group (every rank holds its share of the draws):

    1. training data: the method's own steady solutions.  With boot > 0 the
       first `boot` draws run cold (from rest), a network trained on them
       warm-starts the remaining draws, and every draw still runs to the
       tolerance, so the data are the method's results either way;
    2. training on the GPU with the library's kernels (gradients averaged
       over ranks);
    3. held-out draws run to the tolerance from rest (cold) and from the
       network's prediction (warm), next to a long-run reference from rest
       (tolerance ref_tol, at most ref_factor times the cold run's steps), in
       one batch.  A run that hits the step cap counts at the cap.

    Returns the summary on rank 0 (per-case rows in global order) and None on
    the other ranks."""
    import time
    import torch
    from .distributed import gather_indexed, shard_indices, world_and_rank
    if world is None or rank is None:
        world, rank = world_and_rank()
    t0 = time.perf_counter()
    tr, te = draws(n_train, seed), draws(n_test, seed + 1000)
    mine_tr = shard_indices(len(tr), rank, world)
    mine_te = shard_indices(len(te), rank, world)
    n_boot = 0 if boot <= 0 else len(shard_indices(min(boot, n_train), rank, world))
    net = UNet(c=c, batch=batch, H=n, W=n, device=device, seed=seed)
    # 1. training data (this rank's share)
    d_cold = [tr[i] for i in mine_tr[:n_boot]] if n_boot else [tr[i] for i in mine_tr]
    Xc, Tc, steps_c = _steady_data(d_cold, n, [_rest(n) for _ in d_cold], tol, max_steps, device)
    t_cold = time.perf_counter() - t0
    log(f"rank {rank}: {len(steps_c)}/{len(d_cold)} cold cavities converged in {t_cold:.1f} s")
    X_all, T_all, steps_w, t_boot_train, t_warm = Xc, Tc, [], 0.0, 0.0
    if n_boot:
        Xd = torch.from_numpy(Xc).to(torch.bfloat16).to(device)
        Td = torch.from_numpy(Tc).to(device)
        t1 = time.perf_counter()
        train(net, Xd, Td, boot_epochs or epochs, world=world, rank=rank)
        torch.cuda.synchronize()
        t_boot_train = time.perf_counter() - t1
        del Xd, Td
        d_warm = [tr[i] for i in mine_tr[n_boot:]]
        t2 = time.perf_counter()
        pred = predict(net, _inputs(d_warm, n, device)) if d_warm else None
        starts = [warm_fields(pred[k], d) for k, d in enumerate(d_warm)]
        del pred
        Xw, Tw, steps_w = _steady_data(d_warm, n, starts, tol, max_steps, device)
        del starts
        t_warm = time.perf_counter() - t2
        log(f"rank {rank}: {len(steps_w)}/{len(d_warm)} warm-started cavities converged in {t_warm:.1f} s")
        X_all, T_all = np.concatenate([Xc, Xw]), np.concatenate([Tc, Tw])
    # 2. training on everything this rank holds
    Xd = torch.from_numpy(X_all).to(torch.bfloat16).to(device)
    Td = torch.from_numpy(T_all).to(device)
    del X_all, T_all
    t3 = time.perf_counter()
    hist = train(net, Xd, Td, epochs, seed=seed + 1, world=world, rank=rank,
                 log=lambda e, l: log(f"epoch {e} loss {l:.4e}") if e % 10 == 0 and rank == 0 else None)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t3
    n_train_ok = int(round(_sum_over_ranks(float(Xd.shape[0]), world, device)))
    del Xd, Td
    # 3. held-out: cold, warm and the long-run reference side by side
    ds = [te[i] for i in mine_te]
    rows = {}
    if ds:
        t4 = time.perf_counter()
        pred = predict(net, _inputs(ds, n, device))
        k_ = len(ds)
        cfgs = [cavity_config(d, n) for d in ds] * 2
        starts = [_rest(n) for _ in ds] + [warm_fields(pred[k], d) for k, d in enumerate(ds)]
        b, st = run_to_steady(cfgs, starts, tol=tol, max_steps=max_steps, device=device)
        capped = lambda i: int(st["steps_to_tol"][i]) if st["flags"][i] == D.INST_CONVERGED else max_steps
        cold = [capped(k) for k in range(k_)]
        warm = [capped(k + k_) for k in range(k_)]
        fc = [steady_fields(b, k) for k in range(k_)]
        fw = [steady_fields(b, k + k_) for k in range(k_)]
        ok_c = [bool(st["flags"][k] == D.INST_CONVERGED) for k in range(k_)]
        ok_w = [bool(st["flags"][k + k_] == D.INST_CONVERGED) for k in range(k_)]
        del b
        # long-run reference from rest: ref_tol, at most ref_factor x the cold steps
        rb = D.Batch([cavity_config(d, n) for d in ds], device=device).set_run(
            tol=ref_tol, steps_per_launch=2000, scalar_residual=True)
        rb.autotune(trial_steps=4, cache=True)
        for k in range(k_):
            rb.set_instance_run(k, ref_tol, ref_factor * cold[k])
            rb.init(k, *_rest(n))
        while True:
            rb.step(20000)
            rs = rb.stats()
            if (rs["flags"] != 0).all():
                break
        fr = [steady_fields(rb, k) for k in range(k_)]
        rsteps = [int(rs["state_time"][k] - rs["init_time"][k]) for k in range(k_)]
        del rb
        t_eval = time.perf_counter() - t4
        for k, d in enumerate(ds):
            tgt = targets(fc[k], d, n)
            pk = pred[k].float().cpu().numpy()
            rows[mine_te[k]] = dict(
                k=mine_te[k], cold=cold[k], warm=warm[k], cold_converged=ok_c[k],
                warm_converged=ok_w[k], ratio=cold[k] / max(warm[k], 1),
                omega_err_cold=_omega_err(fc[k], fr[k]), omega_err_warm=_omega_err(fw[k], fr[k]),
                omega_rel_diff=_omega_err(fw[k], fc[k]), ref_steps=rsteps[k],
                ref_converged=bool(rs["flags"][k] == D.INST_CONVERGED),
                pred_rel_err=float(np.linalg.norm(pk[..., :4] - tgt[..., :4]) /
                                   np.linalg.norm(tgt[..., :4])), **d)
        log(f"rank {rank}: held-out evaluation in {t_eval:.1f} s")
    timing = dict(data_cold=t_cold, boot_train=t_boot_train, data_warm=t_warm, train=t_train)
    allrows = gather_indexed(rows, world)
    times = gather_indexed({rank: timing}, world)
    data_steps = gather_indexed({rank: (sum(steps_c), len(steps_c), sum(steps_w), len(steps_w))}, world)
    if allrows is None:
        return None
    ratios = [r["ratio"] for r in allrows]
    cold_sum = sum(r["cold"] for r in allrows)
    warm_sum = sum(r["warm"] for r in allrows)
    med = lambda v: float(np.median(v)) if v else None
    sc = sum(x[0] for x in data_steps); nc = sum(x[1] for x in data_steps)
    sw = sum(x[2] for x in data_steps); nw = sum(x[3] for x in data_steps)
    return dict(
        grid=n, world=world, n_train=n_train_ok, n_train_drawn=len(tr), n_boot=min(boot, n_train),
        n_test=len(te), n_test_cold_converged=sum(r["cold_converged"] for r in allrows),
        n_test_warm_converged=sum(r["warm_converged"] for r in allrows),
        n_test_both_converged=sum(r["cold_converged"] and r["warm_converged"] for r in allrows),
        params=net.numel, epochs=epochs, final_loss=hist[-1] if hist else None,
        steps_cold_total=cold_sum, steps_warm_total=warm_sum,
        steps_saved_ratio=cold_sum / max(warm_sum, 1), median_ratio=med(ratios),
        capped_counted_at=max_steps,
        omega_err_cold_median=med([r["omega_err_cold"] for r in allrows]),
        omega_err_warm_median=med([r["omega_err_warm"] for r in allrows]),
        omega_err_cold_max=max(r["omega_err_cold"] for r in allrows),
        omega_err_warm_max=max(r["omega_err_warm"] for r in allrows),
        omega_rel_diff_max=max(r["omega_rel_diff"] for r in allrows),
        ref_tol=ref_tol, ref_factor=ref_factor,
        ref_converged=sum(r["ref_converged"] for r in allrows),
        pred_rel_err_median=med([r["pred_rel_err"] for r in allrows]),
        data_steps_cold_mean=sc / max(nc, 1), data_steps_warm_mean=sw / max(nw, 1),
        seconds=max(sum(t.values()) for t in times), timing_rank0=times[0], rows=allrows)


def _sum_over_ranks(v: float, world: int, device) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
