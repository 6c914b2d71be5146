"""Surrogate network kernels against FP64 references: the tensor-core GEMM
against a float64 matrix product of the same BF16 inputs, and the full U-Net
(output and every parameter gradient) against the FP64 network oracle run on
the GPU's BF16 weights and input.  BF16 rounding of the activations between
layers bounds the agreement (about 2^-9 per layer)."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as OU
from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture
def gemm_path():
    """Select a GEMM kernel for one test, then restore the default."""
    lib = D.load()
    yield lambda p: D._check(lib.ddflb_nn_set_gemm_path(p))
    D._check(lib.ddflb_nn_set_gemm_path(S.GEMM_PATH))


def take_error():
    e = ctypes.c_int32(-1)
    D._check(D.load().ddflb_nn_take_error(ctypes.byref(e), None))
    return e.value


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("M,N,K,splits,bias,act", [
    (1, 1, 8, 1, False, 0), (130, 70, 40, 1, True, 1), (257, 129, 136, 1, True, 0),
    (1000, 64, 4096, 7, False, 0), (64, 2304, 8192, 16, True, 1), (300, 8, 32, 1, True, 0),
    (4096, 128, 576, 1, True, 1), (513, 256, 1152, 3, False, 0),
    # more tiles than SMs (the persistent kernel), ragged in M, N and K
    (40000, 96, 200, 1, True, 1), (20000, 32, 72, 1, False, 0), (1300, 64, 8192, 16, False, 0)])
def test_gemm_against_float64(M, N, K, splits, bias, act, path, gemm_path):
    """The GEMM kernels (0: tcgen05 persistent, 1: mma.sync, 2: tcgen05 one
    tile per CTA) against a float64 product of the same BF16 operands, over
    ragged multi-tile shapes and split-K."""
    gemm_path(path)
    g = torch.Generator().manual_seed(M * 7 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bm = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    b = torch.randn(N, generator=g).float().cuda() if bias else None
    Cf = torch.empty(M, N, device="cuda")
    Cb = torch.empty(M, N, dtype=torch.bfloat16, device="cuda") if splits == 1 else None
    part = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
    lib = D.load()
    D._check(lib.ddflb_nn_gemm(A.data_ptr(), Bm.data_ptr(), M, N, K, K, K, Cf.data_ptr(), N,
                               Cb.data_ptr() if Cb is not None else None, N,
                               b.data_ptr() if b is not None else None, act, 0, splits,
                               part.data_ptr() if part is not None else None,
                               torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    ref = A.double().cpu().numpy() @ Bm.double().cpu().numpy().T
    if bias:
        ref = ref + b.double().cpu().numpy()
    if act == 1:
        ref = np.where(ref > 0, ref, 0.02 * ref)
    got = Cf.double().cpu().numpy()
    # FP32 accumulation of exact BF16 products: relative error ~ sqrt(K) * 2^-24
    assert np.abs(got - ref).max() <= 1e-5 * (np.abs(ref).max() + 1) * max(1, math.sqrt(K / 64)), \
        np.abs(got - ref).max()
    if Cb is not None:
        assert rel(Cb.double().cpu().numpy(), ref) < 4e-3
    assert take_error() == 0


@pytest.mark.parametrize("path", [0, 1, 2])
def test_gemm_accumulate_and_strides(path, gemm_path):
    """accumulate = 1 adds to Cf; lda, ldb, ldc larger than K and N."""
    gemm_path(path)
    M, N, K, lda, ldb, ldc = 333, 96, 200, 216, 208, 100
    g = torch.Generator().manual_seed(5)
    A = torch.randn(M, lda, generator=g).to(torch.bfloat16).cuda()
    Bm = torch.randn(N, ldb, generator=g).to(torch.bfloat16).cuda()
    C0 = torch.randn(M, ldc, generator=g).cuda()
    Cf = C0.clone()
    D._check(D.load().ddflb_nn_gemm(A.data_ptr(), Bm.data_ptr(), M, N, K, lda, ldb, Cf.data_ptr(),
                                    ldc, None, 0, None, 0, 1, 1, None,
                                    torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    ref = C0.double().cpu().numpy()
    ref[:, :N] += A[:, :K].double().cpu().numpy() @ Bm[:, :K].double().cpu().numpy().T
    got = Cf.double().cpu().numpy()
    assert np.abs(got - ref).max() < 1e-4
    assert take_error() == 0


def test_gemm_rejects_bad_shapes():
    lib = D.load()
    st = lib.ddflb_nn_gemm(16, 16, 4, 4, 12, 12, 12, 16, 4, None, 0, None, 0, 0, 1, None, None)
    assert st == D.EINVAL and b"multiples of 8" in lib.ddflb_last_error()


def make_net(c=8, batch=2, H=16, seed=0):
    net = S.UNet(c=c, batch=batch, H=H, W=H, seed=seed)
    r = np.random.default_rng(seed + 1)
    x = np.zeros((batch, H, H, S.CIN), np.float32)
    x[..., :5] = r.standard_normal((batch, H, H, 5))
    t = np.zeros((batch, H, H, S.COUT), np.float32)
    t[..., :5] = r.standard_normal((batch, H, H, 5))
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    return net, xb, torch.from_numpy(t).cuda()


def oracle_params(net):
    """The GPU's BF16 weights (what its GEMMs use) and FP32 biases, in FP64."""
    P = {}
    for name, ci, co in net.specs:
        p = net.p[name]
        w = p["wb"].double().cpu().numpy()
        P[name] = (w if name == "head" else w.reshape(co, 3, 3, ci), p["b"].double().cpu().numpy())
    return P


def test_unet_forward_and_gradients_match_oracle():
    net, xb, t = make_net()
    out = net.forward(xb)
    loss = net.backward(t)
    torch.cuda.synchronize()
    P = oracle_params(net)
    x64 = xb.double().cpu().numpy()
    ref_out, cache = OU.forward(P, x64)
    G = OU.backward(P, cache, ref_out, t.double().cpu().numpy())
    e_out = rel(out.double().cpu().numpy(), ref_out)
    assert e_out < 2e-2, e_out
    assert abs(float(loss.item()) - OU.loss(ref_out, t.double().cpu().numpy())) < 2e-2 * float(loss.item())
    got = net.grads()
    worst = {}
    for name, _, _ in net.specs:
        for k in (0, 1):
            worst[(name, k)] = rel(got[name][k], G[name][k])
    print("gradient relative errors", {f"{n}{'.b' if k else '.w'}": round(v, 4) for (n, k), v in worst.items()})
    assert max(worst.values()) < 6e-2, worst


def test_training_reduces_loss():
    """A few hundred Adam steps on a fixed smooth target: the loss falls by an
    order of magnitude (the network and its gradients are wired correctly)."""
    net, xb, _ = make_net(c=8, batch=4, H=32, seed=3)
    H = 32
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, H), indexing="ij")
    t = np.zeros((4, H, H, S.COUT), np.float32)
    for k in range(4):
        t[k, ..., 0] = np.sin(np.pi * xx * (k + 1) / 2) * yy
        t[k, ..., 1] = np.cos(np.pi * yy) * 0.5
    tt = torch.from_numpy(t).cuda()
    first = None
    for it in range(400):
        net.forward(xb)
        loss = float(net.backward(tt).item())
        first = first if first is not None else loss
        net.adam(lr=3e-3)
    assert loss < 0.1 * first, (first, loss)


def im2col_np(X, C):
    """col[p][(kh*3 + kw)*C + c] = X[b][h+kh-1][w+kw-1][c], zero padding."""
    B, H, W, _ = X.shape
    Xp = np.zeros((B, H + 2, W + 2, C), X.dtype)
    Xp[:, 1:-1, 1:-1] = X[..., :C]
    cols = [Xp[:, kh:kh + H, kw:kw + W] for kh in range(3) for kw in range(3)]
    return np.concatenate(cols, axis=-1).reshape(B * H * W, 9 * C)


@pytest.mark.parametrize("C,cs", [(16, 16), (32, 48), (6, 10)])
def test_im2col_both_layouts(C, cs):
    """Vector (C, cs multiples of 8) and scalar paths, plain and transposed."""
    B, H, W = 3, 17, 23
    g = torch.Generator().manual_seed(C + cs)
    X = torch.randn(B, H, W, cs, generator=g).to(torch.bfloat16).cuda()
    want = im2col_np(X.float().cpu().numpy(), C)
    lib = D.load()
    for transposed in (0, 1):
        out = torch.empty(want.size, dtype=torch.bfloat16, device="cuda")
        D._check(lib.ddflb_nn_im2col(X.data_ptr(), B, H, W, C, cs, out.data_ptr(), transposed, None))
        torch.cuda.synchronize()
        got = out.float().cpu().numpy().reshape(want.T.shape if transposed else want.shape)
        np.testing.assert_array_equal(got, want.T if transposed else want)


@pytest.mark.parametrize("C,cs", [(32, 32), (8, 12), (5, 5)])
def test_col2im_adjoint_of_im2col(C, cs):
    """col2im sums the taps back: <im2col(x), d> = <x, col2im(d)> (adjoint)."""
    B, H, W = 2, 19, 21
    g = torch.Generator().manual_seed(C)
    dcol = torch.randn(B * H * W, 9 * C, generator=g).cuda()
    dX = torch.zeros(B, H, W, cs, device="cuda")
    D._check(D.load().ddflb_nn_col2im(dcol.data_ptr(), B, H, W, C, dX.data_ptr(), cs, None))
    torch.cuda.synchronize()
    x = np.random.default_rng(C).standard_normal((B, H, W, C))
    lhs = np.sum(im2col_np(x, C) * dcol.double().cpu().numpy())
    rhs = np.sum(x * dX.double().cpu().numpy()[..., :C])
    assert abs(lhs - rhs) < 1e-9 * np.sum(np.abs(dcol.double().cpu().numpy())) * 10


@pytest.mark.parametrize("rows,C,cs", [(100000, 32, 48), (5000, 130, 130), (300, 7, 9)])
def test_bias_grad_column_sums(rows, C, cs):
    g = torch.Generator().manual_seed(rows)
    G = torch.randn(rows, cs, generator=g).cuda()
    db = torch.empty(C, device="cuda")
    D._check(D.load().ddflb_nn_bias_grad(G.data_ptr(), rows, C, cs, db.data_ptr(), None))
    torch.cuda.synchronize()
    want = G.double().cpu().numpy()[:, :C].sum(axis=0)
    np.testing.assert_allclose(db.double().cpu().numpy(), want, rtol=0,
                               atol=1e-5 * np.sqrt(rows))


# --------------------------------------------------------------- implicit 3x3 convolution
def _conv_ref(X, Wt, B, H, Wd, C, cs, N, bias, act, s):
    """im2col + the tcgen05 GEMM: the path the implicit convolution replaces."""
    lib = D.load()
    col = torch.empty(B * H * Wd, 9 * C, dtype=torch.bfloat16, device="cuda")
    D._check(lib.ddflb_nn_im2col(X.data_ptr(), B, H, Wd, C, cs, col.data_ptr(), 0, s))
    Yf = torch.empty(B * H * Wd, N, device="cuda")
    Yb = torch.empty(B * H * Wd, N, dtype=torch.bfloat16, device="cuda")
    D._check(lib.ddflb_nn_gemm(col.data_ptr(), Wt.data_ptr(), B * H * Wd, N, 9 * C, 9 * C, 9 * C,
                               Yf.data_ptr(), N, Yb.data_ptr(), N,
                               None if bias is None else bias.data_ptr(), act, 0, 1, None, s))
    return Yf, Yb


@pytest.fixture
def conv_path():
    lib = D.load()
    yield lambda p: D._check(lib.ddflb_nn_set_conv_path(p))
    D._check(lib.ddflb_nn_set_conv_path(0))


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("B,H,Wd,C,cs,off,N,act", [
    (2, 16, 16, 64, 64, 0, 32, 1), (16, 8, 8, 128, 192, 64, 128, 0), (1, 4, 256, 64, 72, 8, 64, 1),
    (4, 32, 32, 64, 128, 64, 96, 1), (16, 64, 64, 64, 64, 0, 64, 0), (2, 5, 128, 128, 128, 0, 48, 1),
    (1, 3, 384, 192, 256, 64, 128, 0), (3, 2, 256, 64, 64, 0, 32, 0), (1, 1, 128, 64, 64, 0, 32, 1),
    (1, 2, 256, 128, 128, 0, 128, 1), (1, 2, 128, 128, 128, 0, 160, 0)])
def test_conv3x3_equals_im2col_gemm(B, H, Wd, C, cs, off, N, act, path, conv_path):
    """The implicit convolution (zero padding from the tensor map) against
    im2col + GEMM on the same BF16 data, bit for bit, with one box per tap
    (path 1) and with halo bands (path 0, where W is a multiple of 128 and
    C >= 128; per-tap boxes elsewhere): row segments (W = 128, 256, 384; one to three channel
    chunks; one-row images), bands with the weights resident in shared memory
    and with a ring of weight tiles (C = N = 128; N = 160 over two column
    tiles), whole rows (W = 16, 32, 64) and two images (8 x 8),
    channel-strided input read from a channel offset of a wider buffer, N
    below, at and between tile widths, bias and activation."""
    conv_path(path)
    g = torch.Generator().manual_seed(B * H + C + N)
    buf = torch.randn(B, H, Wd, cs, generator=g).to(torch.bfloat16).cuda()
    X = buf[..., off:]                     # channels [off, off + C) of the buffer, stride cs
    Xc = X[..., :C].contiguous().view(-1)  # only for the reference's im2col (stride C)
    Wt = (0.1 * torch.randn(N, 9 * C, generator=g)).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).cuda()
    s = torch.cuda.current_stream().cuda_stream
    lib = D.load()
    Yf = torch.full((B * H * Wd, N), 7.0, device="cuda")
    Yb = torch.empty(B * H * Wd, N, dtype=torch.bfloat16, device="cuda")
    D._check(lib.ddflb_nn_conv3x3(X.data_ptr(), B, H, Wd, C, cs, Wt.data_ptr(), N, Yf.data_ptr(),
                                  N, Yb.data_ptr(), N, bias.data_ptr(), act, 0, s))
    Rf, Rb = _conv_ref(Xc, Wt, B, H, Wd, C, C, N, bias, act, s)
    torch.cuda.synchronize()
    assert take_error() == 0
    assert torch.equal(Yf, Rf) and torch.equal(Yb, Rb)


def test_conv3x3_flip_gives_the_input_gradient():
    """dX = conv3x3(dY, flip(W)) equals the im2col path's input gradient
    (GEMM dY . W into patch columns, then col2im), up to the order of the FP32
    additions (the implicit form sums all 9 taps and channels in one
    accumulator)."""
    B, H, Wd, Ci, Co = 4, 32, 32, 64, 128
    g = torch.Generator().manual_seed(11)
    dY = torch.randn(B, H, Wd, Co, generator=g).to(torch.bfloat16).cuda()
    Wt = (0.1 * torch.randn(Co, 9 * Ci, generator=g)).to(torch.bfloat16).cuda()
    s = torch.cuda.current_stream().cuda_stream
    lib = D.load()
    Wf = torch.empty(Ci, 9 * Co, dtype=torch.bfloat16, device="cuda")
    D._check(lib.ddflb_nn_conv3x3_flip(Wt.data_ptr(), Co, Ci, Wf.data_ptr(), s))
    dX = torch.empty(B * H * Wd, Ci, device="cuda")
    D._check(lib.ddflb_nn_conv3x3(dY.data_ptr(), B, H, Wd, Co, Co, Wf.data_ptr(), Ci,
                                  dX.data_ptr(), Ci, None, 0, None, 0, 0, s))
    # reference: dcol = dY . W  ([P][Co] x [Co][9 Ci]), then the col2im adjoint
    WT = Wt.t().contiguous()                                 # [9 Ci][Co]
    dcol = torch.empty(B * H * Wd, 9 * Ci, device="cuda")
    D._check(lib.ddflb_nn_gemm(dY.data_ptr(), WT.data_ptr(), B * H * Wd, 9 * Ci, Co, Co, Co,
                               dcol.data_ptr(), 9 * Ci, None, 0, None, 0, 0, 1, None, s))
    ref = torch.empty(B * H * Wd, Ci, device="cuda")
    D._check(lib.ddflb_nn_col2im(dcol.data_ptr(), B, H, Wd, Ci, ref.data_ptr(), Ci, s))
    torch.cuda.synchronize()
    assert take_error() == 0
    d = (dX - ref).abs().max().item()
    assert d <= 1e-5 * ref.abs().max().item(), d


def test_conv3x3_rejects_unsupported_shapes():
    lib = D.load()
    x = torch.zeros(2, 8, 8, 64, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(32, 9 * 64, dtype=torch.bfloat16, device="cuda")
    y = torch.empty(128, 32, device="cuda")
    with pytest.raises(D.DdflbError, match="multiple of 64"):
        D._check(lib.ddflb_nn_conv3x3(x.data_ptr(), 2, 8, 8, 32, 64, w.data_ptr(), 32,
                                      y.data_ptr(), 32, None, 0, None, 0, 0, None))
    with pytest.raises(D.DdflbError, match="128-pixel tiles"):
        D._check(lib.ddflb_nn_conv3x3(x.data_ptr(), 2, 8, 6, 64, 64, w.data_ptr(), 32,
                                      y.data_ptr(), 32, None, 0, None, 0, 0, None))


def test_unet_implicit_conv_matches_im2col_path_and_oracle():
    """The U-Net with its 3x3 convolutions of >= 64 input channels as implicit
    GEMMs (forward and input gradient): the forward pass is bit-identical to
    the im2col + GEMM network, every gradient agrees with it up to the order
    of FP32 additions (1e-3) and with the FP64 network oracle within the BF16
    bound of the other test (width 32, so levels 1-3 use the implicit path)."""
    nets = []
    for implicit in (True, False):
        net, xb, t = make_net(c=32, batch=4, H=32, seed=3)
        net.implicit = implicit
        out = net.forward(xb).clone()
        loss = net.backward(t)
        torch.cuda.synchronize()
        nets.append((net, out, float(loss.item()), net.grads()))
    (ni, oi, li, gi), (ne, oe, le, ge) = nets
    assert sum(ni._implicit_ok(ci, *ni.L[lv]) for (n, lv, *_), (_, ci, _) in
               zip(ni.layers, ni.specs)) >= 6            # the implicit path is in use
    assert torch.equal(oi, oe) and li == le
    for name, _, _ in ni.specs:
        for k in (0, 1):
            assert rel(gi[name][k], ge[name][k]) < 1e-3, (name, k, rel(gi[name][k], ge[name][k]))
    P = oracle_params(ni)
    ref_out, cache = OU.forward(P, xb.double().cpu().numpy())
    G = OU.backward(P, cache, ref_out, t.double().cpu().numpy())
    worst = max(rel(gi[name][k], G[name][k]) for name, _, _ in ni.specs for k in (0, 1))
    print("implicit U-Net: worst gradient error against the oracle", worst)
    assert rel(oi.double().cpu().numpy(), ref_out) < 2e-2 and worst < 6e-2
