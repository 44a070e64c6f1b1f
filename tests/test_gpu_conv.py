"""The warm-start network's convolution kernels (include/warmstart_conv.h)
against the FP64 oracle layers on BF16-exact inputs: the forward (tcgen05
tensor cores for 32 -> 32, CUDA cores for the edge layers, ragged tiles of
128 pixels), both gradients, the autograd wrapper, and exact integer sums
that pin the tensor-core operand layouts (shared-memory descriptors, tensor
memory lanes) of the forward and of the weight gradient."""
import numpy as np
import pytest

from oracle.conv import conv3x3, conv3x3_grad_input, conv3x3_grad_weight

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_20907_gb300")

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(torch.bfloat16)


def _exact(t):
    return t.float().cpu().numpy().astype(np.float64)


def _fwd(x, w, b, relu, cout, d=1):
    from paper_2503_20907_gb300 import _lib
    B, H, W, cin = x.shape
    y = torch.empty((B, H, W, cout) if cout > 1 else (B, H, W), device=DEV,
                    dtype=torch.bfloat16 if cout > 1 else torch.float32)
    _lib._check(_lib.load().sp_conv3x3_fwd(B, H, W, cin, cout, d, x.data_ptr(), w.data_ptr(),
                                           b.data_ptr() if b is not None else None, int(relu), y.data_ptr(), None))
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("H,W,d", [(5, 70, 1), (3, 64, 1), (4, 17, 1), (9, 70, 4), (20, 40, 16), (3, 256, 1),
                                   (4, 130, 5), (35, 129, 16)])
def test_conv32_exact_integer_sums(H, W, d):
    # small integers: every product and partial sum is exact in FP32 and the
    # result (|y| < 256) exact in BF16, so the tensor-core result must equal
    # the definition bit for bit
    rng = np.random.default_rng(H * W)
    x = rng.integers(-2, 3, size=(2, H, W, 32)).astype(np.float32)
    w = rng.integers(-1, 2, size=(32, 3, 3, 32)).astype(np.float32)
    y = _fwd(_bf16(x), _bf16(w), None, False, 32, d)
    ref = conv3x3(x, w, d=d)
    assert np.abs(ref).max() < 256
    assert np.array_equal(_exact(y), ref)


@pytest.mark.parametrize("cin,cout,relu,d", [(32, 32, True, 1), (32, 32, False, 2), (1, 32, True, 1), (1, 32, True, 3),
                                             (32, 1, False, 1), (32, 1, False, 8)])
def test_conv_forward_matches_oracle(cin, cout, relu, d):
    rng = np.random.default_rng(cin + 7 * cout + relu)
    x = _bf16(rng.standard_normal((3, 6, 75, cin)))
    w = _bf16(rng.standard_normal((cout, 3, 3, cin)) * 0.2)
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).to(DEV)
    y = _fwd(x, w, b, relu, cout, d)
    ref = conv3x3(_exact(x), _exact(w), b.cpu().numpy(), d=d)
    if relu:
        ref = np.maximum(ref, 0.0)
    got = _exact(y).reshape(ref.shape)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # BF16 outputs carry a relative rounding of 2^-9 RMS; FP32 outputs ~1e-7
    assert err < (3e-3 if cout > 1 else 1e-5)


@pytest.mark.parametrize("cin,cout,d,W", [(32, 32, 1, 33), (1, 32, 1, 33), (32, 1, 1, 33), (32, 32, 4, 33),
                                           (1, 32, 2, 33), (32, 1, 16, 33), (32, 32, 16, 150), (32, 32, 3, 64)])
def test_conv_gradients_match_oracle(cin, cout, d, W):
    from paper_2503_20907_gb300 import _lib
    rng = np.random.default_rng(11 * cin + cout + d)
    B, H = 2, 5
    x = _bf16(rng.standard_normal((B, H, W, cin)))
    w = _bf16(rng.standard_normal((cout, 3, 3, cin)) * 0.2)
    g = torch.from_numpy(rng.standard_normal((B, H, W, cout)).astype(np.float32)).to(DEV)
    lib = _lib.load()
    dw = torch.empty((cout, 3, 3, cin), device=DEV)
    db = torch.empty(cout, device=DEV)
    _lib._check(lib.sp_conv3x3_bwd_weight(B, H, W, cin, cout, d, x.data_ptr(), g.data_ptr(), dw.data_ptr(),
                                          db.data_ptr(), None))
    # the 32 -> 32 gradients run on the tensor cores, which take g rounded to
    # BF16 (products and sums in FP32); the others take g in FP32.  The bias
    # gradient sums g in FP32 either way.
    g_in = _exact(g.to(torch.bfloat16)) if (cin, cout) == (32, 32) else g.cpu().numpy()
    ref_w, _ = conv3x3_grad_weight(_exact(x), g_in, d=d)
    _, ref_b = conv3x3_grad_weight(_exact(x), g.cpu().numpy(), d=d)
    assert np.linalg.norm(dw.cpu().numpy() - ref_w) / np.linalg.norm(ref_w) < 1e-5
    assert np.allclose(db.cpu().numpy(), ref_b, rtol=1e-5, atol=1e-4)
    dx = torch.empty((B, H, W, cin), device=DEV)
    gate = _bf16(rng.standard_normal((B, H, W, cin)))
    _lib._check(lib.sp_conv3x3_bwd_data(B, H, W, cin, cout, d, g.data_ptr(), w.data_ptr(), gate.data_ptr(),
                                        dx.data_ptr(), None))
    ref_x = conv3x3_grad_input(g_in, _exact(w), d=d) * (_exact(gate) > 0)
    assert np.linalg.norm(dx.cpu().numpy() - ref_x) / np.linalg.norm(ref_x) < 1e-5


@pytest.mark.parametrize("B,H,W,d", [(1, 3, 33, 1), (2, 35, 129, 16), (1, 4, 256, 1), (2, 5, 300, 5),
                                     (3, 200, 20, 2), (1, 1, 1, 1)])
def test_conv32_weight_gradient_exact_integer_sums(B, H, W, d):
    # small integers in x and g: every product and sum is exact in FP32, so
    # the tensor-core weight gradient (taps x input channels as M, pixels as
    # K, several 128-pixel segments and blocks of several rows) must equal
    # the definition bit for bit
    from paper_2503_20907_gb300 import _lib
    rng = np.random.default_rng(B * 1000 + H * W + d)
    x = rng.integers(-2, 3, size=(B, H, W, 32)).astype(np.float32)
    g = rng.integers(-2, 3, size=(B, H, W, 32)).astype(np.float32)
    dw = torch.empty((32, 3, 3, 32), device=DEV)
    db = torch.empty(32, device=DEV)
    gd = torch.from_numpy(g).to(DEV)
    _lib._check(_lib.load().sp_conv3x3_bwd_weight(B, H, W, 32, 32, d, _bf16(x).data_ptr(), gd.data_ptr(),
                                                  dw.data_ptr(), db.data_ptr(), None))
    ref_w, ref_b = conv3x3_grad_weight(x.astype(np.float64), g.astype(np.float64), d=d)
    assert np.abs(ref_w).max() < 2 ** 24
    assert np.array_equal(dw.cpu().numpy().astype(np.float64), ref_w)
    assert np.array_equal(db.cpu().numpy().astype(np.float64), ref_b)


def test_flip_weights():
    from paper_2503_20907_gb300 import _lib
    rng = np.random.default_rng(5)
    w = _bf16(rng.standard_normal((32, 3, 3, 32)))
    wf = torch.empty_like(w)
    _lib._check(_lib.load().sp_conv3x3_flip_weights(32, 32, w.data_ptr(), wf.data_ptr(), None))
    ref = _exact(w)[:, ::-1, ::-1, :].transpose(3, 1, 2, 0)
    assert np.array_equal(_exact(wf), ref)


def test_autograd_layer_gradients():
    from paper_2503_20907_gb300.warmstart import conv3x3 as layer
    rng = np.random.default_rng(9)
    x = _bf16(rng.standard_normal((2, 6, 40, 32))).requires_grad_(True)
    w = torch.from_numpy((rng.standard_normal((32, 3, 3, 32)) * 0.1).astype(np.float32)).to(DEV).requires_grad_(True)
    b = torch.from_numpy(rng.standard_normal(32).astype(np.float32)).to(DEV).requires_grad_(True)
    R = torch.from_numpy(rng.standard_normal((2, 6, 40, 32)).astype(np.float32)).to(DEV)
    y = layer(x, w, b, True, 2)
    (y.float() * R).sum().backward()
    wb = w.detach().to(torch.bfloat16)
    pre = conv3x3(_exact(x.detach()), _exact(wb), b.detach().cpu().numpy(), d=2)
    # the gradient reaching a BF16 output is BF16 (autograd keeps the dtype)
    g = _exact(R.to(torch.bfloat16)) * (pre > 0) * (_exact(y.detach()) > 0)
    ref_w, ref_b = conv3x3_grad_weight(_exact(x.detach()), g, d=2)
    assert np.linalg.norm(w.grad.cpu().numpy() - ref_w) / np.linalg.norm(ref_w) < 1e-5
    assert np.allclose(b.grad.cpu().numpy(), ref_b, rtol=1e-5, atol=1e-4)
    ref_x = conv3x3_grad_input(g, _exact(wb), d=2)
    got_x = x.grad.float().cpu().numpy()
    assert np.linalg.norm(got_x - ref_x) / np.linalg.norm(ref_x) < 5e-3    # BF16 gradient of a BF16 input
