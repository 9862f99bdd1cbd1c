"""The U-Net kernels (include/sgn_unet.h) against the FP64 oracle.

Bars. FP32 activations: every value is an FP32 sum of at most 160 x 9
products (relative error ~1e-6 typically), so the output and each layer's
gradient match the oracle to 1e-5 and 1e-4 relative L2.

One tensor-core layer (sgn_conv3_relu_bf16) against the oracle's convolution
of the same BF16 values, rounded to BF16 the same way: the GPU's FP32 sum and
the oracle's FP64 sum differ by ~1e-7 relative (the accumulator was measured
FP32-accurate), so an output differs only where the exact value lies that
close to a BF16 rounding boundary - then by one BF16 step. At least 99.9% of
the outputs are bit-identical and every other one is within one BF16 step.

Whole networks with BF16 activations: the oracle rounds what the GPU stores
at the same places (oracle.unet_oracle.forward(bf16=True)), but one output
that flips across a rounding boundary nudges the sums of the next layer, some
of which flip in turn, so two correct BF16 evaluations of a deep network end
up as far apart as BF16 rounding takes either from the exact network. The
bars are therefore twice the oracle's own BF16-to-FP64 distance (and at least
1e-3 for outputs, 1e-2 for gradients); a wrong term, layer or scale is off by
far more.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPEC = (4, (32, 64, 64, 96))
SMALL4 = (4, (16, 16, 32, 32))


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def layer_slices(arch):
    off = 0
    for ci, co, k in U.layers(arch):
        n = ci * co * k * k + co
        yield slice(off, off + n)
        off += n


def make_net(n, B, bf16, arch):
    from paper_2306_09731_gb300.unet import UNet
    return UNet(n, max_batch=B, bf16=bf16, seed=1, arch=None if arch == U.DEFAULT_ARCH else arch)


def run_pair(n, B, bf16, seed, arch=U.DEFAULT_ARCH):
    rng = np.random.default_rng(seed)
    p = U.init_params(seed, arch).astype(np.float32)
    x = rng.standard_normal((B, 4, n, n)).astype(np.float32)
    t = (0.1 * rng.standard_normal((B, 1, n, n))).astype(np.float32)
    net = make_net(n, B, bf16, arch)
    assert net.num_params() == U.num_params(arch)
    assert net.arch() == (arch[0], tuple(arch[1]))
    net.set_params(torch.tensor(p, device="cuda"))
    xd = torch.tensor(x, device="cuda")
    out = net.forward(xd)
    loss = net.backward(torch.tensor(t, device="cuda"))
    g = net.grads().cpu().numpy()
    out = out.cpu().numpy()
    net.close()
    p64, x64, t64 = p.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    ro, cache = U.forward(p64, x64, arch, bf16=bf16)
    rloss, rg = U.backward(p64, ro, cache, t64, arch)
    ro64, cache64 = U.forward(p64, x64, arch)
    _, rg64 = U.backward(p64, ro64, cache64, t64, arch)
    return out, loss, g, ro, rloss, rg, ro64, rg64


@pytest.mark.parametrize("n,B,arch", [(16, 1, U.DEFAULT_ARCH), (32, 3, U.DEFAULT_ARCH), (32, 2, SMALL4),
                                      (32, 1, SPEC), (16, 2, (2, (16, 32)))])
def test_unet_fp32_matches_oracle(n, B, arch):
    out, loss, g, ro, rloss, rg, _, _ = run_pair(n, B, False, 5 + n, arch)
    assert rel(out, ro) < 1e-5
    assert abs(loss - rloss) < 1e-5 * rloss
    for i, sl in enumerate(layer_slices(arch)):
        assert rel(g[sl], rg[sl]) < 1e-4, i


@pytest.mark.parametrize("n,B,arch,seed", [(32, 2, U.DEFAULT_ARCH, 11), (32, 1, SPEC, 11), (64, 2, SPEC, 12)])
def test_unet_bf16_matches_bf16_oracle(n, B, arch, seed):
    out, loss, g, ro, rloss, rg, ro64, rg64 = run_pair(n, B, True, seed, arch)
    noise = rel(ro, ro64)
    assert 1e-4 < noise < 5e-2  # the oracle's BF16 rounding is in effect
    assert rel(out, ro) < max(1e-3, 2 * noise)
    assert abs(loss - rloss) < max(1e-3, 4 * noise) * rloss
    for i, sl in enumerate(layer_slices(arch)):
        assert rel(g[sl], rg[sl]) < max(1e-2, 2 * rel(rg[sl], rg64[sl])), i


def to_nchw(a):
    return np.ascontiguousarray(np.transpose(a, (0, 3, 1, 2)))


# (B, H, W, C0, up0, C1, Co): a plain layer; the decoder's upsample + concatenation; a split K loop (336
# channels in three blocks of 112) on a ragged grid of 192 pixels; a non-square grid with the widest N;
# 1024 input channels on a 16-pixel grid. Rows of >= 128 pixels take the halo-staged row kernel: a plain
# layer, upsample + concatenation in two channel blocks, and five channel blocks over two images
LAYER_CASES = [(2, 32, 32, 32, 0, 0, 32), (1, 16, 16, 64, 1, 32, 64), (3, 8, 8, 256, 1, 80, 80),
               (1, 8, 64, 16, 0, 0, 256), (1, 4, 4, 512, 0, 512, 16),
               (1, 4, 128, 64, 0, 0, 64), (1, 4, 256, 32, 1, 32, 48), (2, 8, 128, 96, 1, 64, 64)]


@pytest.mark.parametrize("B,H,W,C0,up0,C1,Co", LAYER_CASES)
def test_tensor_core_layer_matches_oracle_convolution(B, H, W, C0, up0, C1, Co):
    from paper_2306_09731_gb300.unet import conv3_relu_bf16
    rng = np.random.default_rng(B * H * W + C0 + C1 + Co)
    h0, w0 = (H // 2, W // 2) if up0 else (H, W)
    s0 = torch.tensor(rng.standard_normal((B, h0, w0, C0)), dtype=torch.bfloat16, device="cuda")
    s1 = None if C1 == 0 else torch.tensor(rng.standard_normal((B, H, W, C1)), dtype=torch.bfloat16, device="cuda")
    Ci = C0 + C1
    wt = (rng.standard_normal((Co, Ci, 3, 3)) / np.sqrt(9 * Ci)).astype(np.float32)
    bs = (0.1 * rng.standard_normal(Co)).astype(np.float32)
    got = conv3_relu_bf16(s0, torch.tensor(wt, device="cuda"), torch.tensor(bs, device="cuda"), s1, bool(up0))
    got = got.float().cpu().numpy().astype(np.float64)
    x = to_nchw(s0.float().cpu().numpy().astype(np.float64))
    if up0:
        x = U.up(x)
    if s1 is not None:
        x = np.concatenate([x, to_nchw(s1.float().cpu().numpy().astype(np.float64))], axis=1)
    wb = U.bf16_round(wt.astype(np.float64))
    v = U.conv3(x, wb, bs.astype(np.float64))  # exact (FP64) pre-activation
    # any FP32 summation of the K = 9 Ci products and the bias, rounded to
    # nearest or toward zero, is within 2 (K + 1) 2^-24 sum |p| of the exact
    # sum; ReLU and BF16 rounding are monotone, so
    # the GPU's output lies between the roundings of the two ends
    tol = 2 * (9 * Ci + 1) * 2.0 ** -24 * (U.conv3(np.abs(x), np.abs(wb), np.zeros(Co)) + np.abs(bs)[None, :, None, None])
    nhwc = lambda a: np.transpose(a, (0, 2, 3, 1))
    ref, lo, hi = (nhwc(U.bf16_round(U.relu(a))) for a in (v, v - tol, v + tol))
    assert np.all((lo <= got) & (got <= hi))
    # and nearly all of them are the rounding of the exact value
    assert (got == ref).mean() >= 0.95
    assert np.count_nonzero(ref) > 0.3 * ref.size  # the ReLU leaves a real test


def test_tensor_core_wait_runs_out_and_the_context_survives():
    """A barrier that never completes (armed for more bytes than its copy
    delivers) makes each kernel's bounded wait run out: the launch reports it
    and the same context then runs the layer normally (sgn_conv3_wait_selftest);
    a full layer afterwards still matches the oracle."""
    import time
    from paper_2306_09731_gb300 import unet as UN
    lib = UN.load_library()
    t0 = time.perf_counter()
    assert lib.sgn_conv3_wait_selftest(torch.cuda.current_stream().cuda_stream) == 0
    assert time.perf_counter() - t0 < 60
    test_tensor_core_layer_matches_oracle_convolution(1, 4, 128, 64, 0, 0, 64)


def run_infer(n, B, arch, seed):
    rng = np.random.default_rng(seed)
    p = U.init_params(seed, arch).astype(np.float32)
    x = rng.standard_normal((B, 4, n, n)).astype(np.float32)
    net = make_net(n, B, True, arch)
    net.set_params(torch.tensor(p, device="cuda"))
    xd = torch.tensor(x, device="cuda")
    out = net.infer(xd)
    net.check()
    fwd = net.forward(xd)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), fwd.cpu().numpy()
    net.close()
    p64, x64 = p.astype(np.float64), x.astype(np.float64)
    ro, _ = U.forward(p64, x64, arch, bf16=True, weights_bf16=True)
    ro64, _ = U.forward(p64, x64, arch)
    return res[0], res[1], ro, ro64


# the coarsest level of (64, SPEC) has 64 pixels (one partial tile); (128, SPEC, 3) spans several tiles at
# every level; n = 16 with the default net ends on 4 x 4
@pytest.mark.parametrize("n,B,arch", [(16, 1, U.DEFAULT_ARCH), (32, 2, U.DEFAULT_ARCH), (64, 1, SPEC),
                                      (128, 3, SPEC), (32, 2, (2, (16, 32))), (64, 2, (3, (48, 80, 256)))])
def test_infer_tensor_cores_match_bf16_oracle(n, B, arch):
    out, fwd, ro, ro64 = run_infer(n, B, arch, 21 + n + B)
    assert np.all(np.isfinite(out))
    noise = rel(ro, ro64)
    assert 1e-4 < noise < 5e-2
    assert rel(out, ro) < max(1e-3, 2 * noise)
    assert rel(out, ro64) < 3 * noise
    # the CUDA-core forward keeps FP32 weights: the same network to BF16 rounding
    assert rel(out, fwd) < 4 * noise


@pytest.mark.parametrize("n,arch", [(64, SPEC), (16, U.DEFAULT_ARCH)])
def test_infer_partial_batches_match_the_full_batch(n, arch):
    """Each pixel's sums are the same dot products whatever the batch (an MMA
    row is one pixel, its K order fixed), so sample i of a call with fewer
    samples than max_batch equals sample i of the full call bit for bit; the
    full call meets the BF16-emulating oracle."""
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(n + 7)
    B = 3
    p = U.init_params(13, arch).astype(np.float32)
    x = rng.standard_normal((B, 4, n, n)).astype(np.float32)
    net = UNet(n, max_batch=B, bf16=True, seed=1, arch=None if arch == U.DEFAULT_ARCH else arch)
    net.set_params(torch.tensor(p, device="cuda"))
    xd = torch.tensor(x, device="cuda")
    full = net.infer(xd).clone()
    one = net.infer(xd[:1].contiguous()).clone()
    two = net.infer(xd[1:3].contiguous()).clone()
    net.check()
    net.close()
    assert torch.equal(one[0], full[0])
    assert torch.equal(two, full[1:3])
    ro, _ = U.forward(p.astype(np.float64), x.astype(np.float64), arch, bf16=True, weights_bf16=True)
    ro64, _ = U.forward(p.astype(np.float64), x.astype(np.float64), arch)
    assert rel(full.cpu().numpy(), ro) < max(1e-3, 2 * rel(ro, ro64))


def test_infer_is_deterministic_and_graph_capturable():
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(4)
    net = UNet(64, max_batch=2, bf16=True, seed=3, arch=SPEC)
    x = torch.tensor(rng.standard_normal((2, 4, 64, 64)).astype(np.float32), device="cuda")
    a = net.infer(x).clone()
    out = torch.empty_like(a)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        net.infer(x, out)  # warm-up on the capture stream
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            net.infer(x, out)
    torch.cuda.current_stream().wait_stream(s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    net.check()
    assert torch.equal(a, out)
    net.close()


def test_adam_step_follows_its_formula():
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(3)
    net = UNet(16, max_batch=1, bf16=False, seed=4)
    p0 = net.params().cpu().numpy().astype(np.float64)
    x = torch.tensor(rng.standard_normal((1, 4, 16, 16)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.standard_normal((1, 1, 16, 16)).astype(np.float32), device="cuda")
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    p = p0.copy()
    for step in (1, 2):
        net.forward(x)
        net.backward(t)
        g = net.grads().cpu().numpy().astype(np.float64)
        net.adam_step(1e-3, step)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p = p - 1e-3 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    got = net.params().cpu().numpy().astype(np.float64)
    net.close()
    assert np.max(np.abs(got - p)) < 1e-6


@pytest.mark.parametrize("arch", [None, SPEC])
def test_training_reduces_the_loss(arch):
    """200 Adam steps on a fixed batch fit a smooth function of the input."""
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(8)
    x = rng.standard_normal((4, 4, 32, 32)).astype(np.float32)
    t = 0.25 * (x[:, :1] + np.roll(x[:, :1], 1, axis=2) + np.roll(x[:, 1:2], -1, axis=3) - x[:, 3:4])
    net = UNet(32, max_batch=4, bf16=True, seed=9, arch=arch)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t.astype(np.float32), device="cuda")
    losses = []
    for step in range(1, 201):
        net.forward(xd)
        losses.append(net.backward(td))
        net.adam_step(3e-3 if arch is None else 1e-3, step)
    # the trained network evaluated on the tensor cores fits as well
    inf = net.infer(xd).cpu().numpy()
    net.close()
    assert losses[-1] < 0.1 * losses[0]
    assert float(np.mean((inf - t) ** 2)) < 0.15 * losses[0]
