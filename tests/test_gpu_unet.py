"""The U-Net kernels (include/sgn_unet.h) against the FP64 oracle.

Bars. FP32 activations: every value is an FP32 sum of at most 64 x 9 products
(relative error ~ 576 x 6e-8 in the worst case, ~1e-6 typically), so the
output and each layer's gradient match the oracle to 1e-5 and 1e-4 relative
L2. BF16 activations: each stored activation carries a relative rounding of
2^-9 = 2e-3, and an output passes 9 stored layers (up to 2e-2 relative); the
gradients also flip ReLU masks of activations within that rounding of zero,
so each layer's gradient gets 1e-1.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def layer_slices():
    off = 0
    for ci, co, k in U.LAYERS:
        n = ci * co * k * k + co
        yield slice(off, off + n)
        off += n


def run_pair(n, B, bf16, seed):
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(seed)
    p = U.init_params(seed).astype(np.float32)
    x = rng.standard_normal((B, 4, n, n)).astype(np.float32)
    t = (0.1 * rng.standard_normal((B, 1, n, n))).astype(np.float32)
    net = UNet(n, max_batch=B, bf16=bf16, seed=1)
    net.set_params(torch.tensor(p, device="cuda"))
    xd = torch.tensor(x, device="cuda")
    out = net.forward(xd)
    loss = net.backward(torch.tensor(t, device="cuda"))
    g = net.grads().cpu().numpy()
    out = out.cpu().numpy()
    net.close()
    ro, cache = U.forward(p.astype(np.float64), x.astype(np.float64))
    rloss, rg = U.backward(p.astype(np.float64), ro, cache, t.astype(np.float64))
    return out, loss, g, ro, rloss, rg


@pytest.mark.parametrize("n,B", [(16, 1), (32, 3)])
def test_unet_fp32_matches_oracle(n, B):
    out, loss, g, ro, rloss, rg = run_pair(n, B, False, 5 + n)
    assert rel(out, ro) < 1e-5
    assert abs(loss - rloss) < 1e-5 * rloss
    for i, sl in enumerate(layer_slices()):
        assert rel(g[sl], rg[sl]) < 1e-4, i


def test_unet_bf16_matches_oracle_to_bf16_rounding():
    out, loss, g, ro, rloss, rg = run_pair(32, 2, True, 11)
    assert rel(out, ro) < 2e-2
    for i, sl in enumerate(layer_slices()):
        assert rel(g[sl], rg[sl]) < 1e-1, i


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


def test_training_reduces_the_loss():
    """200 Adam steps on a fixed batch fit a smooth function of the input."""
    from paper_2306_09731_gb300.unet import UNet
    rng = np.random.default_rng(8)
    x = rng.standard_normal((4, 4, 32, 32)).astype(np.float32)
    t = 0.25 * (x[:, :1] + np.roll(x[:, :1], 1, axis=2) + np.roll(x[:, 1:2], -1, axis=3) - x[:, 3:4])
    net = UNet(32, max_batch=4, bf16=True, seed=9)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t.astype(np.float32), device="cuda")
    losses = []
    for step in range(1, 201):
        net.forward(xd)
        losses.append(net.backward(td))
        net.adam_step(3e-3, step)
    net.close()
    assert losses[-1] < 0.1 * losses[0]
