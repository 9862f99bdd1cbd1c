"""Pins of the U-Net oracle (oracle/unet_oracle.py), CPU only.

The backward pass is derived by hand in the oracle; it is pinned here by
central finite differences of the loss, the periodic convolution by an FFT
circular correlation, and the pooling / upsampling gradients by the adjoint
identity <A x, y> = <x, A^T y>.
"""
import numpy as np

from oracle import unet_oracle as U


def test_parameter_count_matches_layer_table():
    # e0, s0, e1, (s1, b0, b1), d1, d0, out: weights Co*Ci*k*k plus Co biases
    assert U.num_params() == (4 * 16 * 9 + 16) + (16 * 16 * 9 + 16) + (16 * 32 * 9 + 32) + 3 * (32 * 32 * 9 + 32) \
        + (64 * 32 * 9 + 32) + (48 * 16 * 9 + 16) + (16 + 1) == 60705
    assert sum(w.size + b.size for w, b in U.unpack(np.zeros(U.num_params()))) == U.num_params()


def test_conv3_is_fft_circular_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 16, 16))
    W = rng.standard_normal((4, 3, 3, 3))
    out = U.conv3(x, W, np.zeros(4))
    ref = np.zeros_like(out)
    for o in range(4):
        for c in range(3):
            k = np.zeros((16, 16))
            for ky in range(3):
                for kx in range(3):
                    k[(ky - 1) % 16, (kx - 1) % 16] = W[o, c, ky, kx]
            ref[:, o] += np.real(np.fft.ifft2(np.conj(np.fft.fft2(k))[None] * np.fft.fft2(x[:, c])))
    assert np.max(np.abs(out - ref)) < 1e-12


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 8, 8))
    y = rng.standard_normal((2, 3, 4, 4))
    assert abs(np.sum(U.pool(x) * y) - np.sum(x * U.pool_bwd(y))) < 1e-12
    z = rng.standard_normal((2, 3, 16, 16))
    assert abs(np.sum(U.up(x) * z) - np.sum(x * U.up_bwd(z))) < 1e-12


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    p = U.init_params(3)
    x = rng.standard_normal((2, 4, 16, 16))
    t = rng.standard_normal((2, 1, 16, 16)) * 0.1
    out, cache = U.forward(p, x)
    loss, g = U.backward(p, out, cache, t)
    idx = rng.choice(p.size, 60, replace=False)
    # the last layer's bias and a few weights of every layer
    offs = np.cumsum([0] + [ci * co * k * k + co for ci, co, k in U.LAYERS])
    idx = np.concatenate([idx, offs[1:] - 1, offs[:-1] + 3])
    eps = 1e-6
    for i in idx:
        pp = p.copy()
        pp[i] += eps
        lp = U.backward(pp, *U.forward(pp, x), t)[0]
        pp[i] -= 2 * eps
        lm = U.backward(pp, *U.forward(pp, x), t)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * max(abs(g[i]), 1e-3 * np.max(np.abs(g))), (i, fd, g[i])


def test_four_level_layer_table_and_count():
    arch = (4, (32, 64, 64, 96))
    assert U.layers(arch) == [(4, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 64, 3), (64, 64, 3),
                              (64, 96, 3), (96, 96, 3), (96 + 64, 64, 3), (64 + 64, 64, 3), (64 + 32, 32, 3),
                              (32, 1, 1)]
    # 9 (4*32 + 32*32 + 32*64 + 64*64 + 64*64 + 64*64 + 64*96 + 96*96 + 160*64 + 128*64 + 96*32) + 32 + 1 weights,
    # 32+32+64+64+64+64+96+96+64+64+32+1 biases
    assert U.num_params(arch) == 9 * 52352 + 32 + 673 == 471873
    assert U.layers() == U.LAYERS and U.num_params() == 60705


def _fd_check(arch, n, B, seed, count):
    rng = np.random.default_rng(seed)
    p = U.init_params(seed, arch)
    x = rng.standard_normal((B, 4, n, n))
    t = rng.standard_normal((B, 1, n, n)) * 0.1
    out, cache = U.forward(p, x, arch)
    loss, g = U.backward(p, out, cache, t, arch)
    offs = np.cumsum([0] + [ci * co * k * k + co for ci, co, k in U.layers(arch)])
    idx = np.concatenate([rng.choice(p.size, count, replace=False), offs[1:] - 1, offs[:-1] + 3])
    eps = 1e-6
    for i in idx:
        pp = p.copy()
        pp[i] += eps
        lp = U.backward(pp, *U.forward(pp, x, arch), t, arch)[0]
        pp[i] -= 2 * eps
        lm = U.backward(pp, *U.forward(pp, x, arch), t, arch)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * max(abs(g[i]), 1e-3 * np.max(np.abs(g))), (arch, i, fd, g[i])


def test_backward_matches_central_differences_four_levels():
    # widths of the oracle need not be multiples of 16; level 3 works on 2 x 2
    _fd_check((4, (6, 8, 10, 12)), 16, 1, 5, 30)


def test_backward_matches_central_differences_two_levels():
    _fd_check((2, (5, 7)), 8, 2, 6, 30)


def test_bf16_round_matches_a_library_conversion():
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        # exact ties between two BF16 neighbours go to the even one
                        np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0, -0.0])])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(x), ref)
    assert U.bf16_round(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert U.bf16_round(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6


def test_bf16_forward_stores_rounded_activations():
    arch = (3, (16, 32, 32))
    rng = np.random.default_rng(8)
    p = U.init_params(8, arch)
    x = rng.standard_normal((1, 4, 16, 16))
    out, c = U.forward(p, x, arch, bf16=True, weights_bf16=True)
    for k in ("a0", "s0", "q0", "a1", "u1", "u0", "cat0"):
        assert np.array_equal(U.bf16_round(c[k]), c[k]), k
    ref, _ = U.forward(p, x, arch)
    r = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert 1e-4 < r < 3e-2
