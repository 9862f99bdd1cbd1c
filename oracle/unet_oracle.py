"""Plain FP64 CPU oracle of the periodic U-Net of include/sgn_unet.h.

TEST INFRASTRUCTURE. Only ``tests/`` and the training checks may import this
module; the GPU library never calls it and shares no code with it.

The network is the one the header specifies, for any depth D (resolution
levels) and widths w[0..D-1]: at each level l < D-1 two 3x3 convolutions
(e_l: in -> w_l, s_l: w_l -> w_l) and a 2x2 average pool; at level D-1 two
convolutions (b0, b1); on the way up a nearest 2x upsample of the level below,
concatenated (upsampled channels first) with s_l, and one convolution
d_l: w_{l+1} + w_l -> w_l; then a 1x1 convolution w_0 -> 1. Every 3x3
convolution is followed by a ReLU. The default architecture is D = 3,
w = (16, 32, 32).

The periodic 3x3 convolution is written as a sum over the nine shifted copies
of the input (numpy.roll) and the backward pass is derived by hand: for
out = b + sum_k W_k * roll(x, -d_k), the input gradient is
sum_k W_k^T * roll(dout, +d_k) and the weight gradient
sum over pixels of dout * roll(x, -d_k). The loss is the mean squared error.

``forward(..., bf16=True)`` rounds what the GPU's BF16 path stores to BF16
(round to nearest even) at the same places: every activation a layer writes,
the pooled tensors, and - for the tensor-core inference path, ``weights_bf16``
- the convolution weights of the 3x3 layers after the first. Sums stay FP64.
"""
import numpy as np

DEFAULT_ARCH = (3, (16, 32, 32))


def layers(arch=DEFAULT_ARCH):
    """(Ci, Co, k) of every layer in parameter order: e_0, s_0, ..., e_{D-2},
    s_{D-2}, b0, b1, d_{D-2}, ..., d_0, out."""
    D, w = arch
    assert D >= 2 and len(w) == D
    out = []
    for l in range(D - 1):
        out.append((4 if l == 0 else w[l - 1], w[l], 3))
        out.append((w[l], w[l], 3))
    out.append((w[D - 2], w[D - 1], 3))
    out.append((w[D - 1], w[D - 1], 3))
    for l in range(D - 2, -1, -1):
        out.append((w[l + 1] + w[l], w[l], 3))
    out.append((w[0], 1, 1))
    return out


# the default network's layer table: e0, s0, e1, s1, b0, b1, d1, d0, out
LAYERS = layers()


def num_params(arch=DEFAULT_ARCH):
    return sum(co * ci * k * k + co for ci, co, k in layers(arch))


def unpack(p, arch=DEFAULT_ARCH):
    """List of (W [Co][Ci][k][k], b [Co]) views into the flat parameter array."""
    out, off = [], 0
    for ci, co, k in layers(arch):
        nw = co * ci * k * k
        out.append((p[off:off + nw].reshape(co, ci, k, k), p[off + nw:off + nw + co]))
        off += nw + co
    return out


def bf16_round(x):
    """Round FP64 values to the nearest BF16 (ties to even), through FP32 as a
    GPU conversion of an FP32 sum does: the FP64 value is first rounded to
    FP32, then its 16 low bits are rounded off."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3(x, W, b):
    out = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for ky in range(3):
        for kx in range(3):
            xs = np.roll(x, (-(ky - 1), -(kx - 1)), axis=(2, 3))
            out += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], xs)
    return out + b[None, :, None, None]


def conv3_bwd(x, W, dout):
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            dx += np.roll(np.einsum("oc,bohw->bchw", W[:, :, ky, kx], dout), (ky - 1, kx - 1), axis=(2, 3))
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dout, np.roll(x, (-(ky - 1), -(kx - 1)), axis=(2, 3)))
    return dx, dW, dout.sum(axis=(0, 2, 3))


def pool(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_bwd(d):
    return 0.25 * np.repeat(np.repeat(d, 2, axis=2), 2, axis=3)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_bwd(d):
    B, C, H, W = d.shape
    return d.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def forward(p, x, arch=DEFAULT_ARCH, bf16=False, weights_bf16=False):
    """Output [B][1][n][n] and the activations the backward pass needs."""
    D, w = arch
    L = unpack(np.asarray(p, dtype=np.float64), arch)
    if weights_bf16:  # the 3x3 layers after the first run on BF16 weights
        L = [(bf16_round(W) if (i > 0 and W.shape[2] == 3) else W, b) for i, (W, b) in enumerate(L)]
    st = bf16_round if bf16 else (lambda a: a)
    x = np.asarray(x, dtype=np.float64)
    c = dict(x=x)
    inp = x
    for l in range(D - 1):
        c[f"a{l}"] = st(relu(conv3(inp, *L[2 * l])))
        c[f"s{l}"] = st(relu(conv3(c[f"a{l}"], *L[2 * l + 1])))
        c[f"q{l}"] = st(pool(c[f"s{l}"]))
        inp = c[f"q{l}"]
    c[f"a{D - 1}"] = st(relu(conv3(inp, *L[2 * (D - 1)])))
    below = c[f"u{D - 1}"] = st(relu(conv3(c[f"a{D - 1}"], *L[2 * (D - 1) + 1])))
    for l in range(D - 2, -1, -1):
        c[f"cat{l}"] = np.concatenate([up(below), c[f"s{l}"]], axis=1)
        below = c[f"u{l}"] = st(relu(conv3(c[f"cat{l}"], *L[2 * D + (D - 2 - l)])))
    Wo, bo = L[-1]
    out = np.einsum("oc,bchw->bohw", Wo[:, :, 0, 0], below) + bo[None, :, None, None]
    return out, c


def backward(p, out, cache, target, arch=DEFAULT_ARCH):
    """Mean squared error and its gradient for every parameter (flat, FP64).

    The ReLU masks are those of the stored activations in the cache, so with
    a BF16 forward the gradient is that of the network the GPU evaluates."""
    D, w = arch
    L = unpack(np.asarray(p, dtype=np.float64), arch)
    c = cache
    diff = out - target
    loss = float(np.mean(diff ** 2))
    dout = 2.0 * diff / diff.size
    grads = [None] * len(L)
    Wo = L[-1][0]
    grads[-1] = (np.einsum("bohw,bchw->oc", dout, c["u0"])[:, :, None, None], dout.sum(axis=(0, 2, 3)))
    d = np.einsum("oc,bohw->bchw", Wo[:, :, 0, 0], dout) * (c["u0"] > 0)
    dcat = {}
    for l in range(D - 1):  # decoder, from the top level down the U
        li = 2 * D + (D - 2 - l)
        dcat[l], dW, db = conv3_bwd(c[f"cat{l}"], L[li][0], d)
        grads[li] = (dW, db)
        d = up_bwd(dcat[l][:, :w[l + 1]]) * (c[f"u{l + 1}"] > 0)
    ib = 2 * (D - 1)
    d, dW, db = conv3_bwd(c[f"a{D - 1}"], L[ib + 1][0], d)
    grads[ib + 1] = (dW, db)
    d = d * (c[f"a{D - 1}"] > 0)
    d, dW, db = conv3_bwd(c[f"q{D - 2}"], L[ib][0], d)
    grads[ib] = (dW, db)
    for l in range(D - 2, -1, -1):  # encoder, back up to the input
        d = (pool_bwd(d) + dcat[l][:, w[l + 1]:]) * (c[f"s{l}"] > 0)
        d, dW, db = conv3_bwd(c[f"a{l}"], L[2 * l + 1][0], d)
        grads[2 * l + 1] = (dW, db)
        d = d * (c[f"a{l}"] > 0)
        d, dW, db = conv3_bwd(c["x"] if l == 0 else c[f"q{l - 1}"], L[2 * l][0], d)
        grads[2 * l] = (dW, db)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])
    return loss, flat


def init_params(seed, arch=DEFAULT_ARCH):
    """A reproducible initialisation in the style of the GPU one (Kaiming-uniform)."""
    rng = np.random.default_rng(seed)
    parts = []
    lay = layers(arch)
    for i, (ci, co, k) in enumerate(lay):
        bound = np.sqrt(6.0 / (ci * k * k)) * (0.1 if i == len(lay) - 1 else 1.0)
        parts.append(rng.uniform(-bound, bound, co * ci * k * k))
        parts.append(rng.uniform(-0.1, 0.1, co))
    return np.concatenate(parts)
