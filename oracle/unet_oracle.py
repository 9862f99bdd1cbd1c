"""Plain FP64 CPU oracle of the periodic U-Net of include/sgn_unet.h.

TEST INFRASTRUCTURE. Only ``tests/`` and the training checks may import this
module; the GPU library never calls it and shares no code with it.

The network is the one the header specifies, layer by layer, with the periodic
3x3 convolution written as a sum over the nine shifted copies of the input
(numpy.roll) and the backward pass derived by hand: for
out = b + sum_k W_k * roll(x, -d_k), the input gradient is
sum_k W_k^T * roll(dout, +d_k) and the weight gradient
sum over pixels of dout * roll(x, -d_k). The loss is the mean squared error.
"""
import numpy as np

# (Ci, Co, k) of e0, s0, e1, s1, b0, b1, d1, d0, out
LAYERS = [(4, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 32, 3), (32, 32, 3), (64, 32, 3), (48, 16, 3),
          (16, 1, 1)]


def num_params():
    return sum(co * ci * k * k + co for ci, co, k in LAYERS)


def unpack(p):
    """List of (W [Co][Ci][k][k], b [Co]) views into the flat parameter array."""
    out, off = [], 0
    for ci, co, k in LAYERS:
        nw = co * ci * k * k
        out.append((p[off:off + nw].reshape(co, ci, k, k), p[off + nw:off + nw + co]))
        off += nw + co
    return out


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


def forward(p, x):
    """Output [B][1][n][n] and the activations the backward pass needs."""
    L = unpack(np.asarray(p, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    a0 = relu(conv3(x, *L[0]))
    s0 = relu(conv3(a0, *L[1]))
    q0 = pool(s0)
    a1 = relu(conv3(q0, *L[2]))
    s1 = relu(conv3(a1, *L[3]))
    q1 = pool(s1)
    a2 = relu(conv3(q1, *L[4]))
    a3 = relu(conv3(a2, *L[5]))
    cat1 = np.concatenate([up(a3), s1], axis=1)
    a4 = relu(conv3(cat1, *L[6]))
    cat0 = np.concatenate([up(a4), s0], axis=1)
    a5 = relu(conv3(cat0, *L[7]))
    W8, b8 = L[8]
    out = np.einsum("oc,bchw->bohw", W8[:, :, 0, 0], a5) + b8[None, :, None, None]
    cache = dict(x=x, a0=a0, s0=s0, q0=q0, a1=a1, s1=s1, q1=q1, a2=a2, a3=a3, cat1=cat1, a4=a4, cat0=cat0, a5=a5)
    return out, cache


def backward(p, out, cache, target):
    """Mean squared error and its gradient for every parameter (flat, FP64)."""
    L = unpack(np.asarray(p, dtype=np.float64))
    c = cache
    diff = out - target
    loss = float(np.mean(diff ** 2))
    dout = 2.0 * diff / diff.size
    grads = [None] * len(LAYERS)
    W8 = L[8][0]
    grads[8] = (np.einsum("bohw,bchw->oc", dout, c["a5"])[:, :, None, None], dout.sum(axis=(0, 2, 3)))
    d = np.einsum("oc,bohw->bchw", W8[:, :, 0, 0], dout) * (c["a5"] > 0)
    dcat0, dW, db = conv3_bwd(c["cat0"], L[7][0], d)
    grads[7] = (dW, db)
    d = up_bwd(dcat0[:, :32]) * (c["a4"] > 0)
    dcat1, dW, db = conv3_bwd(c["cat1"], L[6][0], d)
    grads[6] = (dW, db)
    d = up_bwd(dcat1[:, :32]) * (c["a3"] > 0)
    d, dW, db = conv3_bwd(c["a2"], L[5][0], d)
    grads[5] = (dW, db)
    d = d * (c["a2"] > 0)
    d, dW, db = conv3_bwd(c["q1"], L[4][0], d)
    grads[4] = (dW, db)
    d = (pool_bwd(d) + dcat1[:, 32:]) * (c["s1"] > 0)
    d, dW, db = conv3_bwd(c["a1"], L[3][0], d)
    grads[3] = (dW, db)
    d = d * (c["a1"] > 0)
    d, dW, db = conv3_bwd(c["q0"], L[2][0], d)
    grads[2] = (dW, db)
    d = (pool_bwd(d) + dcat0[:, 32:]) * (c["s0"] > 0)
    d, dW, db = conv3_bwd(c["a0"], L[1][0], d)
    grads[1] = (dW, db)
    d = d * (c["a0"] > 0)
    _, dW, db = conv3_bwd(c["x"], L[0][0], d)
    grads[0] = (dW, db)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])
    return loss, flat


def init_params(seed):
    """A reproducible initialisation in the style of the GPU one (Kaiming-uniform)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co, k) in enumerate(LAYERS):
        bound = np.sqrt(6.0 / (ci * k * k)) * (0.1 if i == len(LAYERS) - 1 else 1.0)
        parts.append(rng.uniform(-bound, bound, co * ci * k * k))
        parts.append(rng.uniform(-0.1, 0.1, co))
    return np.concatenate(parts)
