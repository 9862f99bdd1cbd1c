"""ctypes binding of include/sgn_unet.h (the learned-guess U-Net).

Argument marshalling only: every computation runs in the library's kernels.
Tensors are CUDA float32 torch tensors (or raw device pointers as ints).
"""
import ctypes

from . import sgn as S

# every symbol include/sgn_unet.h declares
UNET_EXPORTS = ["sgn_unet_create", "sgn_unet_create_arch", "sgn_unet_destroy", "sgn_unet_set_stream",
                "sgn_unet_last_error", "sgn_unet_num_params", "sgn_unet_side", "sgn_unet_levels", "sgn_unet_width",
                "sgn_unet_set_params", "sgn_unet_get_params", "sgn_unet_get_grads", "sgn_unet_forward",
                "sgn_unet_infer", "sgn_unet_check", "sgn_unet_backward", "sgn_unet_adam_step",
                "sgn_conv3_relu_bf16", "sgn_conv3_workspace_bytes", "sgn_conv3_wait_selftest"]

# the default network and the four-level one of 471,873 parameters
DEFAULT_ARCH = (3, (16, 32, 32))
SPEC_ARCH = (4, (32, 64, 64, 96))

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_ready = False


def load_library():
    global _ready
    lib = S.load_library()
    if not _ready:
        sig = {
            "sgn_unet_create": (_I, [_I, _I, _I, ctypes.c_ulonglong, ctypes.POINTER(_P)]),
            "sgn_unet_create_arch": (_I, [_I, _I, _I, ctypes.c_ulonglong, _I, ctypes.POINTER(_I),
                                          ctypes.POINTER(_P)]),
            "sgn_unet_levels": (_I, [_P]),
            "sgn_unet_width": (_I, [_P, _I]),
            "sgn_unet_infer": (_I, [_P, _P, _P, _I]),
            "sgn_unet_check": (_I, [_P]),
            "sgn_conv3_relu_bf16": (_I, [_I, _I, _I, _P, _I, _I, _P, _I, _P, _P, _I, _P, _P, ctypes.c_size_t, _P]),
            "sgn_conv3_workspace_bytes": (ctypes.c_size_t, [_I, _I]),
            "sgn_conv3_wait_selftest": (_I, [_P]),
            "sgn_unet_destroy": (_I, [_P]),
            "sgn_unet_set_stream": (_I, [_P, _P]),
            "sgn_unet_last_error": (ctypes.c_char_p, [_P]),
            "sgn_unet_num_params": (ctypes.c_longlong, [_P]),
            "sgn_unet_side": (_I, [_P]),
            "sgn_unet_set_params": (_I, [_P, _P]),
            "sgn_unet_get_params": (_I, [_P, _P]),
            "sgn_unet_get_grads": (_I, [_P, _P]),
            "sgn_unet_forward": (_I, [_P, _P, _P, _I]),
            "sgn_unet_backward": (_I, [_P, _P, _P]),
            "sgn_unet_adam_step": (_I, [_P, _F, _F, _F, _F, _I]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _ready = True
    return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _on_current_stream(net):
    """The solver re-points an attached network to its own stream: every call
    from Python puts it back on torch's current stream first."""
    import torch
    load_library().sgn_unet_set_stream(net, torch.cuda.current_stream().cuda_stream)


def _check(net, st):
    if st != 0:
        msg = load_library().sgn_unet_last_error(net) if net else b""
        raise S.SGNError(st, (msg or b"").decode())


def conv3_relu_bf16(src0, weight, bias, src1=None, up0=False):
    """One periodic 3x3 convolution + bias + ReLU on the tensor cores.

    src0 [B][h][w][C0] (h = H/2, w = W/2 when up0) and src1 [B][H][W][C1]:
    torch.bfloat16 CUDA tensors (NHWC); weight [Co][C0+C1][3][3] and bias [Co]
    float32. Returns out [B][H][W][Co] bfloat16."""
    import torch
    lib = load_library()
    B = src0.shape[0]
    H, W = (src0.shape[1] * 2, src0.shape[2] * 2) if up0 else (src0.shape[1], src0.shape[2])
    C0 = src0.shape[3]
    C1 = 0 if src1 is None else src1.shape[3]
    Co = weight.shape[0]
    ws_bytes = int(lib.sgn_conv3_workspace_bytes(C0 + C1, Co))
    ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, H, W, Co), dtype=torch.bfloat16, device="cuda")
    src0, weight, bias = src0.contiguous(), weight.contiguous().float(), bias.contiguous().float()
    src1 = None if src1 is None else src1.contiguous()
    st = lib.sgn_conv3_relu_bf16(int(B), int(H), int(W), _ptr(src0), int(C0), 1 if up0 else 0, _ptr(src1), int(C1),
                                 _ptr(weight), _ptr(bias), int(Co), _ptr(out), _ptr(ws), ws_bytes,
                                 torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise S.SGNError(st, "sgn_conv3_relu_bf16 failed")
    return out


class UNet:
    """One network (coarse grid side n, up to max_batch samples per call);
    arch = (levels, widths), None for the library's default network."""

    def __init__(self, n, max_batch=8, bf16=True, seed=0, arch=None):
        import torch
        self._torch = torch
        lib = load_library()
        h = _P()
        if arch is None:
            _check(None, lib.sgn_unet_create(int(n), int(max_batch), 1 if bf16 else 0, int(seed), ctypes.byref(h)))
        else:
            levels, widths = arch
            wa = (_I * len(widths))(*[int(x) for x in widths])
            _check(None, lib.sgn_unet_create_arch(int(n), int(max_batch), 1 if bf16 else 0, int(seed), int(levels),
                                                  wa, ctypes.byref(h)))
        self.handle = h
        self.n = n
        self.max_batch = max_batch
        self.bf16 = bf16
        lib.sgn_unet_set_stream(self.handle, torch.cuda.current_stream().cuda_stream)

    def close(self):
        if self.handle:
            load_library().sgn_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(load_library().sgn_unet_num_params(self.handle))

    def arch(self):
        lib = load_library()
        levels = int(lib.sgn_unet_levels(self.handle))
        return levels, tuple(int(lib.sgn_unet_width(self.handle, i)) for i in range(levels))

    def params(self):
        p = self._torch.empty(self.num_params(), dtype=self._torch.float32, device="cuda")
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_get_params(self.handle, _ptr(p)))
        return p

    def set_params(self, p):
        p = p.to(device="cuda", dtype=self._torch.float32).contiguous()
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_set_params(self.handle, _ptr(p)))
        self._keep = p

    def grads(self):
        g = self._torch.empty(self.num_params(), dtype=self._torch.float32, device="cuda")
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_get_grads(self.handle, _ptr(g)))
        return g

    def forward(self, x):
        """x: [B][4][n][n] float32 CUDA tensor -> [B][1][n][n]."""
        self._x = x.contiguous()
        out = self._torch.empty((x.shape[0], 1, self.n, self.n), dtype=self._torch.float32, device="cuda")
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_forward(self.handle, _ptr(self._x), _ptr(out), int(x.shape[0])))
        return out

    def infer(self, x, out=None):
        """Tensor-core BF16 forward: x [B][4][n][n] float32 CUDA tensor -> [B][1][n][n]."""
        x = x.contiguous()
        if out is None:
            out = self._torch.empty((x.shape[0], 1, self.n, self.n), dtype=self._torch.float32, device="cuda")
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_infer(self.handle, _ptr(x), _ptr(out), int(x.shape[0])))
        return out

    def check(self):
        """Raises SGNError if an infer call since the last check gave up waiting."""
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_check(self.handle))

    def backward(self, target):
        """MSE against target [B][1][n][n] after forward; returns the loss (host float)."""
        self._t = target.contiguous()
        loss = self._torch.zeros(1, dtype=self._torch.float64, device="cuda")
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_backward(self.handle, _ptr(self._t), _ptr(loss)))
        return float(loss.item())

    def adam_step(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        _on_current_stream(self.handle)
        _check(self.handle, load_library().sgn_unet_adam_step(self.handle, lr, beta1, beta2, eps, int(t)))
