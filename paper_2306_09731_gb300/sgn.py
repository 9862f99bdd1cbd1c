"""Thin ctypes binding of libsgn.so (include/sgn.h): argument marshalling only.

Functions keep the C names (``sgn_create``, ``sgn_rhs``, ...). Field arguments
are CUDA tensors (float64, contiguous, shape (Ny, Nx)) or raw integer device
pointers; every computation runs in the library's CUDA kernels. The library is
loaded on first use and a missing or unloadable library raises: there is no
CPU fallback.

``Solver`` wraps a handle for convenient use from PyTorch.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SGN_OK, SGN_EINVAL, SGN_ENOTCONV, SGN_ECAVITATION, SGN_ENONFINITE, SGN_ECUDA, SGN_ENOMEM = range(7)
STATUS_NAMES = {0: "SGN_OK", 1: "SGN_EINVAL", 2: "SGN_ENOTCONV", 3: "SGN_ECAVITATION",
                4: "SGN_ENONFINITE", 5: "SGN_ECUDA", 6: "SGN_ENOMEM"}

# every symbol include/sgn.h declares
EXPORTS = ["sgn_default_options", "sgn_create", "sgn_destroy", "sgn_set_stream",
           "sgn_spectral_derivative", "sgn_fft2_r2c", "sgn_fft2_c2r", "sgn_elliptic_apply",
           "sgn_gmres_solve", "sgn_rhs", "sgn_rk4_step", "sgn_rk4_step_host", "sgn_invariants",
           "sgn_get_stats", "sgn_set_profiling", "sgn_get_profile", "sgn_elliptic_apply_noalloc",
           "sgn_diagnostics", "sgn_set_learned_guess", "sgn_record_learned", "sgn_recorded_count",
           "sgn_coarse_sample", "sgn_coarse_embed", "sgn_rk4_step_batch", "sgn_autotune", "sgn_set_tuning",
           "sgn_last_error"]

# index names of sgn_tuning's [type][pass] arrays
TUNE_TYPES = ["fp32", "fp64", "dfl"]
TUNE_PASSES = ["mv_yinv", "mv_yfwd", "rhs_yinv", "rhs_yfwd", "mv_x", "rhs_x"]

PROFILE_CLASSES = ["coef", "mv_yinv", "mv_x", "mv_yfwd", "rhs_yinv", "rhs_x", "rhs_yfwd", "krylov", "io",
                   "ref_yinv", "ref_x", "ref_yfwd", "rk"]


class SGNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sgn_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("tol", ctypes.c_double), ("krasny", ctypes.c_int), ("krasny_thr", ctypes.c_double),
                ("dealias", ctypes.c_int), ("guess", ctypes.c_int), ("graph", ctypes.c_int)]


class sgn_diag(ctypes.Structure):
    _fields_ = [("h_max", ctypes.c_double), ("i_max", ctypes.c_longlong), ("x_s", ctypes.c_double),
                ("y_s", ctypes.c_double), ("c_fit", ctypes.c_double), ("dev_h", ctypes.c_double),
                ("dev_vx", ctypes.c_double), ("max_vy", ctypes.c_double), ("tail", ctypes.c_double * 3)]


class sgn_tuning(ctypes.Structure):
    _fields_ = [("threads", (ctypes.c_int * 6) * 3), ("default_threads", (ctypes.c_int * 6) * 3),
                ("us_tuned", (ctypes.c_float * 6) * 3), ("us_default", (ctypes.c_float * 6) * 3),
                ("plan", (ctypes.c_int * 6) * 3)]


class sgn_stats(ctypes.Structure):
    _fields_ = [("matvecs", ctypes.c_longlong), ("solves", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("last_relres", ctypes.c_double), ("last_iters", ctypes.c_int),
                ("refinements", ctypes.c_longlong)]


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def load_library(path: str | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libsgn.so (building it in-tree first if it is absent or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if path is None:
        path = _build.lib_path()
        if build_if_missing and not _build.up_to_date():
            _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsgn.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "sgn_default_options": (None, [ctypes.POINTER(sgn_options)]),
        "sgn_create": (_I, [_I, _I, _D, _D, _D, ctypes.POINTER(sgn_options), ctypes.POINTER(_P)]),
        "sgn_destroy": (_I, [_P]),
        "sgn_set_stream": (_I, [_P, _P]),
        "sgn_spectral_derivative": (_I, [_P, _P, _P, _P]),
        "sgn_fft2_r2c": (_I, [_P, _P, _P]),
        "sgn_fft2_c2r": (_I, [_P, _P, _P]),
        "sgn_elliptic_apply": (_I, [_P, _P, _P, _P]),
        "sgn_gmres_solve": (_I, [_P, _P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
        "sgn_rhs": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
        "sgn_rk4_step": (_I, [_P, _P, _P, _P, _P, _D, _I]),
        "sgn_rk4_step_host": (_I, [_P, _P, _P, _P, _P, _D, _I]),
        "sgn_invariants": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_D)]),
        "sgn_get_stats": (_I, [_P, ctypes.POINTER(sgn_stats)]),
        "sgn_set_profiling": (_I, [_P, _I]),
        "sgn_get_profile": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), _I,
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "sgn_elliptic_apply_noalloc": (_I, [_I, _I, _D, _D, _P, _P, _P, _P]),
        "sgn_diagnostics": (_I, [_P, _P, _P, _P, ctypes.POINTER(sgn_diag)]),
        "sgn_autotune": (_I, [_P, _I, ctypes.POINTER(sgn_tuning)]),
        "sgn_set_tuning": (_I, [_P, ctypes.POINTER(sgn_tuning)]),
        "sgn_set_learned_guess": (_I, [_P, _P, _I, ctypes.POINTER(ctypes.c_float), ctypes.c_float, _I]),
        "sgn_record_learned": (_I, [_P, _I, _P, _I, _I]),
        "sgn_recorded_count": (_I, [_P, ctypes.POINTER(_I)]),
        "sgn_coarse_sample": (_I, [_P, _P, _I, _P]),
        "sgn_coarse_embed": (_I, [_P, _P, _I, _D, _P]),
        "sgn_rk4_step_batch": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(_I)]),
        "sgn_last_error": (ctypes.c_char_p, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_cuda or x.dtype.itemsize != 8 or not x.is_contiguous():
            raise ValueError("expected a contiguous CUDA float64 tensor")
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy array (host variants only)
        if x.dtype.itemsize != 8 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(handle, status):
    if status != SGN_OK:
        msg = load_library().sgn_last_error(handle)
        raise SGNError(status, msg.decode() if msg else "")


# ------------------------------------------------------------ C-named calls

def sgn_default_options() -> sgn_options:
    o = sgn_options()
    load_library().sgn_default_options(ctypes.byref(o))
    return o


def sgn_create(Nx, Ny, Lx, Ly, g=1.0, opt: sgn_options | None = None):
    h = _P()
    st = load_library().sgn_create(int(Nx), int(Ny), float(Lx), float(Ly), float(g),
                                   ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(None, st)
    return h


def sgn_destroy(handle):
    _check(handle, load_library().sgn_destroy(handle))


def sgn_set_stream(handle, stream):
    _check(handle, load_library().sgn_set_stream(handle, int(stream) if stream else None))


def sgn_spectral_derivative(handle, f, fx, fy):
    _check(handle, load_library().sgn_spectral_derivative(handle, _ptr(f), _ptr(fx), _ptr(fy)))


def sgn_fft2_r2c(handle, f, fhat):
    _check(handle, load_library().sgn_fft2_r2c(handle, _ptr(f), _ptr(fhat)))


def sgn_fft2_c2r(handle, fhat, f):
    _check(handle, load_library().sgn_fft2_c2r(handle, _ptr(fhat), _ptr(f)))


def sgn_elliptic_apply(handle, h, sigma, out):
    _check(handle, load_library().sgn_elliptic_apply(handle, _ptr(h), _ptr(sigma), _ptr(out)))


def sgn_gmres_solve(handle, h, b, sigma):
    it = _I(0)
    rr = _D(0.0)
    st = load_library().sgn_gmres_solve(handle, _ptr(h), _ptr(b), _ptr(sigma), ctypes.byref(it),
                                        ctypes.byref(rr))
    if st not in (SGN_OK, SGN_ENOTCONV):
        _check(handle, st)
    return st, it.value, rr.value


def sgn_rhs(handle, h, vx, vy, sigma, ht, vxt, vyt):
    _check(handle, load_library().sgn_rhs(handle, _ptr(h), _ptr(vx), _ptr(vy), _ptr(sigma), _ptr(ht),
                                          _ptr(vxt), _ptr(vyt)))


def sgn_rk4_step(handle, h, vx, vy, sigma, dt, nsteps=1):
    _check(handle, load_library().sgn_rk4_step(handle, _ptr(h), _ptr(vx), _ptr(vy), _ptr(sigma),
                                               float(dt), int(nsteps)))


def sgn_rk4_step_host(handle, h, vx, vy, sigma, dt, nsteps=1):
    _check(handle, load_library().sgn_rk4_step_host(handle, _ptr(h), _ptr(vx), _ptr(vy), _ptr(sigma),
                                                    float(dt), int(nsteps)))


def sgn_invariants(handle, h, vx, vy, sigma):
    out = (_D * 4)()
    _check(handle, load_library().sgn_invariants(handle, _ptr(h), _ptr(vx), _ptr(vy), _ptr(sigma), out))
    return [out[i] for i in range(4)]


def sgn_diagnostics(handle, h, vx, vy) -> dict:
    """Monitoring quantities of the paper's experiments; see include/sgn.h."""
    d = sgn_diag()
    _check(handle, load_library().sgn_diagnostics(handle, _ptr(h), _ptr(vx), _ptr(vy), ctypes.byref(d)))
    return dict(h_max=d.h_max, i_max=d.i_max, x_s=d.x_s, y_s=d.y_s, c_fit=d.c_fit, dev_h=d.dev_h,
                dev_vx=d.dev_vx, max_vy=d.max_vy, tail=[d.tail[i] for i in range(3)])


def sgn_autotune(handle, reps=5) -> dict:
    """Times the launch shapes of the handle's transform passes and keeps the
    fastest; see include/sgn.h. Returns {type: {pass: {...}}} for the passes
    the handle runs."""
    t = sgn_tuning()
    _check(handle, load_library().sgn_autotune(handle, int(reps), ctypes.byref(t)))
    out = {}
    for i, ty in enumerate(TUNE_TYPES):
        for j, ps in enumerate(TUNE_PASSES):
            if t.threads[i][j] > 0:
                out.setdefault(ty, {})[ps] = dict(threads=t.threads[i][j], default_threads=t.default_threads[i][j],
                                                  us=t.us_tuned[i][j], us_default=t.us_default[i][j],
                                                  plan=t.plan[i][j])
    return out


def sgn_set_tuning(handle, tuning: dict):
    """Applies {type: {pass: {"threads": t, "plan": p}}} (the form sgn_autotune
    returns; missing passes keep their built-in shape and plan 0)."""
    t = sgn_tuning()
    for i, ty in enumerate(TUNE_TYPES):
        for j, ps in enumerate(TUNE_PASSES):
            r = tuning.get(ty, {}).get(ps)
            if r:
                t.threads[i][j] = int(r.get("threads", 0))
                t.plan[i][j] = int(r.get("plan", 0))
    _check(handle, load_library().sgn_set_tuning(handle, ctypes.byref(t)))


def _ptr32(x):
    if x is None or isinstance(x, int):
        return x
    if not x.is_cuda or x.dtype.itemsize != 4 or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32 tensor")
    return x.data_ptr()


def sgn_set_learned_guess(handle, net, n, in_scale, out_scale, tau_power):
    """Attach (net = a UNet handle) or detach (net = None) the learned start; see include/sgn.h."""
    sc = (ctypes.c_float * 4)(*[float(v) for v in in_scale])
    _check(handle, load_library().sgn_set_learned_guess(handle, net, int(n), sc, float(out_scale), int(tau_power)))


def sgn_record_learned(handle, n, buf, capacity, tau_power):
    _check(handle, load_library().sgn_record_learned(handle, int(n), _ptr32(buf), int(capacity), int(tau_power)))


def sgn_recorded_count(handle) -> int:
    c = _I(0)
    _check(handle, load_library().sgn_recorded_count(handle, ctypes.byref(c)))
    return c.value


def sgn_coarse_sample(handle, f, n, out):
    _check(handle, load_library().sgn_coarse_sample(handle, _ptr(f), int(n), _ptr32(out)))


def sgn_coarse_embed(handle, fc, n, scale, f):
    _check(handle, load_library().sgn_coarse_embed(handle, _ptr32(fc), int(n), float(scale), _ptr(f)))


def sgn_rk4_step_batch(handles, fields, dt, nsteps):
    """fields: per member [h, vx, vy, sigma] (CUDA float64 tensors); returns the member statuses.
    Raises SGNError with the first failing member's status."""
    n = len(handles)
    arr = lambda vals: (_P * n)(*vals)
    hs = arr([h.value if hasattr(h, "value") else h for h in handles])
    ps = [arr([_ptr(f[k]) for f in fields]) for k in range(4)]
    st = (_I * n)()
    rc = load_library().sgn_rk4_step_batch(hs, n, ps[0], ps[1], ps[2], ps[3], float(dt), int(nsteps), st)
    statuses = [st[i] for i in range(n)]
    if rc != 0:
        bad = next(i for i in range(n) if statuses[i] != 0)
        raise SGNError(rc, f"member {bad}: {sgn_last_error(handles[bad])}")
    return statuses


def sgn_get_stats(handle) -> dict:
    s = sgn_stats()
    _check(handle, load_library().sgn_get_stats(handle, ctypes.byref(s)))
    return dict(matvecs=s.matvecs, solves=s.solves, max_iters=s.max_iters,
                last_relres=s.last_relres, last_iters=s.last_iters, refinements=s.refinements)


def sgn_set_profiling(handle, on: bool):
    _check(handle, load_library().sgn_set_profiling(handle, 1 if on else 0))


def sgn_get_profile(handle) -> dict:
    n = len(PROFILE_CLASSES)
    ms = (_D * n)()
    cnt = (ctypes.c_longlong * n)()
    launches = ctypes.c_longlong(0)
    _check(handle, load_library().sgn_get_profile(handle, ms, cnt, n, ctypes.byref(launches)))
    return dict(ms={k: ms[i] for i, k in enumerate(PROFILE_CLASSES)},
                counts={k: cnt[i] for i, k in enumerate(PROFILE_CLASSES)}, launches=launches.value)


def sgn_elliptic_apply_noalloc(Nx, Ny, Lx, Ly, h, sigma, out, stream=None):
    """L[sigma] with no device allocation; see include/sgn.h."""
    st = load_library().sgn_elliptic_apply_noalloc(int(Nx), int(Ny), float(Lx), float(Ly), _ptr(h),
                                                     _ptr(sigma), _ptr(out), int(stream) if stream else None)
    _check(None, st)


def sgn_last_error(handle) -> str:
    m = load_library().sgn_last_error(handle)
    return m.decode() if m else ""


# ------------------------------------------------------------------ wrapper

class Solver:
    """One grid + options; methods take and return CUDA float64 tensors (Ny, Nx)."""

    def __init__(self, Nx, Ny, Lx, Ly, g=1.0, **opts):
        import torch
        o = sgn_default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.Nx, self.Ny, self.Lx, self.Ly, self.g = Nx, Ny, Lx, Ly, g
        self.options = o
        self.handle = sgn_create(Nx, Ny, Lx, Ly, g, o)
        self._torch = torch
        sgn_set_stream(self.handle, torch.cuda.current_stream().cuda_stream)

    def close(self):
        if self.handle:
            sgn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new(self):
        return self._torch.empty((self.Ny, self.Nx), dtype=self._torch.float64, device="cuda")

    def set_stream(self, stream):
        sgn_set_stream(self.handle, stream.cuda_stream)

    def derivative(self, f):
        fx, fy = self._new(), self._new()
        sgn_spectral_derivative(self.handle, f, fx, fy)
        return fx, fy

    def fft2(self, f):
        out = self._torch.empty((self.Ny, self.Nx // 2 + 1), dtype=self._torch.complex128, device="cuda")
        _check(self.handle, load_library().sgn_fft2_r2c(self.handle, _ptr(f), out.data_ptr()))
        return out

    def ifft2(self, fhat):
        f = self._new()
        _check(self.handle, load_library().sgn_fft2_c2r(self.handle, fhat.contiguous().data_ptr(), _ptr(f)))
        return f

    def elliptic_apply(self, h, sigma):
        out = self._new()
        sgn_elliptic_apply(self.handle, h, sigma, out)
        return out

    def gmres_solve(self, h, b, sigma0=None):
        sigma = self._torch.zeros_like(b) if sigma0 is None else sigma0.clone()
        st, its, rr = sgn_gmres_solve(self.handle, h, b, sigma)
        return sigma, its, rr, st == SGN_OK

    def rhs(self, h, vx, vy, sigma):
        ht, vxt, vyt = self._new(), self._new(), self._new()
        sgn_rhs(self.handle, h, vx, vy, sigma, ht, vxt, vyt)
        return ht, vxt, vyt

    def rk4_step(self, h, vx, vy, sigma, dt, nsteps=1):
        sgn_rk4_step(self.handle, h, vx, vy, sigma, dt, nsteps)

    def invariants(self, h, vx, vy, sigma):
        return sgn_invariants(self.handle, h, vx, vy, sigma)

    def stats(self):
        return sgn_get_stats(self.handle)

    def diagnostics(self, h, vx, vy):
        return sgn_diagnostics(self.handle, h, vx, vy)

    def autotune(self, reps=5):
        return sgn_autotune(self.handle, reps)

    def set_tuning(self, tuning):
        sgn_set_tuning(self.handle, tuning)

    def coarse_sample(self, f, n):
        out = self._torch.empty((n, n), dtype=self._torch.float32, device="cuda")
        sgn_coarse_sample(self.handle, f, n, out)
        return out

    def coarse_embed(self, fc, n, scale, f):
        sgn_coarse_embed(self.handle, fc.contiguous(), n, scale, f)

    def set_learned_guess(self, net, n=None, in_scale=(1.0, 1.0, 1.0, 1.0), out_scale=1.0, tau_power=1):
        """net: a unet.UNet (kept alive by the solver) or None."""
        self._net = net
        sgn_set_learned_guess(self.handle, net.handle if net is not None else None,
                              n if n is not None else (net.n if net is not None else 0), in_scale, out_scale,
                              tau_power)

    def record_learned(self, n, capacity, tau_power=1):
        """Start recording; returns the device buffer [capacity][5][n][n] that fills as stages run."""
        buf = self._torch.zeros((capacity, 5, n, n), dtype=self._torch.float32, device="cuda")
        sgn_record_learned(self.handle, n, buf, capacity, tau_power)
        self._rec = buf
        return buf

    def stop_recording(self):
        sgn_record_learned(self.handle, 0, None, 0, 1)
        return sgn_recorded_count(self.handle)

    def set_profiling(self, on=True):
        sgn_set_profiling(self.handle, on)

    def profile(self):
        return sgn_get_profile(self.handle)
