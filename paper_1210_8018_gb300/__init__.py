"""Fourier-accelerated steepest-descent Landau gauge fixing of SU(3) lattice gauge fields on GB300.

A thin Python binding over the C ABI of liblgf.so (include/lgf.h): it only marshals arguments. Every
step of the iteration (Cardoso, Silva, Oliveira, Bicudo, Lattice 2012, Algorithm 1) runs in the CUDA
kernels of that library; there is no Python or CPU fallback, and importing this module fails if the
library is missing.

Links are complex128 arrays of shape (4, Nt, Nz, Ny, Nx, 3, 3) (direction, site with x fastest, row,
column): torch tensors on the GPU (used in place) or numpy arrays / CPU tensors (copied through the
library's device buffers).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liblgf.so")

if not os.path.exists(_SO):
    raise ImportError("liblgf.so is not built; run __graft_entry__.build() (needs nvcc for sm_103a)")
_lib = ctypes.CDLL(_SO)

LGF_OK, LGF_EINVAL, LGF_ENOMEM, LGF_ECUDA, LGF_ENOCONV, LGF_ENONFINITE = range(6)
FP64, MIXED, FP32 = 0, 1, 2
_PREC = {"fp64": FP64, "mixed": MIXED, "fp32": FP32, FP64: FP64, MIXED: MIXED, FP32: FP32}
_STATUS = {0: "LGF_OK", 1: "LGF_EINVAL", 2: "LGF_ENOMEM", 3: "LGF_ECUDA", 4: "LGF_ENOCONV", 5: "LGF_ENONFINITE"}


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("theta_switch", ctypes.c_double), ("reunit_period", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_len", ctypes.c_int), ("fft32_final", ctypes.c_int)]


_vp, _d, _i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
_P = ctypes.POINTER
_SIGS = {
    "lgf_default_options": (None, [_P(Options)]),
    "lgf_create": (_i, [_i, _i, _i, _i, _P(_vp)]),
    "lgf_destroy": (None, [_vp]),
    "lgf_last_error": (ctypes.c_char_p, [_vp]),
    "lgf_set_stream": (_i, [_vp, _vp]),
    "lgf_fix": (_i, [_vp, _vp, _d, _d, _P(Options), _P(_d), _P(_d), _P(_i)]),
    "lgf_measure": (_i, [_vp, _vp, _P(_d), _P(_d), _P(_d)]),
    "lgf_load": (_i, [_vp, _vp, _i]),
    "lgf_iterate": (_i, [_vp, _i, _d, _d, _P(Options), _P(_d), _P(_d), _P(_i)]),
    "lgf_store": (_i, [_vp, _vp]),
    "lgf_delta": (_i, [_vp, _vp, _vp, _P(_d), _P(_d), _i]),
    "lgf_filter": (_i, [_vp, _vp, _vp, _i]),
    "lgf_filter_coeffs": (_i, [_vp, _vp, _vp, _i]),
    "lgf_gauge": (_i, [_vp, _vp, _d, _vp, _i]),
    "lgf_update": (_i, [_vp, _vp, _vp, _i]),
    "lgf_functional": (_i, [_vp, _vp, _vp, _P(_d), _vp]),
    "lgf_functional_grad": (_i, [_vp, _vp, _vp, _d, _vp]),
    "lgf_batch_create": (_i, [_i, _P(_i), _P(_vp)]),
    "lgf_batch_destroy": (None, [_vp]),
    "lgf_batch_last_error": (ctypes.c_char_p, [_vp]),
    "lgf_batch_fix": (_i, [_vp, _P(_vp), _d, _d, _P(Options), _P(_d), _P(_d), _P(_i), _P(_i)]),
    "lgf_batch_describe": (_i, [_vp, ctypes.c_char_p, _i]),
    "lgf_enable_timing": (_i, [_vp, _i]),
    "lgf_kernel_times": (_i, [_vp, _P(ctypes.c_char_p), _P(ctypes.c_long), _P(_d), _i, _P(_i)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class LgfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


def library_path():
    return _SO


_CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def _torch_stream_handle():
    """Raw handle of torch's current CUDA stream (the legacy default stream as cudaStreamLegacy)."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return h if h else _CUDA_STREAM_LEGACY


def _ptr(a, real=False):
    """Device or host address of a C-contiguous torch tensor or numpy array (complex128, or float64
    when real=True)."""
    if isinstance(a, np.ndarray):
        want = np.float64 if real else np.complex128
        if a.dtype != want or not a.flags.c_contiguous:
            raise ValueError("numpy arrays must be %s and C-contiguous" % np.dtype(want).name)
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        want = torch.float64 if real else torch.complex128
        if a.dtype != want or not a.is_contiguous():
            raise ValueError("tensors must be %s and contiguous" % want)
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


def dims_of(U):
    nt, nz, ny, nx = tuple(U.shape[1:5])
    return (int(nx), int(ny), int(nz), int(nt))


class Lattice:
    """A gauge-fixing context for one lattice shape (Nx, Ny, Nz, Nt) on the current CUDA device."""

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        h = ctypes.c_void_p()
        st = _lib.lgf_create(*self.dims, ctypes.byref(h))
        if st != LGF_OK:
            raise LgfError(st, _lib.lgf_last_error(None).decode())
        self._h = h
        self._stream = None

    def close(self):
        if getattr(self, "_h", None):
            _lib.lgf_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _bind(self, *arrays):
        """Order the library's work after torch's: unless set_stream() chose a stream, issue on torch's
        current stream whenever a CUDA tensor is passed."""
        if self._stream is not None:
            return
        for a in arrays:
            if not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
                self._check(_lib.lgf_set_stream(self._h, _torch_stream_handle()))
                return

    def _check(self, st, allow=(LGF_OK,)):
        if st not in allow:
            raise LgfError(st, _lib.lgf_last_error(self._h).decode())
        return st

    def set_stream(self, stream):
        """Issue work on a torch.cuda.Stream (or a raw cudaStream_t as int); None = own stream."""
        raw = None
        if stream is not None:
            raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            raw = raw if raw else _CUDA_STREAM_LEGACY
        self._stream = stream
        self._check(_lib.lgf_set_stream(self._h, raw))

    @staticmethod
    def options(precision="fp64", theta_switch=1e-11, reunit_period=16, max_iter=100000, history=None,
                fft32_final=False):
        o = Options()
        _lib.lgf_default_options(ctypes.byref(o))
        o.fft32_final = 1 if fft32_final else 0
        o.precision = _PREC[precision]
        o.theta_switch = theta_switch
        o.reunit_period = reunit_period
        o.max_iter = max_iter
        if history is not None:
            o.history = history.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.history_len = history.shape[0]
        return o

    def fix(self, U, alpha=0.08, eps=1e-15, precision="fp64", max_iter=100000, theta_switch=1e-11,
            reunit_period=16, history_len=0, fft32_final=False):
        """Algorithm 1: fix U in place. Returns dict(theta, F, iters, converged, history)."""
        hist = np.zeros((history_len, 2), dtype=np.float64) if history_len > 0 else None
        o = self.options(precision, theta_switch, reunit_period, max_iter, hist, fft32_final)
        th, F, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        self._bind(U)
        st = self._check(_lib.lgf_fix(self._h, _ptr(U), alpha, eps, ctypes.byref(o), ctypes.byref(th),
                                      ctypes.byref(F), ctypes.byref(it)), (LGF_OK, LGF_ENOCONV))
        out = dict(theta=th.value, F=F.value, iters=it.value, converged=(st == LGF_OK))
        if hist is not None:
            out["history"] = hist[:min(it.value + 1, history_len)]
        return out

    def measure(self, U):
        th, F, pl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._bind(U)
        self._check(_lib.lgf_measure(self._h, _ptr(U), ctypes.byref(th), ctypes.byref(F), ctypes.byref(pl)))
        return dict(theta=th.value, F=F.value, plaquette=pl.value)

    # session interface
    def load(self, U, precision="fp64"):
        self._bind(U)
        self._check(_lib.lgf_load(self._h, _ptr(U), _PREC[precision]))

    def iterate(self, max_new, alpha=0.08, eps=1e-15, theta_switch=1e-11, reunit_period=16, history_len=0,
                fft32_final=False):
        hist = np.zeros((history_len, 2), dtype=np.float64) if history_len > 0 else None
        o = self.options("fp64", theta_switch, reunit_period, 0, hist, fft32_final)
        th, F, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        st = self._check(_lib.lgf_iterate(self._h, int(max_new), alpha, eps, ctypes.byref(o), ctypes.byref(th),
                                          ctypes.byref(F), ctypes.byref(it)), (LGF_OK, LGF_ENOCONV))
        out = dict(theta=th.value, F=F.value, iters=it.value, converged=(st == LGF_OK))
        if hist is not None:
            out["history"] = hist
        return out

    def store(self, U):
        self._bind(U)
        self._check(_lib.lgf_store(self._h, _ptr(U)))

    # single steps
    def delta(self, U, out, precision="fp64"):
        th, F = ctypes.c_double(), ctypes.c_double()
        self._bind(U, out)
        self._check(_lib.lgf_delta(self._h, _ptr(U), _ptr(out), ctypes.byref(th), ctypes.byref(F),
                                   _PREC[precision]))
        return th.value, F.value

    def filter(self, delta, out, precision="fp64"):
        self._bind(delta, out)
        self._check(_lib.lgf_filter(self._h, _ptr(delta), _ptr(out), _PREC[precision]))

    def filter_coeffs(self, coef, out, precision="fp64"):
        """The p^2_max/p^2 filter of Algorithm 1 on each of the eight real fields coef[:, a] (float64,
        (V, 8) or (Nt, Nz, Ny, Nx, 8)); out may be coef itself."""
        self._bind(coef, out)
        self._check(_lib.lgf_filter_coeffs(self._h, _ptr(coef, True), _ptr(out, True), _PREC[precision]))

    def gauge(self, dtilde, alpha, out, precision="fp64"):
        self._bind(dtilde, out)
        self._check(_lib.lgf_gauge(self._h, _ptr(dtilde), float(alpha), _ptr(out), _PREC[precision]))

    def update(self, U, g, precision="fp64"):
        self._bind(U, g)
        self._check(_lib.lgf_update(self._h, _ptr(U), _ptr(g), _PREC[precision]))

    # the functional of a Lie-algebra field omega (V x 8 float64, site-major)
    def functional(self, U, omega, g_out=None):
        """F_U[exp(i omega)] (Eq. 1); fills g_out (complex128, (Nt, Nz, Ny, Nx, 3, 3)) if given."""
        F = ctypes.c_double()
        self._bind(U, omega)
        self._check(_lib.lgf_functional(self._h, _ptr(U), _ptr(omega, True), ctypes.byref(F),
                                        None if g_out is None else _ptr(g_out)))
        return F.value

    def functional_grad(self, U, omega, grad_out, scale=1.0):
        """grad_out[s, a] = scale * dF/d omega^a(s) (hand-written backward kernel)."""
        self._bind(U, omega, grad_out)
        self._check(_lib.lgf_functional_grad(self._h, _ptr(U), _ptr(omega, True), float(scale),
                                             _ptr(grad_out, True)))

    # timing
    def enable_timing(self, on=True):
        self._check(_lib.lgf_enable_timing(self._h, 1 if on else 0))

    def kernel_times(self):
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_long * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        self._check(_lib.lgf_kernel_times(self._h, names, launches, ms, cap, ctypes.byref(n)))
        return {names[i].decode(): (launches[i], ms[i]) for i in range(min(n.value, cap))}


class Batch:
    """Several configurations, of possibly different lattice shapes, fixed together: equal shapes share
    kernel launches (one per group), the iteration loop is a replayed CUDA graph, and FFT passes are
    autotuned per (shape, precision)."""

    def __init__(self, dims_list):
        self.dims = [tuple(int(v) for v in d) for d in dims_list]
        flat = (ctypes.c_int * (4 * len(self.dims)))(*[v for d in self.dims for v in d])
        h = ctypes.c_void_p()
        st = _lib.lgf_batch_create(len(self.dims), flat, ctypes.byref(h))
        if st != LGF_OK:
            raise LgfError(st, _lib.lgf_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lgf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def fix(self, Us, alpha=0.08, eps=1e-15, precision="fp64", max_iter=100000, theta_switch=1e-11,
            reunit_period=16):
        """Fix every configuration of Us (list of links, device tensors or numpy arrays) in place.
        Returns a list of dict(theta, F, iters, status)."""
        n = len(self.dims)
        assert len(Us) == n
        for U, d in zip(Us, self.dims):
            assert dims_of(U) == d
            if not isinstance(U, np.ndarray) and getattr(U, "is_cuda", False):
                import torch
                torch.cuda.current_stream().synchronize()  # the batch runs on its own stream
        ptrs = (ctypes.c_void_p * n)(*[_ptr(U) for U in Us])
        o = Lattice.options(precision, theta_switch, reunit_period, max_iter)
        th, F = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        it, stt = (ctypes.c_int * n)(), (ctypes.c_int * n)()
        st = _lib.lgf_batch_fix(self._h, ptrs, alpha, eps, ctypes.byref(o), th, F, it, stt)
        if st not in (LGF_OK, LGF_ENOCONV):
            raise LgfError(st, _lib.lgf_batch_last_error(self._h).decode())
        return [dict(theta=th[i], F=F[i], iters=it[i], status=stt[i]) for i in range(n)]

    def describe(self):
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _lib.lgf_batch_describe(self._h, buf, len(buf))
        return json.loads(buf.value.decode())


def _landau_function():
    import torch

    class LandauF(torch.autograd.Function):
        """F_U[exp(i omega)] as a differentiable function of omega (torch float64, (V, 8) or
        (Nt, Nz, Ny, Nx, 8), on the GPU): forward and backward run in the library's kernels.
        Usage: F = LandauF.apply(omega, U, lattice)."""

        @staticmethod
        def forward(ctx, omega, U, lattice):
            omega = omega.contiguous()
            F = lattice.functional(U, omega)
            ctx.save_for_backward(omega, U)
            ctx.lattice = lattice
            return torch.tensor(F, dtype=torch.float64, device=omega.device)

        @staticmethod
        def backward(ctx, gF):
            omega, U = ctx.saved_tensors
            grad = torch.empty_like(omega)
            ctx.lattice.functional_grad(U, omega, grad, float(gF))
            return grad, None, None

    return LandauF


_LandauF = None


def LandauF():
    """The torch.autograd.Function for F_U[exp(i omega)] (created on first use; needs torch)."""
    global _LandauF
    if _LandauF is None:
        _LandauF = _landau_function()
    return _LandauF


def adam_fix(U, target=1e-10, lr=1e-2, max_steps=20000, check_every=20, lr_decay=0.5, min_lr=1e-12,
             omega0=None, precondition=False, optimizer="adam", rebase_every=0, keep_moments=True,
             betas=(0.9, 0.999), amsgrad=False, adam_eps=1e-8, patience=0):
    """Maximise F_U[exp(i omega)] over omega with a torch optimiser, using the library's forward and
    backward kernels, until theta of the transformed links g U g^+ falls to `target`.

    The optimiser minimises the loss -24 V F (V sites): its gradient with respect to omega^a(x) at omega = 0
    is i Tr[T^a Delta(x)], of the size of Delta itself, so Adam's epsilon stays negligible down to small
    theta. omega starts at omega0 (default 0). Every `check_every` steps F and theta are evaluated, and the
    learning rate is multiplied by `lr_decay` once F has not risen above its best value for more than
    `patience` consecutive checks (patience = 0: whenever F did not increase). A momentum method such as
    Adam does not raise F at every step even when it converges, so with frequent checks give it some
    patience.

    optimizer="adam": torch.optim.Adam (betas, amsgrad and adam_eps are passed through); "sgd":
    torch.optim.SGD. With precondition=True the gradient first passes through the p^2_max/p^2 filter of
    Algorithm 1 (lgf_filter_coeffs, the library's FFT kernels), which removes the critical slowing down of
    the plain gradient. SGD with lr = alpha on the preconditioned gradient and re-basing after every step
    is the step of Algorithm 1 with the exponential in place of its first-order expansion.

    Re-basing (every `rebase_every` steps, 0 = never) applies g = exp(i omega) to U exactly (FP64,
    lgf_update) and resets omega to 0, so the gradient is always taken near omega = 0, where its
    coordinates are those of the Lie algebra at the current links. With keep_moments=True the optimiser's
    state (Adam's first and second moments) is carried over unchanged: both coordinate systems are the Lie
    algebra at nearby points, identified by left translation, and they differ by O(|omega|) per component
    (|omega| is one step). With keep_moments=False a new optimiser starts after each re-basing.
    At the end g is applied to U in place. Returns dict(theta, F, F0, steps, lr, history=[(step, theta, F,
    lr)])."""
    import torch
    dims = dims_of(U)
    V = int(np.prod(dims))
    LF = LandauF()
    hist = []
    scale = 24.0 * V

    def make_opt(rate):
        if optimizer == "sgd":
            return torch.optim.SGD([omega], lr=rate)
        return torch.optim.Adam([omega], lr=rate, betas=betas, amsgrad=amsgrad, eps=adam_eps)

    with Lattice(dims) as lat:
        omega = torch.zeros((V, 8), dtype=torch.float64, device=U.device) if omega0 is None else omega0.clone()
        omega = omega.contiguous().requires_grad_(True)
        g = torch.empty(U.shape[1:], dtype=torch.complex128, device=U.device)
        Ut = torch.empty_like(U)

        def evaluate():
            with torch.no_grad():
                F = lat.functional(U, omega.detach(), g)
                Ut.copy_(U)
                lat.update(Ut, g)
                return F, lat.measure(Ut)["theta"]

        F0 = lat.measure(U)["F"]
        F, theta = evaluate()
        hist.append((0, theta, F, lr))
        opt = make_opt(lr)
        step = 0
        best, stale = F, 0
        while step < max_steps and theta > target and opt.param_groups[0]["lr"] > min_lr:
            opt.zero_grad(set_to_none=False)
            loss = -scale * LF.apply(omega, U, lat)
            loss.backward()
            if precondition:
                with torch.no_grad():
                    lat.filter_coeffs(omega.grad, omega.grad)
            opt.step()
            step += 1
            rebase = rebase_every > 0 and step % rebase_every == 0
            if step % check_every == 0 or rebase:
                F, theta = evaluate()
                if F > best:
                    best, stale = F, 0
                else:
                    stale += 1
                    if stale > patience:
                        for pg in opt.param_groups:
                            pg["lr"] *= lr_decay
                        stale = 0
                hist.append((step, theta, F, opt.param_groups[0]["lr"]))
                if rebase:
                    U.copy_(Ut)
                    with torch.no_grad():
                        omega.zero_()
                    if not keep_moments:
                        opt = make_opt(opt.param_groups[0]["lr"])
        F, theta = evaluate()
        U.copy_(Ut)
    return dict(theta=theta, F=F, F0=F0, steps=step, lr=opt.param_groups[0]["lr"], history=hist)


def fix(U, alpha=0.08, eps=1e-15, precision="fp64", **kw):
    """Fix the links U (complex128, (4, Nt, Nz, Ny, Nx, 3, 3)) to Landau gauge in place."""
    with Lattice(dims_of(U)) as lat:
        return lat.fix(U, alpha, eps, precision, **kw)
