"""PyTorch-facing API over the C ABI: plans, analysis/synthesis calls on CUDA tensors,
dual/tight windows, and a torch.autograd.Function whose backward is the library's
hand-written adjoint (synthesis with the analysis window) plus its window gradient.

Every computation runs in libdgt.so; this module only checks tensors and passes
pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _capi as K

_ROUTES = {"auto": K.ROUTE_AUTO, "coset": K.ROUTE_COSET, "shear": K.ROUTE_SHEAR, "fir": K.ROUTE_FIR}
_ROUTE_NAMES = {v: k for k, v in _ROUTES.items()}
_SYN = {"adjoint": K.SYN_ADJOINT, "dual": K.SYN_DUAL, "tight": K.SYN_TIGHT}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """A DGT plan for the lattice (L, a, M, lambda = lam1/lam2) and a window.

    window: 1-D numpy array / CPU tensor, real or complex; full length L, or FIR taps
    when `fir_center` is given (tap t sits at time t - fir_center).
    precision: "f32" or "f64".  route: "auto", "coset", "shear" or "fir".
    block_len: blockwise (overlap-add) plan for an FIR window: blocks of block_len samples
    transformed by the coset or shear route ("auto", "coset", "shear") on the zero-extended
    block, the same results as the plain plan (dgt_plan_create_ola).
    """

    def __init__(self, L, a, M, lam1, lam2, window, route="auto", precision="f32", fir_center=None, stream=None,
                 block_len=None):
        w = np.asarray(window.detach().cpu().numpy() if torch.is_tensor(window) else window)
        self.is_real_window = not np.iscomplexobj(w)
        data = np.ascontiguousarray(w.astype(np.float64) if self.is_real_window
                                    else w.astype(np.complex128).view(np.float64))
        self._window_host = data
        win = K.Window(K.WINDOW_FIR if fir_center is not None else K.WINDOW_FULL, len(w),
                       int(fir_center or 0), data.ctypes.data_as(C.POINTER(C.c_double)), int(self.is_real_window))
        self.precision = precision
        prec = K.F64 if precision == "f64" else K.F32
        h = C.c_void_p()
        if block_len is not None:
            if fir_center is None:
                raise ValueError("a blockwise plan needs FIR taps (fir_center)")
            K.check(K.lib().dgt_plan_create_ola(C.byref(h), L, a, M, lam1, lam2, C.byref(win), int(block_len),
                                                 _ROUTES[route], prec, _stream(stream)))
        else:
            K.check(K.lib().dgt_plan_create(C.byref(h), L, a, M, lam1, lam2, C.byref(win), _ROUTES[route], prec,
                                             _stream(stream)))
        self._h = h
        info = K.PlanInfo()
        K.check(K.lib().dgt_plan_get_info(self._h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in K.PlanInfo._fields_}
        self.info["route_name"] = _ROUTE_NAMES[info.route]
        self.L, self.a, self.M, self.N = L, a, M, L // a
        self.lam1, self.lam2 = lam1, lam2
        self.rdtype = torch.float64 if precision == "f64" else torch.float32
        self.cdtype = torch.complex128 if precision == "f64" else torch.complex64

    # ------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            K.lib().dgt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def route(self) -> str:
        return self.info["route_name"]

    def _check_signal(self, f):
        if not f.is_cuda or not f.is_contiguous():
            raise ValueError("signal must be a contiguous CUDA tensor")
        if f.dtype not in (self.rdtype, self.cdtype):
            raise TypeError("signal dtype %s does not match the plan precision %s" % (f.dtype, self.precision))
        if f.shape[-1] != self.L:
            raise ValueError("signal length %d != L=%d" % (f.shape[-1], self.L))

    def dgt(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Coefficients c[..., n, m] (complex) of signals f[..., L]."""
        self._check_signal(f)
        B = int(np.prod(f.shape[:-1])) if f.dim() > 1 else 1
        if out is None:
            out = torch.empty(tuple(f.shape[:-1]) + (self.N, self.M), dtype=self.cdtype, device=f.device)
        K.check(K.lib().dgt_exec(self._h, f.data_ptr(), int(not f.is_complex()), out.data_ptr(), B,
                                 _stream(stream)))
        return out

    def idgt(self, c: torch.Tensor, window: str = "dual", real: bool = False, out=None, stream=None) -> torch.Tensor:
        """Synthesis f = C_gamma^* c with gamma = g ("adjoint"), S^-1 g ("dual") or S^-1/2 g ("tight")."""
        if not c.is_cuda or not c.is_contiguous() or c.dtype != self.cdtype:
            raise TypeError("coefficients must be a contiguous CUDA %s tensor" % self.cdtype)
        if tuple(c.shape[-2:]) != (self.N, self.M):
            raise ValueError("coefficient shape %s != (N, M)=(%d, %d)" % (tuple(c.shape), self.N, self.M))
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        if out is None:
            out = torch.empty(tuple(c.shape[:-2]) + (self.L,), dtype=self.rdtype if real else self.cdtype,
                              device=c.device)
        K.check(K.lib().idgt_exec(self._h, c.data_ptr(), out.data_ptr(), int(real), B, _SYN[window],
                                  _stream(stream)))
        return out

    def idgt_window(self, c: torch.Tensor, gamma: torch.Tensor, real: bool = False, out=None, stream=None):
        """Synthesis with the caller's window gamma (CUDA tensor of the plan precision, real or
        complex; L samples, or the FIR taps for an FIR-route plan)."""
        if not c.is_cuda or not c.is_contiguous() or c.dtype != self.cdtype:
            raise TypeError("coefficients must be a contiguous CUDA %s tensor" % self.cdtype)
        if tuple(c.shape[-2:]) != (self.N, self.M):
            raise ValueError("coefficient shape %s != (N, M)=(%d, %d)" % (tuple(c.shape), self.N, self.M))
        if not gamma.is_cuda or not gamma.is_contiguous() or gamma.dtype not in (self.rdtype, self.cdtype):
            raise TypeError("window must be a contiguous CUDA tensor of the plan precision")
        want = self.info["fir_len"] if self.info["route_name"] == "fir" else self.L
        if gamma.numel() != want:
            raise ValueError("window length %d != %d" % (gamma.numel(), want))
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        if out is None:
            out = torch.empty(tuple(c.shape[:-2]) + (self.L,), dtype=self.rdtype if real else self.cdtype,
                              device=c.device)
        K.check(K.lib().idgt_exec_window(self._h, c.data_ptr(), out.data_ptr(), int(real), B, gamma.data_ptr(),
                                         int(not gamma.is_complex()), _stream(stream)))
        return out

    def dgtreal(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Channels 0..M/2 of the coefficients of real signals f[..., L] (real window,
        lambda2 <= 2, M even): c[..., n, m], m <= M/2."""
        self._check_signal(f)
        if f.is_complex():
            raise TypeError("dgtreal needs real signals")
        B = int(np.prod(f.shape[:-1])) if f.dim() > 1 else 1
        if out is None:
            out = torch.empty(tuple(f.shape[:-1]) + (self.N, self.M // 2 + 1), dtype=self.cdtype, device=f.device)
        K.check(K.lib().dgt_exec_real(self._h, f.data_ptr(), out.data_ptr(), B, _stream(stream)))
        return out

    def idgtreal(self, c: torch.Tensor, window: str = "dual", out=None, stream=None) -> torch.Tensor:
        """Real synthesis from channels 0..M/2 (the inverse of dgtreal with the dual window)."""
        if not c.is_cuda or not c.is_contiguous() or c.dtype != self.cdtype:
            raise TypeError("coefficients must be a contiguous CUDA %s tensor" % self.cdtype)
        if tuple(c.shape[-2:]) != (self.N, self.M // 2 + 1):
            raise ValueError("coefficient shape %s != (N, M/2+1)" % (tuple(c.shape),))
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        if out is None:
            out = torch.empty(tuple(c.shape[:-2]) + (self.L,), dtype=self.rdtype, device=c.device)
        K.check(K.lib().idgt_exec_real(self._h, c.data_ptr(), out.data_ptr(), B, _SYN[window], _stream(stream)))
        return out

    def dual_window(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.L, dtype=self.cdtype, device="cuda")
        K.check(K.lib().dgt_window_dual(self._h, out.data_ptr(), _stream(stream)))
        return out

    def tight_window(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.L, dtype=self.cdtype, device="cuda")
        K.check(K.lib().dgt_window_tight(self._h, out.data_ptr(), _stream(stream)))
        return out

    def set_window(self, g: torch.Tensor, stream=None):
        if not g.is_cuda or not g.is_contiguous() or g.dtype not in (self.rdtype, self.cdtype):
            raise TypeError("window must be a contiguous CUDA tensor of the plan precision")
        K.check(K.lib().dgt_plan_set_window(self._h, g.data_ptr(), int(not g.is_complex()), _stream(stream)))

    def grad_window(self, f: torch.Tensor, G: torch.Tensor, real: bool = True, stream=None) -> torch.Tensor:
        """Window gradient of a real loss with coefficient gradient G, summed over the batch."""
        self._check_signal(f)
        B = int(np.prod(f.shape[:-1])) if f.dim() > 1 else 1
        out = torch.empty(self.L, dtype=self.rdtype if real else self.cdtype, device=f.device)
        K.check(K.lib().dgt_grad_window(self._h, f.data_ptr(), int(not f.is_complex()), G.data_ptr(),
                                        out.data_ptr(), int(real), B, _stream(stream)))
        return out

    def logmag_loss(self, c: torch.Tensor, eps: float = 1e-6, need_grad: bool = True, stream=None):
        """Per-signal sum log(|c|^2 + eps) (float64) and its coefficient gradient 2c/(|c|^2+eps)."""
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        loss = torch.empty(B, dtype=torch.float64, device=c.device)
        G = torch.empty_like(c) if need_grad else None
        K.check(K.lib().dgt_logmag_loss(self._h, c.data_ptr(), G.data_ptr() if G is not None else None,
                                        loss.data_ptr(), eps, B, _stream(stream)))
        return loss, G

    def workspace_bytes(self, batch: int) -> int:
        v = C.c_size_t()
        K.check(K.lib().dgt_workspace_bytes(self._h, batch, C.byref(v)))
        return v.value

    def dgt_ws(self, f, out, workspace: torch.Tensor, stream=None):
        B = int(np.prod(f.shape[:-1])) if f.dim() > 1 else 1
        K.check(K.lib().dgt_exec_ws(self._h, f.data_ptr(), int(not f.is_complex()), out.data_ptr(), B,
                                    workspace.data_ptr() if workspace is not None else None, _stream(stream)))
        return out

    def idgt_ws(self, c, out, window: str, real: bool, workspace: torch.Tensor, stream=None):
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        K.check(K.lib().idgt_exec_ws(self._h, c.data_ptr(), out.data_ptr(), int(real), B, _SYN[window],
                                     workspace.data_ptr() if workspace is not None else None, _stream(stream)))
        return out

    def dgt_host(self, f: torch.Tensor, out: torch.Tensor | None = None, chunk: int = 0, stream=None):
        """Analysis of HOST signals f[..., L] into HOST coefficients (dgt_exec_host): chunks of
        `chunk` signals are copied in, transformed and copied out on overlapping streams.  With
        pinned tensors the call returns before the copies end; synchronise `stream` first."""
        if f.is_cuda or not f.is_contiguous() or f.dtype not in (self.rdtype, self.cdtype):
            raise TypeError("signal must be a contiguous host tensor of the plan precision")
        if f.shape[-1] != self.L:
            raise ValueError("signal length %d != L=%d" % (f.shape[-1], self.L))
        B = int(np.prod(f.shape[:-1])) if f.dim() > 1 else 1
        if out is None:
            out = torch.empty(tuple(f.shape[:-1]) + (self.N, self.M), dtype=self.cdtype, pin_memory=f.is_pinned())
        K.check(K.lib().dgt_exec_host(self._h, f.data_ptr(), int(not f.is_complex()), out.data_ptr(), B, int(chunk),
                                      _stream(stream)))
        return out

    def idgt_host(self, c: torch.Tensor, window: str = "dual", real: bool = False, out=None, chunk: int = 0,
                  stream=None):
        """Synthesis from HOST coefficients c[..., N, M] into HOST signals (idgt_exec_host)."""
        if c.is_cuda or not c.is_contiguous() or c.dtype != self.cdtype:
            raise TypeError("coefficients must be a contiguous host %s tensor" % self.cdtype)
        if tuple(c.shape[-2:]) != (self.N, self.M):
            raise ValueError("coefficient shape %s != (N, M)=(%d, %d)" % (tuple(c.shape), self.N, self.M))
        B = int(np.prod(c.shape[:-2])) if c.dim() > 2 else 1
        if out is None:
            out = torch.empty(tuple(c.shape[:-2]) + (self.L,), dtype=self.rdtype if real else self.cdtype,
                              pin_memory=c.is_pinned())
        K.check(K.lib().idgt_exec_host(self._h, c.data_ptr(), out.data_ptr(), int(real), B, _SYN[window],
                                       int(chunk), _stream(stream)))
        return out

    def status(self, stream=None) -> None:
        """Synchronise and raise DGTError(DGT_ERR_TIMEOUT) if a bounded device wait of this
        plan's calls without a caller workspace expired (the plan's next call raises it too)."""
        K.check(K.lib().dgt_plan_status(self._h, _stream(stream)))

    def workspace_status(self, workspace: torch.Tensor, stream=None) -> None:
        """Synchronise `stream` and raise DGTError(DGT_ERR_TIMEOUT) if the last synthesis that
        used `workspace` (idgt_ws) had a kernel give up waiting for its tile copies."""
        K.check(K.lib().dgt_workspace_status(self._h, workspace.data_ptr(), _stream(stream)))

    def plan_bytes(self) -> int:
        v = C.c_size_t()
        K.check(K.lib().dgt_plan_bytes(self._h, C.byref(v)))
        return v.value


def _window_struct(window, fir_center):
    w = np.asarray(window.detach().cpu().numpy() if torch.is_tensor(window) else window)
    real = not np.iscomplexobj(w)
    data = np.ascontiguousarray(w.astype(np.float64) if real else w.astype(np.complex128).view(np.float64))
    win = K.Window(K.WINDOW_FIR if fir_center is not None else K.WINDOW_FULL, len(w), int(fir_center or 0),
                   data.ctypes.data_as(C.POINTER(C.c_double)), int(real))
    return win, data


class Plan2:
    """Two-dimensional DGT on the tensor-product lattice lattice1 x lattice2 with the separable
    window g1 (x) g2 (dgt2_plan_create).  lattice_i = (L_i, a_i, M_i, lam1_i, lam2_i); signals
    f[..., L1, L2]; coefficients c[..., N1, M1, N2, M2]."""

    def __init__(self, lattice1, window1, lattice2, window2, route="auto", precision="f32", fir_center1=None,
                 fir_center2=None, stream=None):
        (L1, a1, M1, p1, q1), (L2, a2, M2, p2, q2) = lattice1, lattice2
        w1, d1 = _window_struct(window1, fir_center1)
        w2, d2 = _window_struct(window2, fir_center2)
        self._keep = (d1, d2)
        prec = K.F64 if precision == "f64" else K.F32
        h = C.c_void_p()
        K.check(K.lib().dgt2_plan_create(C.byref(h), L1, a1, M1, p1, q1, C.byref(w1), L2, a2, M2, p2, q2, C.byref(w2),
                                          _ROUTES[route], prec, _stream(stream)))
        self._h = h
        self.L1, self.L2, self.N1, self.M1, self.N2, self.M2 = L1, L2, L1 // a1, M1, L2 // a2, M2
        self.precision = precision
        self.rdtype = torch.float64 if precision == "f64" else torch.float32
        self.cdtype = torch.complex128 if precision == "f64" else torch.complex64

    def close(self):
        if getattr(self, "_h", None):
            K.lib().dgt2_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dgt(self, f: torch.Tensor, stream=None) -> torch.Tensor:
        if not f.is_cuda or not f.is_contiguous() or f.dtype not in (self.rdtype, self.cdtype):
            raise TypeError("signals must be contiguous CUDA tensors of the plan precision")
        if tuple(f.shape[-2:]) != (self.L1, self.L2):
            raise ValueError("signal shape %s != (L1, L2)" % (tuple(f.shape),))
        B = int(np.prod(f.shape[:-2])) if f.dim() > 2 else 1
        out = torch.empty(tuple(f.shape[:-2]) + (self.N1, self.M1, self.N2, self.M2), dtype=self.cdtype,
                          device=f.device)
        K.check(K.lib().dgt2_exec(self._h, f.data_ptr(), int(not f.is_complex()), out.data_ptr(), B, _stream(stream)))
        return out

    def idgt(self, c: torch.Tensor, window: str = "dual", real: bool = False, stream=None) -> torch.Tensor:
        if not c.is_cuda or not c.is_contiguous() or c.dtype != self.cdtype:
            raise TypeError("coefficients must be a contiguous CUDA %s tensor" % self.cdtype)
        if tuple(c.shape[-4:]) != (self.N1, self.M1, self.N2, self.M2):
            raise ValueError("coefficient shape %s != (N1, M1, N2, M2)" % (tuple(c.shape),))
        B = int(np.prod(c.shape[:-4])) if c.dim() > 4 else 1
        out = torch.empty(tuple(c.shape[:-4]) + (self.L1, self.L2), dtype=self.rdtype if real else self.cdtype,
                          device=c.device)
        K.check(K.lib().idgt2_exec(self._h, c.data_ptr(), out.data_ptr(), int(real), B, _SYN[window],
                                   _stream(stream)))
        return out

    def status(self, stream=None) -> None:
        K.check(K.lib().dgt2_plan_status(self._h, _stream(stream)))


def debug_status():
    """Guard-zone report of the DGT_DEBUG build (``DGT_DEBUG=1`` loads libdgt_debug.so):
    (violations, kernel, zone_offset) -- guard words found overwritten since the previous call,
    the launch after which the first was found and its byte offset in its zone.  Synchronises
    the device.  Raises DGTError (DGT_ERR_UNSUPPORTED) in the release build."""
    v, off = C.c_ulonglong(0), C.c_longlong(-1)
    name = C.create_string_buffer(128)
    K.check(K.lib().dgt_debug_status(C.byref(v), C.byref(off), name, 128))
    return int(v.value), name.value.decode(), int(off.value)


def fft_selftest(x: torch.Tensor, direction: int = -1) -> torch.Tensor:
    """Library FFT building block on rows of x (contiguous complex CUDA tensor)."""
    prec = K.F64 if x.dtype == torch.complex128 else K.F32
    out = torch.empty_like(x)
    n = x.shape[-1]
    K.check(K.lib().dgt_fft_selftest(n, prec, direction, x.data_ptr(), out.data_ptr(), x.numel() // n,
                                     _stream(None)))
    return out


class DGTFunction(torch.autograd.Function):
    """c = DGT_g(f) with gradients in the signal f and a full-length window g.

    backward: grad_f = C_g^* grad_c (the library's synthesis with the analysis window,
    real part for a real signal); grad_g = the library's window gradient."""

    @staticmethod
    def forward(ctx, f, g, plan: Plan):
        if g is not None and g.requires_grad:
            plan.set_window(g.detach().contiguous())
        c = plan.dgt(f.detach().contiguous())
        ctx.plan = plan
        ctx.save_for_backward(f, g)
        return c

    @staticmethod
    def backward(ctx, grad_c):
        f, g = ctx.saved_tensors
        plan = ctx.plan
        grad_c = grad_c.contiguous()
        gf = gg = None
        if ctx.needs_input_grad[0]:
            gf = plan.idgt(grad_c, window="adjoint", real=not f.is_complex())
        if g is not None and ctx.needs_input_grad[1]:
            gg = plan.grad_window(f.detach().contiguous(), grad_c, real=not g.is_complex())
        return gf, gg, None


def dgt(f, g, plan: Plan):
    return DGTFunction.apply(f, g, plan)


class LogMagLoss(torch.autograd.Function):
    """l = sum over the batch and every coefficient of log(|c|^2 + eps), from one pass of the
    library's kernel that also writes dl/dc = 2 c / (|c|^2 + eps) (the gradient convention
    d/dRe + i d/dIm); backward scales it by the incoming gradient.  The value is float64."""

    @staticmethod
    def forward(ctx, c, plan: Plan, eps: float):
        per_signal, G = plan.logmag_loss(c.detach().contiguous(), eps=eps, need_grad=c.requires_grad)
        ctx.save_for_backward(G)
        return per_signal.sum()

    @staticmethod
    def backward(ctx, grad):
        (G,) = ctx.saved_tensors
        return G * grad.to(G.real.dtype), None, None


def log_magnitude_loss(c, plan: Plan, eps: float = 1e-6):
    """sum log(|c|^2 + eps) with the fused forward / gradient kernel (see LogMagLoss)."""
    return LogMagLoss.apply(c, plan, eps)
