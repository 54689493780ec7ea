"""Python face of the Dichotomy solver: the C entry points with torch tensors.

Functions named after the C ABI (``dichotomy_plan``, ``dichotomy_solve``, ...) marshal
torch CUDA tensors to device pointers and torch's current stream to a cudaStream_t.  The
classes ``Plan`` and ``Batch`` own the device workspace (a uint8 torch tensor) that the
library needs; ``DichotomySolve`` / ``DichotomySolveBatched`` are autograd Functions whose
backward is the library's adjoint kernel (Not in the paper: dL/dF = T^-T w,
dL/dt = -(sum lambda_i x_{i-1}, sum lambda_i x_i, sum lambda_i x_{i+1})).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (FLAG_ALLOW_NOT_DOMINANT, FLAG_CHECK_FINITE, FLAG_DEVICE_PRELIM, FLAG_FORCE_GENERAL, FLAG_HOST_PRELIM, FLAG_REG_PATH, FLAG_SMEM_PATH, PREC_AUTO, PREC_F64, PREC_MIXED, DichotomyError,
                   check, make_opts)

__all__ = [
    "dichotomy_plan", "dichotomy_plan_quasi", "dichotomy_plan_info", "dichotomy_plan_workspace_bytes", "dichotomy_plan_bind",
    "dichotomy_solve", "dichotomy_solve_series", "dichotomy_solve_host", "dichotomy_adjoint", "dichotomy_status", "dichotomy_destroy",
    "dichotomy_batch_prepare", "dichotomy_batch_workspace_bytes", "dichotomy_batch_bind",
    "dichotomy_solve_batched", "dichotomy_adjoint_batched", "dichotomy_batch_status", "dichotomy_batch_info",
    "dichotomy_batch_destroy", "Plan", "Batch", "GenPlan", "solve", "DichotomySolve", "DichotomySolveQuasi", "DichotomySolveBatched", "DichotomySolveBatchedQuasi",
    "PREC_F64", "PREC_MIXED", "PREC_AUTO", "FLAG_FORCE_GENERAL", "FLAG_CHECK_FINITE", "FLAG_HOST_PRELIM", "FLAG_DEVICE_PRELIM", "FLAG_ALLOW_NOT_DOMINANT", "FLAG_REG_PATH", "FLAG_SMEM_PATH", "DichotomyError",
]


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t: torch.Tensor, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the solver has no CPU path)")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C entry points
def dichotomy_plan(t_m1: float, t_0: float, t_1: float, N: int, opts=None) -> ctypes.c_void_p:
    L = _lib.load()
    h = ctypes.c_void_p()
    if opts is None:
        check(L.dichotomy_plan(float(t_m1), float(t_0), float(t_1), int(N), ctypes.byref(h)), "dichotomy_plan")
    else:
        check(L.dichotomy_plan_ex(float(t_m1), float(t_0), float(t_1), int(N), ctypes.byref(opts), ctypes.byref(h)),
              "dichotomy_plan_ex")
    return h


def dichotomy_plan_quasi(t_m1: float, t_0: float, t_1: float, psi: float, chi: float, N: int,
                         opts=None) -> ctypes.c_void_p:
    """Plan for the quasi-Toeplitz matrix of eq. 21 (t_0 + psi in the first row, t_0 + chi in the last)."""
    h = ctypes.c_void_p()
    o = make_opts() if opts is None else opts
    check(_lib.load().dichotomy_plan_quasi(float(t_m1), float(t_0), float(t_1), float(psi), float(chi), int(N),
                                          ctypes.byref(o), ctypes.byref(h)), "dichotomy_plan_quasi")
    return h


def dichotomy_plan_info(plan) -> dict:
    info = _lib.dich_plan_info()
    check(_lib.load().dichotomy_plan_info(plan, ctypes.byref(info)), "dichotomy_plan_info")
    return {name: getattr(info, name) for name, _ in info._fields_}


def dichotomy_plan_workspace_bytes(plan) -> int:
    n = ctypes.c_size_t()
    check(_lib.load().dichotomy_plan_workspace_bytes(plan, ctypes.byref(n)), "dichotomy_plan_workspace_bytes")
    return int(n.value)


def dichotomy_plan_bind(plan, workspace: torch.Tensor, stream=None) -> None:
    if not workspace.is_cuda:
        raise TypeError("workspace must be a CUDA tensor")
    check(_lib.load().dichotomy_plan_bind(plan, ctypes.c_void_p(workspace.data_ptr()),
                                          workspace.numel() * workspace.element_size(), _stream(stream)),
          "dichotomy_plan_bind")


def dichotomy_solve(plan, F: torch.Tensor, x: torch.Tensor, stream=None) -> None:
    check(_lib.load().dichotomy_solve(plan, _dev(F, "F"), _dev(x, "x"), _stream(stream)), "dichotomy_solve")


def _dev_rows(t: torch.Tensor, name: str):
    """Pointer and row stride (in elements) of a 2-D float64 CUDA tensor with unit column stride."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the solver has no CPU path)")
    if t.dtype != torch.float64 or t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1):
        raise TypeError(f"{name} must be a 2-D float64 tensor with contiguous rows")
    return ctypes.c_void_p(t.data_ptr()), int(t.stride(0))


def dichotomy_solve_series(plan, F: torch.Tensor, x: torch.Tensor, stream=None) -> None:
    """x[k] = T^-1 F[k] for every row k of the [M, N] tensors F and x (rows may be strided)."""
    pF, ldf = _dev_rows(F, "F")
    px, ldx = _dev_rows(x, "x")
    if F.shape != x.shape:
        raise ValueError("F and x must have the same shape")
    check(_lib.load().dichotomy_solve_series(plan, int(F.shape[0]), pF, ldf, px, ldx, _stream(stream)),
          "dichotomy_solve_series")


def _host(t: torch.Tensor, name: str, n: int):
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CPU tensor")
    if t.numel() != n:
        raise ValueError(f"{name} must hold {n} values")
    return ctypes.c_void_p(t.data_ptr())


def dichotomy_solve_host(plan, F: torch.Tensor, x: torch.Tensor, dF: torch.Tensor | None, dx: torch.Tensor | None,
                         chunks=0, stream=None) -> None:
    """Enqueue x = T^-1 F for host tensors F, x: directly from and to pinned memory (chunks = 0),
    else through the device staging tensors dF, dx; x is complete once the stream has synchronized."""
    n = F.numel()
    pF = _dev(dF, "dF") if dF is not None else None
    px = _dev(dx, "dx") if dx is not None else None
    check(_lib.load().dichotomy_solve_host(plan, _host(F, "F", n), _host(x, "x", n), pF, px, int(chunks),
                                           _stream(stream)), "dichotomy_solve_host")


def dichotomy_adjoint(plan, w: torch.Tensor, x: torch.Tensor, gF: torch.Tensor, gt: torch.Tensor,
                      stream=None) -> None:
    check(_lib.load().dichotomy_adjoint(plan, _dev(w, "w"), _dev(x, "x"), _dev(gF, "gF"), _dev(gt, "gt"),
                                        _stream(stream)), "dichotomy_adjoint")


def dichotomy_status(plan, stream=None) -> int:
    s = ctypes.c_int(0)
    check(_lib.load().dichotomy_status(plan, _stream(stream), ctypes.byref(s)), "dichotomy_status")
    return int(s.value)


def dichotomy_destroy(plan) -> None:
    _lib.load().dichotomy_destroy(plan)


def _host_i64(a):
    import numpy as np
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _host_f64(a):
    import numpy as np
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def dichotomy_batch_prepare(N, offset, t_m1, t_0, t_1, opts=None, psi=None, chi=None) -> ctypes.c_void_p:
    """Prepare a batch; with psi / chi arrays, a batch of quasi-Toeplitz systems (eq. 21)."""
    N, offset = _host_i64(N), _host_i64(offset)
    tm1, t0, tp1 = _host_f64(t_m1), _host_f64(t_0), _host_f64(t_1)
    nsys = N.size
    if not (offset.size == tm1.size == t0.size == tp1.size == nsys):
        raise ValueError("batch arrays must have one entry per system")
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    o = ctypes.byref(opts) if opts is not None else None
    if psi is None and chi is None:
        check(_lib.load().dichotomy_batch_prepare(nsys, p(N), p(offset), p(tm1), p(t0), p(tp1), o, ctypes.byref(h)),
              "dichotomy_batch_prepare")
        return h
    import numpy as np
    ps = _host_f64(psi if psi is not None else np.zeros(nsys))
    ch = _host_f64(chi if chi is not None else np.zeros(nsys))
    if not (ps.size == ch.size == nsys):
        raise ValueError("psi and chi must have one entry per system")
    check(_lib.load().dichotomy_batch_prepare_quasi(nsys, p(N), p(offset), p(tm1), p(t0), p(tp1), p(ps), p(ch), o,
                                                    ctypes.byref(h)), "dichotomy_batch_prepare_quasi")
    return h


def dichotomy_batch_workspace_bytes(batch) -> int:
    n = ctypes.c_size_t()
    check(_lib.load().dichotomy_batch_workspace_bytes(batch, ctypes.byref(n)), "dichotomy_batch_workspace_bytes")
    return int(n.value)


def dichotomy_batch_bind(batch, workspace: torch.Tensor, stream=None) -> None:
    check(_lib.load().dichotomy_batch_bind(batch, ctypes.c_void_p(workspace.data_ptr()),
                                           workspace.numel() * workspace.element_size(), _stream(stream)),
          "dichotomy_batch_bind")


def dichotomy_solve_batched(batch, F: torch.Tensor, x: torch.Tensor, stream=None) -> None:
    check(_lib.load().dichotomy_solve_batched(batch, _dev(F, "F"), _dev(x, "x"), _stream(stream)),
          "dichotomy_solve_batched")


def dichotomy_adjoint_batched(batch, w, x, gF, gt, stream=None) -> None:
    check(_lib.load().dichotomy_adjoint_batched(batch, _dev(w, "w"), _dev(x, "x"), _dev(gF, "gF"), _dev(gt, "gt"),
                                                _stream(stream)), "dichotomy_adjoint_batched")


def dichotomy_batch_status(batch, stream=None) -> int:
    s = ctypes.c_int(0)
    check(_lib.load().dichotomy_batch_status(batch, _stream(stream), ctypes.byref(s)), "dichotomy_batch_status")
    return int(s.value)


def dichotomy_batch_info(batch) -> dict:
    import numpy as np
    ns, nw = ctypes.c_int64(), ctypes.c_int64()
    check(_lib.load().dichotomy_batch_info(batch, ctypes.byref(ns), ctypes.byref(nw), None), "dichotomy_batch_info")
    forms = np.zeros(ns.value, dtype=np.int32)
    check(_lib.load().dichotomy_batch_info(batch, None, None, forms.ctypes.data_as(ctypes.c_void_p)),
          "dichotomy_batch_info")
    return {"nsys": ns.value, "windows": nw.value, "form": forms}


def dichotomy_batch_destroy(batch) -> None:
    _lib.load().dichotomy_batch_destroy(batch)


# ------------------------------------------------------------------ owning wrappers
class Plan:
    """A bound single-system plan: T = tridiag{t_m1, t_0, t_1} of order N on a CUDA device (with
    psi, chi: the quasi-Toeplitz matrix of eq. 21, t_0 + psi in the first row, t_0 + chi in the last)."""

    def __init__(self, t_m1, t_0, t_1, N, block_size=0, precision=PREC_F64, threads=0, flags=0, trunc_eps=0.0,
                 device=None, stream=None, psi=None, chi=None):
        self.t = (float(t_m1), float(t_0), float(t_1))
        self.N = int(N)
        # psi / chi given (zeros included): a corner plan, whose adjoint also returns dL/dpsi, dL/dchi
        self.quasi = psi is not None or chi is not None
        self.corners = (float(psi or 0.0), float(chi or 0.0))
        self._h = None
        opts = make_opts(block_size, precision, threads, flags, trunc_eps)
        if self.quasi:
            self._h = dichotomy_plan_quasi(t_m1, t_0, t_1, self.corners[0], self.corners[1], N, opts)
        else:
            self._h = dichotomy_plan(t_m1, t_0, t_1, N, opts)
        self.info = dichotomy_plan_info(self._h)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(max(1, self.info["workspace_bytes"]), dtype=torch.uint8, device=dev)
        dichotomy_plan_bind(self._h, self.workspace, stream)

    @property
    def handle(self):
        return self._h

    def solve(self, F: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = torch.empty_like(F) if out is None else out
        dichotomy_solve(self._h, F, x, stream)
        return x

    def solve_series(self, F: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Every row of F ([M, N]) solved with this plan (a series with a constant matrix)."""
        x = torch.empty_like(F) if out is None else out
        dichotomy_solve_series(self._h, F, x, stream)
        return x

    def solve_host(self, F: torch.Tensor, out: torch.Tensor | None = None, chunks: int = 0, stream=None) -> torch.Tensor:
        """x = T^-1 F for a CPU tensor F: with pinned F and x (and chunks = 0) the kernels read and
        write them directly over the host link; otherwise pipelined copy-in, solve and copy-out
        through device staging tensors kept by the plan.  Returns once x is complete."""
        x = torch.empty(F.shape, dtype=F.dtype, pin_memory=F.is_pinned()) if out is None else out
        direct = chunks == 0 and F.is_pinned() and x.is_pinned() and self.info["path"] != 2
        if not direct and getattr(self, "_staging", None) is None:
            dev = self.workspace.device
            self._staging = (torch.empty(self.N, dtype=torch.float64, device=dev),
                             torch.empty(self.N, dtype=torch.float64, device=dev))
        if direct:
            try:
                dichotomy_solve_host(self._h, F, x, None, None, 0, stream)
                direct = True
            except DichotomyError as err:   # pinned but not mapped into the device's address space
                if err.code != 1:
                    raise
                direct = False
                if getattr(self, "_staging", None) is None:
                    dev = self.workspace.device
                    self._staging = (torch.empty(self.N, dtype=torch.float64, device=dev),
                                     torch.empty(self.N, dtype=torch.float64, device=dev))
        if not direct:
            dichotomy_solve_host(self._h, F, x, self._staging[0], self._staging[1], chunks, stream)
        if isinstance(stream, torch.cuda.Stream):
            stream.synchronize()
        elif stream is None:
            torch.cuda.current_stream(self.workspace.device).synchronize()
        else:
            torch.cuda.synchronize(self.workspace.device)
        return x

    def adjoint(self, w: torch.Tensor, x: torch.Tensor, stream=None):
        """lambda = A^-T w and dL/d(t_-1, t_0, t_1) (then dL/dpsi, dL/dchi for corner plans)."""
        gF = torch.empty_like(w)
        gt = torch.empty(5 if self.quasi else 3, dtype=torch.float64, device=w.device)
        dichotomy_adjoint(self._h, w, x, gF, gt, stream)
        return gF, gt

    def residual(self, F: torch.Tensor, x: torch.Tensor, stream=None):
        """The a posteriori check: (max |F - A x|, norm-wise backward error)."""
        out = (ctypes.c_double * 2)()
        check(_lib.load().dichotomy_residual(self._h, _dev(F, "F"), _dev(x, "x"), out, _stream(stream)),
              "dichotomy_residual")
        return float(out[0]), float(out[1])

    def status(self, stream=None) -> int:
        return dichotomy_status(self._h, stream)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib_obj is not None:
            _lib._lib_obj.dichotomy_destroy(self._h)
            self._h = None


class Batch:
    """A bound batch of independent Toeplitz systems stored back to back in one vector (with psi,
    chi arrays: quasi-Toeplitz systems, eq. 21)."""

    def __init__(self, N, t_m1, t_0, t_1, offset=None, block_size=0, precision=PREC_F64, threads=0, flags=0,
                 trunc_eps=0.0, device=None, stream=None, psi=None, chi=None):
        import numpy as np
        N = _host_i64(N)
        if offset is None:
            offset = np.concatenate([[0], np.cumsum(N)[:-1]]).astype(np.int64) if N.size else np.zeros(0, np.int64)
        self.N = N
        self.offset = _host_i64(offset)
        self.total = int((self.offset + N).max()) if N.size else 0
        self._h = None
        opts = make_opts(block_size, precision, threads, flags, trunc_eps)
        self.corners = psi is not None or chi is not None
        self._h = dichotomy_batch_prepare(N, self.offset, t_m1, t_0, t_1, opts, psi=psi, chi=chi)
        self.info = dichotomy_batch_info(self._h)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(max(1, dichotomy_batch_workspace_bytes(self._h)), dtype=torch.uint8, device=dev)
        dichotomy_batch_bind(self._h, self.workspace, stream)

    @property
    def handle(self):
        return self._h

    @property
    def nsys(self) -> int:
        return int(self.N.size)

    def solve(self, F: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = torch.empty_like(F) if out is None else out
        dichotomy_solve_batched(self._h, F, x, stream)
        return x

    def adjoint(self, w: torch.Tensor, x: torch.Tensor, stream=None):
        gF = torch.empty_like(w)
        gt = torch.empty((self.nsys, 5 if self.corners else 3), dtype=torch.float64, device=w.device)
        dichotomy_adjoint_batched(self._h, w, x, gF, gt, stream)
        return gF, gt

    def status(self, stream=None) -> int:
        return dichotomy_batch_status(self._h, stream)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib_obj is not None:
            _lib._lib_obj.dichotomy_batch_destroy(self._h)
            self._h = None


class GenPlan:
    """A bound plan for a general tridiagonal matrix (sub-diagonal a, diagonal b, super-diagonal c,
    host arrays of N entries; a[0] and c[N-1] are ignored): the general O(N) preliminary step of
    the Dichotomy Algorithm, then any number of FP64 solves."""

    def __init__(self, a, b, c, block_size=0, threads=0, flags=0, trunc_eps=0.0, device=None, stream=None,
                 precision=PREC_F64):
        a, b, c = _host_f64(a), _host_f64(b), _host_f64(c)
        if not (a.size == b.size == c.size):
            raise ValueError("a, b and c must have one entry per row")
        self.N = int(b.size)
        self._h = None
        L = _lib.load()
        h = ctypes.c_void_p()
        opts = make_opts(block_size, precision, threads, flags, trunc_eps)
        check(L.dichotomy_gen_plan(self.N, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                                   c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts), ctypes.byref(h)),
              "dichotomy_gen_plan")
        self._h = h
        info = _lib.dich_plan_info()
        check(L.dichotomy_gen_info(h, ctypes.byref(info)), "dichotomy_gen_info")
        self.info = {k: getattr(info, k) for k, _ in info._fields_}
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(max(1, self.info["workspace_bytes"]) + 256, dtype=torch.uint8, device=dev)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        check(L.dichotomy_gen_bind(h, ctypes.c_void_p(base), self.info["workspace_bytes"], _stream(stream)),
              "dichotomy_gen_bind")
        check(L.dichotomy_gen_info(h, ctypes.byref(info)), "dichotomy_gen_info")   # path final after bind
        self.info = {k: getattr(info, k) for k, _ in info._fields_}

    def solve(self, F: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = torch.empty_like(F) if out is None else out
        check(_lib.load().dichotomy_gen_solve(self._h, _dev(F, "F"), _dev(x, "x"), _stream(stream)),
              "dichotomy_gen_solve")
        return x

    def solve_series(self, F: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = torch.empty_like(F) if out is None else out
        pF, ldf = _dev_rows(F, "F")
        px, ldx = _dev_rows(x, "x")
        check(_lib.load().dichotomy_gen_solve_series(self._h, int(F.shape[0]), pF, ldf, px, ldx, _stream(stream)),
              "dichotomy_gen_solve_series")
        return x

    def residual(self, F: torch.Tensor, x: torch.Tensor, stream=None):
        """The a posteriori check: (max |F - A x|, norm-wise backward error)."""
        out = (ctypes.c_double * 2)()
        check(_lib.load().dichotomy_gen_residual(self._h, _dev(F, "F"), _dev(x, "x"), out, _stream(stream)),
              "dichotomy_gen_residual")
        return float(out[0]), float(out[1])

    def status(self, stream=None) -> int:
        s = ctypes.c_int(0)
        check(_lib.load().dichotomy_gen_status(self._h, _stream(stream), ctypes.byref(s)), "dichotomy_gen_status")
        return int(s.value)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib_obj is not None:
            _lib._lib_obj.dichotomy_gen_destroy(self._h)


def solve(t, F: torch.Tensor, **kw) -> torch.Tensor:
    """One-shot x = T^-1 F (plans and binds on every call; keep a Plan for repeated solves)."""
    return Plan(t[0], t[1], t[2], F.numel(), **kw).solve(F)


# ------------------------------------------------------------------ autograd
class DichotomySolve(torch.autograd.Function):
    """x = T(t)^-1 F for one system; t = tensor([t_-1, t_0, t_1]) (float64).

    The backward pass is one adjoint launch: dL/dF = T^-T dL/dx and dL/dt from the fused
    -lambda.x products.  (The coefficients are read on the host to build the plan.)"""

    @staticmethod
    def forward(ctx, F, t, precision=PREC_F64):
        tv = [float(v) for v in t.detach().cpu().tolist()]
        plan = Plan(tv[0], tv[1], tv[2], F.numel(), precision=precision, device=F.device)
        x = plan.solve(F.detach().contiguous())
        ctx.plan = plan
        ctx.t_device = t.device
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        gF, gt = ctx.plan.adjoint(gx.contiguous(), x)
        return gF, gt.to(device=ctx.t_device, dtype=torch.float64), None


class DichotomySolveQuasi(torch.autograd.Function):
    """x = A^-1 F for the quasi-Toeplitz A of eq. 21; t = tensor([t_-1, t_0, t_1]), corners =
    tensor([psi, chi]) (float64).  The backward pass is one adjoint call: dL/dF = A^-T dL/dx,
    dL/dt and dL/d(psi, chi)."""

    @staticmethod
    def forward(ctx, F, t, corners, precision=PREC_F64):
        tv = [float(v) for v in t.detach().cpu().tolist()]
        psi, chi = (float(v) for v in corners.detach().cpu().tolist())
        plan = Plan(tv[0], tv[1], tv[2], F.numel(), precision=precision, device=F.device, psi=psi, chi=chi)
        x = plan.solve(F.detach().contiguous())
        ctx.plan = plan
        ctx.devices = (t.device, corners.device)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        # a corner plan (zero corners included): the library returns all five gradients
        gF, g = ctx.plan.adjoint(gx.contiguous(), x)
        return gF, g[:3].to(ctx.devices[0]), g[3:5].to(ctx.devices[1]), None


class DichotomySolveBatched(torch.autograd.Function):
    """Batched x_s = T(t_s)^-1 F_s; F: [sum N] (systems back to back), t: [nsys, 3]."""

    @staticmethod
    def forward(ctx, F, t, N, precision=PREC_F64):
        tv = t.detach().cpu().double().numpy()
        batch = Batch(N, tv[:, 0], tv[:, 1], tv[:, 2], precision=precision, device=F.device)
        x = batch.solve(F.detach().contiguous())
        ctx.batch = batch
        ctx.t_device = t.device
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        gF, gt = ctx.batch.adjoint(gx.contiguous(), x)
        return gF, gt.to(ctx.t_device), None, None


class DichotomySolveBatchedQuasi(torch.autograd.Function):
    """Batched quasi-Toeplitz solves (eq. 21): F [sum N], t [nsys, 3], corners [nsys, 2] = (psi, chi)."""

    @staticmethod
    def forward(ctx, F, t, corners, N, precision=PREC_F64):
        tv = t.detach().cpu().double().numpy()
        cv = corners.detach().cpu().double().numpy()
        batch = Batch(N, tv[:, 0], tv[:, 1], tv[:, 2], precision=precision, device=F.device, psi=cv[:, 0],
                      chi=cv[:, 1])
        x = batch.solve(F.detach().contiguous())
        ctx.batch = batch
        ctx.devices = (t.device, corners.device)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        gF, g = ctx.batch.adjoint(gx.contiguous(), x)
        return gF, g[:, :3].to(ctx.devices[0]), g[:, 3:].to(ctx.devices[1]), None, None
