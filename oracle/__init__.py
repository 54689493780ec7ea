"""CPU oracle for the Toeplitz tridiagonal solve T x = F (arXiv 1002.2469).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1002_2469_gb300`` and never imports it.

The compiled part (``oracle.c``) is built with plain ``gcc`` on first use (or by
``build()``); everything is FP64 unless named otherwise, plus a binary128
arbiter.  Functions:

* ``thomas(t, F)``            sequential Thomas, FP64 (Sec. 2.2, eq. 7).
* ``thomas_q(t, F)``          the same in binary128, rounded to FP64.
* ``thomas_tridiag(a, b, c, F)`` Thomas for a general tridiagonal matrix (Sec. 2), FP64.
* ``thomas_quasi(t, psi, chi, F)`` the quasi-Toeplitz matrix of eq. 21 through ``thomas_tridiag``.
* ``adjoint_quasi(t, psi, chi, w, x)`` its adjoint: A^-T w and the five parameter gradients.
* ``thomas_batched(...)``     one Thomas per system on a thread pool.
* ``adjoint(t, w, x)``        lambda = T^-T w and dL/d(t_-1, t_0, t_1).
* ``dich_eq15(t, F, starts)`` the paper's formulas eq. 9-16 + eq. 7.
* ``dich_levels(t, F, starts)`` interface values via the level process eq. 17-19.
* ``dich_prelim(t, N, starts)`` the preliminary vectors G (eq. 9) and Z (eq. 10-12).

``t`` is always the triple ``(t_-1, t_0, t_1)``: sub-, main and super-diagonal.
``oracle.poisson`` holds the 2-D Poisson oracle (Sec. 3.2, Sec. 4); ``build_variant`` compiles
the C part with one deliberate mistake planted, for the tests that show the pins catch it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lpthread", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.oracle_thomas_f64.argtypes = [I64, D, D, D, P, P]
            lib.oracle_thomas_q.argtypes = [I64, D, D, D, P, P]
            lib.oracle_thomas_tridiag.argtypes = [I64, P, P, P, P, P]
            lib.oracle_thomas_batched.argtypes = [I64, P, P, P, P, P, P, P, ctypes.c_int]
            lib.oracle_adjoint_f64.argtypes = [I64, D, D, D, P, P, P, P]
            lib.oracle_dich_eq15.argtypes = [I64, D, D, D, P, I64, P, P, P, P, P, P]
            lib.oracle_dich_levels.argtypes = [I64, D, D, D, P, I64, P, P, P]
            lib.oracle_dich_prelim.argtypes = [I64, D, D, D, I64, P, P, P, P, P]
            for f in (lib.oracle_thomas_f64, lib.oracle_thomas_q, lib.oracle_thomas_tridiag, lib.oracle_thomas_batched,
                      lib.oracle_adjoint_f64, lib.oracle_dich_eq15, lib.oracle_dich_levels,
                      lib.oracle_dich_prelim):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ArithmeticError(f"oracle {what} failed with status {rc} (zero pivot or bad input)")


def thomas(t, F) -> np.ndarray:
    """x = T^-1 F by the sequential Thomas algorithm in FP64."""
    F = _f64(F)
    x = np.empty_like(F)
    _check(_load().oracle_thomas_f64(F.size, float(t[0]), float(t[1]), float(t[2]), _ptr(F), _ptr(x)),
           "thomas")
    return x


def thomas_tridiag(sub, dia, sup, F) -> np.ndarray:
    """x = A^-1 F for a general tridiagonal A (row i: sub[i], dia[i], sup[i]) by Thomas, FP64."""
    sub, dia, sup, F = _f64(sub), _f64(dia), _f64(sup), _f64(F)
    if not (sub.size == dia.size == sup.size == F.size):
        raise ValueError("sub, dia, sup and F must have one entry per row")
    x = np.empty_like(F)
    _check(_load().oracle_thomas_tridiag(F.size, _ptr(sub), _ptr(dia), _ptr(sup), _ptr(F), _ptr(x)),
           "thomas_tridiag")
    return x


def thomas_quasi(t, psi, chi, F) -> np.ndarray:
    """x = A^-1 F for the quasi-Toeplitz matrix of eq. 21: tridiag{t_-1, t_0, t_1} with the first
    diagonal entry t_0 + psi and the last t_0 + chi (a single row: t_0 + psi + chi)."""
    F = _f64(F)
    n = F.size
    dia = np.full(n, float(t[1]))
    if n:
        dia[0] += psi
        dia[-1] += chi
    return thomas_tridiag(np.full(n, float(t[0])), dia, np.full(n, float(t[2])), F)


def adjoint_quasi(t, psi, chi, w, x):
    """Adjoint of L(x), x = A^-1 F, for the quasi-Toeplitz A of eq. 21, given w = dL/dx and x:
    lambda = A^-T w (A^T is the quasi-Toeplitz matrix of tridiag{t_1, t_0, t_-1} with the same
    corners) and the gradient (dL/dt_-1, dL/dt_0, dL/dt_1, dL/dpsi, dL/dchi) =
    -(sum lambda_i x_{i-1}, sum lambda_i x_i, sum lambda_i x_{i+1}, lambda_0 x_0, lambda_{N-1} x_{N-1})."""
    w, x = _f64(w), _f64(x)
    lam = thomas_quasi((t[2], t[1], t[0]), psi, chi, w)
    g = np.zeros(5)
    if x.size:
        g[0] = -float(np.dot(lam[1:], x[:-1]))
        g[1] = -float(np.dot(lam, x))
        g[2] = -float(np.dot(lam[:-1], x[1:]))
        g[3] = -lam[0] * x[0]
        g[4] = -lam[-1] * x[-1]
    return lam, g


def thomas_q(t, F) -> np.ndarray:
    """x = T^-1 F by the Thomas algorithm carried out in binary128, rounded to FP64."""
    F = _f64(F)
    x = np.empty_like(F)
    _check(_load().oracle_thomas_q(F.size, float(t[0]), float(t[1]), float(t[2]), _ptr(F), _ptr(x)),
           "thomas_q")
    return x


def thomas_batched(tm1, t0, tp1, N, offsets, F, nthreads: int | None = None) -> np.ndarray:
    """Independent systems stored back to back; system s occupies F[off[s]:off[s]+N[s]]."""
    tm1, t0, tp1, F = _f64(tm1), _f64(t0), _f64(tp1), _f64(F)
    N, offsets = _i64(N), _i64(offsets)
    x = np.zeros_like(F)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    _check(_load().oracle_thomas_batched(N.size, _ptr(N), _ptr(offsets), _ptr(tm1), _ptr(t0), _ptr(tp1),
                                         _ptr(F), _ptr(x), int(nthreads)), "thomas_batched")
    return x


def adjoint(t, w, x):
    """For L = <w, x>, x = T^-1 F: returns (lambda = T^-T w, (dL/dt_-1, dL/dt_0, dL/dt_1))."""
    w, x = _f64(w), _f64(x)
    lam = np.empty_like(w)
    gt = np.zeros(3)
    _check(_load().oracle_adjoint_f64(w.size, float(t[0]), float(t[1]), float(t[2]), _ptr(w), _ptr(x),
                                      _ptr(lam), _ptr(gt)), "adjoint")
    return lam, gt


def dich_eq15(t, F, starts):
    """The Dichotomy solve by eq. 9-16 (preliminary vectors, beta, first/last values) and eq. 7.

    Returns dict(x, beta_L, beta_R, x_first, x_last).
    """
    F, starts = _f64(F), _i64(starts)
    P = starts.size
    x = np.zeros_like(F)
    bL, bR, xs, xe = (np.zeros(P) for _ in range(4))
    _check(_load().oracle_dich_eq15(F.size, float(t[0]), float(t[1]), float(t[2]), _ptr(F), P,
                                    _ptr(starts), _ptr(x), _ptr(bL), _ptr(bR), _ptr(xs), _ptr(xe)),
           "dich_eq15")
    return dict(x=x, beta_L=bL, beta_R=bR, x_first=xs, x_last=xe)


def dich_levels(t, F, starts):
    """The Dichotomy solve by the level process (eq. 17-19) and eq. 7. Returns (x, levels)."""
    F, starts = _f64(F), _i64(starts)
    x = np.zeros_like(F)
    lv = ctypes.c_int(0)
    _check(_load().oracle_dich_levels(F.size, float(t[0]), float(t[1]), float(t[2]), _ptr(F), starts.size,
                                      _ptr(starts), _ptr(x), ctypes.byref(lv)), "dich_levels")
    return x, lv.value


def dich_prelim(t, N: int, starts):
    """Preliminary vectors: G^L, G^R (eq. 9) and Z^L, Z^R (eq. 10-12), each P x N."""
    starts = _i64(starts)
    P = starts.size
    GL, GR, ZL, ZR = (np.zeros((P, N)) for _ in range(4))
    _check(_load().oracle_dich_prelim(int(N), float(t[0]), float(t[1]), float(t[2]), P, _ptr(starts),
                                      _ptr(GL), _ptr(GR), _ptr(ZL), _ptr(ZR)), "dich_prelim")
    return GL, GR, ZL, ZR


def even_starts(N: int, n: int) -> np.ndarray:
    """Block starts for blocks of n rows, the last block taking the remainder.

    A remainder of a single row is merged into the block before it, so every block keeps
    at least 2 rows (Sec. 2.1 asks for sub-vectors of size >= 2)."""
    if N < 2 or n < 2:
        raise ValueError("need N >= 2 and n >= 2")
    P = N // n
    r = N - P * n
    if r >= 2 or P == 0:
        P += 1
    return np.arange(P, dtype=np.int64) * n


def matvec(t, x) -> np.ndarray:
    """T x for the Toeplitz tridiagonal T (used to manufacture right-hand sides)."""
    x = _f64(x)
    y = t[1] * x
    y[1:] += t[0] * x[:-1]
    y[:-1] += t[2] * x[1:]
    return y


class _Variant:
    """thomas/adjoint bound to a separately built copy of oracle.c (used by pin-strength tests)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.oracle_thomas_f64.argtypes = [I64, D, D, D, P, P]
        lib.oracle_adjoint_f64.argtypes = [I64, D, D, D, P, P, P, P]
        lib.oracle_thomas_f64.restype = ctypes.c_int
        lib.oracle_adjoint_f64.restype = ctypes.c_int
        self._lib = lib

    def thomas(self, t, F):
        F = _f64(F)
        x = np.empty_like(F)
        _check(self._lib.oracle_thomas_f64(F.size, float(t[0]), float(t[1]), float(t[2]), _ptr(F), _ptr(x)),
               "thomas")
        return x

    def adjoint(self, t, w, x):
        w, x = _f64(w), _f64(x)
        lam = np.empty_like(w)
        gt = np.zeros(3)
        _check(self._lib.oracle_adjoint_f64(w.size, float(t[0]), float(t[1]), float(t[2]), _ptr(w), _ptr(x),
                                            _ptr(lam), _ptr(gt)), "adjoint")
        return lam, gt


def build_variant(mutant: int, out_dir: str) -> _Variant:
    """Compile oracle.c with -DORACLE_MUTANT=<mutant> (0 = the real oracle) into out_dir."""
    os.makedirs(out_dir, exist_ok=True)
    path = os.path.join(out_dir, "liboracle_m%d.so" % mutant)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-DORACLE_MUTANT=%d" % mutant,
                    "-o", path, _SRC, "-lpthread", "-lm"], check=True)
    return _Variant(path)
