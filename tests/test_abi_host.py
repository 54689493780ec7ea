"""CPU tests of the C ABI boundary: the library loads, exports every symbol that
include/dichotomy.h declares, and its host-only planning logic (the Toeplitz preliminary
step, block partition, path choice, argument validation) behaves.  No GPU calls."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1002_2469_gb300 import _lib as L
    return L, L.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dichotomy.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dichotomy_\w+)\s*\(", text)))


def test_header_declares_the_solver_entry_points():
    syms = declared_symbols()
    for s in ("dichotomy_plan", "dichotomy_solve", "dichotomy_solve_batched", "dichotomy_adjoint"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    L, lib = _lib()
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} not exported"
    assert sorted(L.EXPORTS) == declared_symbols()
    assert lib.dichotomy_version().decode().count(".") == 2


def test_exports_are_c_symbols_in_the_binary():
    L, _ = _lib()
    out = os.popen(f"nm -D --defined-only {L.lib_path()}").read()
    names = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for s in declared_symbols():
        assert s in names


def test_library_targets_sm_103a_only():
    L, _ = _lib()
    out = os.popen(f"cuobjdump --list-elf {L.lib_path()} 2>/dev/null").read()
    if not out:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_\d+a?", out))
    assert archs == {"sm_103a"}


def plan_info(t, N, **kw):
    from paper_1002_2469_gb300 import dichotomy as D
    h = D.dichotomy_plan(t[0], t[1], t[2], N, D.make_opts(**kw) if kw else None)
    try:
        return D.dichotomy_plan_info(h)
    finally:
        D.dichotomy_destroy(h)


def status_of(t, N, **kw):
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()
    h = ctypes.c_void_p()
    opts = L.make_opts(**kw)
    rc = lib.dichotomy_plan_ex(t[0], t[1], t[2], N, ctypes.byref(opts), ctypes.byref(h))
    if rc == 0:
        lib.dichotomy_destroy(h)
    return rc


def test_roots_match_characteristic_polynomial():
    for t in [(-1.2, 2.5, -0.8), (-1.0, 4.0, -1.0), (0.7, 2.5, -1.1), (-1.0, 2.001, -1.0), (0.0, 2.0, -1.0)]:
        info = plan_info(t, 1000)
        tm1, t0, tp1 = t
        roots = np.roots([tp1, t0, tm1]) if tp1 != 0 else np.array([-tm1 / t0])
        small = roots[np.argmin(np.abs(roots))]
        assert abs(info["rs"] - small) < 1e-13 * max(1.0, abs(small))
        if tp1 != 0 and tm1 != 0:
            big = roots[np.argmax(np.abs(roots))]
            assert abs(info["ib"] - 1.0 / big) < 1e-13
        assert abs(info["z"] - info["rs"] * info["ib"]) < 1e-15
        assert abs(info["rs"]) <= 1.0 and abs(info["ib"]) <= 1.0


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7, 64, 65, 129, 1000, 4097, 65537, 1 << 20, (1 << 26) + 1])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_partition_every_block_has_two_rows(N, threads):
    info = plan_info((-1.2, 2.5, -0.8), N, threads=threads)
    n, P, nl = info["n"], info["P"], info["n_last"]
    assert n >= 2 and nl >= 2 and nl <= n
    assert (P - 1) * n + nl == N
    assert info["tiles"] >= 1
    if P <= threads:
        assert info["path"] == 0 and info["tiles"] == 1


def test_halo_path_and_general_path():
    strong = plan_info((-1.2, 2.5, -0.8), 1 << 24)
    assert strong["path"] == 1 and strong["halo_l"] >= 1 and strong["halo_r"] >= 1
    # the halo covers the decay of the coupling: |rs|^(n * halo_l) is below 2^-64
    assert abs(strong["rs"]) ** (strong["n"] * strong["halo_l"]) < 2.0 ** -64
    assert abs(strong["ib"]) ** (strong["n"] * strong["halo_r"]) < 2.0 ** -64
    # MIXED plans truncate at 2^-56 unless the caller sets a threshold
    mixed = plan_info((-1.2, 2.5, -0.8), 1 << 24, precision=1)
    assert mixed["precision"] == 1
    assert abs(mixed["rs"]) ** (mixed["n"] * mixed["halo_l"]) < 2.0 ** -56
    assert abs(mixed["ib"]) ** (mixed["n"] * mixed["halo_r"]) < 2.0 ** -56
    tight = plan_info((-1.2, 2.5, -0.8), 1 << 24, precision=1, trunc_eps=2.0 ** -64)
    assert abs(tight["rs"]) ** (tight["n"] * tight["halo_l"]) < 2.0 ** -64
    assert mixed["halo_l"] + mixed["halo_r"] < tight["halo_l"] + tight["halo_r"]
    forced = plan_info((-1.2, 2.5, -0.8), 1 << 24, flags=1)
    assert forced["path"] == 2 and forced["halo_l"] == 0
    # the 1-D Laplacian has a double root on the unit circle: no decay, general path
    lap = plan_info((-1.0, 2.0, -1.0), 1 << 20)
    assert lap["path"] == 2
    assert lap["kl"] == lap["P"]          # every block keeps end-dependent ratios


def test_spike_truncation_lengths():
    info = plan_info((-1.0, 4.0, -1.0), 1 << 22)
    rs = abs(info["rs"])
    # v_i ~ rs^{i+1}: the first dropped term is below 2^-64
    assert rs ** (info["Lv"]) < 2.0 ** -64 * 4
    assert info["Lv"] < info["n"]


@pytest.mark.parametrize("t,code", [
    ((-1.0, 1.5, -1.0), 2),        # not diagonally dominant (eq. 32-33)
    ((0.0, 0.0, 0.0), 3),          # singular
    ((float("nan"), 2.0, -1.0), 1),
    ((-1.0, float("inf"), -1.0), 1),
])
def test_plan_rejects_bad_coefficients(t, code):
    assert status_of(t, 100) == code


def test_plan_argument_validation():
    assert status_of((-1.0, 4.0, -1.0), -1) == 1
    assert status_of((-1.0, 4.0, -1.0), 100, block_size=1) == 1
    assert status_of((-1.0, 4.0, -1.0), 100, threads=96) == 1
    assert status_of((-1.0, 4.0, -1.0), 100, precision=7) == 1
    assert status_of((-1.0, 4.0, -1.0), 0) == 0
    assert status_of((-1.0, 4.0, -1.0), 1) == 0
    # dominance with equality is accepted (end rows strict)
    assert status_of((-1.2, 2.0, -0.8), 100) == 0


def test_precision_policy_auto():
    strong = plan_info((-1.2, 2.5, -0.8), 1 << 20, precision=2)
    weak = plan_info((-1.0, 2.0 + 1e-6, -1.0), 1 << 20, precision=2)
    assert strong["precision"] == 1 and weak["precision"] == 0


def test_precision_policy_scale_range():
    """MIXED keeps g X at the window scale of F: |g| = 1/|q| within 2^-60..2^60.  Outside it AUTO
    takes FP64 and an explicit MIXED request is refused (DICH_ERR_UNSUPPORTED)."""
    t = np.array([-1.2, 2.5, -0.8])
    for k in (-40, 0, 40):
        assert plan_info(tuple(t * 2.0 ** k), 1 << 16, precision=2)["precision"] == 1
        assert status_of(tuple(t * 2.0 ** k), 1 << 16, precision=1) == 0
    for k in (-80, 80):
        assert plan_info(tuple(t * 2.0 ** k), 1 << 16, precision=2)["precision"] == 0
        assert status_of(tuple(t * 2.0 ** k), 1 << 16, precision=1) == 11
        assert status_of(tuple(t * 2.0 ** k), 1 << 16, precision=0) == 0
    from paper_1002_2469_gb300 import dichotomy as D
    N = np.array([1000, 2000])
    with pytest.raises(D.DichotomyError):
        D.dichotomy_batch_prepare(N, np.array([0, 1000]), np.array([-1.2, -1.2 * 2.0 ** 80]),
                                  np.array([2.5, 2.5 * 2.0 ** 80]), np.array([-0.8, -0.8 * 2.0 ** 80]),
                                  D.make_opts(precision=1))


def test_batch_prepare_host_only():
    from paper_1002_2469_gb300 import dichotomy as D
    N = np.array([0, 1, 2, 100, 5000, 300000])
    tm1 = np.full(N.size, -0.8)
    t0 = np.full(N.size, 2.5)
    tp1 = np.full(N.size, -1.2)
    h = D.dichotomy_batch_prepare(N, np.concatenate([[0], np.cumsum(N)[:-1]]), tm1, t0, tp1)
    try:
        info = D.dichotomy_batch_info(h)
        assert info["nsys"] == N.size
        assert info["windows"] >= 4
        assert D.dichotomy_batch_workspace_bytes(h) > 0
    finally:
        D.dichotomy_batch_destroy(h)


def test_unbound_and_null_arguments_are_rejected_without_a_gpu():
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.dichotomy_plan(-1.0, 4.0, -1.0, 10, ctypes.byref(h)) == 0
    try:
        assert lib.dichotomy_solve(h, None, None, None) == 8          # DICH_ERR_UNBOUND
        assert lib.dichotomy_plan_bind(h, None, 0, None) == 1         # NULL workspace
        assert lib.dichotomy_plan(-1.0, 4.0, -1.0, 10, None) == 1     # NULL out
    finally:
        lib.dichotomy_destroy(h)
    assert lib.dichotomy_strerror(2).decode().startswith("matrix is not")


def test_quasi_plan_validation_and_series_arguments_without_a_gpu():
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()
    o = L.make_opts()

    def quasi(t, psi, chi, N):
        h = ctypes.c_void_p()
        rc = lib.dichotomy_plan_quasi(t[0], t[1], t[2], psi, chi, N, ctypes.byref(o), ctypes.byref(h))
        if rc == 0:
            lib.dichotomy_destroy(h)
        return rc

    t = (-1.0, 2.5, -1.0)
    assert quasi(t, -1.0, -1.0, 1000) == 0          # Neumann-type end rows (1.5, -1): dominant
    assert quasi(t, -2.0, 0.0, 1000) == 2           # |t_0 + psi| < |t_1|: first row not dominant
    assert quasi(t, 0.0, -2.0, 1000) == 2           # last row not dominant
    assert quasi(t, -1.0, -1.5, 1) == 3             # one row: t_0 + psi + chi = 0
    assert quasi(t, float("nan"), 0.0, 10) == 1
    assert quasi(t, 0.0, 0.0, 1000) == 0            # plain Toeplitz
    h = ctypes.c_void_p()
    assert lib.dichotomy_plan_quasi(*t, 0.3, 0.2, 100, ctypes.byref(o), ctypes.byref(h)) == 0
    try:
        assert lib.dichotomy_adjoint(h, None, None, None, None, None) == 8    # unbound
        assert lib.dichotomy_solve_series(h, 2, None, 100, None, 100, None) == 8   # unbound
        assert lib.dichotomy_solve_series(h, -1, None, 100, None, 100, None) == 1  # M < 0
        assert lib.dichotomy_solve_host(h, None, None, None, None, 0, None) == 8    # unbound
        assert lib.dichotomy_solve_host(h, None, None, None, None, -1, None) == 1   # chunks < 0
    finally:
        lib.dichotomy_destroy(h)


def test_general_plan_validation_and_geometry_without_a_gpu():
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()

    def gen(a, b, c, **kw):
        a, b, c = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c))
        h = ctypes.c_void_p()
        o = L.make_opts(**kw)
        rc = lib.dichotomy_gen_plan(b.size, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                                    c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o), ctypes.byref(h))
        info = None
        if rc == 0:
            info = L.dich_plan_info()
            assert lib.dichotomy_gen_info(h, ctypes.byref(info)) == 0
            lib.dichotomy_gen_destroy(h)
        return rc, info

    rng = np.random.default_rng(0)
    N = 1 << 18
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.5, 1.0, N)
    rc, info = gen(a, b, c, flags=4)
    assert rc == 0 and info.path == 1 and info.halo_l >= 1          # strong dominance: halo windows
    rc, info = gen(a, b, c, flags=1 | 4)
    assert rc == 0 and info.path == 2
    rc, dinfo = gen(a, b, c)                                        # device preliminary: path known at bind
    assert rc == 0 and dinfo.path == 2 and dinfo.halo_l == 0 and dinfo.P == info.P
    assert dinfo.workspace_bytes > info.workspace_bytes            # block composites, scan chunks
    assert info.workspace_bytes >= 40 * N + 24 * N                   # factors and spikes, the matrix
    assert info.growth == 1.0                                        # dominant: maps contract
    rc, info = gen(a[:1000], b[:1000], c[:1000])
    assert rc == 0 and (info.P - 1) * info.n + info.n_last == 1000
    bad = b.copy()
    bad[17] = 0.5 * (abs(a[17]) + abs(c[17]))
    assert gen(a, bad, c)[0] == 2                                   # a row without dominance
    rc, info = gen(a, bad, c, flags=16 | 4)                         # ... accepted when waived
    assert rc == 0 and info.growth >= 1.0
    z = b.copy()
    z[0] = 0.0
    assert gen(np.zeros(N), z, np.zeros(N))[0] == 3                 # zero row: singular
    nan = b.copy()
    nan[5] = np.nan
    assert gen(a, nan, c)[0] == 1
    rc, info = gen(a, b, c, precision=1, flags=4)                   # MIXED (float-float rows)
    assert rc == 0 and info.precision == 1
    rc, info = gen(a, b, c, precision=2, flags=4)                   # AUTO: strongly dominant -> MIXED
    assert rc == 0 and info.precision == 1 and info.n == 16 and info.threads == 128
    wb = np.abs(a) + np.abs(c) + 1e-6                               # weakly dominant: AUTO -> FP64
    rc, info = gen(a, wb, c, precision=2, flags=4)
    assert rc == 0 and info.precision == 0
    rc, info = gen(a * 1e30, b * 1e30, c * 1e30, precision=1, flags=4)   # factors beyond 2^40: refused
    assert rc == 11
    assert gen([0.0], [2.0], [0.0])[0] == 0


def test_batch_with_long_coupling_prepares_without_a_gpu():
    """A system whose coupling outlasts half a window (here the 1-D Laplacian) is planned on the
    general path inside the batch instead of being refused."""
    from paper_1002_2469_gb300 import dichotomy as D
    N = np.array([1 << 20, 5000])
    h = D.dichotomy_batch_prepare(N, np.array([0, 1 << 20]), np.array([-1.0, -1.0]), np.array([2.0, 4.0]),
                                  np.array([-1.0, -1.0]), D.make_opts(precision=2))
    try:
        assert D.dichotomy_batch_workspace_bytes(h) > 32 * (1 << 20) // 16   # beta and first/last values
    finally:
        D.dichotomy_batch_destroy(h)


def test_quasi_batch_validation_without_a_gpu():
    from paper_1002_2469_gb300 import dichotomy as D
    N = np.array([1000, 1, 50], dtype=np.int64)
    tm1, t0, tp1 = np.array([-1.0, -1.0, -1.2]), np.array([2.5, 4.0, 2.5]), np.array([-1.0, -1.0, -0.8])
    o = D.make_opts(precision=2)
    h = D.dichotomy_batch_prepare(N, np.array([0, 1000, 1001]), tm1, t0, tp1, o,
                                  psi=np.array([-1.0, 0.5, 0.0]), chi=np.array([-1.0, 0.25, 0.7]))
    try:
        plain = D.dichotomy_batch_prepare(N, np.array([0, 1000, 1001]), tm1, t0, tp1, o)
        assert D.dichotomy_batch_workspace_bytes(h) > D.dichotomy_batch_workspace_bytes(plain)   # corner data
        D.dichotomy_batch_destroy(plain)
    finally:
        D.dichotomy_batch_destroy(h)
    with pytest.raises(D.DichotomyError) as e:      # first row of system 0 loses dominance
        D.dichotomy_batch_prepare(N, np.array([0, 1000, 1001]), tm1, t0, tp1, o, psi=np.array([-2.0, 0, 0]),
                                  chi=np.zeros(3))
    assert e.value.code == 2
    with pytest.raises(D.DichotomyError) as e:      # one row with t_0 + psi + chi = 0
        D.dichotomy_batch_prepare(N, np.array([0, 1000, 1001]), tm1, t0, tp1, o, psi=np.array([0, -3.0, 0]),
                                  chi=np.array([0, -1.0, 0]))
    assert e.value.code == 3
    with pytest.raises(D.DichotomyError) as e:
        D.dichotomy_batch_prepare(N, np.array([0, 1000, 1001]), tm1, t0, tp1, o, psi=np.array([np.nan, 0, 0]),
                                  chi=np.zeros(3))
    assert e.value.code == 1


def test_toeplitz_without_dominance_needs_split_roots():
    """Without dominance a Toeplitz plan is accepted only on request, and only when the roots of
    t_1 r^2 + t_0 r + t_-1 are real and separated by the unit circle."""
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()

    def plan(t, flags):
        h = ctypes.c_void_p()
        o = L.make_opts(flags=flags)
        rc = lib.dichotomy_plan_ex(*t, 1000, ctypes.byref(o), ctypes.byref(h))
        if rc == 0:
            lib.dichotomy_destroy(h)
        return rc

    assert plan((1.0, 1.5, -1.0), 0) == 2            # |1.5| < 2: not dominant
    assert plan((1.0, 1.5, -1.0), 16) == 0           # roots -0.5 and 2: split
    assert plan((1.0, 0.3, -1.0), 16) == 0
    assert plan((1.0, 1.0, 1.0), 16) == 2            # complex roots
    assert plan((-1.0, 1.0, -1.0), 16) == 2          # roots on one side of the unit circle
    assert plan((1.0, 0.0, 1.0), 16) == 2            # roots +-i


def test_kernel_path_flags():
    """The MIXED window kernel's register and shared-memory paths are chosen by flags: each alone
    is accepted, both together are refused."""
    t = (-1.2, 2.5, -0.8)
    assert status_of(t, 100000, precision=1, flags=32) == 0
    assert status_of(t, 100000, precision=1, flags=64) == 0
    assert status_of(t, 100000, precision=1, flags=96) == 1
