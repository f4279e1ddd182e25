"""FP64 CPU oracle for the explicit 5/9/13-point schemes of arXiv:1904.04048.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(``paper_1904_04048_gb300``) never imports it and shares no code with it.

Contents
--------
* ``wave_oracle.c`` (loaded here through ctypes): the first-step and two-step
  updates of Section 6 written as printed, the standing-wave / plane-wave exact
  solutions and the relative space-time error E(n, n_t) of Section 6.1.2.
* ``derive.py``: the derivation of Sections 4-5 (McKinney node map, the order
  g, the matrix D and its inverse, the exact integrals of the operators A and
  B) in exact rational arithmetic.
* ``plane_wave.py``: the closed-form discrete solution of the schemes for a
  periodic plane wave (a consequence of the two-step recursion).

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself: the printed Tables 1-3, the Section 4-5 derivation,
polynomial exactness, the discrete dispersion relation, energy conservation,
D4 symmetry and a brute-force dense evaluation.  One result is not pinned by
a printed value: the E_P9 column of Table 2 does not reproduce (the 9-point
new scheme is pinned instead by the derivation, polynomial exactness and the
dense evaluation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wave_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

BC_ZERO = 0
BC_PERIODIC = 1
BC_ODD = 2
EXACT_NONE = 0
EXACT_STANDING = 1
EXACT_PLANE = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.oracle_coeffs.argtypes = [i, i, d, dp, dp]
        lib.oracle_first_step.argtypes = [i, i, i, i, i, d, d, dp, dp, dp]
        lib.oracle_two_step.argtypes = [i, i, i, i, i, d, dp, dp, dp]
        lib.oracle_run.argtypes = [i, i, i, i, i, d, d, dp, dp, i64, d, d, i, dp, d, dp, dp, dp]
        lib.oracle_continue.argtypes = [i, i, i, i, i, d, dp, dp, i64]
        lib.oracle_error_sums.argtypes = [dp, i, i, d, d, i, dp, d, d, dp]
        lib.oracle_error_sums.restype = None
        lib.oracle_set_threads.argtypes = [i]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_run_nodes.argtypes = [i, i, i, i, ip, ip, dp, dp, d, dp, dp, i64, dp, dp]
        for name in ("oracle_coeffs", "oracle_first_step", "oracle_two_step", "oracle_run",
                     "oracle_continue", "oracle_set_threads"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _field(a, ny: int, nx: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (ny, nx):
        raise ValueError(f"expected a ({ny}, {nx}) field, got {a.shape}")
    return a


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the oracle; returns the count in use."""
    return _load().oracle_set_threads(int(n))


def coeffs(scheme: int, lam: float, conventional: bool = False):
    """Printed Section 6 coefficients (a10, a11, a20), (b10, b11, b20)."""
    a = np.zeros(3)
    b = np.zeros(3)
    if _load().oracle_coeffs(scheme, int(conventional), float(lam), _ptr(a), _ptr(b)) != 0:
        raise ValueError(f"unknown scheme {scheme}")
    return a, b


def first_step(scheme, u0, v0, lam, tau, bc=BC_ZERO, conventional=False):
    """u^1 from (u^0, v^0): Eq. A1 in the forms comp5.1 / 9.1 / 13.1 (or the
    conventional comp5.1a / 9.1b / 13-point first step)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    ny, nx = u0.shape
    v0 = _field(v0, ny, nx)
    out = np.empty_like(u0)
    if _load().oracle_first_step(scheme, int(conventional), bc, nx, ny, float(lam), float(tau),
                                 _ptr(u0), _ptr(v0), _ptr(out)) != 0:
        raise ValueError("bad arguments")
    return out


def two_step(scheme, uk, ukm1, lam, bc=BC_ZERO, conventional=False):
    """u^{k+1} from (u^k, u^{k-1}): Eq. A2 in the forms comp5.2 / 9.2 / 13.2."""
    uk = np.ascontiguousarray(uk, dtype=np.float64)
    ny, nx = uk.shape
    ukm1 = _field(ukm1, ny, nx)
    out = np.empty_like(uk)
    if _load().oracle_two_step(scheme, int(conventional), bc, nx, ny, float(lam),
                               _ptr(uk), _ptr(ukm1), _ptr(out)) != 0:
        raise ValueError("bad arguments")
    return out


def run(scheme, u0, v0, lam, tau, n_t, bc=BC_ZERO, conventional=False,
        exact=EXACT_NONE, exact_params=(1.0, 1.0, 0.0), c=1.0, h=1.0, x_off=0.0):
    """The algorithm of Section 3: first step then n_t - 1 two-steps.

    Returns (u^{n_t-1}, u^{n_t}, err) where err = (sum (u-u_e)^2, sum u_e^2,
    max |u-u_e|) accumulated over k = 1..n_t when ``exact`` is set (the
    relative error E(n, n_t) of Eq. error is sqrt(err[0] / err[1]))."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    ny, nx = u0.shape
    v0 = _field(v0, ny, nx)
    up = np.empty_like(u0)
    uc = np.empty_like(u0)
    err = np.zeros(3)
    p = np.zeros(3)
    p[:len(exact_params)] = exact_params
    rc = _load().oracle_run(scheme, int(conventional), bc, nx, ny, float(lam), float(tau),
                            _ptr(u0), _ptr(v0), int(n_t), float(h), float(x_off), int(exact),
                            _ptr(p), float(c), _ptr(up), _ptr(uc), _ptr(err))
    if rc != 0:
        raise ValueError("bad arguments")
    return up, uc, err


def continue_run(scheme, u_prev, u_cur, lam, n_more, bc=BC_ZERO, conventional=False):
    """Advance a pair (u^{k-1}, u^k) by n_more two-steps; returns the new pair."""
    a = np.array(u_prev, dtype=np.float64, order="C", copy=True)
    ny, nx = a.shape
    b = np.array(_field(u_cur, ny, nx), copy=True)
    if _load().oracle_continue(scheme, int(conventional), bc, nx, ny, float(lam),
                               _ptr(a), _ptr(b), int(n_more)) != 0:
        raise ValueError("bad arguments")
    return a, b


def run_nodes(nodes, wa, wb, u0, v0, tau, n_t, bc=BC_ZERO):
    """The algorithm of Section 3 in node-weight form (any derived stencil):
    u^1 = sum_q wa_q u^0_{.+q} + tau sum_q wb_q v^0_{.+q}, then
    u^{k+1} = 2 sum_q wa_q u^k_{.+q} - u^{k-1}.  ``nodes`` are (q1, q2)
    offsets, ``wa`` / ``wb`` the weights A phi_q and B phi_q / tau evaluated
    at the Courant number.  Returns (u^{n_t-1}, u^{n_t})."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    ny, nx = u0.shape
    v0 = _field(v0, ny, nx)
    q1 = np.ascontiguousarray([q[0] for q in nodes], dtype=np.intc)
    q2 = np.ascontiguousarray([q[1] for q in nodes], dtype=np.intc)
    wa = np.ascontiguousarray(wa, dtype=np.float64)
    wb = np.ascontiguousarray(wb, dtype=np.float64)
    if not (len(q1) == len(wa) == len(wb)):
        raise ValueError("nodes and weights differ in length")
    up = np.empty_like(u0)
    uc = np.empty_like(u0)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _load().oracle_run_nodes(bc, nx, ny, len(q1), q1.ctypes.data_as(ip), q2.ctypes.data_as(ip),
                                  _ptr(wa), _ptr(wb), float(tau), _ptr(u0), _ptr(v0), int(n_t),
                                  _ptr(up), _ptr(uc))
    if rc != 0:
        raise ValueError("bad arguments")
    return up, uc


def error_sums(u, h, x_off, exact, exact_params, c, t):
    """(sum (u-u_e)^2, sum u_e^2, max |u-u_e|) of one level at time t."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    ny, nx = u.shape
    p = np.zeros(3)
    p[:len(exact_params)] = exact_params
    out = np.zeros(3)
    _load().oracle_error_sums(_ptr(u), nx, ny, float(h), float(x_off), int(exact), _ptr(p),
                              float(c), float(t), _ptr(out))
    return out


def relative_spacetime_error(err) -> float:
    """E(n, n_t) of Eq. error from accumulated sums."""
    return float(np.sqrt(err[0] / err[1]))
