"""ctypes wrapper of the plain-C FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  Arrays are numpy
complex128 in the host layouts of ``paper_1502_04025_gb300.inputs``:
links (V, 4, 3, 3), spinors (V, 4, 3), clover (V, 12, 12).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_long_p = ctypes.POINTER(ctypes.c_long)
_c_double_p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11, -O2, no fast-math)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        for name, args in {
            "ora_gamma": [ctypes.c_int, _c_double_p],
            "ora_field_strength": [_c_int_p, _c_double_p, ctypes.c_long, ctypes.c_int, ctypes.c_int, _c_double_p],
            "ora_clover": [_c_int_p, _c_double_p, ctypes.c_double, ctypes.c_double, _c_double_p],
            "ora_invert_clover": [_c_int_p, _c_double_p, _c_double_p],
            "ora_apply_D": [_c_int_p, _c_double_p, _c_double_p, ctypes.c_double, _c_double_p, _c_double_p],
            "ora_apply_H": [_c_int_p, _c_double_p, _c_double_p, _c_double_p],
            "ora_apply_D_sites": [_c_int_p, _c_double_p, ctypes.c_double, ctypes.c_double, _c_double_p,
                                  ctypes.c_long, _c_long_p, _c_double_p],
            "ora_sap": [_c_int_p, _c_int_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                        _c_double_p, _c_double_p, _c_double_p, ctypes.c_int, ctypes.c_int],
            "ora_fgmres": [_c_int_p, _c_int_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_double,
                           _c_double_p, _c_double_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_int_p, _c_int_p, _c_double_p,
                           _c_double_p, ctypes.c_int, _c_int_p],
            "ora_domain_colour": [_c_int_p, _c_int_p, ctypes.c_int],
        }.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ivec(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _dp(a: np.ndarray):
    assert a.dtype == np.complex128 or a.dtype == np.float64
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_c_double_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _vol(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def gamma(mu: int) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    assert lib().ora_gamma(mu, _dp(out)) == 0
    return out


def field_strength(L, U, n: int, mu: int, nu: int) -> np.ndarray:
    U = _c128(U)
    out = np.zeros((3, 3), dtype=np.complex128)
    assert lib().ora_field_strength(_ivec(L), _dp(U), n, mu, nu, _dp(out)) == 0
    return out


def clover(L, U, csw: float, kappa: float) -> np.ndarray:
    U = _c128(U)
    A = np.zeros((_vol(L), 12, 12), dtype=np.complex128)
    assert lib().ora_clover(_ivec(L), _dp(U), csw, kappa, _dp(A)) == 0
    return A


def invert_clover(L, A) -> np.ndarray:
    A = _c128(A)
    out = np.zeros_like(A)
    assert lib().ora_invert_clover(_ivec(L), _dp(A), _dp(out)) == 0
    return out


def apply_D(L, U, A, kappa: float, x) -> np.ndarray:
    U, A, x = _c128(U), _c128(A), _c128(x)
    y = np.zeros_like(x)
    assert lib().ora_apply_D(_ivec(L), _dp(U), _dp(A), kappa, _dp(x), _dp(y)) == 0
    return y


def apply_H(L, U, x) -> np.ndarray:
    U, x = _c128(U), _c128(x)
    y = np.zeros_like(x)
    assert lib().ora_apply_H(_ivec(L), _dp(U), _dp(x), _dp(y)) == 0
    return y


def apply_D_sites(L, U, csw: float, kappa: float, x, sites) -> np.ndarray:
    U, x = _c128(U), _c128(x)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    y = np.zeros((len(sites), 4, 3), dtype=np.complex128)
    rc = lib().ora_apply_D_sites(_ivec(L), _dp(U), csw, kappa, _dp(x), len(sites),
                                 sites.ctypes.data_as(_c_long_p), _dp(y))
    assert rc == 0
    return y


def sap(L, dom, U, A, Ainv, kappa: float, eta, nmr: int, n_half: int):
    """One application of the Schwarz preconditioner; returns (psi, rho)."""
    U, A, Ainv, eta = _c128(U), _c128(A), _c128(Ainv), _c128(eta)
    psi = np.zeros_like(eta)
    rho = np.zeros_like(eta)
    rc = lib().ora_sap(_ivec(L), _ivec(dom), _dp(U), _dp(A), _dp(Ainv), kappa, _dp(eta), _dp(psi), _dp(rho),
                       nmr, n_half)
    assert rc == 0, rc
    return psi, rho


def fgmres(L, dom, U, A, Ainv, kappa: float, b, tol: float, m: int = 16, max_restarts: int = 50,
           use_sap: bool = True, nmr: int = 4, ncy: int = 4, x0=None, max_hist: int = 4096):
    """Flexible GMRES(m); returns (x, info dict)."""
    U, A, Ainv, b = _c128(U), _c128(A), _c128(Ainv), _c128(b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    iters = ctypes.c_int(0)
    restarts = ctypes.c_int(0)
    true_rel = ctypes.c_double(0)
    hist = np.zeros(max_hist, dtype=np.float64)
    nh = ctypes.c_int(0)
    if dom is None:
        dom = (2, 2, 2, 2)
    rc = lib().ora_fgmres(_ivec(L), _ivec(dom), _dp(U), _dp(A), _dp(Ainv), kappa, _dp(b), _dp(x),
                          0 if x0 is None else 1, tol, m, max_restarts, 1 if use_sap else 0, nmr, ncy,
                          ctypes.byref(iters), ctypes.byref(restarts), ctypes.byref(true_rel), _dp(hist),
                          max_hist, ctypes.byref(nh))
    assert rc >= 0, rc
    return x, {"converged": rc == 0, "iters": iters.value, "restarts": restarts.value,
               "true_rel_res": true_rel.value, "history": hist[: nh.value].copy()}


def domain_colour(L, dom, d: int) -> int:
    return lib().ora_domain_colour(_ivec(L), _ivec(dom), d)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB)
