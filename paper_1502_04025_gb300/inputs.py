"""Seeded synthetic inputs: SU(3) gauge fields and spinor sources.

This module is shared by the tests, the benchmark and the reference
checker.  It holds no part of the solver's arithmetic (no Dirac operator,
no Schwarz sweep, no Krylov step): only the recipes that produce the
inputs the solver is run on.

Host layouts (the library's public layout):

* site index  n = x + Lx*(y + Ly*(z + Lz*t))   (x fastest)
* links       U[n, mu, a, b], mu = 0..3 for x, y, z, t; U_mu(n) joins n to n+mu
* spinors     psi[n, s, c], spin s = 0..3, colour c = 0..2

Gauge recipe: U = exp(i*eps*H) with H = sum_a h_a lambda_a / 2, h_a ~ N(0,1)
(lambda_a the Gell-Mann matrices), then re-unitarised by Gram-Schmidt and
phase-fixed to det U = 1.  Random numbers come from numpy's Philox
counter-based generator keyed by the seed, drawn in site-major order
(n, mu, a).  The matrix exponential and the re-unitarisation run in the
small C helper su3gen.c (Taylor series with scaling and squaring, OpenMP
over links), built with gcc on first use: a 48^3x96 field has 42 million
links, which numpy's per-matrix eigen-decomposition takes minutes for.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

__all__ = [
    "volume",
    "rng",
    "gell_mann",
    "gauge_field",
    "unit_gauge_field",
    "gaussian_source",
    "z2_source",
    "point_source",
    "point_sources",
    "random_su3",
]


def volume(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on the rows of each 3x3 matrix, then fix det to 1."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = u[..., 2, :]
    r2 = r2 - np.sum(np.conj(r0) * r2, axis=-1, keepdims=True) * r0
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    out = np.stack([r0, r1, r2], axis=-2)
    det = np.linalg.det(out)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return out * phase[..., None, None]


_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "su3gen.c")
_GEN_LIB = os.path.join(_HERE, "libsu3gen.so")
_gen = None


def build_generator(force: bool = False) -> str:
    """Compile su3gen.c into libsu3gen.so (gcc, OpenMP, no contracted FMAs)."""
    if not force and os.path.exists(_GEN_LIB) and os.path.getmtime(_GEN_LIB) >= os.path.getmtime(_GEN_SRC):
        return _GEN_LIB
    tmp = _GEN_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                    _GEN_SRC, "-lm"], check=True)
    os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _generator():
    global _gen
    if _gen is None:
        build_generator()
        lib = ctypes.CDLL(_GEN_LIB)
        lib.su3gen_from_normals.argtypes = [ctypes.c_long, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        lib.su3gen_from_normals.restype = ctypes.c_int
        _gen = lib
    return _gen


def _su3_from_normals(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*sum_a h_a lambda_a/2), re-unitarised, for h of shape (..., 8)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    out = np.empty(h.shape[:-1] + (3, 3), dtype=np.complex128)
    assert _generator().su3gen_from_normals(h.size // 8, h.ctypes.data, float(eps), out.ctypes.data) == 0
    return out


def su3_from_normals_eigh(h: np.ndarray, eps: float) -> np.ndarray:
    """The same matrices through numpy's eigen-decomposition of H (slow; a
    cross-check of the C helper in the tests)."""
    lam = gell_mann()
    H = np.einsum("...a,aij->...ij", h, lam) * 0.5
    w, W = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("...ik,...k,...jk->...ij", W, ph, np.conj(W))
    return _reunitarise(U)


def gauge_field(L, eps: float, seed: int, chunk_sites: int = 1 << 18) -> np.ndarray:
    """Random SU(3) links U = exp(i eps H), shape (V, 4, 3, 3) complex128."""
    V = volume(L)
    g = rng(seed)
    out = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk_sites):
        s1 = min(V, s0 + chunk_sites)
        h = g.standard_normal((s1 - s0, 4, 8))
        out[s0:s1] = _su3_from_normals(h, eps)
    return out


def unit_gauge_field(L) -> np.ndarray:
    V = volume(L)
    out = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    out[:, :, 0, 0] = out[:, :, 1, 1] = out[:, :, 2, 2] = 1.0
    return out


def gaussian_source(L, seed: int, nrhs: int = 1) -> np.ndarray:
    """Complex Gaussian source(s): re, im ~ N(0,1) per component.

    Shape (V, 4, 3) for nrhs == 1, else (nrhs, V, 4, 3)."""
    V = volume(L)
    g = rng(seed)
    a = g.standard_normal((nrhs, V, 4, 3, 2))
    out = a[..., 0] + 1j * a[..., 1]
    return out[0] if nrhs == 1 else out


def z2_source(L, seed: int) -> np.ndarray:
    """Z2 x Z2 complex noise: each component (+-1 +-i)/sqrt(2)."""
    V = volume(L)
    g = rng(seed)
    bits = g.integers(0, 2, size=(V, 4, 3, 2))
    v = (1.0 - 2.0 * bits)
    return (v[..., 0] + 1j * v[..., 1]) / np.sqrt(2.0)


def point_source(L, spin: int, colour: int, site: int = 0) -> np.ndarray:
    V = volume(L)
    out = np.zeros((V, 4, 3), dtype=np.complex128)
    out[site, spin, colour] = 1.0
    return out


def point_sources(L, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, shape (12, V, 4, 3)."""
    return np.stack([point_source(L, s, c, site) for s in range(4) for c in range(3)])


def random_su3(shape, seed: int) -> np.ndarray:
    """Haar-random SU(3) matrices (QR of a complex Gaussian), for gauge transforms."""
    g = rng(seed)
    shape = tuple(shape)
    z = g.standard_normal(shape + (3, 3, 2))
    z = (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q * np.exp(-1j * np.angle(det) / 3.0)[..., None, None]
