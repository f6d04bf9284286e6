"""CPU FP64 oracle for the element matrices of arXiv 1711.00984 -- TEST INFRASTRUCTURE ONLY.

The conventional quadrature of the paper (Algorithms 1, 4, 6, 8) in plain C, wrapped
with ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does.

Functions and the passages they follow:

* ``gauss(L)``           -- Gauss-Legendre rule on (0,1), Eq. 2.23 (Newton on Eq. 2.93).
* ``one_d(n, x)``        -- P_i, P_i', L_i, L_i' (Eqs. 2.91-2.101).
* ``geometry(v, xi)``    -- trilinear map, Jacobian (Eq. 2.2) and its determinant.
* ``shape(space, ...)``  -- 3D shape functions (Eqs. 2.17, 2.33, 2.51-2.53, 2.69-2.71) and
                            their master-element grad / curl / div (Eqs. 2.30, 2.67, 2.48).
* ``gram(space, ...)``   -- Gram matrices (Eqs. 2.13, 2.16, 2.31, 2.49, 2.68).
* ``mixed_b(...)``       -- mixed stiffness B (pattern of Eqs. 3.15-3.16).
* ``acoustic_cross(...)`` -- cross terms of the acoustics adjoint graph norm, Eq. 3.18
                            (the coefficient of i*omega).
* ``acoustic_b(...)``    -- ultraweak acoustics stiffness, Eqs. 3.14-3.16, as (part without
                            i*omega, coefficient of i*omega).
* ``load(space, ...)``   -- load vector l_I = (f, v_I)_K (the right-hand side of Eq. 3.7).
* ``condense(G, B, l)``  -- static condensation of the test variables, Eq. 3.8 from Eq. 3.7:
                            B^T G^-1 B and B^T G^-1 l through a Cholesky factorization of G
                            (numpy / scipy routines as the steps).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

SPACES = {"H1": 1, "HCURL": 2, "HDIV": 3, "L2": 4, "B": 5}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain IEEE double: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_gauss.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_gauss.restype = ctypes.c_int
            lib.oracle_1d.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, dp]
            lib.oracle_1d.restype = None
            lib.oracle_geometry.argtypes = [dp, dp, dp, dp]
            lib.oracle_geometry.restype = ctypes.c_double
            lib.oracle_shape.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.oracle_shape.restype = ctypes.c_int
            lib.oracle_dim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_dim.restype = ctypes.c_int64
            lib.oracle_gram.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                        dp, dp, dp, ctypes.c_int]
            lib.oracle_gram.restype = ctypes.c_int64
            lib.oracle_load.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                        dp, dp, dp, ctypes.c_int]
            lib.oracle_load.restype = ctypes.c_int64
            lib.oracle_mixed_b.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                           dp, dp, ctypes.c_int, ctypes.c_int]
            lib.oracle_mixed_b.restype = ctypes.c_int64
            lib.oracle_acoustic_cross.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int]
            lib.oracle_acoustic_cross.restype = ctypes.c_int64
            lib.oracle_acoustic_b.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                              dp, dp, ctypes.c_int]
            lib.oracle_acoustic_b.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _sid(space) -> int:
    return SPACES[space] if isinstance(space, str) else int(space)


def gauss(L: int):
    """L-point Gauss-Legendre nodes and weights on (0,1), nodes increasing."""
    x = np.zeros(L); w = np.zeros(L)
    if _load().oracle_gauss(L, _ptr(x), _ptr(w)) != 0:
        raise ValueError(f"bad L={L}")
    return x, w


def one_d(n: int, x: float):
    """(P, P', L, L') at x, each of length n (indices 0..n-1)."""
    P = np.zeros(n); dP = np.zeros(n); Lv = np.zeros(n); dL = np.zeros(n)
    _load().oracle_1d(n, float(x), _ptr(P), _ptr(dP), _ptr(Lv), _ptr(dL))
    return P, dP, Lv, dL


def geometry(verts8: np.ndarray, xi) -> tuple[np.ndarray, np.ndarray, float]:
    """(x(xi), J(xi) as 3x3 with J[i, d] = dx_i/dxi_d, det J) of one element."""
    v = np.ascontiguousarray(verts8, dtype=np.float64).reshape(8, 3)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    x = np.zeros(3); J = np.zeros(9)
    det = _load().oracle_geometry(_ptr(v), _ptr(xi), _ptr(x), _ptr(J))
    return x, J.reshape(3, 3), det


def dim(space, q: int, p: int = 0) -> int:
    """Number of test functions of a space at order q (rows of B for space 'B')."""
    return int(_load().oracle_dim(_sid(space), q, p))


def shape(space, q: int, xi, p: int = 0):
    """Master-element shape values ``val[n, 3]`` and operator ``op[n, 3]`` at xi.

    ``op`` holds grad (H1), curl (HCURL), div in column 0 (HDIV), nothing (L2).  For
    space 'B' the vector-L2 trial space of order p is evaluated.
    """
    sid = _sid(space)
    n = dim(sid, q, p) if sid != 5 else 3 * p ** 3
    val = np.zeros((n, 3)); op = np.zeros((n, 3))
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    if _load().oracle_shape(sid, q, p, _ptr(xi), _ptr(val), _ptr(op)) != 0:
        raise ValueError("shape failed")
    return val, op


def gram(space, q: int, L: int, verts: np.ndarray, coeffs: np.ndarray | None = None,
         nthreads: int = 0) -> tuple[np.ndarray, int]:
    """Gram matrices ``[n_elem, n, n]`` by conventional FP64 quadrature.

    Returns (G, first_bad) where first_bad is -1 or the first element with det J <= 0
    (its matrix is NaN).
    """
    sid = _sid(space)
    v = np.ascontiguousarray(verts, dtype=np.float64)
    ne = v.shape[0]
    c = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    n = dim(sid, q)
    out = np.empty((ne, n, n))
    r = _load().oracle_gram(sid, q, L, ne, _ptr(v), _ptr(c), _ptr(out), nthreads)
    if r < 0:
        raise ValueError("oracle_gram: bad arguments")
    return out, int(r) - 1


def load(space, q: int, L: int, verts: np.ndarray, coef, nthreads: int = 0) -> tuple[np.ndarray, int]:
    """Load vectors ``[n_elem, n]``, l_I = (f, v_I)_K by conventional FP64 quadrature.

    ``coef``: 10 (H1, L2) or 30 (H(curl), H(div)) coefficients of the source, component c
    being sum_k coef[10 c + k] m_k(x) with m = (1, x1, x2, x3, x1^2, x2^2, x3^2, x1 x2,
    x1 x3, x2 x3).  Returns (l, first_bad) like ``gram``.
    """
    sid = _sid(space)
    v = np.ascontiguousarray(verts, dtype=np.float64)
    c = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    if c.size != (10 if sid in (1, 4) else 30):
        raise ValueError("coef: 10 values for H1 / L2, 30 for H(curl) / H(div)")
    ne = v.shape[0]
    out = np.empty((ne, dim(sid, q)))
    r = _load().oracle_load(sid, q, L, ne, _ptr(v), _ptr(c), _ptr(out), nthreads)
    if r < 0:
        raise ValueError("oracle_load: bad arguments")
    return out, int(r) - 1


def mixed_b(q: int, p: int, L: int, verts: np.ndarray, split: bool = False,
            nthreads: int = 0) -> tuple[np.ndarray, int]:
    """Mixed stiffness ``[n_elem, (2,) n_test, 3p^3]`` (vector-L2 trial p, H(curl) test q)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    ne = v.shape[0]
    nt = dim("HCURL", q)
    nu = 3 * p ** 3
    shp = (ne, 2, nt, nu) if split else (ne, nt, nu)
    out = np.empty(shp)
    r = _load().oracle_mixed_b(q, p, L, ne, _ptr(v), _ptr(out), 1 if split else 0, nthreads)
    if r < 0:
        raise ValueError("oracle_mixed_b: bad arguments")
    return out, int(r) - 1


def acoustic_cross(q: int, L: int, verts: np.ndarray, nthreads: int = 0) -> tuple[np.ndarray, int]:
    """Cross block ``[n_elem, dim H(div), dim H1]`` of the acoustics adjoint graph norm
    (Eq. 3.18, coefficient of i*omega): -(div v_I, q_J) + (v_I, grad q_J)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    ne = v.shape[0]
    out = np.empty((ne, dim("HDIV", q), dim("H1", q)))
    r = _load().oracle_acoustic_cross(q, L, ne, _ptr(v), _ptr(out), nthreads)
    if r < 0:
        raise ValueError("oracle_acoustic_cross: bad arguments")
    return out, int(r) - 1


def acoustic_b(q: int, p: int, L: int, verts: np.ndarray, nthreads: int = 0) -> tuple[np.ndarray, int]:
    """Ultraweak acoustics stiffness ``[n_elem, 2, dim H1 + dim H(div), 4 p^3]`` (Eq. 3.16):
    part 0 = -(p, div v) - (u, grad q), part 1 = coefficient of i*omega: (p, q) + (u, v).
    Rows: H1 test functions then H(div) ones; columns: scalar L2 trial then (L2)^3."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    ne = v.shape[0]
    rows = dim("H1", q) + dim("HDIV", q)
    out = np.empty((ne, 2, rows, 4 * p ** 3))
    r = _load().oracle_acoustic_b(q, p, L, ne, _ptr(v), _ptr(out), nthreads)
    if r < 0:
        raise ValueError("oracle_acoustic_b: bad arguments")
    return out, int(r) - 1


def condense(G: np.ndarray, B: np.ndarray, l: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray | None, int]:
    """Static condensation of Eq. 3.8 per element: K = B^T G^-1 B and F = B^T G^-1 l.

    ``G[n_elem, n, n]`` symmetric positive definite, ``B[n_elem, n, m]``, ``l[n_elem, n]`` or
    None.  Steps as the paper names them: Cholesky factorization G = L L^T, the substitutions
    W = L^-1 B and y = L^-1 l, then the products K = W^T W and F = W^T y (so K = B^T L^-T
    L^-1 B = B^T G^-1 B).  An element whose G is not positive definite (the factorization
    fails) gets NaN in K and F.  Returns (K, F or None, first such element or -1).
    """
    from scipy.linalg import solve_triangular
    G = np.asarray(G, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ne, n, m = B.shape
    K = np.empty((ne, m, m))
    F = None if l is None else np.empty((ne, m))
    bad = -1
    for e in range(ne):
        try:
            Lf = np.linalg.cholesky(G[e])
        except np.linalg.LinAlgError:
            K[e] = np.nan
            if F is not None:
                F[e] = np.nan
            bad = e if bad < 0 else bad
            continue
        W = solve_triangular(Lf, B[e], lower=True)
        K[e] = W.T @ W
        if F is not None:
            F[e] = W.T @ solve_triangular(Lf, np.asarray(l[e], dtype=np.float64), lower=True)
    return K, F, bad
