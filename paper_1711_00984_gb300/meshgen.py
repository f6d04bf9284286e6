"""Seeded synthetic hexahedral meshes: the inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the integration method.  It only produces element
vertex arrays and per-element coefficients, so that the GPU library and the CPU
oracle are fed the identical bytes.

Element map convention (Sec. 2.2, Eq. 2.2 leaves the map unspecified): a hexahedron is
given by its 8 vertices ``x_v`` stored at index ``v = v1 + 2*v2 + 4*v3`` with
``v_d in {0, 1}`` the master-cube corner ``(v1, v2, v3)``; the map is trilinear.

Workloads (shapes follow the paper's element-level experiments, Sec. 3, scaled to a mesh):

* ``jittered_grid(n, seed)``: an ``n x n x nz`` grid of the unit cube, every interior
  vertex moved by ``U[-0.1h, 0.1h]^3``; elements are trilinear, ``|J| > 0`` everywhere
  (each column of ``J`` is ``h e_d`` plus a perturbation of at most ``0.2h`` per entry).
* ``affine_parallelepipeds(n, seed)``: the same grid origins, each element mapped by
  ``x = x0 + h (I + S) xi`` with ``S`` off-diagonal ``U[-0.2, 0.2]`` (constant Jacobian,
  the case of Sec. 2.8.1 with a full matrix).
* ``extruded_prisms(n, seed)``: a jittered ``n x n`` quadrilateral grid of the unit
  square in (x2, x3) extruded along x1 in ``n`` layers of thickness ``h``: every element
  has x1 = x1_0 + h xi1 and (x2, x3) a bilinear function of (xi2, xi3), the second
  Jacobian form of Eq. 2.89.  Interior 2D vertices move by ``U[-0.1h, 0.1h]^2``.
* per-element coefficient ``k_e ~ U[0.5, 2]`` (the Poisson diffusivity of Eq. 3.9).

Random draws use numpy's PCG64 (``numpy.random.default_rng``) in a fixed order, so every
array is a pure function of its seed.
"""
from __future__ import annotations

import numpy as np

# vertex v = v1 + 2 v2 + 4 v3 -> corner offsets (v1, v2, v3)
CORNERS = np.array([[v & 1, (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=np.int64)


def _grid_points(n: int, nz: int) -> np.ndarray:
    """Vertex coordinates of an n x n x nz grid of [0,1]x[0,1]x[0,nz/n], i fastest."""
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    return np.stack([i * h, j * h, k * h], axis=-1).reshape(-1, 3).astype(np.float64)


def _element_origins(n: int, nz: int) -> np.ndarray:
    """Integer (i, j, k) of every element, element index e = i + n j + n^2 k."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([i, j, k], axis=-1).reshape(-1, 3)


def jittered_grid(n: int, seed: int, jitter: float = 0.1, nz: int | None = None,
                  rng: np.random.Generator | None = None) -> np.ndarray:
    """Trilinear elements of a jittered ``n x n x nz`` unit-cube grid.

    Returns ``verts[n_elem, 8, 3]`` (float64, C-contiguous).  Interior vertices of the
    full ``n^3`` cube are jittered by ``U[-jitter*h, jitter*h]^3`` in vertex order
    (i fastest); with ``nz < n`` only the elements with ``k < nz`` are returned, the
    jitter being that of the full ``n^3`` mesh.
    """
    nzf = n
    rng = np.random.default_rng(seed) if rng is None else rng
    h = 1.0 / n
    pts = _grid_points(n, nzf)
    idx = np.arange(pts.shape[0])
    i = idx % (n + 1)
    j = (idx // (n + 1)) % (n + 1)
    k = idx // ((n + 1) * (n + 1))
    interior = (i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < nzf)
    nint = int(interior.sum())
    pts[interior] += rng.uniform(-jitter * h, jitter * h, size=(nint, 3))
    nz = nzf if nz is None else nz
    org = _element_origins(n, nz)
    vid = ((org[:, None, 0] + CORNERS[None, :, 0])
           + (n + 1) * (org[:, None, 1] + CORNERS[None, :, 1])
           + (n + 1) * (n + 1) * (org[:, None, 2] + CORNERS[None, :, 2]))
    return np.ascontiguousarray(pts[vid])


def affine_parallelepipeds(n: int, seed: int, shear: float = 0.2, nz: int | None = None,
                           rng: np.random.Generator | None = None) -> np.ndarray:
    """Parallelepipeds ``x = x0 + h (I + S) xi`` on the origins of an ``n x n x nz`` grid.

    ``S`` has a zero diagonal and off-diagonal entries ``U[-shear, shear]``, one draw of
    shape ``(n_elem, 3, 3)``.  Returns ``verts[n_elem, 8, 3]``.
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    nz = n if nz is None else nz
    h = 1.0 / n
    org = _element_origins(n, nz).astype(np.float64) * h
    ne = org.shape[0]
    S = rng.uniform(-shear, shear, size=(ne, 3, 3))
    S[:, [0, 1, 2], [0, 1, 2]] = 0.0
    A = h * (np.eye(3)[None] + S)                      # columns = images of e_1, e_2, e_3
    verts = org[:, None, :] + np.einsum("eij,vj->evi", A, CORNERS.astype(np.float64))
    return np.ascontiguousarray(verts)


def extruded_prisms(n: int, seed: int, jitter: float = 0.1, nz: int | None = None,
                    rng: np.random.Generator | None = None) -> np.ndarray:
    """Elements of an ``n x n`` jittered quadrilateral grid in (x2, x3) extruded along x1.

    The 2D grid of [0,1]^2 has its interior vertices moved by ``U[-jitter*h, jitter*h]^2``
    (one draw, vertex order with the x2 index fastest); the extrusion has ``nz`` (default
    ``n``) uniform layers of thickness ``h`` along x1.  Element index
    ``e = i1 + nz (i2 + n i3)`` for layer i1 and quadrilateral (i2, i3).  Returns
    ``verts[n_elem, 8, 3]``.
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    nz = n if nz is None else nz
    h = 1.0 / n
    b, a = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")      # a: x2 index
    q2 = np.stack([a * h, b * h], axis=-1).reshape(-1, 2).astype(np.float64)
    interior = ((a > 0) & (a < n) & (b > 0) & (b < n)).reshape(-1)
    q2[interior] += rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 2))
    i3, i2, i1 = np.meshgrid(np.arange(n), np.arange(n), np.arange(nz), indexing="ij")
    i1, i2, i3 = i1.reshape(-1), i2.reshape(-1), i3.reshape(-1)
    verts = np.empty((i1.shape[0], 8, 3), dtype=np.float64)
    for v in range(8):
        c1, c2, c3 = CORNERS[v]
        verts[:, v, 0] = (i1 + c1) * h
        verts[:, v, 1:] = q2[(i2 + c2) + (n + 1) * (i3 + c3)]
    return np.ascontiguousarray(verts)


def uniform_coefficients(n_elem: int, rng: np.random.Generator, lo: float = 0.5,
                         hi: float = 2.0) -> np.ndarray:
    """Per-element scalar k_e ~ U[lo, hi]."""
    return rng.uniform(lo, hi, size=n_elem)


def coeff_pairs(space: str, k: np.ndarray | None, n_elem: int) -> np.ndarray:
    """Per-element (mass weight, derivative weight) pairs, ``coeffs[n_elem, 2]``.

    With a scalar coefficient ``k_e``: H1, H(curl), H(div) weight the derivative term by
    ``k_e`` (as ``(k grad u, grad v)`` in Eq. 3.10); L2, which has no derivative term,
    weights its mass term.  Without ``k`` every pair is ``(1, 1)``.
    """
    c = np.ones((n_elem, 2), dtype=np.float64)
    if k is not None:
        if space == "L2":
            c[:, 0] = k
        else:
            c[:, 1] = k
    return c


def spd_batch(n_elem: int, n: int, cond: float, seed: int) -> np.ndarray:
    """Symmetric positive definite matrices ``[n_elem, n, n]`` with eigenvalues spaced
    geometrically in [1, cond] and a random orthogonal eigenbasis (QR of a standard normal
    draw per matrix), symmetrised exactly: test inputs of the static condensation."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_elem, n, n))
    lam = np.geomspace(1.0, cond, n)
    for e in range(n_elem):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = (Q * lam) @ Q.T
        out[e] = 0.5 * (A + A.T)
    return out


def reference_cube(h: float = 1.0, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """One axis-aligned cube of side h: ``verts[1, 8, 3]``."""
    o = np.asarray(origin, dtype=np.float64)
    return np.ascontiguousarray((o[None, :] + h * CORNERS.astype(np.float64))[None])


def affine_from_matrix(A: np.ndarray, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """One parallelepiped with Jacobian ``A`` (columns = edge vectors): ``verts[1, 8, 3]``."""
    o = np.asarray(origin, dtype=np.float64)
    return np.ascontiguousarray((o[None, :] + CORNERS.astype(np.float64) @ np.asarray(A, np.float64).T)[None])


# ---------------------------------------------------------------------------------------
# The five workloads.  Each returns a dict of arrays; 'verts' are trilinear elements,
# 'verts_affine' parallelepipeds, 'k' the scalar coefficients (or None), plus orders.
# ---------------------------------------------------------------------------------------

def workload(name: str) -> dict:
    if name == "h1_q3_2x2x2":
        # 8 trilinear elements, single interior vertex jittered, q=3 with 4^3 Gauss points
        v = jittered_grid(2, seed=1)
        return dict(verts=v, k=None, q=3, L=4, spaces=["H1"])
    if name == "seq_q5_8x8x8":
        rng = np.random.default_rng(2)
        v = jittered_grid(8, seed=2, rng=rng)
        k = uniform_coefficients(v.shape[0], rng)
        va = affine_parallelepipeds(8, seed=2, rng=rng)
        return dict(verts=v, verts_affine=va, k=k, q=5, L=7, spaces=["H1", "HCURL", "HDIV", "L2"])
    if name == "hcurl_q6_p4_16x16x16":
        v = jittered_grid(16, seed=3)
        return dict(verts=v, k=None, q=6, p=4, L=8, spaces=["HCURL", "B"])
    if name == "hp_q2to8_16x16x16":
        rng = np.random.default_rng(4)
        v = jittered_grid(16, seed=4, rng=rng)
        q = rng.integers(2, 9, size=v.shape[0]).astype(np.int32)
        return dict(verts=v, k=None, q_elem=q, spaces=["H1", "HCURL", "HDIV", "L2"])
    if name == "q9_8x8x4":
        rng = np.random.default_rng(5)
        v = jittered_grid(8, seed=5, nz=4, rng=rng)
        va = affine_parallelepipeds(8, seed=5, nz=4, rng=rng)
        return dict(verts=v, verts_affine=va, k=None, q=9, L=11, spaces=["H1", "HDIV"])
    if name == "ext_q5_8x8x8":
        # the 8^3 mesh of seq_q5_8x8x8 as an extrusion: 8 layers along x1 of a jittered
        # 8 x 8 quadrilateral grid, k_e ~ U[0.5, 2]
        rng = np.random.default_rng(6)
        v = extruded_prisms(8, seed=6, rng=rng)
        k = uniform_coefficients(v.shape[0], rng)
        return dict(verts=v, k=k, q=5, L=7, spaces=["H1", "HCURL", "HDIV", "L2"])
    raise KeyError(name)


WORKLOADS = ["h1_q3_2x2x2", "seq_q5_8x8x8", "hcurl_q6_p4_16x16x16", "hp_q2to8_16x16x16", "q9_8x8x4",
             "ext_q5_8x8x8"]
