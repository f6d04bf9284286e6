"""Entry-wise parity of the O(p^6) paths, beside the per-element Frobenius measure.

The affine and extruded-map kernels skip the exact zeros of the 1D integral tables F
(Eq. 2.90, Sec. 2.8.2), so a wrong small entry, or one that should be exactly zero,
could hide under the Frobenius norm of the whole matrix.  Here:
  * affine elements with a dyadic Jacobian (every value exact in binary) against the exact
    rational Gram matrix (Sec. 2.8.1 with a full constant J): every entry within
    1e-12 max|G| (FP64), and exactly 0.0 wherever every term's product of exact 1D
    integrals has a zero factor (zeros forced by F, not by the geometry; entries that
    vanish only by cancellation between terms are held to the tolerance, not to 0.0);
  * extruded elements against the oracle: every entry within 1e-12 max|G|, exactly 0.0
    wherever the exact xi_1 integral F1 of every term is zero;
  * the FP32 forms: every entry within 1e-5 max|G| (the structural zeros exact as well).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest
import torch

import exact
import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

J_A = [[Fr(3, 4), Fr(1, 8), Fr(-1, 16)], [Fr(1, 16), Fr(5, 8), Fr(1, 8)], [Fr(-1, 8), Fr(1, 16), Fr(7, 8)]]
J_B = [[Fr(5, 8), Fr(-3, 32), Fr(1, 8)], [Fr(3, 16), Fr(7, 8), Fr(-1, 32)], [Fr(1, 32), Fr(-1, 8), Fr(9, 16)]]
C_A, C_B = (Fr(3, 4), Fr(5, 2)), (Fr(7, 4), Fr(1, 2))


def _parallelepiped(J, x0=(0.25, -0.5, 0.125)):
    """Vertices x0 + J (v1, v2, v3), vertex v = v1 + 2 v2 + 4 v3 (J's columns are the edges)."""
    Jf = np.array([[float(x) for x in row] for row in J])
    v = np.zeros((8, 3))
    for k in range(8):
        xi = np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1], dtype=np.float64)
        v[k] = np.array(x0) + Jf @ xi
    return v


def _to_np(G):
    return np.array([[float(x) for x in row] for row in G])


def _structural_zeros(space, q):
    """Entries where every term's product of exact 1D integrals has a zero factor (whatever
    the metric), and the exact Gram matrix of the element with Jacobian J_A."""
    support = np.array(exact.affine_support(space, q))
    A = exact.affine_gram(space, q, J_A, *C_A)
    B = exact.affine_gram(space, q, J_B, *C_B)
    zero = ~support
    # a structural zero is zero in exact arithmetic for any Jacobian
    assert all(A[i][j] == 0 and B[i][j] == 0 for i, j in zip(*np.nonzero(zero)))
    return zero, _to_np(A)


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("fp32", [False, True])
def test_affine_entrywise_and_structural_zeros(gpu_lib, space, q, fp32):
    zero, ref = _structural_zeros(space, q)
    v = _parallelepiped(J_A)[None].copy()
    c = np.array([[float(C_A[0]), float(C_A[1])]])
    gpu_lib.dpg_tables_init(q, space)
    out = gpu_lib.integrate(space, q, torch.from_numpy(v).cuda(), torch.from_numpy(c).cuda(), fp32=fp32,
                            affine=True)
    assert gpu_lib.sync_status()[0] == 0
    got = out.double().cpu().numpy()[0]
    if space == "L2":
        # the L2 Gram matrix of an affine element is diagonal (Eq. 2.95): every
        # off-diagonal entry is a structural zero
        assert zero[~np.eye(zero.shape[0], dtype=bool)].all()
    # (with a full J every H1 entry has a non-zero term at q = 2: the zero set may be empty)
    tol = 1e-5 if fp32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert (got[zero] == 0.0).all(), "entries forced to zero by the 1D integrals must be exactly 0"


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("fp32", [False, True])
def test_extruded_entrywise_and_structural_zeros(gpu_lib, space, fp32):
    q, L = 3, 5
    vn = meshgen.extruded_prisms(3, seed=94, jitter=0.2)[[4, 21]].copy()
    ref, _ = oracle.gram(space, q, L, vn)
    scale = np.abs(ref).max(axis=(1, 2))
    # the xi_1 factor (an exact integral F1) of every term is zero there
    zero = ~np.array(exact.affine_support(space, q, dirs=(0,)))
    assert np.all(np.abs(ref[:, zero]) <= 1e-13 * scale[:, None])     # the oracle agrees
    if space == "L2":                       # nu_i nu_j integrates to delta_ij / (2i + 1) along xi_1
        assert zero.any()
    gpu_lib.dpg_tables_init(q, space)
    out = gpu_lib.integrate(space, q, torch.from_numpy(vn).cuda(), fp32=fp32, extruded=True)
    assert gpu_lib.sync_status()[0] == 0
    got = out.double().cpu().numpy()
    tol = 1e-5 if fp32 else 1e-12
    for e in range(2):
        assert np.abs(got[e] - ref[e]).max() <= tol * scale[e]
        assert (got[e][zero] == 0.0).all()


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
def test_general_path_entrywise(gpu_lib, space):
    """The general O(p^7) path entry by entry on trilinear elements (FP64)."""
    q, L = 4, 6
    vn = meshgen.jittered_grid(3, seed=95, jitter=0.2)[[0, 13, 26]].copy()
    ref, _ = oracle.gram(space, q, L, vn)
    gpu_lib.dpg_tables_init(q, space)
    got = gpu_lib.integrate(space, q, torch.from_numpy(vn).cuda()).cpu().numpy()
    assert gpu_lib.sync_status()[0] == 0
    for e in range(3):
        assert np.abs(got[e] - ref[e]).max() <= 1e-12 * np.abs(ref[e]).max()
