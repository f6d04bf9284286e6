"""Vector- and matrix-valued test spaces V^3 (Sec. 2.7, Eqs. 2.85-2.88).

CPU pin (no GPU): the V^3 Gram matrix is evaluated from its definition by brute-force
quadrature -- the functions e_a (x) v_i are built as 3x3 (or 3-vector) fields from the
oracle's pointwise master shape functions and the Piola maps of Eqs. 2.3-2.6, then
(Phi_I, Phi_J) = int Phi_I : Phi_J + D Phi_I : D Phi_J is summed over the tensor Gauss
rule -- and compared with the block structure delta_ab G_V of Eqs. 2.86 / 2.88 built from
the oracle's scalar-space Gram matrix.

GPU parity (``-m gpu``): DPG_VEC3 through the C ABI against kron(I_3, oracle Gram) for
every Gram space, map (general, affine, extruded) and form.
"""
import numpy as np
import pytest

import oracle
from paper_1711_00984_gb300 import meshgen


def _vec3_by_definition(space, q, L, verts8):
    """[3n][3n] Gram matrix of V^3 on one element by quadrature of the matrix fields."""
    z, w = oracle.gauss(L)
    n = oracle.dim(space, q)
    G = np.zeros((3 * n, 3 * n))
    for l in range(L):
        for m in range(L):
            for k in range(L):
                xi = np.array([z[l], z[m], z[k]])
                _, J, det = oracle.geometry(verts8, xi)
                val, op = oracle.shape(space, q, xi)
                Jit = np.linalg.inv(J).T
                if space == "H1":                    # Eq. 2.3: u = u^, grad u = J^-T grad^ u^
                    f = val[:, :1]                   # scalar values as 1-vectors
                    d = op @ Jit.T                   # physical gradients, rows
                elif space == "HCURL":               # Eq. 2.4: E = J^-T psi^, curl E = J curl^ psi^ / |J|
                    f = val @ Jit.T
                    d = op @ J.T / det
                elif space == "HDIV":                # Eq. 2.5: V = J theta^ / |J|, div V = div^ theta^ / |J|
                    f = val @ J.T / det
                    d = op[:, :1] / det
                else:                                # Eq. 2.6: q = q^ / |J|
                    f = val[:, :1] / det
                    d = np.zeros((n, 1))
                # Phi_(a,i) = e_a (x) f_i: a matrix with row a = f_i (3 x dim f); the same
                # for the derivative field
                Phi = np.zeros((3 * n, 3, f.shape[1]))
                DPhi = np.zeros((3 * n, 3, d.shape[1]))
                for a in range(3):
                    Phi[a * n:(a + 1) * n, a, :] = f
                    DPhi[a * n:(a + 1) * n, a, :] = d
                P = Phi.reshape(3 * n, -1)
                D = DPhi.reshape(3 * n, -1)
                G += w[l] * w[m] * w[k] * abs(det) * (P @ P.T + D @ D.T)
    return G


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
def test_vec3_block_structure_from_definition(space):
    q, L = 2, 4
    v = meshgen.jittered_grid(2, seed=81, jitter=0.2)[3]
    Gv = _vec3_by_definition(space, q, L, v)
    Gs, _ = oracle.gram(space, q, L, v[None])
    ref = np.kron(np.eye(3), Gs[0])
    assert np.linalg.norm(Gv - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.gpu
@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("mp", ["general", "affine", "extruded"])
@pytest.mark.parametrize("fp32", [False, True])
def test_vec3_gpu(gpu_lib, space, mp, fp32):
    import torch
    q = 3
    if mp == "affine":
        v = meshgen.affine_parallelepipeds(2, seed=82)[:5]
    elif mp == "extruded":
        v = meshgen.extruded_prisms(2, seed=83, jitter=0.2)[:5]
    else:
        v = meshgen.jittered_grid(2, seed=84, jitter=0.2)[:5]
    rng = np.random.default_rng(85)
    c = np.stack([rng.uniform(0.5, 2, 5), rng.uniform(0.5, 2, 5)], axis=1)
    gpu_lib.dpg_tables_init(q, space)
    out = gpu_lib.integrate(space, q, torch.from_numpy(v).cuda(), torch.from_numpy(c).cuda(), fp32=fp32,
                            affine=mp == "affine", extruded=mp == "extruded", vec3=True)
    code, bad = gpu_lib.sync_status()
    assert code == 0, (code, bad)
    got = out.double().cpu().numpy()
    ref, _ = oracle.gram(space, q, q + 2, v, c)
    n = ref.shape[1]
    assert got.shape == (5, 3 * n, 3 * n)
    tol = 1e-5 if fp32 else 1e-12
    for e in range(5):
        g = got[e]
        for a in range(3):
            for b in range(3):
                blk = g[a * n:(a + 1) * n, b * n:(b + 1) * n]
                if a == b:
                    assert np.array_equal(blk, g[:n, :n])          # exact copies
                else:
                    assert not blk.any()                           # exact zeros
        assert np.linalg.norm(g[:n, :n] - ref[e]) <= tol * np.linalg.norm(ref[e])


@pytest.mark.gpu
def test_vec3_rejected_where_undefined(gpu_lib):
    """DPG_VEC3 is a Gram-space flag: the mixed stiffness rejects it (DPG_ERR_ARG)."""
    import torch
    gpu_lib.dpg_tables_init(2, "B")
    v = torch.from_numpy(meshgen.jittered_grid(1, seed=86)).cuda()
    o = torch.empty((1, 54, 3), dtype=torch.float64, device="cuda")
    sid = gpu_lib.space_id("B", vec3=True)
    assert gpu_lib._L().dpg_integrate(sid, 1, 2, 1, v.data_ptr(), 0, o.data_ptr(), 0) == 1
