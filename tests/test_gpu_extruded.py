"""Extruded-map path (the second Jacobian form of Eq. 2.89, Algorithm 11) through the C ABI.

On an element extruded along x1 the metric fields do not depend on xi1, so the xi1
integrals are the exact 1D integrals F (Eq. 2.90) and the quadrature runs in (xi2, xi3)
only.  A Gauss rule with L >= q + 1 points integrates the xi1 factors exactly, so the
result is the conventional quadrature sum of the oracle (any trilinear map) on the same
rule.  Tolerances as in ``test_gpu_parity``: FP64 <= 1e-12, FP32 <= 1e-5 relative
Frobenius error per element matrix.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def rel_errs(got, ref):
    got = got.reshape(ref.shape)
    return np.array([np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]) for e in range(ref.shape[0])])


def run(dpg, space, q, verts, coeffs=None, *, L=None, p=0, fp32=False, extruded=True, split=False):
    if L is None:
        dpg.dpg_tables_init(q, space)
    else:
        dpg.dpg_tables_init_L(q, L, space)
    v = torch.from_numpy(np.ascontiguousarray(verts)).cuda()
    c = None if coeffs is None else torch.from_numpy(np.ascontiguousarray(coeffs)).cuda()
    out = dpg.integrate(space, q, v, c, p=p, fp32=fp32, extruded=extruded, split=split)
    code, bad = dpg.sync_status()
    return out.cpu().numpy().astype(np.float64), code, bad


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("fp32", [False, True])
def test_extruded_small_orders(gpu_lib, space, q, fp32):
    v = meshgen.extruded_prisms(3, seed=40 + q, jitter=0.2, nz=2)[:11]     # ragged count
    rng = np.random.default_rng(q)
    c = np.stack([rng.uniform(0.5, 2, 11), rng.uniform(0.5, 2, 11)], axis=1)
    got, code, _ = run(gpu_lib, space, q, v, c, fp32=fp32)
    ref, _ = oracle.gram(space, q, q + 2, v, c)
    assert code == 0
    assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


@pytest.mark.parametrize("space", ["B", "ACOUSTIC_CROSS", "ACOUSTIC_B"])
def test_extruded_non_gram(gpu_lib, space):
    """Mixed stiffness and the acoustics blocks: the same Kronecker structure."""
    q, p = 3, 2
    v = meshgen.extruded_prisms(2, seed=47, jitter=0.2)
    if space == "B":
        ref, _ = oracle.mixed_b(q, p, q + 2, v)
    elif space == "ACOUSTIC_CROSS":
        ref, _ = oracle.acoustic_cross(q, q + 2, v)
    else:
        ref, _ = oracle.acoustic_b(q, p, q + 2, v)
    got, code, _ = run(gpu_lib, space, q, v, p=p if space != "ACOUSTIC_CROSS" else 0)
    assert code == 0
    if space == "ACOUSTIC_B":                    # (part without i omega, coefficient of i omega)
        for part in range(2):
            assert rel_errs(got[:, part], ref[:, part]).max() <= TOL64
    else:
        assert rel_errs(got, ref).max() <= TOL64


def test_extruded_equals_general_path(gpu_lib):
    """The extruded path and the general O(p^7) path give the same matrices (FP64)."""
    w = meshgen.workload("ext_q5_8x8x8")
    v = w["verts"][:64]
    for space in ["H1", "HCURL", "HDIV", "L2"]:
        c = meshgen.coeff_pairs(space, w["k"][:64], 64)
        a, code_a, _ = run(gpu_lib, space, 5, v, c, L=7)
        b, code_b, _ = run(gpu_lib, space, 5, v, c, L=7, extruded=False)
        assert code_a == 0 and code_b == 0
        assert rel_errs(a, b).max() <= TOL64


def test_extruded_workload_sampled(gpu_lib):
    """The benchmark workload (512 elements, q = 5, L = 7) in one launch, sampled against
    the oracle element by element (first and last included)."""
    w = meshgen.workload("ext_q5_8x8x8")
    v, ne = w["verts"], w["verts"].shape[0]
    idx = np.unique(np.concatenate([[0, ne - 1], (np.arange(10) * 53 + 7) % ne]))
    for space in ["H1", "HCURL", "HDIV", "L2"]:
        c = meshgen.coeff_pairs(space, w["k"], ne)
        got, code, _ = run(gpu_lib, space, 5, v, c, L=7)
        ref, _ = oracle.gram(space, 5, 7, v[idx], c[idx])
        assert code == 0
        assert rel_errs(got[idx], ref).max() <= TOL64
        assert np.array_equal(got, got.transpose(0, 2, 1))


def test_not_extruded_reported(gpu_lib):
    """A trilinear element that is not an extrusion is reported by index and NaN-filled;
    the other elements of the call are unaffected."""
    v = meshgen.extruded_prisms(2, seed=48).copy()
    v[5, 3, 0] += 0.01                      # moves x1 of one vertex off its layer
    got, code, bad = run(gpu_lib, "H1", 2, v)
    assert gpu_lib.STATUS[code] == "DPG_ERR_NOT_EXTRUDED"
    assert bad == 5
    assert np.isnan(got[5]).all()
    ok = [e for e in range(v.shape[0]) if e != 5]
    ref, _ = oracle.gram("H1", 2, 4, v[ok])
    assert rel_errs(got[ok], ref).max() <= TOL64


def test_extruded_flags(gpu_lib):
    """DPG_MAP_EXTRUDED is not combinable with DPG_MAP_AFFINE; zero elements do nothing."""
    dpg = gpu_lib
    dpg.dpg_tables_init(2, "H1")
    v1 = torch.from_numpy(meshgen.extruded_prisms(1, seed=49)).cuda()
    o1 = torch.empty((1, 27, 27), dtype=torch.float64, device="cuda")
    sid = dpg.space_id("H1", affine=True, extruded=True)
    assert dpg._L().dpg_integrate(sid, 0, 2, 1, v1.data_ptr(), 0, o1.data_ptr(), 0) == 1   # DPG_ERR_ARG
    out = torch.empty((0, 27, 27), dtype=torch.float64, device="cuda")
    v = torch.empty((0, 8, 3), dtype=torch.float64, device="cuda")
    dpg.integrate("H1", 2, v, extruded=True, out=out)
    assert dpg.sync_status()[0] == 0
