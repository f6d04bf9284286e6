"""Ultraweak acoustics (Sec. 3.3) through the C ABI against the CPU oracle.

DPG_ACOUSTIC_CROSS: the cross block of the adjoint graph norm (Eq. 3.18, coefficient of
i*omega); DPG_ACOUSTIC_B: the stiffness of Eq. 3.16 as (part without i*omega, coefficient
of i*omega).  Both maps, both forms; per element and part the relative Frobenius error is
<= 1e-12 (FP64) / 1e-5 (FP32); the blocks that a part does not contain are exact zeros.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def _rel(got, ref):
    return max(np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]) for e in range(ref.shape[0]))


def _run(dpg, space, q, p, verts, L, fp32=False, affine=False):
    dpg.dpg_tables_init_L(q, L, space)
    v = torch.from_numpy(np.ascontiguousarray(verts)).cuda()
    out = dpg.integrate(space, q, v, p=p, fp32=fp32, affine=affine)
    code, bad = dpg.sync_status()
    assert code == 0, (code, bad)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("affine", [False, True])
def test_cross_block(gpu_lib, q, fp32, affine):
    v = (meshgen.affine_parallelepipeds(2, seed=60 + q) if affine else meshgen.jittered_grid(2, seed=60 + q, jitter=0.2))[:7]
    got = _run(gpu_lib, "ACOUSTIC_CROSS", q, 0, v, q + 2, fp32, affine)
    ref, _ = oracle.acoustic_cross(q, q + 2, v)
    assert _rel(got, ref) <= (TOL32 if fp32 else TOL64)


@pytest.mark.parametrize("q,p", [(1, 1), (2, 1), (3, 2), (4, 2), (4, 4)])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("affine", [False, True])
def test_stiffness(gpu_lib, q, p, fp32, affine):
    v = (meshgen.affine_parallelepipeds(2, seed=70 + q) if affine else meshgen.jittered_grid(2, seed=70 + q, jitter=0.2))[:5]
    got = _run(gpu_lib, "ACOUSTIC_B", q, p, v, q + 2, fp32, affine)
    ref, _ = oracle.acoustic_b(q, p, q + 2, v)
    tol = TOL32 if fp32 else TOL64
    for part in range(2):
        assert _rel(got[:, part], ref[:, part]) <= tol
    nh, npp = oracle.dim("H1", q), p ** 3
    # blocks absent from a part: (H1, L2) and (H(div), (L2)^3) in part 0, the others in part 1
    assert np.all(got[:, 0, :nh, :npp] == 0) and np.all(got[:, 0, nh:, npp:] == 0)
    assert np.all(got[:, 1, :nh, npp:] == 0) and np.all(got[:, 1, nh:, :npp] == 0)


def test_acoustics_q6_p4_sampled(gpu_lib):
    """The benchmark's acoustics workload (16^3 jittered mesh, q = 6, p = 4, L = 8): full
    4096-element launches, sampled elements against the oracle, every value finite."""
    w = meshgen.workload("hcurl_q6_p4_16x16x16")
    idx = np.array([0, 1234, 4095])
    for fp32, tol in [(False, TOL64), (True, TOL32)]:
        gx = _run(gpu_lib, "ACOUSTIC_CROSS", 6, 0, w["verts"], 8, fp32)
        gb = _run(gpu_lib, "ACOUSTIC_B", 6, 4, w["verts"], 8, fp32)
        assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gb))
        rx, _ = oracle.acoustic_cross(6, 8, w["verts"][idx])
        rb, _ = oracle.acoustic_b(6, 4, 8, w["verts"][idx])
        assert _rel(gx[idx], rx) <= tol
        for part in range(2):
            assert _rel(gb[idx, part], rb[:, part]) <= tol


def test_degenerate_element_reported(gpu_lib):
    """An inverted element is reported by index; the blocks of its matrix that depend on
    the geometry are NaN, the blocks a part does not contain stay exact zeros."""
    v = meshgen.jittered_grid(2, seed=1)
    v[3] = v[3][[1, 0, 3, 2, 5, 4, 7, 6]]                                # inverted orientation
    gpu_lib.dpg_tables_init_L(2, 4, "ACOUSTIC_B")
    out = gpu_lib.integrate("ACOUSTIC_B", 2, torch.from_numpy(v).cuda(), p=2)
    code, bad = gpu_lib.sync_status()
    assert code == 5 and bad == 3
    o = out.cpu().numpy()
    nh, npp = oracle.dim("H1", 2), 8
    assert np.all(np.isnan(o[3, 0, :nh, npp:])) and np.all(np.isnan(o[3, 0, nh:, :npp]))
    assert np.all(np.isnan(o[3, 1, :nh, :npp])) and np.all(np.isnan(o[3, 1, nh:, npp:]))
    assert np.all(o[3, 0, :nh, :npp] == 0) and np.all(o[3, 1, nh:, :npp] == 0)
    assert np.all(np.isfinite(np.delete(o, 3, axis=0)))
