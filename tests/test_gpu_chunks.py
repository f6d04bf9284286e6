"""The chunk loops of the general and extruded-map paths, forced by the test hook
dpg_test_set_workspace_limit (a workspace of a few elements per chunk), checked element by
element against the oracle on both sides of every chunk boundary.  Tolerances as in
``test_gpu_parity``: FP64 1e-12, FP32 1e-5 relative Frobenius error per element matrix.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def rel_errs(got, ref):
    return np.array([np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]) for e in range(ref.shape[0])])


@pytest.fixture
def small_workspace(gpu_lib):
    yield gpu_lib
    gpu_lib.dpg_test_set_workspace_limit(0)


@pytest.mark.parametrize("space,q,nfields", [("HCURL", 2, 12), ("H1", 3, 7), ("B", 2, 18)])
@pytest.mark.parametrize("fp32", [False, True])
def test_general_path_over_several_chunks(small_workspace, space, q, nfields, fp32):
    dpg = small_workspace
    L = q + 2
    per_elem = nfields * L ** 3 * (4 if fp32 else 8)
    chunk = 5
    dpg.dpg_tables_init(q, space)
    dpg.dpg_test_set_workspace_limit(chunk * per_elem)            # 5 elements per chunk
    ne = 23                                                       # 4 full chunks and a ragged one
    vn = meshgen.jittered_grid(3, seed=90 + q, jitter=0.2)[:ne].copy()
    rng = np.random.default_rng(91)
    c = np.stack([rng.uniform(0.5, 2, ne), rng.uniform(0.5, 2, ne)], axis=1)
    p = 1 if space == "B" else 0
    cc = None if space == "B" else torch.from_numpy(c).cuda()
    out = dpg.integrate(space, q, torch.from_numpy(vn).cuda(), cc, p=p, fp32=fp32)
    code, bad = dpg.sync_status()
    assert code == 0, (code, bad)
    got = out.double().cpu().numpy()
    # both sides of every boundary (4|5, 9|10, 14|15, 19|20), first and last
    idx = np.array([0, 4, 5, 9, 10, 14, 15, 19, 20, 22])
    if space == "B":
        ref, _ = oracle.mixed_b(q, p, L, vn[idx])
    else:
        ref, _ = oracle.gram(space, q, L, vn[idx], c[idx])
    assert rel_errs(got[idx], ref).max() <= (TOL32 if fp32 else TOL64)
    # the same call in one chunk gives the same matrices
    dpg.dpg_test_set_workspace_limit(0)
    one = dpg.integrate(space, q, torch.from_numpy(vn).cuda(), cc, p=p, fp32=fp32).double().cpu().numpy()
    assert dpg.sync_status()[0] == 0
    assert np.array_equal(one, got)


@pytest.mark.parametrize("space,q,nfields", [("HCURL", 3, 12), ("L2", 2, 1)])
@pytest.mark.parametrize("fp32", [False, True])
def test_extruded_path_over_several_chunks(small_workspace, space, q, nfields, fp32):
    dpg = small_workspace
    L = q + 2
    per_elem = nfields * L ** 2 * (4 if fp32 else 8) + 4
    dpg.dpg_tables_init(q, space)
    dpg.dpg_test_set_workspace_limit(4 * per_elem)                # 4 elements per chunk
    vn = meshgen.extruded_prisms(3, seed=92, jitter=0.2)[:18].copy()
    ne = vn.shape[0]
    rng = np.random.default_rng(93)
    c = np.stack([rng.uniform(0.5, 2, ne), rng.uniform(0.5, 2, ne)], axis=1)
    out = dpg.integrate(space, q, torch.from_numpy(vn).cuda(), torch.from_numpy(c).cuda(), fp32=fp32,
                        extruded=True)
    code, bad = dpg.sync_status()
    assert code == 0, (code, bad)
    got = out.double().cpu().numpy()
    idx = np.array([0, 3, 4, 7, 8, 11, 12, 15, 16, 17])
    ref, _ = oracle.gram(space, q, L, vn[idx], c[idx])
    assert rel_errs(got[idx], ref).max() <= (TOL32 if fp32 else TOL64)
