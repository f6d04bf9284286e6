"""Load vector l_I = (f, v_I)_K through the C ABI against the oracle's conventional
quadrature (same Gauss rule, same source).

The GPU evaluates the pulled-back source at the Gauss points and contracts the three
directions one after the other (Eqs. 2.23-2.25 with one test index); the oracle sums
point by point.  Both compute the same discrete sum, so the FP64 form agrees to rounding:
relative max-norm error <= 1e-12 per element vector; the FP32 form (FP32 contractions)
<= 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
NC = {"H1": 1, "L2": 1, "HCURL": 3, "HDIV": 3}


def rel_errs(got, ref):
    return np.array([np.abs(got[e] - ref[e]).max() / np.abs(ref[e]).max() for e in range(ref.shape[0])])


def source(space, seed):
    return np.random.default_rng(seed).uniform(-1, 1, 10 * NC[space])


def run(dpg, space, q, verts, coef, *, L=None, fp32=False):
    if L is None:
        dpg.dpg_tables_init(q, space)
    else:
        dpg.dpg_tables_init_L(q, L, space)
    v = torch.from_numpy(np.ascontiguousarray(verts)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(coef)).cuda()
    out = dpg.integrate_load(space, q, v, c, fp32=fp32)
    code, bad = dpg.sync_status()
    return out.cpu().numpy().astype(np.float64), code, bad


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("fp32", [False, True])
def test_load_trilinear(gpu_lib, space, q, fp32):
    v = meshgen.jittered_grid(3, seed=60 + q, jitter=0.2)[:23]          # ragged count
    c = source(space, q)
    got, code, _ = run(gpu_lib, space, q, v, c, fp32=fp32)
    ref, bad = oracle.load(space, q, q + 2, v, c)
    assert code == 0 and bad == -1
    assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
def test_load_affine_and_extruded_elements(gpu_lib, space):
    """Parallelepipeds and extruded prisms are trilinear maps too: the same entry point."""
    v = np.concatenate([meshgen.affine_parallelepipeds(2, seed=61), meshgen.extruded_prisms(2, seed=62)])
    c = source(space, 5)
    got, code, _ = run(gpu_lib, space, 4, v, c)
    ref, _ = oracle.load(space, 4, 6, v, c)
    assert code == 0
    assert rel_errs(got, ref).max() <= TOL64


@pytest.mark.parametrize("space", ["H1", "HCURL"])
def test_load_per_element_source(gpu_lib, space):
    """Per-element coefficients (coef_stride = 10 nc), a rule with L = q + 1."""
    v = meshgen.jittered_grid(2, seed=63)
    rng = np.random.default_rng(64)
    c = rng.uniform(-1, 1, (v.shape[0], 10 * NC[space]))
    got, code, _ = run(gpu_lib, space, 3, v, c, L=4)
    ref = np.stack([oracle.load(space, 3, 4, v[e:e + 1], c[e])[0][0] for e in range(v.shape[0])])
    assert code == 0
    assert rel_errs(got, ref).max() <= TOL64


@pytest.mark.parametrize("space", ["H1", "HDIV"])
def test_load_high_order(gpu_lib, space):
    """q = 9 with L = 11 (the order of the q = 9 workload), FP64 and FP32."""
    v = meshgen.jittered_grid(2, seed=67)[:3]
    c = source(space, 68)
    ref, _ = oracle.load(space, 9, 11, v, c)
    for fp32 in (False, True):
        got, code, _ = run(gpu_lib, space, 9, v, c, L=11, fp32=fp32)
        assert code == 0
        assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


def test_load_workload_sampled(gpu_lib):
    """The 512-element q = 5 mesh with L = 7 in one launch, sampled against the oracle."""
    w = meshgen.workload("seq_q5_8x8x8")
    v, ne = w["verts"], w["verts"].shape[0]
    idx = np.unique(np.concatenate([[0, ne - 1], (np.arange(10) * 53 + 7) % ne]))
    for space in ["H1", "HCURL", "HDIV", "L2"]:
        c = source(space, 70)
        got, code, _ = run(gpu_lib, space, 5, v, c, L=7)
        ref, _ = oracle.load(space, 5, 7, v[idx], c)
        assert code == 0
        assert rel_errs(got[idx], ref).max() <= TOL64


def test_load_degenerate_and_args(gpu_lib):
    """An inverted element is NaN-filled and reported; bad arguments are refused."""
    dpg = gpu_lib
    v = meshgen.jittered_grid(2, seed=65).copy()
    v[3] = v[3][[1, 0, 3, 2, 5, 4, 7, 6]]                                 # mirrored: |J| < 0
    c = source("H1", 66)
    got, code, bad = run(dpg, "H1", 2, v, c)
    assert dpg.STATUS[code] == "DPG_ERR_DEGENERATE" and bad == 3
    assert np.isnan(got[3]).all() and np.isfinite(np.delete(got, 3, axis=0)).all()
    ref, _ = oracle.load("H1", 2, 4, np.delete(v, 3, axis=0), c)
    assert rel_errs(np.delete(got, 3, axis=0), ref).max() <= TOL64
    vt = torch.from_numpy(v).cuda()
    ct = torch.from_numpy(c).cuda()
    o = torch.empty((8, 27), dtype=torch.float64, device="cuda")
    L = dpg._L()
    sid = dpg.space_id("H1")
    assert L.dpg_integrate_load(dpg.space_id("B"), 2, 8, vt.data_ptr(), ct.data_ptr(), 0, o.data_ptr(), None) == 1
    assert L.dpg_integrate_load(dpg.space_id("H1", affine=True), 2, 8, vt.data_ptr(), ct.data_ptr(), 0, o.data_ptr(), None) == 1
    assert L.dpg_integrate_load(sid, 2, 8, vt.data_ptr(), ct.data_ptr(), 5, o.data_ptr(), None) == 1     # stride < 10
    assert L.dpg_integrate_load(sid, 2, 8, vt.data_ptr(), None, 0, o.data_ptr(), None) == 1
    assert L.dpg_integrate_load(sid, 11, 8, vt.data_ptr(), ct.data_ptr(), 0, o.data_ptr(), None) == 2   # no tables
    assert L.dpg_integrate_load(sid, 2, 0, None, None, 0, None, None) == 0                             # empty
    assert dpg.sync_status()[0] == 0


@pytest.mark.parametrize("space,q", [("L2", 12), ("HDIV", 11)])
def test_load_largest_orders(gpu_lib, space, q):
    """The largest orders whose tables initialise for the space (L = 14 and 13 points)."""
    v = meshgen.jittered_grid(2, seed=71)[:2]
    c = source(space, 72)
    L = min(q + 2, 14)
    got, code, _ = run(gpu_lib, space, q, v, c, L=L)
    ref, _ = oracle.load(space, q, L, v, c)
    assert code == 0
    assert rel_errs(got, ref).max() <= TOL64


def test_load_fp32_per_element_source(gpu_lib):
    v = meshgen.jittered_grid(2, seed=73)
    c = np.random.default_rng(74).uniform(-1, 1, (v.shape[0], 30))
    got, code, _ = run(gpu_lib, "HDIV", 4, v, c, fp32=True)
    ref = np.stack([oracle.load("HDIV", 4, 6, v[e:e + 1], c[e])[0][0] for e in range(v.shape[0])])
    assert code == 0
    assert rel_errs(got, ref).max() <= TOL32
