"""dpg_integrate_noalloc: the allocation-free entry point, called through the C ABI.

Some callers cannot allocate device memory while they integrate (a solver whose device
memory budget is fixed at start, code running under another framework's allocator, a
call issued where an allocation would stall the stream).  For them the library offers a
variant of the general path whose metric-field scratch is a fixed file-scope device
array.  These tests call it twice in a row, on different spaces, orders and element
counts, and check each result against the regular entry point's within the parity
tolerance of its form (FP64 1e-12, FP32 1e-5, and the FP32 form against the FP64 oracle
too); they check that a repeated call changes the device's free memory by nothing, and
the host-side rejections.  They initialise their own tables, so they pass alone in a
fresh process as well as after the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def _rel(a, b):
    a = np.asarray(a.double().cpu().numpy() if torch.is_tensor(a) else a, dtype=np.float64)
    b = np.asarray(b.double().cpu().numpy() if torch.is_tensor(b) else b, dtype=np.float64)
    return max(np.linalg.norm(a[e] - b[e]) / np.linalg.norm(b[e]) for e in range(b.shape[0]))


def _both(dpg, space, q, verts, coeffs, fp32=False):
    sid = dpg.space_id(space, fp32=fp32)
    shape = (verts.shape[0],) + dpg.matrix_shape(space, q)
    dt = torch.float32 if fp32 else torch.float64
    ref = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    got = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    sh = int(torch.cuda.current_stream().cuda_stream)
    cp = coeffs.data_ptr() if coeffs is not None else 0
    assert dpg.dpg_integrate(sid, 0, q, verts.shape[0], verts.data_ptr(), cp, ref.data_ptr(), sh) == 0
    assert dpg.dpg_integrate_noalloc(sid, 0, q, verts.shape[0], verts.data_ptr(), cp, got.data_ptr(), sh) == 0
    assert dpg.dpg_sync_status(sh) == (0, -1)
    return got, ref


def test_noalloc_matches_dpg_integrate_on_two_calls(gpu_lib):
    dpg = gpu_lib
    dpg.dpg_tables_init(3, "HCURL")
    dpg.dpg_tables_init(4, "H1")
    # call 1: H(curl), q = 3, 27 jittered elements
    v1 = torch.from_numpy(meshgen.jittered_grid(3, seed=50, jitter=0.2)).cuda()
    got, ref = _both(dpg, "HCURL", 3, v1, None)
    assert torch.isfinite(got).all()
    assert _rel(got, ref) <= TOL64
    # call 2 (the scratch still holds call 1's fields): H1, q = 4, 13 elements, coefficients
    v2 = torch.from_numpy(meshgen.jittered_grid(3, seed=51, jitter=0.2)[:13].copy()).cuda()
    rng = np.random.default_rng(51)
    c2 = torch.from_numpy(np.stack([rng.uniform(0.5, 2, 13), rng.uniform(0.5, 2, 13)], 1)).cuda()
    got, ref = _both(dpg, "H1", 4, v2, c2)
    assert torch.isfinite(got).all()
    assert _rel(got, ref) <= TOL64


def test_noalloc_fp32_form_on_two_calls(gpu_lib):
    """The FP32 form runs the FP32 programs of dpg_integrate (tensor-core kernel where the
    blocks fit it): equal to dpg_integrate's FP32 result and within 1e-5 of the oracle."""
    dpg = gpu_lib
    dpg.dpg_tables_init(5, "HCURL")
    dpg.dpg_tables_init(3, "HDIV")
    vn = meshgen.jittered_grid(3, seed=52, jitter=0.2)[:19].copy()
    v1 = torch.from_numpy(vn).cuda()
    got, ref = _both(dpg, "HCURL", 5, v1, None, fp32=True)
    assert torch.isfinite(got).all()
    assert _rel(got, ref) <= TOL32
    o, _ = oracle.gram("HCURL", 5, 7, vn)
    assert _rel(got, o) <= TOL32
    vn2 = meshgen.jittered_grid(3, seed=53, jitter=0.2)[:7].copy()
    got, ref = _both(dpg, "HDIV", 3, torch.from_numpy(vn2).cuda(), None, fp32=True)
    assert _rel(got, ref) <= TOL32
    o, _ = oracle.gram("HDIV", 3, 5, vn2)
    assert _rel(got, o) <= TOL32


def test_noalloc_reserves_no_device_memory_per_call(gpu_lib):
    """After the first call (which loads the array's module), further calls leave the
    device's free memory exactly as it was: no allocation, no pool growth."""
    dpg = gpu_lib
    dpg.dpg_tables_init(3, "HCURL")
    v = torch.from_numpy(meshgen.jittered_grid(3, seed=54, jitter=0.2)).cuda()
    out = torch.empty((v.shape[0],) + dpg.matrix_shape("HCURL", 3), dtype=torch.float64, device="cuda")
    sh = int(torch.cuda.current_stream().cuda_stream)
    sid = dpg.space_id("HCURL")
    assert dpg.dpg_integrate_noalloc(sid, 0, 3, v.shape[0], v.data_ptr(), 0, out.data_ptr(), sh) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert dpg.dpg_integrate_noalloc(sid, 0, 3, v.shape[0], v.data_ptr(), 0, out.data_ptr(), sh) == 0
    assert dpg.dpg_sync_status(sh) == (0, -1)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_host_side_rejections(gpu_lib):
    dpg = gpu_lib
    dpg.dpg_tables_init(3, "HCURL")
    sid = dpg.space_id("HCURL")
    per_elem = 12 * 5 ** 3 * 8                        # fields x L^3 x FP64 at q = 3, L = 5
    too_many = (32 << 20) // per_elem + 1
    # rejected before any launch or pointer use: fake pointers are never dereferenced
    assert dpg.dpg_integrate_noalloc(sid, 0, 3, too_many, 16, 0, 16, 0) == 8       # DPG_ERR_SCRATCH
    assert dpg.dpg_integrate_noalloc(sid | dpg.DPG_FP32, 0, 3, 2 * too_many, 16, 0, 16, 0) == 8
    assert dpg.dpg_integrate_noalloc(sid | dpg.DPG_MAP_AFFINE, 0, 3, 1, 16, 0, 16, 0) == 1
    assert dpg.dpg_integrate_noalloc(sid, 0, 12, 1, 16, 0, 16, 0) == 2             # no tables
    assert dpg.dpg_strerror(8).startswith("request larger")
