"""dpg_integrate_noalloc: the allocation-free entry point, called through the C ABI.

Some callers cannot allocate device memory while they integrate (a solver whose device
memory budget is fixed at start, code running under another framework's allocator, a
call issued where an allocation would stall the stream).  For them the library offers a
variant of the general path whose metric-field scratch is a fixed file-scope device
array.  This test calls it twice in a row, on different spaces, orders and element
counts, and checks each result against the regular entry point's within the FP64 parity
tolerance; it also checks the host-side rejections.  It initialises its own tables, so
it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return max(np.linalg.norm(a[e] - b[e]) / np.linalg.norm(b[e]) for e in range(b.shape[0]))


def _both(dpg, space, q, verts, coeffs):
    sid = dpg.space_id(space)
    shape = (verts.shape[0],) + dpg.matrix_shape(space, q)
    ref = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    got = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
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


def test_noalloc_host_side_rejections(gpu_lib):
    dpg = gpu_lib
    dpg.dpg_tables_init(3, "HCURL")
    sid = dpg.space_id("HCURL")
    per_elem = 12 * 5 ** 3 * 8                        # fields x L^3 x FP64 at q = 3, L = 5
    too_many = (32 << 20) // per_elem + 1
    # rejected before any launch or pointer use: fake pointers are never dereferenced
    assert dpg.dpg_integrate_noalloc(sid, 0, 3, too_many, 16, 0, 16, 0) == 8       # DPG_ERR_SCRATCH
    assert dpg.dpg_integrate_noalloc(sid | dpg.DPG_MAP_AFFINE, 0, 3, 1, 16, 0, 16, 0) == 1
    assert dpg.dpg_integrate_noalloc(sid, 0, 12, 1, 16, 0, 16, 0) == 2             # no tables
    assert dpg.dpg_strerror(8).startswith("request larger")
