"""hp-mixed batches (dpg_integrate_hp): elements of different orders q in one call.

Every element of the packed output must equal the uniform-order path for its q (which
the parity tests pin to the oracle), and a sample of elements is checked against the
oracle directly.  Also: invalid orders are skipped and reported, graph replay reads the
current contents of the input buffers, and the FP32 form stays within its target error.
"""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
SPACES = ["H1", "HCURL", "HDIV", "L2"]


@pytest.fixture(scope="module")
def hp_case(gpu_lib):
    w = meshgen.workload("hp_q2to8_16x16x16")
    idx = np.random.default_rng(44).choice(w["verts"].shape[0], 37, replace=False)
    verts = np.ascontiguousarray(w["verts"][idx])
    q = np.ascontiguousarray(w["q_elem"][idx]).astype(np.int32)
    for s in SPACES:
        for qq in range(2, 9):
            gpu_lib.dpg_tables_init(qq, s)
    return verts, q


def _unpack(out, offsets, q, space, dpg):
    mats = []
    for e in range(len(q)):
        n = dpg.dpg_matrix_rows(space, int(q[e]))
        o = int(offsets[e])
        mats.append(out[o:o + n * n].reshape(n, n))
    return mats


@pytest.mark.parametrize("space", SPACES)
@pytest.mark.parametrize("fp32", [False, True])
def test_hp_matches_uniform_path(gpu_lib, hp_case, space, fp32):
    dpg = gpu_lib
    verts, q = hp_case
    v = torch.from_numpy(verts).cuda()
    qt = torch.from_numpy(q).cuda()
    rng = np.random.default_rng(3)
    c = torch.from_numpy(np.stack([rng.uniform(0.5, 2, len(q)), rng.uniform(0.5, 2, len(q))], 1)).cuda()
    out, off = dpg.integrate_hp(space, v, qt, c, fp32=fp32)
    assert dpg.sync_status() == (0, -1)
    mats = _unpack(out.double().cpu(), off.cpu(), q, space, dpg)
    for e in range(len(q)):
        ref = dpg.integrate(space, int(q[e]), v[e:e + 1].contiguous(), c[e:e + 1].contiguous())[0].cpu()
        err = float(torch.linalg.norm(mats[e] - ref) / torch.linalg.norm(ref))
        assert err <= (TOL32 if fp32 else TOL64), (e, int(q[e]), err)


@pytest.mark.parametrize("space", SPACES)
def test_hp_sampled_against_oracle(gpu_lib, hp_case, space):
    dpg = gpu_lib
    verts, q = hp_case
    v = torch.from_numpy(verts).cuda()
    out, off = dpg.integrate_hp(space, v, torch.from_numpy(q).cuda())
    assert dpg.sync_status() == (0, -1)
    mats = _unpack(out.cpu(), off.cpu(), q, space, dpg)
    qmax = 8 if space in ("H1", "L2") else 5          # keep the O(p^9) oracle in seconds
    picks = [e for e in range(len(q)) if q[e] <= qmax][:6]
    for e in picks:
        ref, _ = oracle.gram(space, int(q[e]), int(q[e]) + 2, verts[e:e + 1])
        err = np.linalg.norm(mats[e].numpy() - ref[0]) / np.linalg.norm(ref[0])
        assert err <= TOL64, (e, int(q[e]), err)


def test_hp_replay_and_invalid_orders(gpu_lib, hp_case):
    dpg = gpu_lib
    verts, q = hp_case
    v = torch.from_numpy(verts).cuda()
    qt = torch.from_numpy(q).cuda()
    out1, off = dpg.integrate_hp("H1", v, qt)
    first = out1.clone()
    sh = int(torch.cuda.current_stream().cuda_stream)
    sid = dpg.space_id("H1")
    # the same argument set again: the captured graph is replayed and reads the new vertices
    v.mul_(2.0)
    assert dpg.dpg_integrate_hp(sid, len(q), v.data_ptr(), 0, qt.data_ptr(), off.data_ptr(), out1.data_ptr(), sh) == 0
    assert dpg.sync_status() == (0, -1)
    n = dpg.dpg_matrix_rows("H1", int(q[0]))
    ref = dpg.integrate("H1", int(q[0]), v[:1].contiguous())[0].flatten()
    assert torch.allclose(out1[:n * n], ref, rtol=1e-12, atol=0)
    assert not torch.equal(first[:n * n], out1[:n * n])
    # an element of order 13: skipped and reported; the others are still integrated
    qb = qt.clone()
    qb[3] = 13
    out2, off2 = dpg.integrate_hp("L2", v, qb)
    code, bad = dpg.sync_status()
    assert code == 3 and bad == 3
    n0 = dpg.dpg_matrix_rows("L2", int(q[0]))
    ref0 = dpg.integrate("L2", int(q[0]), v[:1].contiguous())[0].flatten()
    assert torch.allclose(out2[:n0 * n0], ref0, rtol=1e-12, atol=0)


def test_hp_empty_and_errors(gpu_lib, hp_case):
    dpg = gpu_lib
    v = torch.empty((0, 8, 3), dtype=torch.float64, device="cuda")
    out, off = dpg.integrate_hp("H1", v, torch.empty(0, dtype=torch.int32, device="cuda"))
    assert out.numel() == 0
    assert dpg.dpg_integrate_hp(5, 1, 16, 0, 16, 16, 16, 0) == 1                     # B: not an hp space
    assert dpg.dpg_integrate_hp(1 | dpg.DPG_MAP_AFFINE, 1, 16, 0, 16, 16, 16, 0) == 1


def test_hp_fp32_runs_the_autotuned_kernel_per_order(gpu_lib, hp_case, tmp_path, monkeypatch):
    """FP32 hp batch where the autotuner's cached choice puts some orders on the tcgen05
    kernel with stages B and C on the tensor cores (stage-A chunk nj > 0) and the others on
    the stage-C kernel (nj = 0): the graph launches each order's own kernel over the elements
    of that order, and every matrix matches the uniform path."""
    dpg = gpu_lib
    verts, q = hp_case
    v = torch.from_numpy(verts).cuda()
    qt = torch.from_numpy(q).cuda()
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("DPG_AUTOTUNE_CACHE", str(cache))
    forced = {("HDIV", 3): 4, ("HCURL", 4): 3, ("HCURL", 2): 2}

    def install(choice):
        cache.write_text("".join(
            json.dumps({"space": dpg.space_id(s) & 0xff, "q": qq, "L": qq + 2, "fp32": 1, "nj": nj, "ms": 0.0}) + "\n"
            for (s, qq), nj in choice.items()))
        for (s, qq), nj in choice.items():
            assert dpg.dpg_autotune(qq, s, True) == nj
    install(forced)
    try:
        for space in ("HDIV", "HCURL"):
            out, off = dpg.integrate_hp(space, v, qt, fp32=True)
            assert dpg.sync_status() == (0, -1)
            mats = _unpack(out.double().cpu(), off.cpu(), q, space, dpg)
            for e in range(len(q)):
                ref = dpg.integrate(space, int(q[e]), v[e:e + 1].contiguous())[0].cpu()
                err = float(torch.linalg.norm(mats[e] - ref) / torch.linalg.norm(ref))
                assert err <= TOL32, (space, e, int(q[e]), err)
    finally:
        install({k: 0 for k in forced})              # back to the stage-C kernel
