"""Failure path of the tcgen05 kernels (FP32 contraction, condensation), exercised without a
GPU fault.

Every mbarrier wait of the tcgen05 kernel is bounded (about 2^31 cycles).  The test hook
dpg_test_stall_tc_once makes one CTA of the next launch issue no stage-B MMA, so the
completion its producers wait for never arrives: the wait runs out, the CTA stops,
releases its tensor memory and records DPG_ERR_TIMEOUT.  The test checks the reported
status and element, that the call ends within a few seconds, and that the context is
still usable: the same call afterwards matches the oracle.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_recovers(gpu_lib):
    dpg = gpu_lib
    q, L = 5, 7
    v = meshgen.jittered_grid(3, seed=91, jitter=0.2)[:16]
    dpg.dpg_tables_init_L(q, L, "HCURL")
    vt = torch.from_numpy(v).cuda()
    dpg.integrate("HCURL", q, vt, fp32=True)                   # warm-up (set-up outside the timing)
    assert dpg.sync_status()[0] == 0
    dpg.dpg_test_stall_tc_once()
    t0 = time.perf_counter()
    dpg.integrate("HCURL", q, vt, fp32=True)
    code, bad = dpg.sync_status()
    elapsed = time.perf_counter() - t0
    assert dpg.STATUS[code] == "DPG_ERR_TIMEOUT", (code, bad)
    assert bad == 0
    assert elapsed < 20.0
    # the context is still usable and the next call is correct
    out = dpg.integrate("HCURL", q, vt, fp32=True)
    code, bad = dpg.sync_status()
    assert code == 0, (code, bad)
    ref, _ = oracle.gram("HCURL", q, L, v[:4])
    got = out[:4].double().cpu().numpy()
    err = max(np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]) for e in range(4))
    assert err <= 1e-5


def test_condensation_bounded_wait_reports_timeout_and_recovers(gpu_lib):
    """The tcgen05 condensation: the hook makes CTA 0 issue no product for its first panel
    product; its workers' bounded wait runs out, the CTA stops and reports DPG_ERR_TIMEOUT for
    its first element, and the next call is correct."""
    dpg = gpu_lib
    G = meshgen.spd_batch(4, 100, 1e3, seed=92)
    rng = np.random.default_rng(93)
    B = rng.standard_normal((4, 100, 12))
    l = rng.standard_normal((4, 100))
    dpg.dpg_condense_set_method("tcgen05")

    def run():
        g, b, lt = (torch.from_numpy(a.copy()).cuda() for a in (G, B, l))
        K, F = dpg.condense(g, b, lt)
        return K, F

    run()
    assert dpg.sync_status()[0] == 0
    dpg.dpg_test_stall_tc_once()
    t0 = time.perf_counter()
    run()
    code, bad = dpg.sync_status()
    elapsed = time.perf_counter() - t0
    assert dpg.STATUS[code] == "DPG_ERR_TIMEOUT", (code, bad)
    assert bad == 0
    assert elapsed < 20.0
    K, F = run()
    assert dpg.sync_status()[0] == 0
    Kr, Fr, _ = oracle.condense(G, B, l)
    for e in range(4):
        tol = 8 * 100 * np.finfo(np.float64).eps * np.linalg.cond(G[e])
        assert np.linalg.norm(K[e].cpu().numpy() - Kr[e]) <= tol * np.linalg.norm(Kr[e])
        assert np.linalg.norm(F[e].cpu().numpy() - Fr[e]) <= tol * np.linalg.norm(Fr[e])
