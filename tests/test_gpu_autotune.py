"""Autotuner: the chosen chunk width is valid, results after tuning still match the oracle,
and a cached choice is reinstalled from the DPG_AUTOTUNE_CACHE file without timing."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("space", ["H1", "HCURL"])
@pytest.mark.parametrize("fp32", [False, True])
def test_autotune_keeps_parity(gpu_lib, space, fp32, tmp_path, monkeypatch):
    dpg = gpu_lib
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("DPG_AUTOTUNE_CACHE", str(cache))
    q = 3
    dpg.dpg_tables_init(q, space)
    nj = dpg.dpg_autotune(q, space, fp32)
    assert (0 if fp32 else 1) <= nj <= 8          # FP32: 0 = the stage-C tensor-core kernel
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert lines and lines[-1]["nj"] == nj and lines[-1]["q"] == q and lines[-1]["fp32"] == int(fp32)
    # reinstalled from the cache
    assert dpg.dpg_autotune(q, space, fp32) == nj
    v = meshgen.jittered_grid(2, seed=60, jitter=0.2)
    got = dpg.integrate(space, q, torch.from_numpy(v).cuda(), fp32=fp32).double().cpu().numpy()
    assert dpg.sync_status() == (0, -1)
    ref, _ = oracle.gram(space, q, q + 2, v)
    err = max(np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]) for e in range(8))
    assert err <= (1e-5 if fp32 else 1e-12)


def test_autotune_errors(gpu_lib):
    dpg = gpu_lib
    with pytest.raises(dpg.DpgError):
        dpg.dpg_autotune(11, "L2")          # not initialised
    with pytest.raises(dpg.DpgError):
        dpg.dpg_autotune(3, "B")            # not a Gram space
