"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Tolerances: FP64 form <= 1e-12 relative Frobenius error per element matrix; FP32 form
<= 1e-5 (its stated target).  Inputs are the seeded workloads of ``meshgen``.
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


def run(dpg, space, q, verts, coeffs=None, *, L=None, p=0, fp32=False, affine=False, split=False):
    if L is None:
        dpg.dpg_tables_init(q, space)
    else:
        dpg.dpg_tables_init_L(q, L, space)
    v = torch.from_numpy(np.ascontiguousarray(verts)).cuda()
    c = None if coeffs is None else torch.from_numpy(np.ascontiguousarray(coeffs)).cuda()
    out = dpg.integrate(space, q, v, c, p=p, fp32=fp32, affine=affine, split=split)
    code, bad = dpg.sync_status()
    return out.cpu().numpy().astype(np.float64), code, bad


# ---------------------------------------------------------------- config 1: H1 q=3, L=4

def test_h1_q3_2x2x2_full(gpu_lib):
    w = meshgen.workload("h1_q3_2x2x2")
    got, code, _ = run(gpu_lib, "H1", 3, w["verts"], L=4)
    ref, _ = oracle.gram("H1", 3, 4, w["verts"])
    assert code == 0
    assert rel_errs(got, ref).max() <= TOL64
    assert np.array_equal(got, got.transpose(0, 2, 1))


# ---------------------------------------------------------------- small orders, every space

@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("fp32", [False, True])
def test_general_small_orders(gpu_lib, space, q, fp32):
    v = meshgen.jittered_grid(3, seed=20 + q, jitter=0.2)[:11]          # ragged count
    rng = np.random.default_rng(q)
    c = np.stack([rng.uniform(0.5, 2, 11), rng.uniform(0.5, 2, 11)], axis=1)
    got, code, _ = run(gpu_lib, space, q, v, c, fp32=fp32)
    ref, _ = oracle.gram(space, q, q + 2, v, c)
    assert code == 0
    assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("fp32", [False, True])
def test_affine_small_orders(gpu_lib, space, q, fp32):
    v = meshgen.affine_parallelepipeds(3, seed=30 + q)[:13]
    rng = np.random.default_rng(q)
    c = np.stack([rng.uniform(0.5, 2, 13), rng.uniform(0.5, 2, 13)], axis=1)
    got, code, _ = run(gpu_lib, space, q, v, c, fp32=fp32, affine=True)
    ref, _ = oracle.gram(space, q, q + 2, v, c)
    assert code == 0
    assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


@pytest.mark.parametrize("L", [2, 3, 6])
def test_other_quadrature_sizes(gpu_lib, L):
    """Under-integrated (L < q+1) and over-integrated rules: the GPU reproduces the same
    discrete sum as the oracle (Eqs. 2.23-2.26 are equivalent for any common rule)."""
    q = 3
    v = meshgen.jittered_grid(2, seed=3, jitter=0.2)
    for space in ["H1", "HCURL"]:
        got, code, _ = run(gpu_lib, space, q, v, L=L)
        ref, _ = oracle.gram(space, q, L, v)
        assert code == 0 and rel_errs(got, ref).max() <= TOL64
    gpu_lib.dpg_tables_init(q, "H1")
    gpu_lib.dpg_tables_init(q, "HCURL")


# ---------------------------------------------------------------- config 2: q=5, L=7

@pytest.fixture(scope="module")
def seq_q5():
    return meshgen.workload("seq_q5_8x8x8")


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("affine", [False, True])
def test_seq_q5_sampled_parity(gpu_lib, seq_q5, space, affine):
    """Full 512-element launch as timed by the benchmark; 12 sampled elements (first, last,
    and a seeded spread) against the oracle, all elements symmetric and finite."""
    w = seq_q5
    v = w["verts_affine"] if affine else w["verts"]
    c = meshgen.coeff_pairs(space, w["k"], v.shape[0])
    got, code, _ = run(gpu_lib, space, 5, v, c, L=7, affine=affine)
    assert code == 0
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, got.transpose(0, 2, 1))
    idx = np.unique(np.concatenate([[0, v.shape[0] - 1], np.random.default_rng(7).choice(v.shape[0], 10, replace=False)]))
    ref, _ = oracle.gram(space, 5, 7, v[idx], c[idx])
    assert rel_errs(got[idx], ref).max() <= TOL64


def test_seq_q5_fp32_form(gpu_lib, seq_q5):
    w = seq_q5
    idx = np.arange(0, 512, 37)
    for space in ["H1", "HCURL", "HDIV", "L2"]:
        c = meshgen.coeff_pairs(space, w["k"], 512)
        got, code, _ = run(gpu_lib, space, 5, w["verts"][idx], c[idx], L=7, fp32=True)
        ref, _ = oracle.gram(space, 5, 7, w["verts"][idx], c[idx])
        assert code == 0 and rel_errs(got, ref).max() <= TOL32


# ---------------------------------------------------------------- mixed B

@pytest.mark.parametrize("q,p", [(1, 1), (2, 1), (3, 2), (4, 4)])
@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("affine", [False, True])
def test_mixed_b_small(gpu_lib, q, p, split, affine):
    v = (meshgen.affine_parallelepipeds(2, seed=40) if affine else meshgen.jittered_grid(2, seed=40, jitter=0.2))[:5]
    got, code, _ = run(gpu_lib, "B", q, v, p=p, split=split, affine=affine)
    ref, _ = oracle.mixed_b(q, p, q + 2, v, split=split)
    assert code == 0
    assert rel_errs(got, ref.reshape(ref.shape[0], -1)).max() <= TOL64


def test_mixed_b_config3_shape(gpu_lib):
    """H(curl) q=6 test, vector-L2 p=4 trial, L=8, on a few elements of the 16^3 mesh."""
    v = meshgen.jittered_grid(16, seed=3)[[0, 1234, 4095]]
    for fp32, tol in [(False, TOL64), (True, TOL32)]:
        got, code, _ = run(gpu_lib, "B", 6, v, p=4, fp32=fp32)
        ref, _ = oracle.mixed_b(6, 4, 8, v)
        assert code == 0 and rel_errs(got, ref).max() <= tol


def test_hcurl_config3_shape(gpu_lib):
    v = meshgen.jittered_grid(16, seed=3)[[0, 4095]]
    for fp32, tol in [(False, TOL64), (True, TOL32)]:
        got, code, _ = run(gpu_lib, "HCURL", 6, v, fp32=fp32)
        ref, _ = oracle.gram("HCURL", 6, 8, v)
        assert code == 0 and rel_errs(got, ref).max() <= tol


# ---------------------------------------------------------------- high order (q = 9)

@pytest.mark.parametrize("space", ["H1", "HDIV"])
def test_q9_sampled(gpu_lib, space):
    w = meshgen.workload("q9_8x8x4")
    for affine in [False, True]:
        v = (w["verts_affine"] if affine else w["verts"])[[0, 255]]
        got, code, _ = run(gpu_lib, space, 9, v, L=11, affine=affine)
        ref, _ = oracle.gram(space, 9, 11, v)
        assert code == 0 and rel_errs(got, ref).max() <= TOL64


@pytest.mark.parametrize("fp32", [False, True])
def test_affine_l2_diagonal_q9_unaligned_output(gpu_lib, fp32):
    """The L2 Gram matrix of an affine element is diagonal (Legendre orthogonality, Eq. 2.95)
    and is written by a fill kernel: at q = 9 (729 rows) one element covers many of its CTAs,
    and an output starting one value past a 16-byte boundary takes its unaligned head and
    tail.  Off-diagonal entries are exact zeros; nothing is written before the output."""
    q, L = 9, 11
    gpu_lib.dpg_tables_init_L(q, L, "L2")
    v = meshgen.affine_parallelepipeds(2, seed=81)[:2]
    rng = np.random.default_rng(81)
    c = np.stack([rng.uniform(0.5, 2, 2), rng.uniform(0.5, 2, 2)], axis=1)
    n = gpu_lib.dpg_matrix_rows("L2", q)
    dt = torch.float32 if fp32 else torch.float64
    buf = torch.full((2 * n * n + 1,), float("nan"), dtype=dt, device="cuda")
    out = buf[1:].view(2, n, n)
    gpu_lib.integrate("L2", q, torch.from_numpy(v).cuda(), torch.from_numpy(c).cuda(), fp32=fp32, affine=True,
                      out=out)
    code, _ = gpu_lib.sync_status()
    assert code == 0
    assert torch.isnan(buf[0]).item()
    got = out.double().cpu().numpy()
    for e in range(2):
        assert np.count_nonzero(got[e] - np.diag(np.diagonal(got[e]))) == 0
    ref, _ = oracle.gram("L2", q, L, v, c)
    assert rel_errs(got, ref).max() <= (TOL32 if fp32 else TOL64)


# ---------------------------------------------------------------- edges and device faults

def test_every_entry_written(gpu_lib):
    """Poison the output with NaN: after the call every entry is finite."""
    v = torch.from_numpy(meshgen.jittered_grid(2, seed=2)).cuda()
    for space in ["H1", "HCURL", "HDIV", "L2"]:
        gpu_lib.dpg_tables_init(3, space)
        for affine in [False, True]:
            vv = v if not affine else torch.from_numpy(meshgen.affine_parallelepipeds(2, seed=2)).cuda()
            out = torch.full((8,) + gpu_lib.matrix_shape(space, 3), float("nan"), dtype=torch.float64, device="cuda")
            gpu_lib.integrate(space, 3, vv, out=out, affine=affine)
            assert gpu_lib.sync_status()[0] == 0
            assert torch.isfinite(out).all()


def test_zero_elements_and_host_errors(gpu_lib):
    gpu_lib.dpg_tables_init(2, "H1")
    v = torch.empty((0, 8, 3), dtype=torch.float64, device="cuda")
    out = gpu_lib.integrate("H1", 2, v)
    assert out.shape == (0, 27, 27)
    assert gpu_lib.dpg_integrate(1, 0, 11, 1, 1, 0, 1, 0) == 2          # not initialised
    assert gpu_lib.dpg_integrate(1, 0, 13, 1, 1, 0, 1, 0) == 3          # q out of range
    gpu_lib.dpg_tables_init(2, "B")
    assert gpu_lib.dpg_integrate(5, 3, 2, 1, 1, 0, 1, 0) == 1           # p > q
    assert gpu_lib.dpg_integrate(1 | 0x400, 0, 2, 1, 1, 0, 1, 0) == 1   # split on a Gram


def test_degenerate_element_reported(gpu_lib):
    v = meshgen.jittered_grid(2, seed=1)
    v[5] = v[5][[1, 0, 3, 2, 5, 4, 7, 6]]                                # inverted orientation
    got, code, bad = run(gpu_lib, "HCURL", 2, v)
    assert code == 5 and bad == 5
    assert np.all(np.isnan(got[5])) and np.all(np.isfinite(np.delete(got, 5, axis=0)))
    assert gpu_lib.sync_status() == (0, -1)                               # cleared


@pytest.mark.parametrize("space,fp32", [("H1", False), ("L2", False), ("L2", True)])
def test_non_affine_element_on_affine_path(gpu_lib, space, fp32):
    # L2: the diagonal-matrix kernel of the affine path (Eq. 2.95), its NaN rows included
    v = meshgen.affine_parallelepipeds(2, seed=4)
    v[2] = meshgen.jittered_grid(2, seed=4, jitter=0.2)[2]
    got, code, bad = run(gpu_lib, space, 2, v, affine=True, fp32=fp32)
    assert code == 6 and bad == 2
    assert np.all(np.isnan(got[2])) and np.all(np.isfinite(np.delete(got, 2, axis=0)))


def test_host_buffer_entry_point(gpu_lib):
    """dpg_integrate_host (pinned host buffers, streamed chunks) equals dpg_integrate."""
    dpg = gpu_lib
    w = meshgen.workload("seq_q5_8x8x8")
    for space in ["HCURL", "L2"]:
        dpg.dpg_tables_init_L(5, 7, space)
        v = torch.from_numpy(w["verts"]).pin_memory()
        c = torch.from_numpy(meshgen.coeff_pairs(space, w["k"], 512)).pin_memory()
        shape = (512,) + dpg.matrix_shape(space, 5)
        out = torch.empty(shape, dtype=torch.float64).pin_memory()
        sh = int(torch.cuda.current_stream().cuda_stream)
        assert dpg.dpg_integrate_host(dpg.space_id(space), 0, 5, 512, v.data_ptr(), c.data_ptr(), out.data_ptr(), sh) == 0
        ref = dpg.integrate(space, 5, v.cuda(), c.cuda()).cpu()
        assert torch.equal(out, ref)
