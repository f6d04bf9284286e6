"""Static condensation (Eq. 3.8 from Eq. 3.7) through the C ABI against the oracle.

Both sides factor G by Cholesky and substitute, in FP64 with different summation orders,
so they differ by the forward error of a Cholesky solve: the test allows
||K_gpu - K_oracle||_F <= 8 n eps cond(G) ||K_oracle||_F (and the same for F), with
cond(G) computed here for every element.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_00984_gb300 import meshgen

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(params=["fma", "tc", "tcgen05"])
def method(request, gpu_lib):
    """Every arithmetic of the trailing updates (FP64 FMA; FP64 products from exact BF16
    digits on the tensor cores, mma.sync or tcgen05) meets the same tolerance."""
    gpu_lib.dpg_condense_set_method(request.param)
    yield request.param
    gpu_lib.dpg_condense_set_method("tcgen05")


def run(dpg, G, B, l=None):
    g = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    lt = None if l is None else torch.from_numpy(np.ascontiguousarray(l)).cuda()
    K, F = dpg.condense(g, b, lt)
    code, bad = dpg.sync_status()
    return K.cpu().numpy(), (None if F is None else F.cpu().numpy()), g.cpu().numpy(), code, bad


def check(G, K, F, Kr, Fr):
    n = G.shape[1]
    for e in range(G.shape[0]):
        tol = max(8 * n * EPS * np.linalg.cond(G[e]), 1e-14)
        assert np.linalg.norm(K[e] - Kr[e]) <= tol * np.linalg.norm(Kr[e])
        assert np.array_equal(K[e], K[e].T)
        if F is not None:
            assert np.linalg.norm(F[e] - Fr[e]) <= tol * max(np.linalg.norm(Fr[e]), 1e-300)


@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (31, 7), (32, 64), (33, 65), (64, 1), (65, 2), (100, 130),
                                 (150, 24), (200, 300)])
@pytest.mark.parametrize("with_l", [False, True])
def test_condense_random(gpu_lib, method, n, m, with_l):
    ne = 5
    G = meshgen.spd_batch(ne, n, 1e3, seed=n * 1000 + m)
    rng = np.random.default_rng(n + m)
    B = rng.standard_normal((ne, n, m))
    l = rng.standard_normal((ne, n)) if with_l else None
    K, F, Lg, code, _ = run(gpu_lib, G, B, l)
    Kr, Fr, bad = oracle.condense(G, B, l)
    assert code == 0 and bad == -1
    check(G, K, F, Kr, Fr)
    # G's lower triangle now holds the Cholesky factor; the strict upper triangle is untouched
    iu = np.triu_indices(n, 1)
    for e in range(ne):
        Lr = np.linalg.cholesky(G[e])
        assert np.abs(np.tril(Lg[e]) - Lr).max() <= 8 * n * EPS * np.linalg.cond(G[e]) * np.abs(Lr).max()
        assert np.array_equal(Lg[e][iu], G[e][iu])


def test_condense_element_matrices(gpu_lib, method):
    """H(curl) Gram (q = 3), mixed B (p = 2) and load vector of oracle-built elements."""
    v = meshgen.jittered_grid(2, seed=80)[:6]
    G, _ = oracle.gram("HCURL", 3, 5, v)
    B, _ = oracle.mixed_b(3, 2, 5, v)
    l, _ = oracle.load("HCURL", 3, 5, v, np.random.default_rng(81).uniform(-1, 1, 30))
    K, F, _, code, _ = run(gpu_lib, G, B, l)
    Kr, Fr, _ = oracle.condense(G, B, l)
    assert code == 0
    check(G, K, F, Kr, Fr)


def test_condense_config_sizes(gpu_lib, method):
    """The sizes of the mixed-stiffness workload: H(curl) q = 6 (n = 882), p = 4 (m = 192),
    L = 8, two elements."""
    v = meshgen.jittered_grid(16, seed=3)[[0, 4095]]
    G, _ = oracle.gram("HCURL", 6, 8, v)
    B, _ = oracle.mixed_b(6, 4, 8, v)
    l, _ = oracle.load("HCURL", 6, 8, v, np.random.default_rng(82).uniform(-1, 1, 30))
    K, F, _, code, _ = run(gpu_lib, G, B, l)
    Kr, Fr, _ = oracle.condense(G, B, l)
    assert code == 0
    check(G, K, F, Kr, Fr)


def test_condense_large(gpu_lib, method):
    """n = 1400, m = 300 with the load column: 22 panels, up to 11 row blocks of the factor's
    digits per panel, 3 blocks of W, a ragged last panel (n = 21 64 + 56)."""
    G = meshgen.spd_batch(2, 1400, 1e3, seed=96)
    rng = np.random.default_rng(97)
    B = rng.standard_normal((2, 1400, 300))
    l = rng.standard_normal((2, 1400))
    K, F, _, code, _ = run(gpu_lib, G, B, l)
    Kr, Fr, _ = oracle.condense(G, B, l)
    assert code == 0
    check(G, K, F, Kr, Fr)


def test_condense_not_spd_and_args(gpu_lib, method):
    dpg = gpu_lib
    G = meshgen.spd_batch(4, 40, 1e2, seed=83)
    G[2, 35, 35] = -5.0                                   # a negative pivot late in the factorization
    rng = np.random.default_rng(84)
    B = rng.standard_normal((4, 40, 9))
    l = rng.standard_normal((4, 40))
    K, F, _, code, bad = run(dpg, G, B, l)
    assert dpg.STATUS[code] == "DPG_ERR_NOT_SPD" and bad == 2
    assert np.isnan(K[2]).all() and np.isnan(F[2]).all()
    ok = [0, 1, 3]
    Kr, Fr, _ = oracle.condense(G[ok], B[ok], l[ok])
    check(G[ok], K[ok], F[ok], Kr, Fr)
    g = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    b = torch.zeros((1, 4, 2), dtype=torch.float64, device="cuda")
    k = torch.zeros((1, 2, 2), dtype=torch.float64, device="cuda")
    f = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    L = dpg._L()
    assert L.dpg_condense(1, 4, 2, g.data_ptr(), b.data_ptr(), None, k.data_ptr(), f.data_ptr(), None) == 1
    assert L.dpg_condense(1, 0, 2, g.data_ptr(), b.data_ptr(), None, k.data_ptr(), None, None) == 3
    assert L.dpg_condense(1, 4, 2, None, b.data_ptr(), None, k.data_ptr(), None, None) == 1
    assert L.dpg_condense(0, 4, 2, None, None, None, None, None, None) == 0
    assert dpg.sync_status()[0] == 0


def _chain(dpg, q, p, v, c, src):
    """The stage-by-stage route through the separate entry points."""
    G = dpg.integrate("HCURL", q, v, c)
    B = dpg.integrate("B", q, v, p=p)
    l = dpg.integrate_load("HCURL", q, v, src)
    return dpg.condense(G, B, l)


def test_condensed_system_one_call(gpu_lib, method):
    """dpg_condensed_system equals the separate calls bit for bit, and the oracle's chain."""
    dpg = gpu_lib
    q, p = 3, 2
    dpg.dpg_tables_init(q, "HCURL")
    dpg.dpg_tables_init(q, "B")
    vn = meshgen.jittered_grid(4, seed=85)[:37]
    rng = np.random.default_rng(86)
    cn = np.stack([rng.uniform(0.5, 2, 37), rng.uniform(0.5, 2, 37)], axis=1)
    src = rng.uniform(-1, 1, 30)
    v, c, s = (torch.from_numpy(a).cuda() for a in (vn, cn, src))
    K, F = dpg.condensed_system(q, p, v, c, s)
    K2, F2 = _chain(dpg, q, p, v, c, s)
    code, _ = dpg.sync_status()
    assert code == 0
    assert torch.equal(K, K2) and torch.equal(F, F2)
    idx = [0, 17, 36]
    G, _ = oracle.gram("HCURL", q, q + 2, vn[idx], cn[idx])
    B, _ = oracle.mixed_b(q, p, q + 2, vn[idx])
    l, _ = oracle.load("HCURL", q, q + 2, vn[idx], src)
    Kr, Fr, _ = oracle.condense(G, B, l)
    check(G, K.cpu().numpy()[idx], F.cpu().numpy()[idx], Kr, Fr)
    Kn, Fn = dpg.condensed_system(q, p, v, c)                 # no load vector
    assert Fn is None and torch.equal(Kn, K)


def test_condensed_system_chunks_and_errors(gpu_lib, method):
    """1400 elements of the q = 6 / p = 4 pair run in two workspace chunks (912 and 488 on
    152 SMs): equal to the separate calls; an inverted element in the second chunk is
    reported by its index."""
    dpg = gpu_lib
    q, p = 6, 4
    dpg.dpg_tables_init_L(q, 8, "HCURL")
    dpg.dpg_tables_init_L(q, 8, "B")
    vn = meshgen.jittered_grid(16, seed=3)[:1400].copy()
    src = torch.from_numpy(np.random.default_rng(87).uniform(-1, 1, 30)).cuda()
    v = torch.from_numpy(vn).cuda()
    K, F = dpg.condensed_system(q, p, v, None, src)
    K2, F2 = _chain(dpg, q, p, v, None, src)
    assert dpg.sync_status()[0] == 0
    assert torch.equal(K, K2) and torch.equal(F, F2)
    del K2, F2
    vn[1000] = vn[1000][[1, 0, 3, 2, 5, 4, 7, 6]]
    v = torch.from_numpy(vn).cuda()
    K, F = dpg.condensed_system(q, p, v, None, src)
    code, bad = dpg.sync_status()
    assert dpg.STATUS[code] == "DPG_ERR_DEGENERATE" and bad == 1000
    assert torch.isnan(K[1000]).all() and torch.isfinite(K[999]).all() and torch.isfinite(K[1001]).all()
    L = dpg._L()
    k = torch.empty((1, 192, 192), dtype=torch.float64, device="cuda")
    assert L.dpg_condensed_system(q, 7, 1, v.data_ptr(), None, None, 0, k.data_ptr(), None, None) == 1   # p > q
    assert L.dpg_condensed_system(q, p, 1, v.data_ptr(), None, src.data_ptr(), 0, k.data_ptr(), None, None) == 1
    assert L.dpg_condensed_system(q, p, 0, None, None, None, 0, None, None, None) == 0
    assert dpg.sync_status()[0] == 0


def test_condense_methods_agree_and_nonfinite(gpu_lib):
    """The two arithmetics agree to FP64 rounding on the config-3 sizes; a NaN below the
    first panel (met by the tensor-core digit split) is reported, not absorbed."""
    dpg = gpu_lib
    G = meshgen.spd_batch(3, 300, 1e4, seed=90)
    B = np.random.default_rng(91).standard_normal((3, 300, 40))
    out = {}
    for meth in ("fma", "tc", "tcgen05"):
        dpg.dpg_condense_set_method(meth)
        K, _, _, code, _ = run(dpg, G, B)
        assert code == 0
        out[meth] = K
    dpg.dpg_condense_set_method("tcgen05")
    for e in range(3):
        tol = 8 * 300 * EPS * np.linalg.cond(G[e])
        for meth in ("tc", "tcgen05"):
            assert np.linalg.norm(out[meth][e] - out["fma"][e]) <= tol * np.linalg.norm(out["fma"][e])
    G2 = G.copy()
    G2[1, 200, 40] = G2[1, 40, 200] = np.nan
    for meth in ("tc", "tcgen05"):
        dpg.dpg_condense_set_method(meth)
        K, _, _, code, bad = run(dpg, G2, B)
        assert dpg.STATUS[code] == "DPG_ERR_NOT_SPD" and bad == 1
        assert np.isnan(K[1]).all() and np.isfinite(K[[0, 2]]).all()
    dpg.dpg_condense_set_method("tcgen05")
    assert dpg._L().dpg_condense_set_method(7) == 1
