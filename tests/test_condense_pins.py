"""Pins of the oracle's static condensation (Eq. 3.8 from Eq. 3.7), CPU only.

* B = G: B^T G^-1 B = G and B^T G^-1 l = l (closed form).
* Diagonal G: K_ij = sum_k B_ki B_kj / g_k, written out with loops.
* Eq. 3.7 itself: the saddle-point system [[G, -B], [B^T, 0]] [s; u] = [-l; 0], solved as
  one dense system, gives a u with K u = F -- the condensed system of Eq. 3.8.
* The optimal-test-function characterisation of DPG: u^T K u = max_v (v^T B u)^2 / v^T G v,
  reached at v = G^-1 B u, and no random v exceeds it.
* Oracle-built element matrices (H(curl) Gram, mixed B, load vector): K symmetric positive
  definite; a matrix that is not positive definite is reported and NaN-filled.
"""
import numpy as np
import pytest

import oracle
from paper_1711_00984_gb300 import meshgen


def spd(rng, ne, n, cond=1e3):
    out = np.empty((ne, n, n))
    for e in range(ne):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        out[e] = (Q * np.geomspace(1.0, cond, n)) @ Q.T
    return out


def test_b_equals_g():
    rng = np.random.default_rng(1)
    G = spd(rng, 3, 20)
    l = rng.standard_normal((3, 20))
    K, F, bad = oracle.condense(G, G, l)
    assert bad == -1
    assert np.abs(K - G).max() <= 1e-11 * np.abs(G).max()
    assert np.abs(F - l).max() <= 1e-11 * np.abs(l).max()


def test_diagonal_gram():
    rng = np.random.default_rng(2)
    n, m = 7, 4
    g = rng.uniform(0.5, 3.0, n)
    B = rng.standard_normal((1, n, m))
    l = rng.standard_normal((1, n))
    K, F, _ = oracle.condense(np.diag(g)[None], B, l)
    for i in range(m):
        fi = sum(B[0, k, i] * l[0, k] / g[k] for k in range(n))
        assert abs(F[0, i] - fi) <= 1e-14 * max(1.0, abs(fi))
        for j in range(m):
            kij = sum(B[0, k, i] * B[0, k, j] / g[k] for k in range(n))
            assert abs(K[0, i, j] - kij) <= 1e-14 * max(1.0, abs(kij))


def test_saddle_point_system():
    rng = np.random.default_rng(3)
    n, m = 30, 8
    G = spd(rng, 1, n)
    B = rng.standard_normal((1, n, m))
    l = rng.standard_normal((1, n))
    K, F, _ = oracle.condense(G, B, l)
    A = np.block([[G[0], -B[0]], [B[0].T, np.zeros((m, m))]])
    su = np.linalg.solve(A, np.concatenate([-l[0], np.zeros(m)]))
    u = su[n:]
    assert np.linalg.norm(K[0] @ u - F[0]) <= 1e-10 * np.linalg.norm(F[0])


def test_optimal_test_functions():
    rng = np.random.default_rng(4)
    n, m = 25, 6
    G = spd(rng, 1, n, cond=1e2)[0]
    B = rng.standard_normal((n, m))
    K, _, _ = oracle.condense(G[None], B[None])
    for _ in range(5):
        u = rng.standard_normal(m)
        v = np.linalg.solve(G, B @ u)
        best = (v @ B @ u) ** 2 / (v @ G @ v)
        assert abs(u @ K[0] @ u - best) <= 1e-11 * best
        for _ in range(20):
            w = rng.standard_normal(n)
            assert (w @ B @ u) ** 2 / (w @ G @ w) <= best * (1 + 1e-12)


def test_element_matrices_and_not_spd():
    v = meshgen.jittered_grid(2, seed=5)[:2]
    G, _ = oracle.gram("HCURL", 2, 4, v)
    B, _ = oracle.mixed_b(2, 1, 4, v)
    l, _ = oracle.load("HCURL", 2, 4, v, np.random.default_rng(6).uniform(-1, 1, 30))
    K, F, bad = oracle.condense(G, B, l)
    assert bad == -1 and F.shape == (2, 3)
    for e in range(2):
        assert np.abs(K[e] - K[e].T).max() <= 1e-12 * np.abs(K[e]).max()
        assert np.linalg.eigvalsh(K[e]).min() > 0
    G2 = G.copy()
    G2[1, 0, 0] = -1.0
    K2, F2, bad2 = oracle.condense(G2, B, l)
    assert bad2 == 1 and np.isnan(K2[1]).all() and np.isnan(F2[1]).all()
    assert np.array_equal(K2[0], K[0])
