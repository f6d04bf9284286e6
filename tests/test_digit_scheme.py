"""The arithmetic of the condensation's tensor-core route, modelled on the CPU (no GPU).

The CUDA kernel writes each operand row as x = 2^e sum_{u<7} d_u 2^-(8u+7) with balanced
base-256 digits |d_u| <= 128 and sums the digit products of the diagonals D = u + v <= 6.
This model follows those definitions with Python integers and checks what the design
relies on: the digits are exact in BF16, every diagonal sum stays below 2^22 (exact in
FP32 and in the kernel's integer conversion), and a blocked Cholesky condensation whose
updates use these products reproduces the oracle's K and F to FP64 rounding.
"""
import numpy as np

import oracle
from paper_1711_00984_gb300 import meshgen

S = 7


def digits(row):
    """(e, D[S][len(row)]) of one row, from F = trunc(|x| 2^(55 - e)) and balanced bytes."""
    mx = max(abs(float(x)) for x in row)
    e = int(np.floor(np.log2(mx))) + 1 if mx > 0 else 0
    D = np.zeros((S, len(row)), dtype=np.int64)
    for t, x in enumerate(row):
        f = int(abs(float(x)) * 2.0 ** (55 - e))            # exact: a power-of-two scaling
        dig = [0] * S
        for k in range(S - 1):
            d = f & 255
            f >>= 8
            if d >= 128:
                d -= 256
                f += 1
            dig[S - 1 - k] = d
        dig[0] = f
        sgn = -1 if x < 0 else 1
        for u in range(S):
            D[u, t] = sgn * dig[u]
    return e, D


def product(A, B):
    """A B^T from digits: per diagonal the exact integer sum, then 2^(e_i+e_j) 2^-(8D+14)."""
    dA = [digits(r) for r in A]
    dB = [digits(r) for r in B]
    out = np.zeros((len(A), len(B)))
    for i, (ei, Di) in enumerate(dA):
        assert np.abs(Di).max() <= 128                     # exact in BF16 (8 significant bits)
        for j, (ej, Dj) in enumerate(dB):
            total = 0.0
            for Dg in range(S):
                p = sum(int(Di[u] @ Dj[Dg - u]) for u in range(Dg + 1))
                assert abs(p) < 2 ** 22                    # exact FP32 sum, exact conversion
                total += p * 2.0 ** (-8 * Dg - 14)
            out[i, j] = total * 2.0 ** (ei + ej)
    return out


def condense_model(G, B, l, nb=32):
    A = G.copy()
    n = A.shape[0]
    R = np.concatenate([B, l[:, None]], axis=1)
    for kb in range(0, n, nb):
        w = min(nb, n - kb)
        L11 = np.linalg.cholesky(A[kb:kb + w, kb:kb + w])
        X = np.linalg.inv(L11)
        L21 = product(A[kb + w:, kb:kb + w], X)
        W1 = product(X, R[kb:kb + w].T.copy())
        A[kb + w:, kb:kb + w] = L21
        R[kb:kb + w] = W1
        if kb + w < n:
            A[kb + w:, kb + w:] -= product(L21, L21)
            R[kb + w:] -= product(L21, W1.T.copy())
    W, y = R[:, :-1], R[:, -1]
    return product(W.T.copy(), W.T.copy()), W.T @ y


def test_digit_row_reconstruction():
    rng = np.random.default_rng(1)
    row = rng.standard_normal(32) * np.geomspace(1e-6, 1e3, 32)
    e, D = digits(row)
    back = np.array([sum(int(D[u, t]) * 2.0 ** (-(8 * u + 7)) for u in range(S)) for t in range(32)]) * 2.0 ** e
    assert np.abs(back - row).max() <= 2.0 ** (e - 55)


def test_condensation_model_matches_oracle():
    v = meshgen.jittered_grid(2, seed=80)[:1]
    G, _ = oracle.gram("HCURL", 2, 4, v)
    B, _ = oracle.mixed_b(2, 1, 4, v)
    l, _ = oracle.load("HCURL", 2, 4, v, np.random.default_rng(81).uniform(-1, 1, 30))
    Kr, Fr, _ = oracle.condense(G, B, l)
    K, F = condense_model(G[0], B[0], l[0])
    tol = 8 * G.shape[1] * np.finfo(float).eps * np.linalg.cond(G[0])
    assert np.linalg.norm(K - Kr[0]) <= tol * np.linalg.norm(Kr[0])
    assert np.linalg.norm(F - Fr[0]) <= tol * np.linalg.norm(Fr[0])
    assert np.linalg.norm(K - Kr[0]) <= 1e-13 * np.linalg.norm(Kr[0])    # FP64 rounding, in fact


def test_digit_products_error_is_normwise_in_the_row_maxima():
    """The digit products are accurate relative to the rows' maxima, not entry by entry:
    for rows whose entries span nine decades, every product a_i . b_j is within
    2^-52 * 32 * max|a_i| max|b_j| of the exact value (Python fractions), while an entry
    of small magnitude may keep fewer correct bits than an FP64 dot product."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 32)) * np.geomspace(1e-6, 1e3, 32)
    B = rng.standard_normal((5, 32)) * np.geomspace(1e3, 1e-6, 32)
    P = product(A, B)
    for i in range(4):
        for j in range(5):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[j]))
            bound = 2.0 ** -52 * 32 * np.abs(A[i]).max() * np.abs(B[j]).max()
            assert abs(Fraction(float(P[i, j])) - exact) <= Fraction(bound)
