"""Exact rational arithmetic for the oracle's pins (Python ``fractions``).

Nothing here shares code with the oracle or with the CUDA library.  The 1D families are
built from their definitions, not from the recursions the oracle uses:

* shifted Legendre by Rodrigues' formula  P_n(x) = (1/n!) d^n/dx^n (x^2 - x)^n, which is
  the polynomial that Eqs. 2.91-2.93 generate on [0,1] (P_n(1) = 1);
* integrated Legendre by the integral definition of Eq. 2.97, L_i(x) = int_0^x P_{i-1},
  with L_0 = 1 - x (Eq. 2.101);
* 1D integrals F^{rs} (Eq. 2.90) by exact integration of coefficient lists.

For an affine element (constant Jacobian) every Gram and stiffness entry is a finite sum
of products of such 1D integrals times constant metric entries (Sec. 2.8.1), so the
matrices below are exact rationals.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial

# ---------------------------------------------------------------- polynomial helpers
# A polynomial is a tuple of Fractions, coefficient k multiplies x^k.


def pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return tuple(out)


def padd(a, b, sb=1):
    n = max(len(a), len(b))
    out = [Fraction(0)] * n
    for i, x in enumerate(a):
        out[i] += x
    for i, y in enumerate(b):
        out[i] += sb * y
    return tuple(out)


def pder(a):
    return tuple(Fraction(k) * a[k] for k in range(1, len(a))) or (Fraction(0),)


def pint0(a):
    """Antiderivative vanishing at 0."""
    return (Fraction(0),) + tuple(a[k] / (k + 1) for k in range(len(a)))


def peval(a, x):
    """Exact value at the binary float x (evaluated in rationals), rounded once."""
    xf = Fraction(float(x))
    s = Fraction(0)
    for c in reversed(a):
        s = s * xf + c
    return float(s)


def pintegral01(a):
    return sum((c / (k + 1) for k, c in enumerate(a)), Fraction(0))


@lru_cache(maxsize=None)
def legendre(n: int):
    """Shifted Legendre P_n on [0,1] by Rodrigues' formula."""
    base = (Fraction(0), Fraction(-1), Fraction(1))      # x^2 - x
    p = (Fraction(1),)
    for _ in range(n):
        p = pmul(p, base)
    for _ in range(n):
        p = pder(p)
    return tuple(c / factorial(n) for c in p)


@lru_cache(maxsize=None)
def int_legendre(i: int):
    """chi_i = L_i: L_0 = 1 - x, L_i = int_0^x P_{i-1} (i >= 1)."""
    if i == 0:
        return (Fraction(1), Fraction(-1))
    return pint0(legendre(i - 1))


@lru_cache(maxsize=None)
def family(kind: str, i: int):
    """1D factor of kind 'W' (chi_i = L_i), 'D' (chi'_i) or 'Y' (nu_i = P_i)."""
    if kind == "W":
        return int_legendre(i)
    if kind == "D":
        return pder(int_legendre(i))
    if kind == "Y":
        return legendre(i)
    raise KeyError(kind)


@lru_cache(maxsize=None)
def F(kr: str, kc: str, i: int, j: int) -> Fraction:
    """int_0^1 f^{kr}_i f^{kc}_j  (Eq. 2.90 with kinds instead of binary superscripts)."""
    return pintegral01(pmul(family(kr, i), family(kc, j)))


# ---------------------------------------------------------------- 3x3 rational algebra

def mat_mul(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


def mat_t(A):
    return [[A[j][i] for j in range(3)] for i in range(3)]


def det3(A):
    return (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
            - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
            + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]))


def inv3(A):
    d = det3(A)
    C = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            m = [[A[r][c] for c in range(3) if c != j] for r in range(3) if r != i]
            C[j][i] = ((-1) ** (i + j)) * (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / d
    return C


# ---------------------------------------------------------------- space layouts

def components(space: str, q: int, p: int = 0):
    """[(comp, dims[3], kinds[3], offset)] following Eqs. 2.17, 2.33, 2.52-2.53, 2.70-2.71."""
    if space == "H1":
        return [(0, (q + 1,) * 3, ("W",) * 3, 0)]
    if space == "L2":
        return [(0, (q,) * 3, ("Y",) * 3, 0)]
    if space == "TRIAL_L2VEC":
        return [(c, (p,) * 3, ("Y",) * 3, c * p ** 3) for c in range(3)]
    out, off = [], 0
    for a in range(3):
        if space == "HDIV":
            dims = tuple(q + 1 if d == a else q for d in range(3))
            kinds = tuple("W" if d == a else "Y" for d in range(3))
        elif space == "HCURL":
            dims = tuple(q if d == a else q + 1 for d in range(3))
            kinds = tuple("Y" if d == a else "W" for d in range(3))
        else:
            raise KeyError(space)
        out.append((a, dims, kinds, off))
        off += dims[0] * dims[1] * dims[2]
    return out


def dofs(space: str, q: int, p: int = 0):
    """List of (I, comp, (i1, i2, i3), kinds) in index order."""
    out = []
    for comp, dims, kinds, off in components(space, q, p):
        for i3 in range(dims[2]):
            for i2 in range(dims[1]):
                for i1 in range(dims[0]):
                    out.append((off + i1 + dims[0] * (i2 + dims[1] * i3), comp, (i1, i2, i3), kinds))
    out.sort()
    return out


def _terms_scalar_grad(comp_unused, kinds):
    """Master gradient of f1 f2 f3 (kinds W): component a has 'D' in direction a."""
    return [(a, 1, tuple("D" if d == a else kinds[d] for d in range(3))) for a in range(3)]


def _curl_terms(a, kinds):
    """curl^(f e_a) = grad f x e_a: component a+1 is +d_{a+2} f, component a+2 is -d_{a+1} f."""
    a1, a2 = (a + 1) % 3, (a + 2) % 3
    k1 = tuple("D" if d == a2 else kinds[d] for d in range(3))
    k2 = tuple("D" if d == a1 else kinds[d] for d in range(3))
    return [(a1, 1, k1), (a2, -1, k2)]


def _prod(kr, ir, kc, ic):
    return F(kr[0], kc[0], ir[0], ic[0]) * F(kr[1], kc[1], ir[1], ic[1]) * F(kr[2], kc[2], ir[2], ic[2])


def affine_gram(space: str, q: int, J, c0=Fraction(1), c1=Fraction(1)):
    """Exact Gram matrix (list of lists of Fractions) of an affine element with Jacobian J.

    Reference-element forms with constant metrics (Eqs. 2.16, 2.31, 2.49, 2.68 with J
    constant, Sec. 2.8.1): D = J^-1 J^-T, C = J^T J.
    """
    J = [[Fraction(x) for x in row] for row in J]
    det = det3(J)
    Ji = inv3(J)
    D = mat_mul(Ji, mat_t(Ji))
    C = mat_mul(mat_t(J), J)
    dl = dofs(space, q)
    n = len(dl)
    G = [[Fraction(0)] * n for _ in range(n)]
    for I, ca, ir, ka in dl:
        for Jd, cb, jc, kb in dl:
            if Jd < I:
                continue
            v = Fraction(0)
            if space == "L2":
                v = c0 / det * _prod(ka, ir, kb, jc)
            elif space == "H1":
                v = c0 * det * _prod(ka, ir, kb, jc)
                for a, _, kra in _terms_scalar_grad(0, ka):
                    for b, _, krb in _terms_scalar_grad(0, kb):
                        v += c1 * det * D[a][b] * _prod(kra, ir, krb, jc)
            elif space == "HDIV":
                v = c0 / det * C[ca][cb] * _prod(ka, ir, kb, jc)
                kda = tuple("D" if d == ca else ka[d] for d in range(3))
                kdb = tuple("D" if d == cb else kb[d] for d in range(3))
                v += c1 / det * _prod(kda, ir, kdb, jc)
            elif space == "HCURL":
                v = c0 * det * D[ca][cb] * _prod(ka, ir, kb, jc)
                for xa, sa, kra in _curl_terms(ca, ka):
                    for xb, sb, krb in _curl_terms(cb, kb):
                        v += c1 / det * sa * sb * C[xa][xb] * _prod(kra, ir, krb, jc)
            G[I][Jd] = v
            G[Jd][I] = v
    return G


def _prod_dirs(kr, ir, kc, ic, dirs):
    v = Fraction(1)
    for d in dirs:
        v *= F(kr[d], kc[d], ir[d], ic[d])
    return v


def affine_support(space: str, q: int, dirs=(0, 1, 2)):
    """Boolean matrix: True where at least one term of the affine Gram matrix of `space` has
    a non-zero product of exact 1D integrals F (Eq. 2.90) over the directions `dirs`, i.e.
    where the entry is not forced to zero by the zeros of F whatever the metric (all three
    directions: affine elements; dirs = (0,): elements extruded along x1, whose xi_1
    factors are exact integrals); the terms are those of affine_gram."""
    _prod = lambda kr, ir, kc, ic: _prod_dirs(kr, ir, kc, ic, dirs)  # noqa: E731
    dl = dofs(space, q)
    n = len(dl)
    S = [[False] * n for _ in range(n)]
    for I, ca, ir, ka in dl:
        for Jd, cb, jc, kb in dl:
            prods = []
            if space in ("L2", "H1", "HDIV", "HCURL"):
                prods.append(_prod(ka, ir, kb, jc))
            if space == "H1":
                for _, _, kra in _terms_scalar_grad(0, ka):
                    for _, _, krb in _terms_scalar_grad(0, kb):
                        prods.append(_prod(kra, ir, krb, jc))
            elif space == "HDIV":
                kda = tuple("D" if d == ca else ka[d] for d in range(3))
                kdb = tuple("D" if d == cb else kb[d] for d in range(3))
                prods.append(_prod(kda, ir, kdb, jc))
            elif space == "HCURL":
                for _, _, kra in _curl_terms(ca, ka):
                    for _, _, krb in _curl_terms(cb, kb):
                        prods.append(_prod(kra, ir, krb, jc))
            S[I][Jd] = any(x != 0 for x in prods)
    return S


def affine_mixed_b(q: int, p: int, J, split: bool = False):
    """Exact B (n_test x 3p^3): B_IK = int u^_K.J^-T psi^_I + u^_K.J curl^psi^_I / |J| (affine)."""
    J = [[Fraction(x) for x in row] for row in J]
    det = det3(J)
    Ji = inv3(J)
    rows = dofs("HCURL", q)
    cols = dofs("TRIAL_L2VEC", q, p)
    M = [[Fraction(0)] * len(cols) for _ in rows]
    K = [[Fraction(0)] * len(cols) for _ in rows]
    for I, ca, ir, ka in rows:
        for Kc, cc, kc_idx, kk in cols:
            # u^ = P P P e_cc ; psi^ = f e_ca ; u^ . J^-T psi^ = (J^-T)[cc][ca] = Ji[ca][cc]
            M[I][Kc] = Ji[ca][cc] * _prod(ka, ir, kk, kc_idx)
            s = Fraction(0)
            for xa, sa, kra in _curl_terms(ca, ka):
                s += sa * J[cc][xa] / det * _prod(kra, ir, kk, kc_idx)
            K[I][Kc] = s
    if split:
        return M, K
    return [[M[i][j] + K[i][j] for j in range(len(cols))] for i in range(len(rows))]


# ---------------------------------------------------------------- ultraweak acoustics

def _dkind(kinds, d):
    """Kinds of d/dxi_d of a tensor function (chi -> chi' in direction d)."""
    return tuple("D" if e == d else kinds[e] for e in range(3))


def acoustic_cross(q: int):
    """Exact cross block of the acoustics adjoint graph norm (Eq. 3.18, coefficient of
    i*omega) on the master cube: X[I_v][I_q] = int -(div^ v^) q^ + v^ . grad^ q^.  The
    Piola maps cancel in both products, so this is the value on every element."""
    rows = dofs("HDIV", q)
    cols = dofs("H1", q)
    X = [[Fraction(0)] * len(cols) for _ in rows]
    for I, a, ir, ka in rows:
        for Jd, _, jc, kq in cols:
            X[I][Jd] = -_prod(_dkind(ka, a), ir, kq, jc) + _prod(ka, ir, _dkind(kq, a), jc)
    return X


def affine_acoustic_b(q: int, p: int, J):
    """Exact ultraweak acoustics stiffness (Eq. 3.16) on an affine element with Jacobian J:
    (B0, B1) with B0 = -(p, div v) - (u, grad q) and B1 = (p, q) + (u, v) (coefficient of
    i*omega).  Rows: H1 test functions then H(div); columns: scalar L2 trial (order p)
    then the three L2 components."""
    J = [[Fraction(x) for x in row] for row in J]
    det = det3(J)
    Ji = inv3(J)
    h1, hdiv = dofs("H1", q), dofs("HDIV", q)
    pl = dofs("L2", p)
    ul = dofs("TRIAL_L2VEC", q, p)
    nh, npp = len(h1), len(pl)
    rows, cols = nh + len(hdiv), npp + len(ul)
    B0 = [[Fraction(0)] * cols for _ in range(rows)]
    B1 = [[Fraction(0)] * cols for _ in range(rows)]
    for I, _, ir, kq in h1:
        for K, _, kk, kp in pl:
            B1[I][K] = _prod(kq, ir, kp, kk)                          # (p, q): p^ q^
        for K, cc, kk, ku in ul:
            s = Fraction(0)
            for d in range(3):                                        # u^ . J^-T grad^ q^
                s += Ji[d][cc] * _prod(_dkind(kq, d), ir, ku, kk)
            B0[I][npp + K] = -s
    for I, a, ir, kv in hdiv:
        for K, _, kk, kp in pl:
            B0[nh + I][K] = -_prod(_dkind(kv, a), ir, kp, kk) / det  # p^ div^ v^ / |J|
        for K, cc, kk, ku in ul:
            B1[nh + I][npp + K] = J[cc][a] * _prod(kv, ir, ku, kk) / det   # u^ . J v^ / |J|
    return B0, B1
