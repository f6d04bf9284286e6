"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it checks.  Together they are chosen so that a plausible slip
anywhere in the oracle (a dropped term, a wrong sign or index, a transposed Jacobian, a
wrong Piola factor, a wrong index map) fails at least one of them:

* quadrature and 1D families          -> exactness, closed values, Rodrigues polynomials
* 1D integrals                        -> the paper's printed F tables (Eqs. 2.103-2.114)
* geometry                            -> identity / affine Jacobians, finite differences,
                                         total volume of a jittered unit-cube mesh
* Piola maps and index maps           -> exact rational Gram matrices of affine elements
                                         with a full non-symmetric Jacobian
* curl / div / grad and the spaces    -> exact-sequence identities, pointwise and matrix
* trilinear maps (no exact answer)    -> coordinate functions, symmetry, definiteness
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import exact
import oracle
from paper_1711_00984_gb300 import meshgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac_matrix_to_float(M):
    return np.array([[float(x) for x in row] for row in M])


def _rel_fro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ------------------------------------------------------------------ quadrature, 1D

@pytest.mark.parametrize("L", range(1, 13))
def test_gauss_exact_to_degree_2L_minus_1(L):
    """Eq. 2.23: an L-point rule integrates degree <= 2L-1 exactly, and not degree 2L."""
    x, w = oracle.gauss(L)
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1)) and np.all(w > 0)
    for k in range(2 * L):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 2e-15
    # the degree-2L error of Gauss on (0,1) is (L!)^4 / ((2L+1) ((2L)!)^2) (x^2L has a
    # constant 2L-th derivative (2L)!), so the rule is exact to 2L-1 and no further
    err = 1.0 / (2 * L + 1) - np.sum(w * x ** (2 * L))
    expect = math.factorial(L) ** 4 / ((2 * L + 1) * math.factorial(2 * L) ** 2)
    assert abs(err - expect) <= 1e-15 + 1e-9 * expect
    # symmetric about 1/2
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15, rtol=0)


def test_legendre_closed_values():
    """P_i(1) = 1 (after Eq. 2.93); P_i(0) = (-1)^i; L_i(0) = L_i(1) = 0 for i >= 2
    (bubbles, after Eq. 2.98); L_0 = 1 - x, L_1 = x (Eqs. 2.99, 2.101)."""
    n = 14
    P1, _, L1, _ = oracle.one_d(n, 1.0)
    P0, _, L0, _ = oracle.one_d(n, 0.0)
    assert np.allclose(P1, 1.0, atol=1e-14, rtol=0)
    assert np.allclose(P0, [(-1) ** i for i in range(n)], atol=1e-14, rtol=0)
    assert np.allclose(L1[2:], 0.0, atol=1e-15) and np.allclose(L0[2:], 0.0, atol=1e-15)
    assert L0[0] == 1.0 and L1[0] == 0.0 and L0[1] == 0.0 and L1[1] == 1.0


def test_legendre_orthogonality():
    """Eq. 2.95: int_0^1 P_i P_j = delta_ij / (2i+1), and zero average (Eq. 2.96)."""
    n = 11
    x, w = oracle.gauss(12)
    P = np.array([oracle.one_d(n, xx)[0] for xx in x])        # [L, n]
    M = P.T @ (w[:, None] * P)
    assert np.allclose(M, np.diag(1.0 / (2 * np.arange(n) + 1)), atol=2e-15, rtol=0)


def test_1d_families_match_definitions():
    """Oracle P, P', L, L' (recursions 2.93, 2.100) equal the Rodrigues polynomials and the
    integral definition of Eq. 2.97 at arbitrary points."""
    rng = np.random.default_rng(0)
    n = 12
    for xx in rng.uniform(0, 1, 9):
        P, dP, Lv, dL = oracle.one_d(n, xx)
        for i in range(n):
            assert abs(P[i] - exact.peval(exact.legendre(i), xx)) < 1e-13
            assert abs(dP[i] - exact.peval(exact.pder(exact.legendre(i)), xx)) < 1e-11
            assert abs(Lv[i] - exact.peval(exact.int_legendre(i), xx)) < 1e-13
            assert abs(dL[i] - exact.peval(exact.pder(exact.int_legendre(i)), xx)) < 1e-13


def _paper_F(r, s, i, j):
    """The paper's closed forms for F^{rs}_{ij} (Eqs. 2.103-2.114), written out."""
    Fr = Fraction
    if r == 0 and s == 0:
        if i < j:
            i, j = j, i                                  # symmetric (stated before Eq. 2.103)
        if j >= 2:                                       # Eq. 2.103
            if i == j:
                return Fr(1, 4 * (2 * j - 1) ** 2) * (Fr(1, 2 * j + 1) + Fr(1, 2 * j - 3))
            if i == j + 2:
                return Fr(-1, 4 * (2 * j + 3) * (2 * j - 1) * (2 * j + 1))
            return Fr(0)
        if j == 1:                                       # Eq. 2.104
            return {1: Fr(1, 3), 2: Fr(-1, 12), 3: Fr(-1, 60)}.get(i, Fr(0))
        # j == 0, Eq. 2.105
        if i >= 2:
            return (-1) ** i * _paper_F(0, 0, i, 1)
        return {1: Fr(1, 6), 0: Fr(1, 3)}[i]
    if r == 0 and s == 1:
        if j == 0:                                       # Eq. 2.110
            return -_paper_F(0, 1, i, 1)
        if i == 1:                                       # Eq. 2.106
            return {2: Fr(1, 6), 1: Fr(1, 2)}.get(j, Fr(0))
        if i == 2:                                       # Eq. 2.107
            return {3: Fr(1, 30), 1: Fr(-1, 6)}.get(j, Fr(0))
        if i == 0:                                       # Eq. 2.109
            return {1: Fr(1, 2), 2: Fr(-1, 6)}.get(j, Fr(0))
        # i >= 3, j >= 1, Eq. 2.108
        v = Fr(0)
        if i == j - 1:
            v += Fr(1, 2 * i + 1)
        if i - 1 == j:
            v -= Fr(1, 2 * i - 3)
        return v / (2 * (2 * i - 1))
    if r == 1 and s == 0:                                # Eq. 2.112
        return _paper_F(0, 1, j, i)
    # r == s == 1
    if i < j:
        i, j = j, i
    if j >= 1:                                           # Eq. 2.113
        return Fr(1, 2 * i - 1) if i == j else Fr(0)
    return {0: Fr(1), 1: Fr(-1)}.get(i, Fr(0))           # Eq. 2.114


def test_paper_F_tables_golden_file():
    """Every constant printed in Sec. 2.8.2 equals the exact 1D integral."""
    kinds = {0: "W", 1: "D"}
    with open(os.path.join(GOLDEN, "f_tables_paper.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            r, s, i, j, val = line.split()
            r, s, i, j = int(r), int(s), int(i), int(j)
            assert exact.F(kinds[r], kinds[s], i, j) == Fraction(val), (r, s, i, j)
            assert _paper_F(r, s, i, j) == Fraction(val)


@pytest.mark.parametrize("r,s", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_paper_F_formulas_and_oracle_quadrature(r, s):
    """Eqs. 2.103-2.114 for i, j <= 10 equal the exact integrals, and the oracle's Gauss
    rule with its own 1D functions reproduces them (exact for degree <= 2L-1)."""
    kinds = {0: "W", 1: "D"}
    n = 11
    x, w = oracle.gauss(n + 1)
    vals = np.array([oracle.one_d(n, xx) for xx in x])      # [L, 4, n]
    tab = {0: vals[:, 2, :], 1: vals[:, 3, :]}
    Fq = tab[r].T @ (w[:, None] * tab[s])
    for i in range(n):
        for j in range(n):
            ex = exact.F(kinds[r], kinds[s], i, j)
            assert _paper_F(r, s, i, j) == ex, (r, s, i, j)
            assert abs(Fq[i, j] - float(ex)) < 5e-16


# ------------------------------------------------------------------ geometry

def test_geometry_identity_and_affine():
    """Identity cube: J = I, |J| = 1.  Parallelepiped: J equals its edge matrix at every
    point (Eq. 2.2 for a constant map)."""
    cube = meshgen.reference_cube()[0]
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.2 * rng.uniform(-1, 1, (3, 3))
    par = meshgen.affine_from_matrix(A, origin=(0.3, -0.1, 2.0))[0]
    for xi in rng.uniform(0, 1, (5, 3)):
        x, J, det = oracle.geometry(cube, xi)
        assert np.allclose(J, np.eye(3), atol=1e-15) and abs(det - 1) < 1e-15
        assert np.allclose(x, xi, atol=1e-15)
        x, J, det = oracle.geometry(par, xi)
        assert np.allclose(J, A, atol=1e-14) and abs(det - np.linalg.det(A)) < 1e-13
        assert np.allclose(x, np.array([0.3, -0.1, 2.0]) + A @ xi, atol=1e-14)


def test_geometry_finite_differences():
    """J of a trilinear element equals central differences of the map x(xi)."""
    v = meshgen.jittered_grid(3, seed=7, jitter=0.25)
    rng = np.random.default_rng(2)
    eps = 1e-6
    for e in (0, 13, 26):
        for xi in rng.uniform(0.1, 0.9, (4, 3)):
            _, J, det = oracle.geometry(v[e], xi)
            Jfd = np.zeros((3, 3))
            for d in range(3):
                dx = np.zeros(3); dx[d] = eps
                Jfd[:, d] = (oracle.geometry(v[e], xi + dx)[0] - oracle.geometry(v[e], xi - dx)[0]) / (2 * eps)
            assert np.allclose(J, Jfd, atol=1e-9)
            assert abs(det - np.linalg.det(Jfd)) < 1e-9


def test_total_volume_of_jittered_mesh_is_one():
    """The jittered grid tiles the unit cube exactly (boundary vertices fixed, shared
    bilinear faces).  With q = 1 the H1 basis is L_0, L_1 per direction, whose sum is 1,
    so sum_IJ of the H1 mass matrix is the element volume; the volumes sum to 1."""
    v = meshgen.jittered_grid(4, seed=11, jitter=0.2)
    c = np.tile([1.0, 0.0], (v.shape[0], 1))
    G, bad = oracle.gram("H1", 1, 2, v, c)
    assert bad == -1
    vol = G.sum(axis=(1, 2))
    assert np.all(vol > 0)
    assert abs(vol.sum() - 1.0) < 1e-13


# ------------------------------------------------------------------ reference cube, L2

def test_l2_reference_cube_closed_form():
    """Golden values (Eq. 2.95 on the master cube): diagonal G_II = prod 1/(2 i_d + 1)."""
    G, _ = oracle.gram("L2", 3, 4, meshgen.reference_cube())
    G = G[0]
    with open(os.path.join(GOLDEN, "l2_reference_cube.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                I, i1, i2, i3, val = line.split()
                assert abs(G[int(I), int(I)] - float(Fraction(val))) < 1e-15
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-15
    q = 5
    G5, _ = oracle.gram("L2", q, q + 2, meshgen.reference_cube())
    idx = np.array([[i1, i2, i3] for i3 in range(q) for i2 in range(q) for i1 in range(q)])
    expect = np.prod(1.0 / (2 * idx + 1), axis=1)
    assert np.allclose(np.diag(G5[0]), expect, rtol=1e-14, atol=0)


def test_l2_cube_scaling():
    """L2 Piola (Eq. 2.6): on a cube of side h the L2 Gram scales as h^-3."""
    q = 3
    G1, _ = oracle.gram("L2", q, 5, meshgen.reference_cube(1.0))
    Gh, _ = oracle.gram("L2", q, 5, meshgen.reference_cube(0.25, origin=(1, 2, 3)))
    assert np.allclose(Gh, G1 * 0.25 ** -3, rtol=1e-14, atol=1e-12)


# ------------------------------------------------------------------ affine: exact rationals

_J_RAT = [[Fraction(9, 8), Fraction(1, 8), Fraction(-1, 4)],
          [Fraction(-1, 8), Fraction(7, 8), Fraction(1, 8)],
          [Fraction(1, 4), Fraction(-1, 8), Fraction(5, 4)]]


@pytest.mark.parametrize("space", ["L2", "H1", "HDIV", "HCURL"])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_affine_gram_equals_exact_rational(space, q):
    """On a parallelepiped with a full, non-symmetric Jacobian and coefficients (c0, c1),
    the oracle's quadrature (exact for L >= q+1) equals the exact rational Gram matrix of
    Sec. 2.8.1 (Eqs. 2.16, 2.31, 2.49, 2.68 with D = J^-1 J^-T and C = J^T J constant)."""
    c0, c1 = Fraction(3, 4), Fraction(5, 2)
    Jf = np.array([[float(x) for x in r] for r in _J_RAT])
    verts = meshgen.affine_from_matrix(Jf, origin=(0.5, 0.25, -0.125))
    G, bad = oracle.gram(space, q, q + 1, verts, np.array([[float(c0), float(c1)]]))
    assert bad == -1
    ex = _frac_matrix_to_float(exact.affine_gram(space, q, _J_RAT, c0, c1))
    assert _rel_fro(G[0], ex) < 1e-14
    assert np.abs(G[0] - ex).max() < 1e-14 * np.abs(ex).max()


@pytest.mark.parametrize("space", ["L2", "H1", "HDIV", "HCURL"])
def test_affine_more_points_agree(space):
    """Quadrature is exact for affine maps at L >= q+1 (polynomial integrand of degree
    <= 2q per direction), so L = q+1 and L = q+5 agree: brute force with more points."""
    q = 3
    v = meshgen.affine_parallelepipeds(2, seed=3)[:3]
    a, _ = oracle.gram(space, q, q + 1, v)
    b, _ = oracle.gram(space, q, q + 5, v)
    for e in range(v.shape[0]):
        assert _rel_fro(a[e], b[e]) < 1e-14


@pytest.mark.parametrize("q,p", [(2, 1), (3, 2)])
def test_affine_mixed_b_equals_exact_rational(q, p):
    """B_IK = (u_K, psi_I) + (u_K, curl psi_I) on an affine element (pattern of Eq. 3.16)
    equals its exact rational value; both blocks checked separately."""
    Jf = np.array([[float(x) for x in r] for r in _J_RAT])
    verts = meshgen.affine_from_matrix(Jf)
    B, bad = oracle.mixed_b(q, p, q + 1, verts, split=True)
    assert bad == -1
    M, K = exact.affine_mixed_b(q, p, _J_RAT, split=True)
    assert _rel_fro(B[0, 0], _frac_matrix_to_float(M)) < 1e-14
    assert _rel_fro(B[0, 1], _frac_matrix_to_float(K)) < 1e-14
    Bs, _ = oracle.mixed_b(q, p, q + 1, verts, split=False)
    assert np.allclose(Bs[0], B[0, 0] + B[0, 1], atol=1e-15)


# ------------------------------------------------------------------ exact sequence

def _deriv_expand(i):
    """chi'_i in the nu basis: chi'_0 = -nu_0, chi'_i = nu_{i-1} (Eqs. 2.54, 2.98, 2.101)."""
    return [(-1, 0)] if i == 0 else [(1, i - 1)]


def _index(space, q, comp, idx):
    off = 0
    for c, dims, kinds, o in exact.components(space, q):
        if c == comp:
            return o + idx[0] + dims[0] * (idx[1] + dims[1] * idx[2])
    raise KeyError


def discrete_grad(q):
    """Integer matrix Gd with grad^ phi_I = sum_K Gd[K, I] psi_K (H1 -> H(curl), same q)."""
    n1, nc = oracle.dim("H1", q), oracle.dim("HCURL", q)
    Gd = np.zeros((nc, n1))
    for I, _, ii, _ in exact.dofs("H1", q):
        for a in range(3):
            for s, k in _deriv_expand(ii[a]):
                jj = list(ii); jj[a] = k
                Gd[_index("HCURL", q, a, jj), I] += s
    return Gd


def discrete_curl(q):
    """Integer matrix Cd with curl^ psi_K = sum_M Cd[M, K] theta_M (H(curl) -> H(div))."""
    nc, nd = oracle.dim("HCURL", q), oracle.dim("HDIV", q)
    Cd = np.zeros((nd, nc))
    for K, a, kk, _ in exact.dofs("HCURL", q):
        a1, a2 = (a + 1) % 3, (a + 2) % 3
        for s, m in _deriv_expand(kk[a2]):           # + d_{a+2} f e_{a+1}
            jj = list(kk); jj[a2] = m
            Cd[_index("HDIV", q, a1, jj), K] += s
        for s, m in _deriv_expand(kk[a1]):           # - d_{a+1} f e_{a+2}
            jj = list(kk); jj[a1] = m
            Cd[_index("HDIV", q, a2, jj), K] -= s
    return Cd


def discrete_div(q):
    """Integer matrix Dd with div^ theta_M = sum_N Dd[N, M] v_N (H(div) -> L2)."""
    nd, nl = oracle.dim("HDIV", q), oracle.dim("L2", q)
    Dd = np.zeros((nl, nd))
    for M, a, mm, _ in exact.dofs("HDIV", q):
        for s, k in _deriv_expand(mm[a]):
            jj = list(mm); jj[a] = k
            Dd[_index("L2", q, 0, jj), M] += s
    return Dd


@pytest.mark.parametrize("q", [1, 2, 4])
def test_exact_sequence_pointwise(q):
    """Eq. 2.1 on the master cube: grad^ H1 lies in H(curl) through Gd, curl^ of it is 0
    (Eq. 2.67); curl^ H(curl) lies in H(div) through Cd, div^ of it is 0 (Eq. 2.48);
    div^ H(div) lies in L2 through Dd.  Also Cd Gd = 0 and Dd Cd = 0 exactly."""
    Gd, Cd, Dd = discrete_grad(q), discrete_curl(q), discrete_div(q)
    assert np.all(Cd @ Gd == 0) and np.all(Dd @ Cd == 0)
    rng = np.random.default_rng(q)
    for xi in rng.uniform(0, 1, (4, 3)):
        _, grad_h1 = oracle.shape("H1", q, xi)
        v_c, curl_c = oracle.shape("HCURL", q, xi)
        v_d, div_d = oracle.shape("HDIV", q, xi)
        v_l, _ = oracle.shape("L2", q, xi)
        assert np.allclose(Gd.T @ v_c, grad_h1, atol=1e-13)
        assert np.allclose(Gd.T @ curl_c, 0.0, atol=1e-12)
        assert np.allclose(Cd.T @ v_d, curl_c, atol=1e-13)
        assert np.allclose(Cd.T @ div_d[:, 0], 0.0, atol=1e-12)
        assert np.allclose(Dd.T @ v_l[:, 0], div_d[:, 0], atol=1e-13)


@pytest.mark.parametrize("q", [2, 3])
def test_exact_sequence_matrix_identities(q):
    """For any map and any rule (the Piola maps commute with the operators, Sec. 2.4-2.6):
    K^H1 = Gd^T M^curl Gd,  K^curl = Cd^T M^div Cd,  K^div = Dd^T M^L2 Dd, where M is the
    mass-only Gram (coeffs (1,0)) and K the derivative-only Gram (coeffs (0,1))."""
    v = meshgen.jittered_grid(2, seed=5, jitter=0.3)[:4]
    L = q + 2
    ne = v.shape[0]
    m = np.tile([1.0, 0.0], (ne, 1))
    k = np.tile([0.0, 1.0], (ne, 1))
    Gd, Cd, Dd = discrete_grad(q), discrete_curl(q), discrete_div(q)
    KH1, _ = oracle.gram("H1", q, L, v, k)
    Mc, _ = oracle.gram("HCURL", q, L, v, m)
    Kc, _ = oracle.gram("HCURL", q, L, v, k)
    Md, _ = oracle.gram("HDIV", q, L, v, m)
    Kd, _ = oracle.gram("HDIV", q, L, v, k)
    Ml, _ = oracle.gram("L2", q, L, v, m)
    for e in range(ne):
        assert _rel_fro(KH1[e], Gd.T @ Mc[e] @ Gd) < 1e-13
        assert _rel_fro(Kc[e], Cd.T @ Md[e] @ Cd) < 1e-13
        assert _rel_fro(Kd[e], Dd.T @ Ml[e] @ Dd) < 1e-13


def test_mixed_b_curl_of_gradient_vanishes():
    """(u, curl grad phi) = 0 for every map: Gd^T B_curl = 0 (curl o grad = 0, Eq. 2.1)."""
    q, p = 3, 2
    v = meshgen.jittered_grid(2, seed=6, jitter=0.3)[:3]
    B, _ = oracle.mixed_b(q, p, q + 2, v, split=True)
    Gd = discrete_grad(q)
    for e in range(v.shape[0]):
        assert np.abs(Gd.T @ B[e, 1]).max() < 1e-13 * np.abs(B[e, 1]).max()
        assert np.abs(Gd.T @ B[e, 0]).max() > 1e-3 * np.abs(B[e, 0]).max()


# ------------------------------------------------------------------ trilinear maps

def test_h1_coordinate_functions_on_trilinear_elements():
    """x_i = sum_v x_v[i] L_v1 L_v2 L_v3 lies in the H1 space (q >= 1); with the derivative
    Gram K, c_i^T K c_j = int grad x_i . grad x_j = delta_ij vol(K): pins the J^-T of the
    gradient and |J| on genuinely trilinear elements (the integrand is |J|, exact)."""
    q = 2
    v = meshgen.jittered_grid(2, seed=9, jitter=0.3)
    ne = v.shape[0]
    K, _ = oracle.gram("H1", q, q + 2, v, np.tile([0.0, 1.0], (ne, 1)))
    M, _ = oracle.gram("H1", 1, 3, v, np.tile([1.0, 0.0], (ne, 1)))
    for e in range(ne):
        vol = M[e].sum()
        C = np.zeros((oracle.dim("H1", q), 3))
        for vtx in range(8):
            c = meshgen.CORNERS[vtx]
            C[c[0] + (q + 1) * (c[1] + (q + 1) * c[2]), :] = v[e, vtx]
        assert np.allclose(C.T @ K[e] @ C, vol * np.eye(3), atol=1e-14, rtol=0)


@pytest.mark.parametrize("space", ["L2", "H1", "HDIV", "HCURL"])
def test_gram_symmetric_positive_definite(space):
    """Gram matrices of a basis (Eq. 2.13) are symmetric positive definite."""
    v = meshgen.jittered_grid(2, seed=1)
    G, bad = oracle.gram(space, 3, 5, v, np.tile([1.0, 0.7], (8, 1)))
    assert bad == -1
    assert np.array_equal(G, G.transpose(0, 2, 1))
    for e in range(8):
        np.linalg.cholesky(G[e])


def test_degenerate_element_flagged():
    """|J| <= 0 at a quadrature point: the element is NaN and reported (design choice for
    a diffeomorphic map, Sec. 2.2)."""
    v = meshgen.jittered_grid(2, seed=1)
    bad_v = v.copy()
    bad_v[3] = bad_v[3][[1, 0, 3, 2, 5, 4, 7, 6]]          # mirror: inverted orientation
    G, bad = oracle.gram("H1", 2, 4, bad_v)
    assert bad == 3
    assert np.all(np.isnan(G[3])) and np.all(np.isfinite(G[[0, 1, 2, 4]]))


# ------------------------------------------------------------------ ultraweak acoustics

@pytest.mark.parametrize("q", [1, 2, 3])
def test_acoustic_cross_exact_and_geometry_free(q):
    """Eq. 3.18: -(div v, q) + (v, grad q) computed in physical variables equals the
    master-cube value on every element (the H(div) and H1 Piola maps cancel), pinned
    against exact rational 1D integrals; trilinear elements included."""
    ex = _frac_matrix_to_float(exact.acoustic_cross(q))
    ident = meshgen.reference_cube()
    tri = meshgen.jittered_grid(2, seed=7, jitter=0.3)[:3]
    X, bad = oracle.acoustic_cross(q, q + 2, np.concatenate([ident, tri]))
    assert bad == -1
    for e in range(X.shape[0]):
        assert _rel_fro(X[e], ex) < 1e-13


@pytest.mark.parametrize("q", [2, 3])
def test_acoustic_cross_boundary_form(q):
    """div(q v) = q div v + v . grad q: with (div v_I, q_J) = sum_N Dd[N, I] (w_N, q_J) on
    the master cube (div^ H(div) lies in L2 through the pinned Dd; the Piola maps cancel),
    X + 2 Dd^T M = (div v, q) + (v, grad q) = <v.n, q> on the boundary, which vanishes for
    every H(div) function with v.n = 0 there (chi_i, i >= 2, in its own direction) and not
    for the others; M[N, J] = int w^_N q^_J exactly."""
    v = meshgen.jittered_grid(2, seed=8, jitter=0.3)[:2]
    X, _ = oracle.acoustic_cross(q, q + 2, v)
    Dd = discrete_div(q)
    lw, hq = exact.dofs("L2", q), exact.dofs("H1", q)
    M = np.array([[float(exact._prod(kn, nn, kj, jj)) for _, _, jj, kj in hq] for _, _, nn, kn in lw])
    bnd = X + 2.0 * (Dd.T @ M)[None]
    scale = np.abs(bnd).max()
    for I, a, ir, _ in exact.dofs("HDIV", q):
        row = np.abs(bnd[:, I, :]).max()
        if ir[a] >= 2:
            assert row < 1e-13 * scale
        else:
            assert row > 1e-3 * scale


@pytest.mark.parametrize("q,p", [(1, 1), (2, 1), (3, 2)])
def test_affine_acoustic_b_equals_exact_rational(q, p):
    """Eq. 3.16 on a parallelepiped with a full Jacobian: both parts (without i*omega and
    the coefficient of i*omega) equal their exact rational values."""
    Jf = np.array([[float(x) for x in r] for r in _J_RAT])
    verts = meshgen.affine_from_matrix(Jf, origin=(0.25, -0.5, 0.125))
    B, bad = oracle.acoustic_b(q, p, q + 1, verts)
    assert bad == -1
    B0, B1 = exact.affine_acoustic_b(q, p, _J_RAT)
    assert _rel_fro(B[0, 0], _frac_matrix_to_float(B0)) < 1e-14
    assert _rel_fro(B[0, 1], _frac_matrix_to_float(B1)) < 1e-14


def test_acoustic_b_grad_block_matches_mixed_b_on_trilinear_maps():
    """-(u, grad q_I) = -sum_K Gd[K, I] (u, psi_K) for every map (grad^ H1 lies in H(curl)
    through Gd): the (H1, (L2)^3) block of part 0 equals -Gd^T times the mass part of the
    (separately pinned) mixed stiffness; the (H1, L2) block of part 1 is geometry-free."""
    q, p = 3, 2
    v = meshgen.jittered_grid(2, seed=9, jitter=0.3)[:3]
    B, _ = oracle.acoustic_b(q, p, q + 2, v)
    M, _ = oracle.mixed_b(q, p, q + 2, v, split=True)
    Gd = discrete_grad(q)
    nh, npp = oracle.dim("H1", q), p ** 3
    ex_qp = _frac_matrix_to_float(exact.affine_acoustic_b(q, p, [[1, 0, 0], [0, 1, 0], [0, 0, 1]])[1])[:nh, :npp]
    for e in range(v.shape[0]):
        assert _rel_fro(B[e, 0, :nh, npp:], -Gd.T @ M[e, 0]) < 1e-13
        assert _rel_fro(B[e, 1, :nh, :npp], ex_qp) < 1e-13
        assert np.abs(B[e, 0, :nh, :npp]).max() == 0.0 and np.abs(B[e, 1, nh:, :npp]).max() == 0.0
