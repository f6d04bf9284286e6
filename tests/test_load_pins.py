"""Pins of the oracle's load vector l_I = (f, v_I)_K (CPU, no GPU).

* Reference cube, f = 1: l_I is a product of 1D integrals, int chi_i = 1/2, 1/2, -1/6, 0, ...
  (H1) and int P_i = delta_i0 (L2), Eqs. 2.95-2.101.
* Affine element with a rational Jacobian, a degree-2 polynomial source: every entry is an
  exact rational (f(x0 + J xi) is a polynomial in xi, the Piola maps of Eqs. 2.3-2.6 have
  constant factors), computed here with ``fractions`` from the 1D families' definitions.
  The Gauss rule with L = q + 3 integrates the products exactly, so the oracle must agree
  to rounding.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import components, dofs, family, inv3, det3, pintegral01, pmul
from paper_1711_00984_gb300 import meshgen

MONOMIALS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
             (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def test_load_reference_cube_f1():
    v = meshgen.reference_cube()
    c = np.zeros(10); c[0] = 1.0
    q = 4
    l, _ = oracle.load("H1", q, q + 2, v, c)
    ints = [Fraction(1, 2), Fraction(1, 2), Fraction(-1, 6)] + [Fraction(0)] * 10
    ref = [float(ints[i1] * ints[i2] * ints[i3]) for _, _, (i1, i2, i3), _ in dofs("H1", q)]
    # a sum of L^3 = 216 Gauss-weight products: rounding of a few ulp per term
    assert np.allclose(l[0], ref, rtol=0, atol=1e-14)
    l2, _ = oracle.load("L2", q, q + 2, v, c)
    assert abs(l2[0][0] - 1.0) < 1e-14 and np.abs(l2[0][1:]).max() < 1e-14


def _poly_in_xi(coef, comp, x0, J):
    """f_comp(x0 + J xi) as {(e1, e2, e3): Fraction}."""
    # each physical coordinate x_i = x0_i + sum_d J[i][d] xi_d, as a degree-1 polynomial
    lin = [{(0, 0, 0): x0[i], (1, 0, 0): J[i][0], (0, 1, 0): J[i][1], (0, 0, 1): J[i][2]} for i in range(3)]

    def mul(a, b):
        out = {}
        for ea, ca in a.items():
            for eb, cb in b.items():
                e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
                out[e] = out.get(e, Fraction(0)) + ca * cb
        return out
    res = {}
    for k, (a1, a2, a3) in enumerate(MONOMIALS):
        ck = coef[10 * comp + k]
        if ck == 0:
            continue
        term = {(0, 0, 0): Fraction(1)}
        for i, pw in enumerate((a1, a2, a3)):
            for _ in range(pw):
                term = mul(term, lin[i])
        for e, cv in term.items():
            res[e] = res.get(e, Fraction(0)) + ck * cv
    return res


def _int_xi(poly, kinds, idx):
    """int over the master cube of poly(xi) * prod_d family(kinds[d], idx[d])(xi_d)."""
    s = Fraction(0)
    for (e1, e2, e3), cv in poly.items():
        p = cv
        for d, e in enumerate((e1, e2, e3)):
            mono = tuple([Fraction(0)] * e + [Fraction(1)])
            p *= pintegral01(pmul(mono, family(kinds[d], idx[d])))
        s += p
    return s


def exact_load(space, q, x0, J, coef):
    det = det3(J)
    Ji = inv3(J)
    nc = 1 if space in ("H1", "L2") else 3
    f_xi = [_poly_in_xi(coef, c, x0, J) for c in range(nc)]
    out = []
    for _, comp, idx, kinds in dofs(space, q):
        if space == "H1":                      # int f u^ |J|
            poly, scale = f_xi[0], det
        elif space == "L2":                    # int f (q^ / |J|) |J|
            poly, scale = f_xi[0], Fraction(1)
        else:
            # H(curl): f . J^-T psi^ |J| = (J^-1 f)_a psi^_a |J|; H(div): f . J theta^ = (J^T f)_a theta^_a
            M = Ji if space == "HCURL" else [[J[r][c] for r in range(3)] for c in range(3)]
            poly = {}
            for i in range(3):
                w = M[comp][i]
                for e, cv in f_xi[i].items():
                    poly[e] = poly.get(e, Fraction(0)) + w * cv
            scale = det if space == "HCURL" else Fraction(1)
        out.append(scale * _int_xi(poly, kinds, idx))
    return out


@pytest.mark.parametrize("space", ["H1", "HCURL", "HDIV", "L2"])
@pytest.mark.parametrize("q", [1, 2])
def test_load_affine_exact(space, q):
    J = [[Fraction(1, 3), Fraction(1, 10), Fraction(0)],
         [Fraction(-1, 20), Fraction(1, 4), Fraction(1, 12)],
         [Fraction(1, 15), Fraction(0), Fraction(2, 7)]]
    x0 = [Fraction(1, 5), Fraction(-1, 8), Fraction(3, 10)]
    nc = 1 if space in ("H1", "L2") else 3
    rng = np.random.default_rng(7 + q)
    coef = [Fraction(int(k), 7) for k in rng.integers(-6, 7, size=10 * nc)]
    verts = meshgen.affine_from_matrix(np.array(J, dtype=float), origin=[float(t) for t in x0])
    l, bad = oracle.load(space, q, q + 3, verts, np.array([float(c) for c in coef]))
    assert bad == -1
    ref = np.array([float(t) for t in exact_load(space, q, x0, J, coef)])
    assert np.abs(l[0] - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_load_trilinear_invariants():
    """Trilinear elements, f = 1.  L2: the |J| of Eq. 2.6 cancels, l = (1, 0, ..., 0) for
    any map (Legendre orthogonality).  H1: the 8 vertex functions sum to one, so their
    entries sum to the element volume, computed here with the 2-point Gauss rule (|J| is
    of degree 2 in each xi_d, so that rule is exact)."""
    v = meshgen.jittered_grid(2, seed=11, jitter=0.2)
    c = np.zeros(10); c[0] = 1.0
    l2, _ = oracle.load("L2", 3, 5, v, c)
    assert np.abs(l2[:, 0] - 1.0).max() < 1e-13 and np.abs(l2[:, 1:]).max() < 1e-13
    g = (1 + np.array([-1, 1]) / np.sqrt(3)) / 2
    vol = np.zeros(v.shape[0])
    for a in g:
        for b in g:
            for cc in g:
                t = np.array([a, b, cc])
                dN = np.zeros((8, 3))
                for vi, (c1, c2, c3) in enumerate(meshgen.CORNERS):
                    f = [t[d] if cd else 1 - t[d] for d, cd in enumerate((c1, c2, c3))]
                    s = [1.0 if cd else -1.0 for cd in (c1, c2, c3)]
                    dN[vi] = [s[0] * f[1] * f[2], f[0] * s[1] * f[2], f[0] * f[1] * s[2]]
                J = np.einsum("evi,vd->eid", v, dN)
                vol += np.linalg.det(J) / 8
    l1, _ = oracle.load("H1", 3, 5, v, c)
    vert = [I for I, _, idx, _ in dofs("H1", 3) if max(idx) <= 1]     # chi_0 = 1 - xi, chi_1 = xi
    assert len(vert) == 8
    assert np.abs(l1[:, vert].sum(axis=1) - vol).max() < 1e-14
