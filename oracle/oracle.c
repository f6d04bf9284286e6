/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct FP64 CPU integrator for the element matrices of
 * Mora & Demkowicz, "Fast integration of DPG matrices based on tensorization"
 * (arXiv 1711.00984).  It is the conventional algorithm of the paper (Algorithms 1, 4,
 * 6 and 8): at every tensor Gauss point it evaluates every 3D shape function, maps it
 * to the physical element with the Piola maps of Eqs. 2.3-2.6, and accumulates the
 * O(n^2) pairs of the inner product.  No sum factorization, no metric tensors D and C
 * (Eqs. 2.32, 2.50): physical fields are formed explicitly and dotted, which keeps this
 * code independent of the shortcuts the fast path relies on.
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark may load this
 * file.  It shares no code, header or table with the CUDA library.
 *
 * Conventions (the paper leaves these open; each reading is listed in the design notes):
 *   - element map: trilinear from 8 vertices, vertex v = v1 + 2 v2 + 4 v3 at corner
 *     (v1, v2, v3) of the master cube (0,1)^3 (Sec. 2.2; map itself unspecified);
 *   - quadrature: L-point Gauss-Legendre rule on (0,1) in every direction (Eqs. 2.23-2.26);
 *   - coefficients (c0, c1) weight the mass and derivative terms of each inner product;
 *   - output: dense n x n row-major per element, both triangles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_H1 = 1, OR_HCURL = 2, OR_HDIV = 3, OR_L2 = 4, OR_B = 5 };

/* ------------------------------------------------------------------------------------
 * 1D polynomials on [0,1]
 * ---------------------------------------------------------------------------------- */

/* Shifted Legendre P_0..P_{n-1} at x, Eqs. 2.91-2.93. */
static void legendre(int n, double x, double *P) {
    if (n <= 0) return;
    P[0] = 1.0;
    if (n == 1) return;
    P[1] = 2.0 * x - 1.0;
    for (int i = 2; i < n; ++i)
        P[i] = ((2.0 * i - 1.0) * (2.0 * x - 1.0) * P[i - 1] - (i - 1.0) * P[i - 2]) / i;
}

/* Derivatives P'_0..P'_{n-1}: Eq. 2.93 differentiated term by term. */
static void legendre_deriv(int n, double x, const double *P, double *dP) {
    if (n <= 0) return;
    dP[0] = 0.0;
    if (n == 1) return;
    dP[1] = 2.0;
    for (int i = 2; i < n; ++i)
        dP[i] = ((2.0 * i - 1.0) * (2.0 * P[i - 1] + (2.0 * x - 1.0) * dP[i - 1])
                 - (i - 1.0) * dP[i - 2]) / i;
}

/* Integrated Legendre chi_i = L_i, i = 0..n-1, and chi'_i (Eqs. 2.97-2.101):
 * L_0 = 1 - x, L_1 = x, 2(2i-1) L_i = P_i - P_{i-2} (i >= 2); L'_0 = -1, L'_i = P_{i-1}. */
static void int_legendre(int n, double x, double *Lv, double *dL) {
    double P[64];
    legendre(n > 1 ? n : 1, x, P);
    for (int i = 0; i < n; ++i) {
        if (i == 0) { Lv[0] = 1.0 - x; dL[0] = -1.0; }
        else if (i == 1) { Lv[1] = x; dL[1] = 1.0; }
        else { Lv[i] = (P[i] - P[i - 2]) / (2.0 * (2.0 * i - 1.0)); dL[i] = P[i - 1]; }
    }
}

/* Exported for the pins: values of P, P', L, L' at x (arrays of n). */
void oracle_1d(int n, double x, double *P, double *dP, double *Lv, double *dL) {
    double Pt[64];
    legendre(n, x, Pt);
    if (P) memcpy(P, Pt, sizeof(double) * n);
    if (dP) legendre_deriv(n, x, Pt, dP);
    if (Lv || dL) {
        double a[64], b[64];
        int_legendre(n, x, a, b);
        if (Lv) memcpy(Lv, a, sizeof(double) * n);
        if (dL) memcpy(dL, b, sizeof(double) * n);
    }
}

/* Gauss-Legendre rule with L points on (0,1) (Eq. 2.23: exact to degree 2L-1).
 * Newton's method on the shifted P_L of Eq. 2.93, in long double; weights
 * w = 1 / (x (1-x) P_L'(x)^2).  Nodes in increasing order.  Returns 0 on success. */
int oracle_gauss(int L, double *x, double *w) {
    if (L < 1 || L > 60) return -1;
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < L; ++k) {
        long double t = cosl(pi * (k + 0.75L) / (L + 0.5L)); /* root guess on [-1,1] */
        long double xi = (1.0L - t) / 2.0L;
        long double P = 0, dP = 0;
        for (int it = 0; it < 200; ++it) {
            long double p0 = 1.0L, p1 = 2.0L * xi - 1.0L, d0 = 0.0L, d1 = 2.0L;
            if (L == 1) { P = p1; dP = d1; }
            else {
                for (int i = 2; i <= L; ++i) {
                    long double p2 = ((2.0L * i - 1.0L) * (2.0L * xi - 1.0L) * p1 - (i - 1.0L) * p0) / i;
                    long double d2 = ((2.0L * i - 1.0L) * (2.0L * p1 + (2.0L * xi - 1.0L) * d1)
                                      - (i - 1.0L) * d0) / i;
                    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
                }
                P = p1; dP = d1;
            }
            long double dx = P / dP;
            xi -= dx;
            if (fabsl(dx) < 1e-30L) break;
        }
        /* final derivative at the converged node */
        {
            long double p0 = 1.0L, p1 = 2.0L * xi - 1.0L, d0 = 0.0L, d1 = 2.0L;
            for (int i = 2; i <= L; ++i) {
                long double p2 = ((2.0L * i - 1.0L) * (2.0L * xi - 1.0L) * p1 - (i - 1.0L) * p0) / i;
                long double d2 = ((2.0L * i - 1.0L) * (2.0L * p1 + (2.0L * xi - 1.0L) * d1)
                                  - (i - 1.0L) * d0) / i;
                p0 = p1; p1 = p2; d0 = d1; d1 = d2;
            }
            dP = d1;
        }
        x[k] = (double)xi;
        w[k] = (double)(1.0L / (xi * (1.0L - xi) * dP * dP));
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Geometry: trilinear element map (Eq. 2.2, map of Sec. 2.2 taken trilinear)
 * ---------------------------------------------------------------------------------- */

/* J[i][d] = d x_i / d xi_d at xi; returns det J by cofactor expansion. */
static double trilinear_jacobian(const double *verts /*[8][3]*/, const double *xi, double J[3][3]) {
    for (int i = 0; i < 3; ++i) for (int d = 0; d < 3; ++d) J[i][d] = 0.0;
    for (int v = 0; v < 8; ++v) {
        int c[3] = { v & 1, (v >> 1) & 1, (v >> 2) & 1 };
        double l[3], dl[3];
        for (int d = 0; d < 3; ++d) { l[d] = c[d] ? xi[d] : 1.0 - xi[d]; dl[d] = c[d] ? 1.0 : -1.0; }
        double g[3] = { dl[0] * l[1] * l[2], l[0] * dl[1] * l[2], l[0] * l[1] * dl[2] };
        for (int i = 0; i < 3; ++i) for (int d = 0; d < 3; ++d) J[i][d] += verts[3 * v + i] * g[d];
    }
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Exported for the pins: x(xi), J, det J. */
double oracle_geometry(const double *verts, const double *xi, double *x, double *J9) {
    double J[3][3];
    double det = trilinear_jacobian(verts, xi, J);
    if (x) {
        for (int i = 0; i < 3; ++i) x[i] = 0.0;
        for (int v = 0; v < 8; ++v) {
            int c[3] = { v & 1, (v >> 1) & 1, (v >> 2) & 1 };
            double s = 1.0;
            for (int d = 0; d < 3; ++d) s *= c[d] ? xi[d] : 1.0 - xi[d];
            for (int i = 0; i < 3; ++i) x[i] += s * verts[3 * v + i];
        }
    }
    if (J9) for (int i = 0; i < 3; ++i) for (int d = 0; d < 3; ++d) J9[3 * i + d] = J[i][d];
    return det;
}

static void inverse3(const double J[3][3], double det, double Ji[3][3]) {
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* ------------------------------------------------------------------------------------
 * 3D shape functions on the master cube (Eqs. 2.17, 2.33, 2.51-2.53, 2.69-2.71)
 * ---------------------------------------------------------------------------------- */

/* Per-direction 1D factor kind of a 3D shape function: 'W' = chi (L_i), 'Y' = nu (P_i). */
typedef struct { int comp; int n[3]; char kind[3]; int offset; } comp_t;

/* Component layout of each space at order q (trial order p for the vector-L2 trial). */
static int space_layout(int space, int q, int p, comp_t comps[3]) {
    int nc = 0;
    switch (space) {
    case OR_H1:   /* W^q = Q^{q,q,q}, I = i1 + (q+1) i2 + (q+1)^2 i3 */
        comps[0] = (comp_t){ 0, { q + 1, q + 1, q + 1 }, { 'W', 'W', 'W' }, 0 }; nc = 1; break;
    case OR_L2:   /* Y^q = Q^{q-1,q-1,q-1}, nu_i = P_i, I = i1 + q i2 + q^2 i3 */
        comps[0] = (comp_t){ 0, { q, q, q }, { 'Y', 'Y', 'Y' }, 0 }; nc = 1; break;
    case OR_HDIV: /* component a: chi in direction a, nu elsewhere (Eq. 2.52), index Eq. 2.53 */
    case OR_HCURL:/* component a: nu in direction a, chi elsewhere (Eq. 2.70), index Eq. 2.71 */
    {
        int off = 0;
        for (int a = 0; a < 3; ++a) {
            comp_t c; c.comp = a; c.offset = off;
            for (int d = 0; d < 3; ++d) {
                int same = (d == a);
                if (space == OR_HDIV) { c.n[d] = same ? q + 1 : q; c.kind[d] = same ? 'W' : 'Y'; }
                else                  { c.n[d] = same ? q : q + 1; c.kind[d] = same ? 'Y' : 'W'; }
            }
            comps[a] = c; off += c.n[0] * c.n[1] * c.n[2];
        }
        nc = 3; break;
    }
    case -OR_B:   /* vector-L2 trial of order p: each component P_k1 P_k2 P_k3 e_c */
    {
        for (int c = 0; c < 3; ++c)
            comps[c] = (comp_t){ c, { p, p, p }, { 'Y', 'Y', 'Y' }, c * p * p * p };
        nc = 3; break;
    }
    default: return 0;
    }
    return nc;
}

static int64_t space_dim(int space, int q, int p) {
    comp_t c[3]; int nc = space_layout(space, q, p, c);
    int64_t n = 0;
    for (int k = 0; k < nc; ++k) n += (int64_t)c[k].n[0] * c[k].n[1] * c[k].n[2];
    return n;
}

int64_t oracle_dim(int space, int q, int p) {
    if (space == OR_B) return space_dim(OR_HCURL, q, 0);
    return space_dim(space, q, p);
}

/* Evaluate every shape function of a space at xi on the master cube.
 *   val[I][c]   : value of component c (c = 0 only for scalar spaces)
 *   der[I][c][d]: d/dxi_d of component c
 * Scalar spaces fill component 0 only; vector spaces have a single non-zero component. */
static void shape3(int space, int q, int p, const double *xi, double *val, double *der) {
    comp_t comps[3];
    int nc = space_layout(space, q, p, comps);
    int nmax = (q > p ? q : p) + 2;
    double Wv[3][64], Wd[3][64], Yv[3][64], Yd[3][64];
    for (int d = 0; d < 3; ++d) {
        int_legendre(nmax, xi[d], Wv[d], Wd[d]);
        legendre(nmax, xi[d], Yv[d]);
        legendre_deriv(nmax, xi[d], Yv[d], Yd[d]);
    }
    for (int k = 0; k < nc; ++k) {
        const comp_t *c = &comps[k];
        for (int i3 = 0; i3 < c->n[2]; ++i3)
        for (int i2 = 0; i2 < c->n[1]; ++i2)
        for (int i1 = 0; i1 < c->n[0]; ++i1) {
            int idx[3] = { i1, i2, i3 };
            int64_t I = c->offset + i1 + (int64_t)c->n[0] * (i2 + (int64_t)c->n[1] * i3);
            double f[3], df[3];
            for (int d = 0; d < 3; ++d) {
                if (c->kind[d] == 'W') { f[d] = Wv[d][idx[d]]; df[d] = Wd[d][idx[d]]; }
                else                   { f[d] = Yv[d][idx[d]]; df[d] = Yd[d][idx[d]]; }
            }
            double *v = val + 3 * I, *g = der + 9 * I;
            for (int cc = 0; cc < 3; ++cc) { v[cc] = 0.0; for (int d = 0; d < 3; ++d) g[3 * cc + d] = 0.0; }
            v[c->comp] = f[0] * f[1] * f[2];
            g[3 * c->comp + 0] = df[0] * f[1] * f[2];
            g[3 * c->comp + 1] = f[0] * df[1] * f[2];
            g[3 * c->comp + 2] = f[0] * f[1] * df[2];
        }
    }
}

/* Reference-element differential operator of each space, from the component derivatives:
 *   H1   : grad (Eq. 2.30)                      -> 3 values
 *   HCURL: curl (Eq. 2.67)                      -> 3 values
 *   HDIV : div  (Eq. 2.48, with the d3 V3 term) -> 1 value
 *   L2   : none. */
static void ref_operator(int space, const double *v, const double *g, double *out) {
    (void)v;
    if (space == OR_H1) { out[0] = g[0]; out[1] = g[1]; out[2] = g[2]; }
    else if (space == OR_HCURL) {
        /* g[3*c + d] = d_d F_c */
        out[0] = g[3 * 2 + 1] - g[3 * 1 + 2];
        out[1] = g[3 * 0 + 2] - g[3 * 2 + 0];
        out[2] = g[3 * 1 + 0] - g[3 * 0 + 1];
    } else if (space == OR_HDIV) {
        out[0] = g[3 * 0 + 0] + g[3 * 1 + 1] + g[3 * 2 + 2];
    }
}

/* Exported for the pins: reference values (n x 3) and reference operator (n x 3) of a
 * space at xi (for OR_B the vector-L2 trial space of order p). */
int oracle_shape(int space, int q, int p, const double *xi, double *val, double *op) {
    int sp = space == OR_B ? -OR_B : space;
    int64_t n = space_dim(sp, q, p);
    if (n <= 0) return -1;
    double *der = (double *)malloc(sizeof(double) * 9 * n);
    double *v = (double *)malloc(sizeof(double) * 3 * n);
    if (!der || !v) { free(der); free(v); return -2; }
    shape3(sp, q, p, xi, v, der);
    for (int64_t I = 0; I < n; ++I) {
        if (val) for (int c = 0; c < 3; ++c) val[3 * I + c] = v[3 * I + c];
        if (op) { double o[3] = { 0, 0, 0 }; ref_operator(space, v + 3 * I, der + 9 * I, o);
                  for (int c = 0; c < 3; ++c) op[3 * I + c] = o[c]; }
    }
    free(der); free(v);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Conventional integration (Algorithms 1, 4, 6, 8 with the Piola maps of Eqs. 2.3-2.6)
 * ---------------------------------------------------------------------------------- */

/* Physical fields of every shape function at one point.
 *   phys0[I][3]: the mapped function  (H1: u, 1 entry; L2: q; HCURL: E = J^-T psi;
 *                                      HDIV: V = J theta / |J|)
 *   phys1[I][3]: the mapped operator  (H1: grad u = J^-T grad^ u (Eq. 2.29 by the chain
 *                rule); HCURL: curl E = J curl^ psi / |J|; HDIV: div V = div^ theta / |J|) */
static void map_to_physical(int space, int64_t n, const double *val, const double *der,
                            const double J[3][3], double det, const double Ji[3][3],
                            double *phys0, double *phys1) {
    for (int64_t I = 0; I < n; ++I) {
        const double *v = val + 3 * I, *g = der + 9 * I;
        double *a = phys0 + 3 * I, *b = phys1 + 3 * I;
        double op[3] = { 0, 0, 0 };
        ref_operator(space == -OR_B ? OR_L2 : space, v, g, op);
        for (int c = 0; c < 3; ++c) { a[c] = 0.0; b[c] = 0.0; }
        switch (space) {
        case OR_H1:
            a[0] = v[0];                                          /* T^grad, Eq. 2.3 */
            for (int i = 0; i < 3; ++i)                           /* J^-T grad^ u */
                for (int k = 0; k < 3; ++k) b[i] += Ji[k][i] * op[k];
            break;
        case OR_L2:
            a[0] = v[0] / det;                                    /* T, Eq. 2.6 */
            break;
        case OR_HCURL:
            for (int i = 0; i < 3; ++i)                           /* T^curl, Eq. 2.4 */
                for (int k = 0; k < 3; ++k) a[i] += Ji[k][i] * v[k];
            for (int i = 0; i < 3; ++i)                           /* curl E = T^div curl^ */
                for (int k = 0; k < 3; ++k) b[i] += J[i][k] * op[k] / det;
            break;
        case OR_HDIV:
            for (int i = 0; i < 3; ++i)                           /* T^div, Eq. 2.5 */
                for (int k = 0; k < 3; ++k) a[i] += J[i][k] * v[k] / det;
            b[0] = op[0] / det;                                   /* div V = T div^ */
            break;
        case -OR_B:                                               /* vector L2: T per comp. */
            for (int c = 0; c < 3; ++c) a[c] = v[c] / det;
            break;
        }
    }
}

static int ncomp_value(int space) { return (space == OR_H1 || space == OR_L2) ? 1 : 3; }
static int ncomp_op(int space) { return space == OR_HDIV ? 1 : (space == OR_L2 ? 0 : 3); }

/* Gram matrices: G_IJ = sum_lmn w_lmn |J| [c0 (phys0_I . phys0_J) + c1 (phys1_I . phys1_J)]
 * (Eqs. 2.16, 2.31, 2.49, 2.68 before the reduction to master-element metrics).
 * verts: [n_elem][8][3]; coeffs: [n_elem][2] or NULL for (1,1); out: [n_elem][n][n].
 * Returns the index of the first element with det J <= 0 at a point + 1 (element filled
 * with NaN), or 0. */
int64_t oracle_gram(int space, int q, int L, int64_t n_elem, const double *verts,
                    const double *coeffs, double *out, int nthreads) {
    if (space < OR_H1 || space > OR_L2 || q < 1 || L < 1) return -1;
    int64_t n = space_dim(space, q, 0);
    double zeta[64], wq[64];
    if (oracle_gauss(L, zeta, wq) != 0) return -1;
    int64_t first_bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel
    {
        double *val = (double *)malloc(sizeof(double) * 3 * n);
        double *der = (double *)malloc(sizeof(double) * 9 * n);
        double *p0 = (double *)malloc(sizeof(double) * 3 * n);
        double *p1 = (double *)malloc(sizeof(double) * 3 * n);
        int n0 = ncomp_value(space), n1 = ncomp_op(space);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_elem; ++e) {
            const double *ve = verts + 24 * e;
            double c0 = coeffs ? coeffs[2 * e] : 1.0, c1 = coeffs ? coeffs[2 * e + 1] : 1.0;
            double *G = out + e * n * n;
            memset(G, 0, sizeof(double) * n * n);
            int bad = 0;
            for (int l = 0; l < L && !bad; ++l)
            for (int m = 0; m < L && !bad; ++m)
            for (int k = 0; k < L && !bad; ++k) {
                double xi[3] = { zeta[l], zeta[m], zeta[k] };
                double w = wq[l] * wq[m] * wq[k];
                double J[3][3], Ji[3][3];
                double det = trilinear_jacobian(ve, xi, J);
                if (!(det > 0.0) || !isfinite(det)) { bad = 1; break; }
                inverse3(J, det, Ji);
                shape3(space, q, 0, xi, val, der);
                map_to_physical(space, n, val, der, J, det, Ji, p0, p1);
                double s0 = c0 * w * det, s1 = c1 * w * det;
                for (int64_t I = 0; I < n; ++I) {             /* lower triangle J <= I */
                    const double *a0 = p0 + 3 * I, *a1 = p1 + 3 * I;
                    double *row = G + I * n;
                    for (int64_t Jd = 0; Jd <= I; ++Jd) {
                        const double *b0 = p0 + 3 * Jd, *b1 = p1 + 3 * Jd;
                        double t0 = 0.0, t1 = 0.0;
                        for (int c = 0; c < n0; ++c) t0 += a0[c] * b0[c];
                        for (int c = 0; c < n1; ++c) t1 += a1[c] * b1[c];
                        row[Jd] += s0 * t0 + s1 * t1;
                    }
                }
            }
            if (bad) {
                for (int64_t i = 0; i < n * n; ++i) G[i] = NAN;
                #pragma omp critical
                { if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1; }
                continue;
            }
            for (int64_t I = 0; I < n; ++I)                   /* mirror (fillsymmetric) */
                for (int64_t Jd = I + 1; Jd < n; ++Jd) G[I * n + Jd] = G[Jd * n + I];
        }
        free(val); free(der); free(p0); free(p1);
    }
    return first_bad;
}

/* Polynomial source of total degree <= 2 in the physical coordinates: component c is
 * f_c(x) = sum_k coef[10 c + k] m_k(x) with the monomials
 * m = (1, x1, x2, x3, x1^2, x2^2, x3^2, x1 x2, x1 x3, x2 x3). */
static double source_value(const double *coef, int c, const double *x) {
    const double m[10] = { 1.0, x[0], x[1], x[2], x[0] * x[0], x[1] * x[1], x[2] * x[2],
                           x[0] * x[1], x[0] * x[2], x[1] * x[2] };
    double f = 0.0;
    for (int k = 0; k < 10; ++k) f += coef[10 * c + k] * m[k];
    return f;
}

/* Load vector of the test space (the right-hand side l_I = ell(v_I) of the DPG system,
 * Sec. 3, Eq. 3.2): l_I = (f, v_I)_K = sum_lmn w_lmn |J| f(x) . phys0_I with the physical
 * test functions of map_to_physical (Eqs. 2.3-2.6); f is scalar for H1 and L2 (coef[10]),
 * a vector for H(curl) and H(div) (coef[30]).  verts: [n_elem][8][3]; out: [n_elem][n].
 * Returns the index of the first element with det J <= 0 at a point + 1 (NaN-filled), or 0. */
int64_t oracle_load(int space, int q, int L, int64_t n_elem, const double *verts, const double *coef,
                    double *out, int nthreads) {
    if (space < OR_H1 || space > OR_L2 || q < 1 || L < 1 || !coef) return -1;
    int64_t n = space_dim(space, q, 0);
    double zeta[64], wq[64];
    if (oracle_gauss(L, zeta, wq) != 0) return -1;
    const int nc = ncomp_value(space);
    int64_t first_bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel
    {
        double *val = (double *)malloc(sizeof(double) * 3 * n);
        double *der = (double *)malloc(sizeof(double) * 9 * n);
        double *p0 = (double *)malloc(sizeof(double) * 3 * n);
        double *p1 = (double *)malloc(sizeof(double) * 3 * n);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_elem; ++e) {
            const double *ve = verts + 24 * e;
            double *l_e = out + e * n;
            memset(l_e, 0, sizeof(double) * n);
            int bad = 0;
            for (int l = 0; l < L && !bad; ++l)
            for (int m = 0; m < L && !bad; ++m)
            for (int k = 0; k < L && !bad; ++k) {
                double xi[3] = { zeta[l], zeta[m], zeta[k] };
                double x[3], J9[9];
                double det = oracle_geometry(ve, xi, x, J9);
                if (!(det > 0.0) || !isfinite(det)) { bad = 1; break; }
                double J[3][3], Ji[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int d = 0; d < 3; ++d) J[i][d] = J9[3 * i + d];
                inverse3(J, det, Ji);
                shape3(space, q, 0, xi, val, der);
                map_to_physical(space, n, val, der, J, det, Ji, p0, p1);
                double f[3];
                for (int c = 0; c < nc; ++c) f[c] = source_value(coef, c, x);
                const double s = wq[l] * wq[m] * wq[k] * det;
                for (int64_t I = 0; I < n; ++I) {
                    double t = 0.0;
                    for (int c = 0; c < nc; ++c) t += f[c] * p0[3 * I + c];
                    l_e[I] += s * t;
                }
            }
            if (bad) {
                for (int64_t i = 0; i < n; ++i) l_e[i] = NAN;
                #pragma omp critical
                { if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1; }
            }
        }
        free(val); free(der); free(p0); free(p1);
    }
    return first_bad;
}

/* Mixed stiffness B (pattern of Eqs. 3.15-3.16 for a vector-L2 trial u of order p and an
 * H(curl) test psi of order q):  B_IK = (u_K, psi_I)_K + (u_K, curl psi_I)_K, with
 * u_K = T(P_k1 P_k2 P_k3) e_c componentwise (Eq. 2.6) and psi_I = T^curl psi^_I.
 * out: [n_elem][parts][n_test][3 p^3], parts = 1 (sum) or 2 (split: mass, curl). */
int64_t oracle_mixed_b(int q, int p, int L, int64_t n_elem, const double *verts,
                       double *out, int split, int nthreads) {
    if (q < 1 || p < 1 || p > q || L < 1) return -1;
    int64_t nt = space_dim(OR_HCURL, q, 0), nu = space_dim(-OR_B, q, p);
    double zeta[64], wq[64];
    if (oracle_gauss(L, zeta, wq) != 0) return -1;
    int parts = split ? 2 : 1;
    int64_t first_bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel
    {
        double *tv = (double *)malloc(sizeof(double) * 3 * nt), *td = (double *)malloc(sizeof(double) * 9 * nt);
        double *uv = (double *)malloc(sizeof(double) * 3 * nu), *ud = (double *)malloc(sizeof(double) * 9 * nu);
        double *E = (double *)malloc(sizeof(double) * 3 * nt), *cE = (double *)malloc(sizeof(double) * 3 * nt);
        double *u = (double *)malloc(sizeof(double) * 3 * nu), *dummy = (double *)malloc(sizeof(double) * 3 * nu);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_elem; ++e) {
            const double *ve = verts + 24 * e;
            double *Be = out + e * parts * nt * nu;
            memset(Be, 0, sizeof(double) * parts * nt * nu);
            int bad = 0;
            for (int l = 0; l < L && !bad; ++l)
            for (int m = 0; m < L && !bad; ++m)
            for (int k = 0; k < L && !bad; ++k) {
                double xi[3] = { zeta[l], zeta[m], zeta[k] };
                double w = wq[l] * wq[m] * wq[k];
                double J[3][3], Ji[3][3];
                double det = trilinear_jacobian(ve, xi, J);
                if (!(det > 0.0) || !isfinite(det)) { bad = 1; break; }
                inverse3(J, det, Ji);
                shape3(OR_HCURL, q, 0, xi, tv, td);
                map_to_physical(OR_HCURL, nt, tv, td, J, det, Ji, E, cE);
                shape3(-OR_B, q, p, xi, uv, ud);
                map_to_physical(-OR_B, nu, uv, ud, J, det, Ji, u, dummy);
                double s = w * det;
                for (int64_t I = 0; I < nt; ++I) {
                    const double *a = E + 3 * I, *b = cE + 3 * I;
                    for (int64_t K = 0; K < nu; ++K) {
                        const double *c = u + 3 * K;
                        double t0 = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
                        double t1 = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
                        if (split) { Be[I * nu + K] += s * t0; Be[nt * nu + I * nu + K] += s * t1; }
                        else Be[I * nu + K] += s * (t0 + t1);
                    }
                }
            }
            if (bad) {
                for (int64_t i = 0; i < parts * nt * nu; ++i) Be[i] = NAN;
                #pragma omp critical
                { if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1; }
            }
        }
        free(tv); free(td); free(uv); free(ud); free(E); free(cE); free(u); free(dummy);
    }
    return first_bad;
}

/* ------------------------------------------------------------------------------------
 * Ultraweak acoustics (Sec. 3.3), real arithmetic: the i*omega factors are kept apart
 * ---------------------------------------------------------------------------------- */

/* Cross terms of the adjoint graph norm (Eq. 3.18): the coefficient of i*omega in
 * -i w (div dv, q) + i w (dv, grad q), i.e.
 *   X_{IJ} = ( -(div v_I) q_J + v_I . grad q_J )_K
 * with v_I the H(div) test functions of order q (rows) and q_J the H1 test functions of
 * order q (columns), both mapped to the physical element (Eqs. 2.3, 2.5) and integrated
 * there.  out: [n_elem][dim H(div)][dim H1]. */
int64_t oracle_acoustic_cross(int q, int L, int64_t n_elem, const double *verts, double *out, int nthreads) {
    if (q < 1 || L < 1) return -1;
    int64_t nv = space_dim(OR_HDIV, q, 0), nh = space_dim(OR_H1, q, 0);
    double zeta[64], wq[64];
    if (oracle_gauss(L, zeta, wq) != 0) return -1;
    int64_t first_bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel
    {
        double *vv = (double *)malloc(sizeof(double) * 3 * nv), *vd = (double *)malloc(sizeof(double) * 9 * nv);
        double *hv = (double *)malloc(sizeof(double) * 3 * nh), *hd = (double *)malloc(sizeof(double) * 9 * nh);
        double *V = (double *)malloc(sizeof(double) * 3 * nv), *dV = (double *)malloc(sizeof(double) * 3 * nv);
        double *u = (double *)malloc(sizeof(double) * 3 * nh), *gu = (double *)malloc(sizeof(double) * 3 * nh);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_elem; ++e) {
            const double *ve = verts + 24 * e;
            double *X = out + e * nv * nh;
            memset(X, 0, sizeof(double) * nv * nh);
            int bad = 0;
            for (int l = 0; l < L && !bad; ++l)
            for (int m = 0; m < L && !bad; ++m)
            for (int k = 0; k < L && !bad; ++k) {
                double xi[3] = { zeta[l], zeta[m], zeta[k] };
                double w = wq[l] * wq[m] * wq[k];
                double J[3][3], Ji[3][3];
                double det = trilinear_jacobian(ve, xi, J);
                if (!(det > 0.0) || !isfinite(det)) { bad = 1; break; }
                inverse3(J, det, Ji);
                shape3(OR_HDIV, q, 0, xi, vv, vd);
                map_to_physical(OR_HDIV, nv, vv, vd, J, det, Ji, V, dV);
                shape3(OR_H1, q, 0, xi, hv, hd);
                map_to_physical(OR_H1, nh, hv, hd, J, det, Ji, u, gu);
                double s = w * det;
                for (int64_t I = 0; I < nv; ++I) {
                    const double *a = V + 3 * I;
                    const double dv = dV[3 * I];
                    double *row = X + I * nh;
                    for (int64_t Jd = 0; Jd < nh; ++Jd) {
                        const double *g = gu + 3 * Jd;
                        row[Jd] += s * (-dv * u[3 * Jd] + (a[0] * g[0] + a[1] * g[1] + a[2] * g[2]));
                    }
                }
            }
            if (bad) {
                for (int64_t i = 0; i < nv * nh; ++i) X[i] = NAN;
                #pragma omp critical
                { if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1; }
            }
        }
        free(vv); free(vd); free(hv); free(hd); free(V); free(dV); free(u); free(gu);
    }
    return first_bad;
}

/* Stiffness of the ultraweak acoustics formulation (Eqs. 3.14-3.16):
 *   b((p,u),(q,v)) = (i w u, v) - (p, div v) + (i w p, q) - (u, grad q)
 * with test (q, v) in H1 x H(div) of order q and trial (p, u) in L2 x (L2)^3 of order p
 * (the scalar P_k1 P_k2 P_k3 and each vector component mapped by T, Eq. 2.6).
 * Rows: the H1 test functions, then the H(div) ones; columns: the scalar L2 trial
 * functions, then the three vector components.  out: [n_elem][2][rows][cols]:
 *   part 0 (terms without i w): -(p_K, div v_I) and -(u_K, grad q_I);
 *   part 1 (coefficient of i w): (p_K, q_I) and (u_K, v_I). */
int64_t oracle_acoustic_b(int q, int p, int L, int64_t n_elem, const double *verts, double *out, int nthreads) {
    if (q < 1 || p < 1 || p > q || L < 1) return -1;
    int64_t nh = space_dim(OR_H1, q, 0), nv = space_dim(OR_HDIV, q, 0);
    int64_t np = space_dim(OR_L2, p, 0), nu = space_dim(-OR_B, q, p);
    int64_t rows = nh + nv, cols = np + nu;
    double zeta[64], wq[64];
    if (oracle_gauss(L, zeta, wq) != 0) return -1;
    int64_t first_bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel
    {
        double *hv = (double *)malloc(sizeof(double) * 3 * nh), *hd = (double *)malloc(sizeof(double) * 9 * nh);
        double *vv = (double *)malloc(sizeof(double) * 3 * nv), *vd = (double *)malloc(sizeof(double) * 9 * nv);
        double *pv = (double *)malloc(sizeof(double) * 3 * np), *pd = (double *)malloc(sizeof(double) * 9 * np);
        double *uv = (double *)malloc(sizeof(double) * 3 * nu), *ud = (double *)malloc(sizeof(double) * 9 * nu);
        double *qf = (double *)malloc(sizeof(double) * 3 * nh), *gq = (double *)malloc(sizeof(double) * 3 * nh);
        double *V = (double *)malloc(sizeof(double) * 3 * nv), *dV = (double *)malloc(sizeof(double) * 3 * nv);
        double *pf = (double *)malloc(sizeof(double) * 3 * np), *pdum = (double *)malloc(sizeof(double) * 3 * np);
        double *uf = (double *)malloc(sizeof(double) * 3 * nu), *udum = (double *)malloc(sizeof(double) * 3 * nu);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_elem; ++e) {
            const double *ve = verts + 24 * e;
            double *B0 = out + e * 2 * rows * cols, *B1 = B0 + rows * cols;
            memset(B0, 0, sizeof(double) * 2 * rows * cols);
            int bad = 0;
            for (int l = 0; l < L && !bad; ++l)
            for (int m = 0; m < L && !bad; ++m)
            for (int k = 0; k < L && !bad; ++k) {
                double xi[3] = { zeta[l], zeta[m], zeta[k] };
                double w = wq[l] * wq[m] * wq[k];
                double J[3][3], Ji[3][3];
                double det = trilinear_jacobian(ve, xi, J);
                if (!(det > 0.0) || !isfinite(det)) { bad = 1; break; }
                inverse3(J, det, Ji);
                shape3(OR_H1, q, 0, xi, hv, hd);
                map_to_physical(OR_H1, nh, hv, hd, J, det, Ji, qf, gq);
                shape3(OR_HDIV, q, 0, xi, vv, vd);
                map_to_physical(OR_HDIV, nv, vv, vd, J, det, Ji, V, dV);
                shape3(OR_L2, p, 0, xi, pv, pd);
                map_to_physical(OR_L2, np, pv, pd, J, det, Ji, pf, pdum);
                shape3(-OR_B, q, p, xi, uv, ud);
                map_to_physical(-OR_B, nu, uv, ud, J, det, Ji, uf, udum);
                double s = w * det;
                for (int64_t I = 0; I < nh; ++I) {                    /* H1 test rows */
                    const double qi = qf[3 * I], *g = gq + 3 * I;
                    double *r0 = B0 + I * cols, *r1 = B1 + I * cols;
                    for (int64_t K = 0; K < np; ++K) r1[K] += s * pf[3 * K] * qi;
                    for (int64_t K = 0; K < nu; ++K) {
                        const double *c = uf + 3 * K;
                        r0[np + K] -= s * (c[0] * g[0] + c[1] * g[1] + c[2] * g[2]);
                    }
                }
                for (int64_t I = 0; I < nv; ++I) {                    /* H(div) test rows */
                    const double *a = V + 3 * I, dv = dV[3 * I];
                    double *r0 = B0 + (nh + I) * cols, *r1 = B1 + (nh + I) * cols;
                    for (int64_t K = 0; K < np; ++K) r0[K] -= s * pf[3 * K] * dv;
                    for (int64_t K = 0; K < nu; ++K) {
                        const double *c = uf + 3 * K;
                        r1[np + K] += s * (c[0] * a[0] + c[1] * a[1] + c[2] * a[2]);
                    }
                }
            }
            if (bad) {
                for (int64_t i = 0; i < 2 * rows * cols; ++i) B0[i] = NAN;
                #pragma omp critical
                { if (first_bad == 0 || e + 1 < first_bad) first_bad = e + 1; }
            }
        }
        free(hv); free(hd); free(vv); free(vd); free(pv); free(pd); free(uv); free(ud);
        free(qf); free(gq); free(V); free(dV); free(pf); free(pdum); free(uf); free(udum);
    }
    return first_bad;
}
