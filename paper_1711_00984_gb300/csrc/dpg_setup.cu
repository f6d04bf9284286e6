// dpg_setup.cu -- host set-up: Gauss rule, 1D tables, exact 1D integrals, and the term
// programs (blocks, terms, groups, work units) of every space.
//
// Everything here runs once per (space, q, L) in dpg_tables_init; nothing here runs per
// element.
#include "dpg_setup.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

namespace dpg {

// ---------------------------------------------------------------------------------------
// Gauss-Legendre rule on (0,1): Newton's method on the classical Legendre polynomial
// P_L(t) on [-1,1] (three-term recurrence (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}),
// P_L'(t) = L (t P_L - P_{L-1}) / (t^2 - 1), initial guesses from Tricomi's asymptotic
// form; then t -> (1 - t)/2 (ascending nodes), weights w = 1 / ((1 - t^2) P_L'(t)^2).
// The rule integrates degree <= 2L-1 exactly (Eq. 2.23).
// ---------------------------------------------------------------------------------------
void gauss_rule(int L, double *z, double *w) {
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= L; ++k) {
        double t = (1.0 - (L - 1.0) / (8.0 * L * L * L)) * std::cos(pi * (4.0 * k - 1.0) / (4.0 * L + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int n = 1; n < L; ++n) {
                double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0);
                p0 = p1; p1 = p2;
            }
            if (L == 1) { p0 = 1.0; }
            dp = L * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        double p0 = 1.0, p1 = t;
        for (int n = 1; n < L; ++n) {
            double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0);
            p0 = p1; p1 = p2;
        }
        if (L == 1) p0 = 1.0;
        dp = L * (t * p1 - p0) / (t * t - 1.0);
        z[k - 1] = 0.5 * (1.0 - t);
        w[k - 1] = 1.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Values of the three 1D kinds at x for indices 0..n-1:
//   Y_i = P_i(x) (Eqs. 2.91-2.93, written with t = 2x - 1), W_i = L_i (Eqs. 2.99-2.101),
//   D_i = L_i' (Eq. 2.98: D_0 = -1, D_i = P_{i-1}).
static void families(int n, double x, double *W, double *Dv, double *Y) {
    double P[NQ1 + 2];
    double t = 2.0 * x - 1.0;
    int np = n + 1;
    P[0] = 1.0;
    if (np > 1) P[1] = t;
    for (int i = 1; i + 1 < np; ++i) P[i + 1] = ((2.0 * i + 1.0) * t * P[i] - i * P[i - 1]) / (i + 1.0);
    for (int i = 0; i < n; ++i) {
        Y[i] = P[i];
        if (i == 0) { W[0] = 1.0 - x; Dv[0] = -1.0; }
        else if (i == 1) { W[1] = x; Dv[1] = 1.0; }
        else { W[i] = (P[i] - P[i - 2]) / (2.0 * (2.0 * i - 1.0)); Dv[i] = P[i - 1]; }
    }
}

HostTables make_tables(int q, int L) {
    HostTables t;
    t.q = q; t.L = L;
    t.zeta.assign(L, 0.0); t.w.assign(L, 0.0);
    gauss_rule(L, t.zeta.data(), t.w.data());
    // 1D values at the nodes: X[kind][i][l]
    std::vector<double> X((size_t)NKIND * NQ1 * L, 0.0);
    for (int l = 0; l < L; ++l) {
        double W[NQ1], Dv[NQ1], Y[NQ1];
        families(q + 1, t.zeta[l], W, Dv, Y);
        for (int i = 0; i <= q; ++i) {
            X[((size_t)KW * NQ1 + i) * L + l] = W[i];
            X[((size_t)KD * NQ1 + i) * L + l] = Dv[i];
            X[((size_t)KY * NQ1 + i) * L + l] = Y[i];
        }
    }
    // pair products: pp[pair][i][j][l] = X[kr][i][l] X[kc][j][l]
    t.pp.assign((size_t)NPAIR * NQ1 * NQ1 * L, 0.0);
    for (int kr = 0; kr < NKIND; ++kr)
    for (int kc = 0; kc < NKIND; ++kc)
    for (int i = 0; i <= q; ++i)
    for (int j = 0; j <= q; ++j)
    for (int l = 0; l < L; ++l)
        t.pp[(((size_t)(3 * kr + kc) * NQ1 + i) * NQ1 + j) * L + l] =
            X[((size_t)kr * NQ1 + i) * L + l] * X[((size_t)kc * NQ1 + j) * L + l];
    // exact 1D integrals F (Eq. 2.90) with a rule of q+2 points (exact to degree 2q+3)
    int LF = q + 2;
    std::vector<double> zf(LF), wf(LF);
    gauss_rule(LF, zf.data(), wf.data());
    t.F.assign((size_t)NPAIR * NQ1 * NQ1, 0.0);
    for (int l = 0; l < LF; ++l) {
        double V[NKIND][NQ1];
        families(q + 1, zf[l], V[KW], V[KD], V[KY]);
        for (int kr = 0; kr < NKIND; ++kr)
        for (int kc = 0; kc < NKIND; ++kc)
        for (int i = 0; i <= q; ++i)
        for (int j = 0; j <= q; ++j)
            t.F[((size_t)(3 * kr + kc) * NQ1 + i) * NQ1 + j] += wf[l] * V[kr][i] * V[kc][j];
    }
    // integrals of products of polynomials of degree <= 2q whose exact value is 0 come
    // out of the rule at rounding level; store them as exact zeros (orthogonality,
    // Eqs. 2.95-2.96 and Sec. 2.8.2): the affine path relies on exact zeros.
    for (size_t k = 0; k < t.F.size(); ++k)
        if (std::fabs(t.F[k]) < 1e-13) t.F[k] = 0.0;
    return t;
}

// ---------------------------------------------------------------------------------------
// Term programs
// ---------------------------------------------------------------------------------------
struct CompLayout { int n[3]; int kind[3]; int offset; };

// Component layouts (Eqs. 2.17, 2.33, 2.52-2.53, 2.70-2.71).
static int layout(int space, int q, int p, CompLayout c[4]) {
    if (space == S_H1) { c[0] = { { q + 1, q + 1, q + 1 }, { KW, KW, KW }, 0 }; return 1; }
    if (space == S_L2) { c[0] = { { q, q, q }, { KY, KY, KY }, 0 }; return 1; }
    if (space == -S_B) {           // vector-L2 trial of order p
        for (int k = 0; k < 3; ++k) c[k] = { { p, p, p }, { KY, KY, KY }, k * p * p * p };
        return 3;
    }
    if (space == -S_AB) {          // acoustics trial: scalar L2 then vector L2, order p
        for (int k = 0; k < 4; ++k) c[k] = { { p, p, p }, { KY, KY, KY }, k * p * p * p };
        return 4;
    }
    if (space == S_AB) {           // acoustics test: H1 then H(div), order q
        c[0] = { { q + 1, q + 1, q + 1 }, { KW, KW, KW }, 0 };
        layout(S_HDIV, q, 0, c + 1);
        for (int k = 1; k < 4; ++k) c[k].offset += (q + 1) * (q + 1) * (q + 1);
        return 4;
    }
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        for (int d = 0; d < 3; ++d) {
            bool same = d == a;
            if (space == S_HDIV) { c[a].n[d] = same ? q + 1 : q; c[a].kind[d] = same ? KW : KY; }
            else { c[a].n[d] = same ? q : q + 1; c[a].kind[d] = same ? KY : KW; }
        }
        c[a].offset = off;
        off += c[a].n[0] * c[a].n[1] * c[a].n[2];
    }
    return 3;
}

static int dim_of(int space, int q, int p) {
    CompLayout c[4];
    int nc = layout(space, q, p, c);
    int n = 0;
    for (int k = 0; k < nc; ++k) n += c[k].n[0] * c[k].n[1] * c[k].n[2];
    return n;
}

int64_t rows_of(int space, int q) {
    if (q < 1 || q > MAXQ) return -1;
    if (space == S_B) return dim_of(S_HCURL, q, 0);
    if (space == S_AX) return dim_of(S_HDIV, q, 0);
    if (space == S_AB) return dim_of(S_AB, q, 0);
    if (space < S_H1 || space > S_L2) return -1;
    return dim_of(space, q, 0);
}

int64_t cols_of(int space, int p, int q) {
    if (space == S_B || space == S_AB) {
        if (p < 1 || p > q || q < 1 || q > MAXQ) return -1;
        return (space == S_B ? 3LL : 4LL) * p * p * p;
    }
    if (space == S_AX) return rows_of(S_H1, q);
    return rows_of(space, q);
}

struct TermSpec { int field, sign; int kr[3], kc[3]; };

// curl^(f e_a) = grad f x e_a (Eq. 2.67 applied to Eq. 2.74): component a+1 is
// +d_{a+2} f, component a+2 is -d_{a+1} f; the derivative replaces chi by chi' (kind D)
// in that direction (Eqs. 2.73, 2.75).
static void curl_parts(int a, const int base[3], int comp[2], int sign[2], int kinds[2][3]) {
    int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    comp[0] = a1; sign[0] = +1; comp[1] = a2; sign[1] = -1;
    for (int d = 0; d < 3; ++d) {
        kinds[0][d] = (d == a2) ? KD : base[d];
        kinds[1][d] = (d == a1) ? KD : base[d];
    }
}

static void finish_block(BlockDesc &b, const std::vector<TermSpec> &ts, const int dir[3]) {
    b.nterm = (int)ts.size();
    for (int k = 0; k < 3; ++k) b.dir[k] = dir[k];
    std::map<std::pair<int, int>, int> hmap;
    std::map<int, int> gmap, p2map;
    b.nh = b.ng = b.np2 = 0;
    const int dC = dir[0], dB = dir[1];
    for (int t = 0; t < b.nterm; ++t) {
        const TermSpec &s = ts[t];
        TermDesc &d = b.term[t];
        d.field = s.field; d.sign = s.sign;
        for (int k = 0; k < 3; ++k) { d.kr[k] = s.kr[k]; d.kc[k] = s.kc[k]; }
        int p1 = 3 * s.kr[dC] + s.kc[dC], p2 = 3 * s.kr[dB] + s.kc[dB];
        auto key = std::make_pair(p1, p2);
        if (!hmap.count(key)) {
            int h = b.nh++;
            hmap[key] = h;
            if (!gmap.count(p1)) { int g = b.ng++; gmap[p1] = g; b.g_pair[g] = p1; }
            if (!p2map.count(p2)) { int s2 = b.np2++; p2map[p2] = s2; b.p2_pair[s2] = p2; }
            b.h_g[h] = gmap[p1];
            b.h_p2[h] = p2map[p2];
            b.h_pair1[h] = p1;
            b.h_pair2[h] = p2;
        }
        d.h = hmap[key];
    }
    for (int g = 0; g < MAXG; ++g) b.g_nterm[g] = b.g_nh[g] = 0;
    for (int h = 0; h < MAXH; ++h) b.h_nterm[h] = 0;
    b.nslot = 0;
    for (int t = 0; t < b.nterm; ++t) {
        const int h = b.term[t].h, g = b.h_g[h];
        b.g_terms[g][b.g_nterm[g]++] = (signed char)t;
        b.h_terms[h][b.h_nterm[h]++] = (signed char)t;
        int sl = -1;
        for (int u = 0; u < b.nslot; ++u)
            if (b.slot_field[u] == b.term[t].field) sl = u;
        if (sl < 0) { sl = b.nslot; b.slot_field[b.nslot++] = (signed char)b.term[t].field; }
        b.term_slot[t] = (signed char)sl;
    }
    for (int h = 0; h < b.nh; ++h) b.g_hs[b.h_g[h]][b.g_nh[b.h_g[h]]++] = (signed char)h;
}

// Multiply-adds of one block of the general path: per tile (iA, jA) stage A costs
// nterm L^3, stage B nh L^2 nB nB', stage C ng L (outputs of the tile); a diagonal
// block of a symmetric matrix computes tiles jA >= iA, and its iA == jA tiles count
// the upper triangle only.
static double block_fmas(const BlockDesc &b, int L) {
    const int dC = b.dir[0], dB = b.dir[1], dA = b.dir[2];
    const double mr = (double)b.nr[dC] * b.nr[dB], mc = (double)b.nc[dC] * b.nc[dB];
    double f = 0.0;
    for (int i3 = 0; i3 < b.nr[dA]; ++i3)
        for (int j3 = (b.sym == 1 ? i3 : 0); j3 < b.nc[dA]; ++j3) {
            f += (double)b.nterm * L * L * L;
            f += (double)b.nh * L * L * b.nr[dB] * b.nc[dB];
            f += (double)b.ng * L * ((b.sym == 1 && j3 == i3) ? 0.5 * mr * (mr + 1.0) : mr * mc);
        }
    return f;
}

static size_t smem_values(const BlockDesc &b, int L, int nj) {
    auto r4 = [](size_t v) { return (v + 3) & ~size_t(3); };
    const int dC = b.dir[0], dB = b.dir[1];
    size_t P1 = r4((size_t)b.ng * b.nr[dC] * b.nc[dC] * L);
    size_t P2 = r4((size_t)b.np2 * b.nr[dB] * b.nc[dB] * L);
    size_t P3 = r4((size_t)b.nterm * nj * L);
    size_t A = r4((size_t)b.nh * L * L * nj);
    size_t B = r4((size_t)b.ng * L * b.nr[dB] * b.nc[dB] * nj);
    return P1 + P2 + P3 + A + B;
}

Program make_program(int space, int q, int L, int p, bool split, const HostTables &tab, int order, int force_nj,
                     size_t smem_budget, int force_nj_sym) {
    Program pr;
    std::memset(pr.blocks, 0, sizeof(pr.blocks));
    pr.space = space; pr.q = q; pr.L = L; pr.p = p; pr.split = split;
    pr.rows = (int)rows_of(space, q);
    pr.cols = (int)cols_of(space, p, q);
    pr.parts = ((space == S_B && split) || space == S_AB) ? 2 : 1;
    pr.nfields = nfields_of(space);
    pr.nblock = 0;

    CompLayout R[4], C[4];
    const int rspace = space == S_B ? S_HCURL : (space == S_AX ? S_HDIV : space);
    const int cspace = space == S_B ? -S_B : (space == S_AX ? S_H1 : (space == S_AB ? -S_AB : space));
    int nR = layout(rspace, q, 0, R);
    int nC = layout(cspace, q, p, C);

    for (int a = 0; a < nR; ++a)
    for (int b = 0; b < nC; ++b) {
        bool symmetric = space <= S_L2 && order != ORDER_PANEL && order != ORDER_TC && order != ORDER_TCC;
        if (symmetric && b < a) continue;             // lower blocks come from mirroring
        for (int part = 0; part < pr.parts; ++part) {
            std::vector<TermSpec> ts;
            auto add = [&](int field, int sign, const int kr[3], const int kc[3]) {
                TermSpec s; s.field = field; s.sign = sign;
                for (int d = 0; d < 3; ++d) { s.kr[d] = kr[d]; s.kc[d] = kc[d]; }
                ts.push_back(s);
            };
            const int *ka = R[a].kind, *kb = C[b].kind;
            switch (space) {
            case S_L2:                                 // Eq. 2.19: nu nu nu |J|^-1
                add(0, 1, ka, kb);
                break;
            case S_H1: {                               // Eqs. 2.41-2.44 and 2.38-2.40
                add(0, 1, ka, kb);
                for (int aa = 0; aa < 3; ++aa)
                for (int bb = 0; bb < 3; ++bb) {
                    int kr[3], kc[3];
                    for (int d = 0; d < 3; ++d) { kr[d] = d == aa ? KD : KW; kc[d] = d == bb ? KD : KW; }
                    add(1 + sym_index(aa, bb), 1, kr, kc);
                }
                break;
            }
            case S_HDIV: {                             // Eqs. 2.60-2.63 and the div term 2.59
                add(sym_index(a, b), 1, ka, kb);
                int kr[3], kc[3];
                for (int d = 0; d < 3; ++d) { kr[d] = d == a ? KD : ka[d]; kc[d] = d == b ? KD : kb[d]; }
                add(6, 1, kr, kc);
                break;
            }
            case S_HCURL: {                            // Eqs. 2.76-2.84
                add(sym_index(a, b), 1, ka, kb);
                int ca[2], sa[2], kra[2][3], cb[2], sb[2], krb[2][3];
                curl_parts(a, ka, ca, sa, kra);
                curl_parts(b, kb, cb, sb, krb);
                for (int al = 0; al < 2; ++al)
                for (int be = 0; be < 2; ++be)
                    add(6 + sym_index(ca[al], cb[be]), sa[al] * sb[be], kra[al], krb[be]);
                break;
            }
            case S_AX: {                               // Eq. 3.18: -div^v^ q^ + v^ . grad^ q^
                int kr[3], kc[3];
                for (int d = 0; d < 3; ++d) { kr[d] = d == a ? KD : ka[d]; kc[d] = kb[d]; }
                add(0, -1, kr, kc);
                for (int d = 0; d < 3; ++d) { kr[d] = ka[d]; kc[d] = d == a ? KD : kb[d]; }
                add(0, 1, kr, kc);
                break;
            }
            case S_AB: {                               // Eq. 3.16, part 0 / part 1 (i omega)
                // rows: a = 0 the H1 test, a = 1..3 H(div) component a-1;
                // columns: b = 0 the scalar L2 trial, b = 1..3 vector component b-1
                const int ra = a - 1, cb = b - 1;
                int kr[3];
                if (a == 0 && b == 0) { if (part == 1) add(0, 1, ka, kb); }          // (p, q)
                else if (a == 0) {                                                  // -(u, grad q)
                    if (part == 0)
                        for (int d = 0; d < 3; ++d) {
                            for (int e = 0; e < 3; ++e) kr[e] = e == d ? KD : ka[e];
                            add(1 + 3 * d + cb, -1, kr, kb);
                        }
                } else if (b == 0) {                                                // -(p, div v)
                    if (part == 0) {
                        for (int e = 0; e < 3; ++e) kr[e] = e == ra ? KD : ka[e];
                        add(10, -1, kr, kb);
                    }
                } else if (part == 1) {                                             // (u, v)
                    add(11 + 3 * cb + ra, 1, ka, kb);
                }
                break;
            }
            case S_B: {                                // u^.J^-T psi^ + u^.J curl^psi^ / |J|
                if (part == 0 || !split) add(3 * a + b, 1, ka, kb);
                if (part == 1 || !split) {
                    int cc[2], sc[2], kr[2][3];
                    curl_parts(a, ka, cc, sc, kr);
                    for (int al = 0; al < 2; ++al) add(9 + 3 * b + cc[al], sc[al], kr[al], kb);
                }
                break;
            }
            }
            BlockDesc &bd = pr.blocks[pr.nblock++];
            for (int d = 0; d < 3; ++d) { bd.nr[d] = R[a].n[d]; bd.nc[d] = C[b].n[d]; }
            bd.row_off = R[a].offset;
            bd.col_off = C[b].offset;
            bd.base = part * pr.rows * pr.cols;
            bd.sym = symmetric ? (a == b ? 1 : 2) : 0;
            // stage order: the permutation of directions with the fewest multiply-adds
            // (ties keep the paper's order: stage A over xi_3, B over xi_2, C over xi_1);
            // ORDER_A3 keeps stage A on xi_3, ORDER_NATURAL keeps the paper's order
            static const int perms[6][3] = { { 0, 1, 2 }, { 1, 0, 2 }, { 0, 2, 1 },
                                             { 2, 0, 1 }, { 1, 2, 0 }, { 2, 1, 0 } };
            const int nperm = (order == ORDER_NATURAL || order == ORDER_PANEL || order == ORDER_TC ||
                               order == ORDER_EXTRUDED || order == ORDER_TCC)
                                  ? 1 : (order == ORDER_A3 ? 2 : 6);
            double best = 0.0; int bi = 0;
            for (int k = 0; k < nperm; ++k) {
                finish_block(bd, ts, perms[k]);
                const double f = block_fmas(bd, L);
                if (k == 0 || f < best * (1.0 - 1e-12)) { best = f; bi = k; }
            }
            finish_block(bd, ts, perms[bi]);
        }
    }

    // stage-A chunk: the largest nj whose shared memory fits the budget (FP64 general
    // kernel model, or the FP32 kernel's layout for ORDER_A3 programs)
    auto smem_bytes = [&](const BlockDesc &b, int njv) -> size_t {
        if (order == ORDER_A3) return (size_t)f32_layout(b, L, njv).total * sizeof(float);
        if (order == ORDER_PANEL) return (size_t)panel_layout(b, L, njv).total * sizeof(float);
        if (order == ORDER_TC) {
            const TcLayout t = tc_layout(b, L, njv);
            return t.ok ? (size_t)t.total : SIZE_MAX;
        }
        if (order == ORDER_NATURAL) return (size_t)aff_layout_block(b, njv).total * sizeof(double);
        if (order == ORDER_EXTRUDED) return (size_t)ext_layout(b, L, njv).total * sizeof(double);
        if (order == ORDER_TCC) {
            const TccLayout t = tcc_layout(b, L);
            return t.ok ? (size_t)t.total : SIZE_MAX;
        }
        return smem_values(b, L, njv) * sizeof(double);
    };
    // (ORDER_PANEL: the largest chunk that fits one CTA per SM; the launch takes two
    // 8-warp CTAs per SM where the chunk fits PANEL_SMEM_2CTA, else one of 16 warps)
    const size_t budget = smem_budget ? smem_budget
                                      : (order == ORDER_BEST ? 160 * 1024
                                         : (order == ORDER_PANEL ? (size_t)200 * 1024
                                         : (order == ORDER_TC ? (size_t)220 * 1024 : 110 * 1024)));
    int maxnA = 1;
    for (int k = 0; k < pr.nblock; ++k) maxnA = std::max(maxnA, pr.blocks[k].nc[pr.blocks[k].dir[2]]);
    int nj = std::min(NJMAX, maxnA);
    if (force_nj > 0) {
        nj = std::min(force_nj, nj);                       // autotuned chunk (caller checks smem)
    } else {
        for (; nj > 1; --nj) {
            size_t m = 0;
            for (int k = 0; k < pr.nblock; ++k) m = std::max(m, smem_bytes(pr.blocks[k], nj));
            if (m <= budget) break;
        }
    }
    pr.nj = nj;
    // the diagonal blocks of a symmetric matrix may take a smaller chunk (general FP64
    // kernel only: its units carry their own width)
    pr.nj_sym = (order == ORDER_BEST && force_nj_sym > 0) ? std::min(force_nj_sym, nj) : nj;
    auto njb = [&](const BlockDesc &b) { return b.sym == 1 ? pr.nj_sym : nj; };
    size_t m = 0, mb = 0;
    for (int k = 0; k < pr.nblock; ++k) {
        m = std::max(m, smem_values(pr.blocks[k], L, njb(pr.blocks[k])));
        mb = std::max(mb, smem_bytes(pr.blocks[k], njb(pr.blocks[k])));
    }
    pr.smem_values = m;
    pr.smem_bytes = mb;

    // work units (element-local): one per (block, iA, chunk of jA); algorithmic flops
    pr.units.clear();
    double fmas = 0.0;
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        const int dA = b.dir[2];
        const int nju = njb(b);
        for (int i3 = 0; i3 < b.nr[dA]; ++i3) {
            int jlo = b.sym == 1 ? i3 : 0;
            for (int j = jlo; j < b.nc[dA]; j += nju) {
                Unit u;
                u.block = (int16_t)k; u.i3 = (int16_t)i3; u.j3b = (int16_t)j;
                u.nj = (int16_t)std::min(nju, b.nc[dA] - j);
                pr.units.push_back(u);
            }
        }
        fmas += block_fmas(b, L);
    }
    pr.flops = 2.0 * fmas;

    // affine path: non-zero products of the Kronecker sums (Sec. 2.8.1)
    double aff = 0.0;
    auto Fv = [&](int pair, int i, int j) { return tab.F[((size_t)pair * NQ1 + i) * NQ1 + j]; };
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        const int dC = b.dir[0], dB = b.dir[1], dA = b.dir[2];
        for (int i3 = 0; i3 < b.nr[dA]; ++i3)
        for (int j3 = (b.sym == 1 ? i3 : 0); j3 < b.nc[dA]; ++j3) {
            // Q_g(iB, jB) = sum_{t in g} c_t F_B,t F_A,t
            std::vector<char> qnz((size_t)b.ng * b.nr[dB] * b.nc[dB], 0);
            for (int t = 0; t < b.nterm; ++t) {
                const TermDesc &d = b.term[t];
                double f3 = Fv(3 * d.kr[dA] + d.kc[dA], i3, j3);
                if (f3 == 0.0) continue;
                int g = b.h_g[d.h];
                for (int i2 = 0; i2 < b.nr[dB]; ++i2)
                for (int j2 = 0; j2 < b.nc[dB]; ++j2)
                    if (Fv(3 * d.kr[dB] + d.kc[dB], i2, j2) != 0.0) {
                        aff += 2.0;
                        qnz[((size_t)g * b.nr[dB] + i2) * b.nc[dB] + j2] = 1;
                    }
            }
            for (int g = 0; g < b.ng; ++g)
            for (int i1 = 0; i1 < b.nr[dC]; ++i1)
            for (int j1 = 0; j1 < b.nc[dC]; ++j1) {
                if (Fv(b.g_pair[g], i1, j1) == 0.0) continue;
                for (int i2 = 0; i2 < b.nr[dB]; ++i2)
                for (int j2 = 0; j2 < b.nc[dB]; ++j2)
                    if (qnz[((size_t)g * b.nr[dB] + i2) * b.nc[dB] + j2]) aff += 2.0;
            }
        }
    }
    pr.flops_affine = aff;

    // extruded-map path: per (i3, j3) tile stage A over xi_3 (2D fields), stage B over xi_2,
    // stage C by the exact 1D integrals of xi_1 (non-zero products only)
    double ext = 0.0;
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        const int dC = b.dir[0], dB = b.dir[1], dA = b.dir[2];
        const double n22 = (double)b.nr[dB] * b.nc[dB];
        double nzC = 0.0;
        for (int g = 0; g < b.ng; ++g)
            for (int i1 = 0; i1 < b.nr[dC]; ++i1)
                for (int j1 = 0; j1 < b.nc[dC]; ++j1)
                    if (Fv(b.g_pair[g], i1, j1) != 0.0) nzC += 1.0;
        double tiles = 0.0;
        for (int i3 = 0; i3 < b.nr[dA]; ++i3) tiles += b.sym == 1 ? b.nc[dA] - i3 : b.nc[dA];
        ext += 2.0 * tiles * ((double)b.nterm * L * L + (double)b.nh * n22 * L + nzC * n22);
    }
    pr.flops_extruded = ext;
    return pr;
}

// TF32 high / low parts of x: hi keeps 10 mantissa bits (rounded to nearest, ties away
// from zero), lo = x - hi is exact in FP32.
static void split_tf32(float x, float &hi, float &lo) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    std::memcpy(&hi, &u, 4);
    lo = x - hi;
}

void build_panel_tables(const Program &pr, const HostTables &tab, std::vector<float> &ctab, std::vector<int> &off) {
    ctab.clear();
    off.assign(pr.nblock, 0);
    const int L = pr.L;
    auto ppv = [&](int pair, int i, int j, int l) -> float {
        return (float)tab.pp[(((size_t)pair * NQ1 + i) * NQ1 + j) * L + l];
    };
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        const PanelLayout f = panel_layout(b, L, 1);
        off[k] = (int)ctab.size();
        std::vector<float> t((size_t)f.oA, 0.0f);
        // P1 as the B operand of stage C: per k-step ks and row n = (i1, j1 padded to
        // nt1*8), per lane column tg the values {hi(k0), hi(k0+4), lo(k0), lo(k0+4)},
        // k0 = 8 ks + tg
        auto p1 = [&](int kk, int i1, int j1) -> float {
            const int g = kk / f.lpad, l = kk % f.lpad;
            return (j1 < f.nc1 && l < L) ? ppv(b.g_pair[g], i1, j1, l) : 0.0f;
        };
        for (int ks = 0; ks < f.ks1; ++ks)
            for (int n = 0; n < f.n1p; ++n) {
                const int i1 = n / (f.nt1 * 8), j1 = n % (f.nt1 * 8);
                for (int tg = 0; tg < 4; ++tg) {
                    float *d = &t[(size_t)f.oP1 + ((size_t)ks * f.n1p + n) * 16 + tg * 4];
                    split_tf32(p1(ks * 8 + tg, i1, j1), d[0], d[2]);
                    split_tf32(p1(ks * 8 + tg + 4, i1, j1), d[1], d[3]);
                }
            }
        // P2 as the A operand of stage B: per (slot, m-tile, k-step) and lane (gid, tg) the
        // values {hi(a0..a3), lo(a0..a3)} of rows gid, gid+8 and columns tg, tg+4
        auto p2 = [&](int s2, int r, int m) -> float {
            return (r < f.n22 && m < L) ? ppv(b.p2_pair[s2], r / f.nc2, r % f.nc2, m) : 0.0f;
        };
        for (int s2 = 0; s2 < b.np2; ++s2)
            for (int mt = 0; mt < f.mtb; ++mt)
                for (int ks = 0; ks < f.ksh; ++ks)
                    for (int lane = 0; lane < 32; ++lane) {
                        const int gid = lane >> 2, tg = lane & 3;
                        const int r0 = mt * 16 + gid, m0 = ks * 8 + tg;
                        float *d = &t[(size_t)f.oP2 + (((size_t)s2 * f.mtb + mt) * f.ksh + ks) * 256 + lane * 8];
                        split_tf32(p2(s2, r0, m0), d[0], d[4]);
                        split_tf32(p2(s2, r0 + 8, m0), d[1], d[5]);
                        split_tf32(p2(s2, r0, m0 + 4), d[2], d[6]);
                        split_tf32(p2(s2, r0 + 8, m0 + 4), d[3], d[7]);
                    }
        ctab.insert(ctab.end(), t.begin(), t.end());
    }
}

void build_tc_tables(const Program &pr, const HostTables &tab, std::vector<float> &ctab, std::vector<int> &off) {
    ctab.clear();
    off.assign(pr.nblock, 0);
    const int L = pr.L;
    auto ppv = [&](int pair, int i, int j, int l) -> float {
        return (float)tab.pp[(((size_t)pair * NQ1 + i) * NQ1 + j) * L + l];
    };
    // float index of element (r, k) of a K-major canonical operand with row-group stride sbo
    auto at = [](int r, int k, int sbo) { return ((r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4) / 4; };
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        off[k] = (int)ctab.size();
        if (b.ng == 0) continue;                          // no terms: the kernel writes zeros
        const TcLayout f = tc_layout(b, L, pr.nj);
        std::vector<float> t((size_t)f.oAh / 4, 0.0f);
        // P1 (B operand of stage C): row n = i1 nc1p + j1, k = g lpad + l
        for (int n = 0; n < f.NC; ++n)
            for (int kk = 0; kk < b.ng * f.lpad; ++kk) {
                const int g = kk / f.lpad, l = kk % f.lpad, i1 = n / f.nc1p, j1 = n % f.nc1p;
                const float v = (i1 < f.nr1 && j1 < f.nc1 && l < L) ? ppv(b.g_pair[g], i1, j1, l) : 0.0f;
                const int i = at(n, kk, f.sboC);
                split_tf32(v, t[f.oP1 / 4 + i], t[(f.oP1 + f.p1b) / 4 + i]);
            }
        // P2 slots (A operand of stage B): row r = i2 nc2 + j2, k = m
        for (int s2 = 0; s2 < b.np2; ++s2)
            for (int r = 0; r < ((f.n22 + 7) & ~7); ++r)
                for (int m = 0; m < f.lpad; ++m) {
                    const float v = (r < f.n22 && m < L) ? ppv(b.p2_pair[s2], r / f.nc2, r % f.nc2, m) : 0.0f;
                    const int i = at(r, m, f.sbo2);
                    split_tf32(v, t[(f.oP2 + 2 * s2 * f.p2b) / 4 + i], t[(f.oP2 + (2 * s2 + 1) * f.p2b) / 4 + i]);
                }
        ctab.insert(ctab.end(), t.begin(), t.end());
    }
    if (ctab.empty()) ctab.push_back(0.0f);
}

void build_tcc_tables(const Program &pr, const HostTables &tab, std::vector<float> &img, std::vector<int> &off) {
    img.clear();
    off.assign(pr.nblock + 1, 0);
    const int L = pr.L;
    auto ppv = [&](int pair, int i, int j, int l) -> float {
        return (float)tab.pp[(((size_t)pair * NQ1 + i) * NQ1 + j) * L + l];
    };
    auto at = [](int r, int k, int sbo) { return ((r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4) / 4; };
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        off[k] = (int)img.size();
        const TccLayout f = tcc_layout(b, L);
        std::vector<float> t((size_t)f.oC / 4, 0.0f);
        // P1 (B operand of stage C): row n = i1 nc1 + j1, k = g lpad + l
        for (int n = 0; n < f.N; ++n)
            for (int kk = 0; kk < f.K; ++kk) {
                const int g = kk / f.lpad, l = kk % f.lpad, i1 = n / f.nc1, j1 = n % f.nc1;
                const float v = (n < f.nr1 * f.nc1 && g < b.ng && l < L) ? ppv(b.g_pair[g], i1, j1, l) : 0.0f;
                const int i = at(n, kk, f.sbo);
                split_tf32(v, t[f.oP1 / 4 + i], t[(f.oP1 + f.p1b) / 4 + i]);
            }
        // P2 (stage B factors): [slot][m][(i2, j2)] padded to n22p
        for (int s2 = 0; s2 < b.np2; ++s2)
            for (int m = 0; m < L; ++m)
                for (int ij = 0; ij < f.n22; ++ij)
                    t[f.oP2 / 4 + (s2 * L + m) * f.n22p + ij] = ppv(b.p2_pair[s2], ij / f.nc2, ij % f.nc2, m);
        img.insert(img.end(), t.begin(), t.end());
    }
    off[pr.nblock] = (int)img.size();
    if (img.empty()) img.assign(4, 0.0f);
}

template <typename T>
void build_aff_image(const Program &pr, const HostTables &tab, bool extruded, std::vector<unsigned char> &img,
                     std::vector<int> &off16) {
    img.clear();
    off16.assign(pr.nblock + 1, 0);
    const int L = pr.L;
    auto Fv = [&](int pair, int i, int j) { return (T)tab.F[((size_t)pair * NQ1 + i) * NQ1 + j]; };
    auto ppv = [&](int pair, int i, int j, int l) { return (T)tab.pp[(((size_t)pair * NQ1 + i) * NQ1 + j) * L + l]; };
    for (int k = 0; k < pr.nblock; ++k) {
        const BlockDesc &b = pr.blocks[k];
        const AffLayout a = extruded ? ext_layout(b, L, pr.nj).a : aff_layout_block(b, pr.nj);
        off16[k] = (int)(img.size() / 16);
        std::vector<unsigned char> t((size_t)a.oC * sizeof(T), 0);
        T *tv = reinterpret_cast<T *>(t.data());
        auto iat = [&](int off_values) { return reinterpret_cast<int *>(t.data() + (size_t)off_values * sizeof(T)); };
        const int n11 = b.nr[0] * b.nc[0], n22 = b.nr[1] * b.nc[1];
        // stage-C factors: the non-zero exact integrals F1_g(i1, j1), row-major order
        for (int g = 0; g < b.ng; ++g) {
            int c = 0;
            for (int i1 = 0; i1 < b.nr[0]; ++i1)
                for (int j1 = 0; j1 < b.nc[0]; ++j1) {
                    const T v = Fv(b.g_pair[g], i1, j1);
                    if (v != T(0)) {
                        tv[a.oF1V + g * n11 + c] = v;
                        iat(a.oF1I)[g * n11 + c] = i1 * a.ldt + j1;
                        ++c;
                    }
                }
            iat(a.oF1C)[g] = c;
        }
        if (!extruded)                                  // F2_t(i2, j2), exact integrals
            for (int t2 = 0; t2 < b.nterm; ++t2)
                for (int ij = 0; ij < n22; ++ij)
                    tv[a.oF2 + t2 * n22 + ij] = Fv(3 * b.term[t2].kr[1] + b.term[t2].kc[1], ij / b.nc[1], ij % b.nc[1]);
        else                                            // P2[slot][(i2, j2)][m] at the Gauss points
            for (int s2 = 0; s2 < b.np2; ++s2)
                for (int ij = 0; ij < n22; ++ij)
                    for (int m = 0; m < L; ++m)
                        tv[a.oP2 + (s2 * n22 + ij) * L + m] = ppv(b.p2_pair[s2], ij / b.nc[1], ij % b.nc[1], m);
        t.resize((t.size() + 15) & ~size_t(15), 0);
        img.insert(img.end(), t.begin(), t.end());
    }
    off16[pr.nblock] = (int)(img.size() / 16);
    if (img.empty()) img.resize(16, 0);
}
template void build_aff_image<double>(const Program &, const HostTables &, bool, std::vector<unsigned char> &,
                                      std::vector<int> &);

bool affine_diagonal(const Program &pa, const HostTables &tab, int max_terms, std::vector<double> &D) {
    D.clear();
    const BlockDesc &b0 = pa.blocks[0];
    bool diag = pa.nblock == 1 && pa.parts == 1 && b0.row_off == 0 && b0.col_off == 0 &&
                b0.nterm <= max_terms && !pa.split;
    for (int d = 0; d < 3 && diag; ++d) diag = b0.nr[d] == b0.nc[d];
    for (int t = 0; t < b0.nterm && diag; ++t)
        for (int d = 0; d < 3 && diag; ++d) {
            const TermDesc &td = b0.term[t];
            const int pair = 3 * td.kr[d] + td.kc[d], nd = b0.nr[d];
            for (int i = 0; i < nd && diag; ++i)
                for (int j = 0; j < nd && diag; ++j)
                    if (i != j && tab.F[((size_t)pair * NQ1 + i) * NQ1 + j] != 0.0) diag = false;
        }
    if (!diag) return false;
    const int n = pa.rows, n1 = b0.nr[0], n2 = b0.nr[1];
    D.assign((size_t)b0.nterm * n, 0.0);
    for (int t = 0; t < b0.nterm; ++t) {
        const TermDesc &td = b0.term[t];
        auto Fd = [&](int d, int i) { return tab.F[((size_t)(3 * td.kr[d] + td.kc[d]) * NQ1 + i) * NQ1 + i]; };
        for (int r = 0; r < n; ++r)
            D[(size_t)t * n + r] = Fd(0, r % n1) * Fd(1, (r / n1) % n2) * Fd(2, r / (n1 * n2));
    }
    return true;
}

bool build_aff_qlists(const Program &pr, const HostTables &tab, std::vector<unsigned> &ql, std::vector<int> &qo) {
    ql.clear();
    qo.assign(pr.units.size() + 1, 0);
    auto nz = [&](int pair, int i, int j) { return tab.F[((size_t)pair * NQ1 + i) * NQ1 + j] != 0.0; };
    for (size_t ui = 0; ui < pr.units.size(); ++ui) {
        const Unit &u = pr.units[ui];
        const BlockDesc &b = pr.blocks[u.block];
        const int nc2 = b.nc[1], n22 = b.nr[1] * b.nc[1];
        if (n22 > 255 || u.nj > 15 || b.ng > 15) return false;
        qo[ui] = (int)ql.size();
        for (int g = 0; g < b.ng; ++g) {
            if (b.g_nterm[g] > 12) return false;
            for (int ij2 = 0; ij2 < n22; ++ij2)
                for (int jj = 0; jj < u.nj; ++jj) {
                    unsigned m = 0;
                    for (int k2 = 0; k2 < b.g_nterm[g]; ++k2) {
                        const TermDesc &td = b.term[b.g_terms[g][k2]];
                        if (nz(3 * td.kr[1] + td.kc[1], ij2 / nc2, ij2 % nc2) &&
                            nz(3 * td.kr[2] + td.kc[2], u.i3, u.j3b + jj))
                            m |= 1u << k2;
                    }
                    if (m) ql.push_back((unsigned)ij2 | (unsigned)jj << 8 | m << 12 | (unsigned)g << 24);
                }
            while (ql.size() % 32) ql.push_back((unsigned)g << 24);   // empty entries: whole warps
        }
    }
    qo[pr.units.size()] = (int)ql.size();
    if (ql.empty()) ql.push_back(0u);
    return true;
}
template void build_aff_image<float>(const Program &, const HostTables &, bool, std::vector<unsigned char> &,
                                     std::vector<int> &);

}  // namespace dpg
