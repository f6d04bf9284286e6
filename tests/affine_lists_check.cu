// Host-only check of the structural stage-B lists of the affine path (build_aff_qlists)
// against the affine flop count that make_program computes by its own loops (Sec. 2.8.1):
// the stage-B products are the set bits of the entries' term masks, the stage-C products
// are, per entry, the non-zero exact integrals F1_g(i1, j1) of its group, and twice their
// sum must be flops_affine.  Also checks the list format: per unit a run of whole 32-entry
// chunks, one group per chunk, indices inside the block.  Then the diagonal-matrix test of
// the affine programs (affine_diagonal, any number of terms): it must hold for L2 and for no
// other space, and the L2 table must be the product of the Legendre norms of Eq. 2.95,
// D(r) = 1 / ((2 i1 + 1)(2 i2 + 1)(2 i3 + 1)).  Prints one JSON line per (space, q, p,
// form); exit status 1 on the first failed check.
#include "dpg_setup.h"

#include <cmath>
#include <cstdio>
#include <vector>

using namespace dpg;

static int fail(const char *what, int space, int q, int p, int prec) {
    std::printf("{\"fail\": \"%s\", \"space\": %d, \"q\": %d, \"p\": %d, \"prec\": %d}\n", what, space, q, p, prec);
    return 1;
}

int main() {
    const int spaces[] = { S_H1, S_HCURL, S_HDIV, S_L2, S_B, S_AX, S_AB };
    for (int space : spaces)
        for (int q = 1; q <= 7; ++q) {
            const int L = q + 2;
            const HostTables tab = make_tables(q, L);
            auto Fnz = [&](int pair, int i, int j) { return tab.F[((size_t)pair * NQ1 + i) * NQ1 + j] != 0.0; };
            const bool mixed = space == S_B || space == S_AB;           // trial order p = 1..q
            for (int p = (mixed ? 1 : 0); p <= (mixed ? q : 0); ++p)
                for (int prec = 0; prec < 2; ++prec) {
                    // the affine programs of both forms, as the library builds them
                    const Program pa = make_program(space, q, L, p, false, tab, ORDER_NATURAL, 0,
                                                    prec == 0 ? 72 * 1024 : 0);
                    std::vector<unsigned> ql;
                    std::vector<int> qo;
                    if (!build_aff_qlists(pa, tab, ql, qo)) return fail("builder refused", space, q, p, prec);
                    if (qo.size() != pa.units.size() + 1) return fail("offset count", space, q, p, prec);
                    double nB = 0.0, nC = 0.0;
                    long entries = 0;
                    for (size_t u = 0; u < pa.units.size(); ++u) {
                        const Unit &un = pa.units[u];
                        const BlockDesc &b = pa.blocks[un.block];
                        if (b.dir[0] != 0 || b.dir[1] != 1 || b.dir[2] != 2) return fail("order", space, q, p, prec);
                        const int n22 = b.nr[1] * b.nc[1];
                        if (qo[u + 1] < qo[u] || (qo[u + 1] - qo[u]) % 32 != 0 || qo[u] % 32 != 0)
                            return fail("padding", space, q, p, prec);
                        for (int c0 = qo[u]; c0 < qo[u + 1]; c0 += 32) {
                            const int g = (int)(ql[c0] >> 24);
                            if (g >= b.ng) return fail("group", space, q, p, prec);
                            int nzF1 = 0;
                            for (int i1 = 0; i1 < b.nr[0]; ++i1)
                                for (int j1 = 0; j1 < b.nc[0]; ++j1) nzF1 += Fnz(b.g_pair[g], i1, j1);
                            for (int k = c0; k < c0 + 32; ++k) {
                                const unsigned code = ql[k];
                                const int ij2 = code & 0xff, jj = (code >> 8) & 0xf;
                                const unsigned m = (code >> 12) & 0xfffu;
                                if ((int)(code >> 24) != g) return fail("mixed chunk", space, q, p, prec);
                                if (m == 0) continue;                           // padding
                                if (ij2 >= n22 || jj >= un.nj || (m >> b.g_nterm[g]) != 0)
                                    return fail("index", space, q, p, prec);
                                nB += __builtin_popcount(m);
                                nC += nzF1;
                                ++entries;
                            }
                        }
                    }
                    if (2.0 * (nB + nC) != pa.flops_affine) return fail("flop count", space, q, p, prec);
                    std::vector<double> D;
                    const bool diag = affine_diagonal(pa, tab, MAXT, D);
                    if (diag != (space == S_L2)) return fail("diagonal test", space, q, p, prec);
                    double derr = 0.0;
                    if (diag) {
                        const BlockDesc &b0 = pa.blocks[0];
                        if (b0.nterm != 1 || (int)D.size() != pa.rows || pa.rows != q * q * q)
                            return fail("diagonal table size", space, q, p, prec);
                        for (int r = 0; r < pa.rows; ++r) {
                            const int i1 = r % q, i2 = (r / q) % q, i3 = r / (q * q);
                            const double ref = 1.0 / ((2.0 * i1 + 1) * (2.0 * i2 + 1) * (2.0 * i3 + 1));
                            derr = std::fmax(derr, std::fabs(D[r] - ref) / ref);
                        }
                        if (!(derr <= 1e-13)) return fail("Legendre norms", space, q, p, prec);
                    }
                    std::printf("{\"space\": %d, \"q\": %d, \"p\": %d, \"prec\": %d, \"units\": %zu, \"entries\": %ld, "
                                "\"stage_b\": %.0f, \"stage_c\": %.0f, \"diagonal\": %d, \"legendre_err\": %.3g}\n",
                                space, q, p, prec, pa.units.size(), entries, nB, nC, (int)diag, derr);
                }
        }
    return 0;
}
