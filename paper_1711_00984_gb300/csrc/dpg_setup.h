// dpg_setup.h -- host-side tables and term programs (internal).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include "dpg_internal.h"

namespace dpg {

struct HostTables {
    int q = 0, L = 0;
    std::vector<double> zeta, w;   // Gauss rule on (0,1), [L]
    std::vector<double> pp;        // [NPAIR][NQ1][NQ1][L]
    std::vector<double> F;         // [NPAIR][NQ1][NQ1]
};

struct Program {
    int space = 0, q = 0, L = 0, p = 0;
    bool split = false;
    int rows = 0, cols = 0, parts = 1, nfields = 0;
    int nblock = 0;
    BlockDesc blocks[MAXBLK];
    std::vector<Unit> units;
    int nj = 1;
    int nj_sym = 1;                // chunk of the diagonal blocks of a symmetric matrix (sym == 1;
                                   // ORDER_BEST programs: may be below nj, their units are uneven)
    size_t smem_values = 0;        // shared-memory values of the FP64-model general kernel
    size_t smem_bytes = 0;         // shared memory of the kernel this program is built for
    double flops = 0.0;            // algorithmic flops per element, general path
    double flops_affine = 0.0;     // algorithmic flops per element, affine path
    double flops_extruded = 0.0;   // algorithmic flops per element, extruded-map path
};

void gauss_rule(int L, double *z, double *w);
HostTables make_tables(int q, int L);
// Contraction order of the blocks: ORDER_BEST picks the cheapest of the six direction
// permutations (FP64 general kernel); ORDER_A3 the cheaper of the two with stage A over
// xi_3 (FP32 general kernel: contiguous tile rows); ORDER_NATURAL the paper's order
// (stage A over xi_3, B over xi_2, C over xi_1; affine kernel).
// ORDER_PANEL: the paper's order and every (a, b) block of a symmetric matrix built (no
// mirrored tiles): the FP32 row-panel kernel writes every output row itself.
// ORDER_TC: the same blocks as ORDER_PANEL, sized for the FP32 tensor-core (tcgen05)
// kernel (tc_layout); a block that does not fit it makes the program's smem_bytes
// SIZE_MAX.
// ORDER_EXTRUDED: the paper's order, sized for the extruded-map kernel (ext_layout).
enum { ORDER_BEST = 0, ORDER_A3 = 1, ORDER_NATURAL = 2, ORDER_PANEL = 3, ORDER_TC = 4, ORDER_EXTRUDED = 5,
       ORDER_TCC = 8 };
// ORDER_TCC: the paper's order and every block built, for the FP32 general kernel with stage C
// on the tensor cores (tcc_layout); a block that does not fit it makes smem_bytes SIZE_MAX.
// force_nj > 0 fixes the stage-A chunk (autotuner); otherwise the largest chunk whose
// shared memory fits the kernel's budget (smem_budget bytes, or the order's default when
// 0) is taken.
Program make_program(int space, int q, int L, int p, bool split, const HostTables &tab, int order = ORDER_BEST,
                     int force_nj = 0, size_t smem_budget = 0, int force_nj_sym = 0);
// Constant operands of the FP32 row-panel kernel for every block of an ORDER_PANEL
// program (the shared-memory image [0, oA) of panel_layout), concatenated; off[k] is the
// first float of block k.
void build_panel_tables(const Program &pr, const HostTables &tab, std::vector<float> &ctab, std::vector<int> &off);
// Constant operands of the FP32 tensor-core kernel for every block of an ORDER_TC program:
// P1 and the P2 slots, each split into TF32 high and low parts, in the canonical K-major
// layout of tc_layout (the shared-memory image [0, oAh)); off[k] is the first float of
// block k.
void build_tc_tables(const Program &pr, const HostTables &tab, std::vector<float> &ctab, std::vector<int> &off);
// Constant shared-memory image of the affine (extruded = false) or extruded-map kernel for
// every block of an ORDER_NATURAL / ORDER_EXTRUDED program in the value type T: the region
// [0, oC) of its layout; block k occupies bytes [16 off16[k], 16 off16[k + 1]).
template <typename T>
void build_aff_image(const Program &pr, const HostTables &tab, bool extruded, std::vector<unsigned char> &img,
                     std::vector<int> &off16);
// Structurally non-zero entries of the affine stage-B products Q_g(i2, j2, jj) of every unit
// (Algorithm 10 with a constant metric): entry (ij2 = i2 nc2 + j2, jj) of group g with the
// mask of the group's terms whose exact integrals F2_t(i2, j2) and F3_t(i3, j3b + jj) are
// both non-zero (bit k2: term g_terms[g][k2]), coded ij2 | jj << 8 | mask << 12 | g << 24.
// Per unit the groups' lists in group order, each in (ij2, jj) order and padded with empty
// entries (mask 0) to a multiple of 32; the list of unit u is [qo[u], qo[u + 1]).  False if a
// block does not fit the code.
bool build_aff_qlists(const Program &pr, const HostTables &tab, std::vector<unsigned> &ql, std::vector<int> &qo);
// Whether the matrix of an affine program is diagonal for every element: one square block at
// the origin, at most max_terms terms, each with diagonal exact 1D integrals in every
// direction (the L2 Gram matrix, by the Legendre orthogonality of Eq. 2.95).  If so, D holds
// per term t the products D[t][r] = F_t1(i1, i1) F_t2(i2, i2) F_t3(i3, i3) of its diagonal
// integrals at r = i1 + nr1 (i2 + nr2 i3), and the element's matrix is
// diag(sum_t sign_t c_t D[t][r]).
bool affine_diagonal(const Program &pa, const HostTables &tab, int max_terms, std::vector<double> &D);
// Constant images of the FP32 tensor-core stage-C kernel for every block of an ORDER_TCC
// program: P1 split into TF32 high and low parts in the canonical K-major layout, then the
// stage-B factors P2 (the region [0, oC) of tcc_layout), in floats; off[k] is the first
// float of block k, off[nblock] the total.
void build_tcc_tables(const Program &pr, const HostTables &tab, std::vector<float> &img, std::vector<int> &off);
int64_t rows_of(int space, int q);
int64_t cols_of(int space, int p, int q);

}  // namespace dpg
