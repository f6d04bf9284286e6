// dpg_internal.h -- data structures shared by the host set-up and the CUDA kernels of the
// library (not part of the public ABI).
//
// Vocabulary (Mora & Demkowicz, arXiv 1711.00984):
//   kind   : a 1D factor family.  W = chi_i = L_i (integrated Legendre, Eqs. 2.97-2.101),
//            D = chi'_i, Y = nu_i = P_i = chi'_{i+1} (Legendre, Eqs. 2.91-2.93, 2.54).
//   term   : one product  sign * field(xi) * prod_d f^{kr_d}_{i_d}(xi_d) f^{kc_d}_{j_d}(xi_d)
//            of an inner product written on the master element, e.g. one D_ab entry of
//            Eq. 2.36, one C_ab entry of Eq. 2.60, one (alpha, beta) curl sub-term of
//            Eq. 2.77 with its sign (-1)^(alpha+beta) (Eq. 2.84).
//   block  : the (row component a, column component b) sub-matrix of a vector space
//            (Eqs. 2.53, 2.71); scalar spaces have one block.
//   stages : A contracts one direction (Eq. 2.23 contracts xi_3), B a second (Eq. 2.24),
//            C the last (Eq. 2.25); which direction each stage takes is a per-block choice
//            (BlockDesc::dir).  Terms with equal stage-C and stage-B kind pairs are summed
//            after stage A ("h groups"), terms with equal stage-C pairs after stage B
//            ("g groups"): the sum of Eq. 2.44 / 2.84 regrouped.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define DPG_HD __host__ __device__
#else
#define DPG_HD
#endif

namespace dpg {

enum Kind : int { KW = 0, KD = 1, KY = 2 };
constexpr int NKIND = 3;
constexpr int NPAIR = NKIND * NKIND;          // pair type = 3 * kr + kc
constexpr int MAXQ = 12;
constexpr int NQ1 = MAXQ + 1;                 // max 1D functions per direction
constexpr int MAXL = 14;
constexpr int MAXT = 12;                      // terms per block (H1 has 10)
constexpr int MAXH = 10;                      // (dir1, dir2)-pair groups per block
constexpr int MAXG = 4;                       // dir1-pair groups per block
constexpr int MAXP2 = 9;                      // distinct dir2 pairs per block
constexpr int MAXBLK = 32;                    // acoustics B: 16 blocks x 2 parts
constexpr int NJMAX = 8;                      // j3 values per work unit

enum SpaceId : int { S_H1 = 1, S_HCURL = 2, S_HDIV = 3, S_L2 = 4, S_B = 5, S_AX = 6, S_AB = 7 };
constexpr int MAXFIELDS = 20;                 // metric fields per point (acoustics B)

struct TermDesc {
    int field;        // index of the per-point metric field
    int sign;         // +1 / -1
    int kr[3], kc[3]; // row / column kinds per direction
    int h;            // (dir1, dir2) group
};

struct BlockDesc {
    int nr[3], nc[3];        // 1D function counts per direction (rows, columns)
    int row_off, col_off;    // position of the block in the element matrix
    int base;                // element-local offset (in values) of the matrix it writes
    int sym;                 // 0: plain; 1: diagonal block of a symmetric matrix (tiles with
                             // jA >= iA computed, the others mirrored); 2: off-diagonal
                             // block of a symmetric matrix (every tile mirrored)
    int dir[3];              // directions contracted by stage C (dir[0], last), stage B
                             // (dir[1]) and stage A (dir[2], first); chosen per block to
                             // minimise the multiply-adds (the paper uses 1, 2, 3)
    int nterm, nh, ng, np2;
    TermDesc term[MAXT];
    int h_g[MAXH];           // g group of each h group
    int h_p2[MAXH];          // dir2 pair slot of each h group
    int p2_pair[MAXP2];      // pair type of each dir2 slot
    int g_pair[MAXG];        // pair type of each g group (dir1)
    int h_pair2[MAXH];       // pair type of each h group's dir2 pair
    int h_pair1[MAXH];       // pair type of each h group's dir1 pair
    // lists derived from the above on the host, read by the kernels as they are
    signed char g_terms[MAXG][MAXT];   // terms of each g group, in term order
    signed char g_nterm[MAXG];
    signed char h_terms[MAXH][MAXT];   // terms of each h group, in term order
    signed char h_nterm[MAXH];
    signed char g_hs[MAXG][MAXH];      // h groups of each g group, in h order
    signed char g_nh[MAXG];
    signed char term_slot[MAXT];       // slot of each term's metric field among the block's
    signed char slot_field[MAXT];      // distinct fields (first-use order) and the field of
    signed char nslot;                 // each slot
};

struct Unit {
    int16_t block, i3, j3b, nj;   // i3 / j3: indices along the stage-A direction dir[2]
};

// Shared-memory layout (in floats, every region a multiple of 4) of the FP32 general
// kernel for one block and a chunk of nj stage-A partners.  The stage-A direction is
// xi_3 (dir[2] == 2), so a tile row is one contiguous run of the output.
struct F32Layout {
    int nr1, nr2, nc1, nc2;          // stage-C / stage-B extents (rows, columns)
    int nc1p, n22, n22p, nx, nx4;    // padded j1 range, (i2,j2) pairs, (j2,jj) pairs
    int nrow, ncol, ldt;             // output tile [nrow][ldt], ncol used columns
    int oP1, oP2, oP3, oA, oB, oT, total;
};
DPG_HD inline int r4i(int v) { return (v + 3) & ~3; }
DPG_HD inline F32Layout f32_layout(const BlockDesc &b, int L, int nj) {
    F32Layout f;
    const int dC = b.dir[0], dB = b.dir[1];
    f.nr1 = b.nr[dC]; f.nr2 = b.nr[dB]; f.nc1 = b.nc[dC]; f.nc2 = b.nc[dB];
    f.nc1p = r4i(f.nc1);
    f.n22 = f.nr2 * f.nc2; f.n22p = r4i(f.n22);
    f.nx = f.nc2 * nj; f.nx4 = r4i(f.nx);
    f.nrow = f.nr1 * f.nr2; f.ncol = f.nc1 * f.nc2 * nj; f.ldt = f.ncol | 1;
    f.oP1 = 0;                                                   // [ng][nr1][L][nc1p]
    f.oP2 = f.oP1 + b.ng * f.nr1 * L * f.nc1p;                   // [np2][L][n22p]
    f.oP3 = f.oP2 + b.np2 * L * f.n22p;                          // [nterm][nj][L]
    f.oA = f.oP3 + r4i(b.nterm * nj * L);                        // [nh][L][L][8]
    f.oB = f.oA + b.nh * L * L * 8;                              // [ng][L][nr2][nx4]
    f.oT = f.oB + b.ng * L * f.nr2 * f.nx4;                      // [nrow][ldt]
    f.total = f.oT + r4i(f.nrow * f.ldt);
    return f;
}

// Shared-memory layout (in values of the output type, every region a multiple of 4) of the
// affine kernel for one block and a chunk of nj partners.  The constant part [0, oC) is a
// per-block image built on the host (build_aff_image) and copied in one pass: the counts of
// the non-zero stage-C factors per group (ints), their values and tile offsets
// i1 ldt + j1 (ints), the stage-B factors F2 (affine: exact 1D integrals per term) or P2
// (extruded maps: pair products at the Gauss points per dir-2 slot).  Then per unit: the
// non-zero list of Q (values, tile offsets) and the output tile [nrow][ldt].  Index lists
// are ints packed at the start of their value-sized regions.
struct AffLayout {
    int ldt, oF1C, oF1V, oF1I, oF2, oP2, oC, oQV, oQI, oT, total;
};
DPG_HD inline AffLayout aff_layout(int ng, int nr1, int nr2, int nc1, int nc2, int nj, int f2vals, int p2vals) {
    AffLayout a;
    const int n22 = nr2 * nc2, n11 = nr1 * nc1, nrow = nr1 * nr2, ncol = nc1 * nc2 * nj;
    a.ldt = ncol | 1;
    a.oF1C = 0;
    a.oF1V = a.oF1C + r4i(MAXG);
    a.oF1I = a.oF1V + r4i(ng * n11);
    a.oF2 = a.oF1I + r4i(ng * n11);
    a.oP2 = a.oF2 + r4i(f2vals);
    a.oC = a.oP2 + r4i(p2vals);
    a.oQV = a.oC;
    a.oQI = a.oQV + r4i(ng * n22 * nj);
    a.oT = a.oQI + r4i(ng * n22 * nj);
    a.total = a.oT + r4i(nrow * a.ldt);
    return a;
}
DPG_HD inline AffLayout aff_layout_block(const BlockDesc &b, int nj) {
    return aff_layout(b.ng, b.nr[0], b.nr[1], b.nc[0], b.nc[1], nj, b.nterm * b.nr[1] * b.nc[1], 0);
}

// Shared-memory layout (in values of the output type) of the extruded-map kernel: the
// affine layout with the stage-B pair products P2[slot][(i2,j2)][m] in its constant part
// (and no F2), followed by the element's 2D metric fields of the block's terms [nfs][L][L],
// the stage-A factors of the unit S3[t][jj][n] and the stage-A output A[h][m][jj].
struct ExtLayout {
    AffLayout a;
    int nfs, oFx, oS3, oA, total;
};
DPG_HD inline int distinct_fields(const BlockDesc &b) {
    int n = 0;
    for (int t = 0; t < b.nterm; ++t) {
        bool seen = false;
        for (int u = 0; u < t; ++u) seen = seen || b.term[u].field == b.term[t].field;
        if (!seen) ++n;
    }
    return n;
}
DPG_HD inline ExtLayout ext_layout(const BlockDesc &b, int L, int nj) {
    ExtLayout x;
    x.a = aff_layout(b.ng, b.nr[0], b.nr[1], b.nc[0], b.nc[1], nj, 0, b.np2 * b.nr[1] * b.nc[1] * L);
    x.nfs = distinct_fields(b);
    x.oFx = x.a.total;
    x.oS3 = x.oFx + r4i(x.nfs * L * L);
    x.oA = x.oS3 + r4i(b.nterm * nj * L);
    x.total = x.oA + r4i(b.nh * L * nj);
    return x;
}

// Shared-memory layout (in floats, every region 16-byte aligned) of the FP32 row-panel
// kernel for one block in the paper's direction order (stage C over xi_1, B over xi_2, A
// over xi_3) and a chunk of nj stage-A partners.  Stages B and C are tensor-core
// products (m16n8k8, TF32 operands split into high and low parts):
//   stage B: D[(i2,j2)][(jj,l)] = sum_{h in g} sum_m P2_h[(i2,j2)][m] A_h[m][(jj,l)]
//   stage C: D[(i2,x)][(i1,j1)] = sum_{g,l} Bs[(i2,x)][(g,l)] P1_g[(g,l)][(i1,j1)],
// with x = j2 + nc2 jj.  The constant operands (P1, P2) are stored pre-split in fragment
// order; the stage outputs A ([k][n], row stride = 8 or 24 mod 32) and Bs ([m][k], row
// stride an odd multiple of 4) are plain FP32 and are split as they are loaded, both
// layouts giving conflict-free fragment loads.
struct PanelLayout {
    int lpad, lsh, ksh;            // L rounded up to 8 (8 or 16), its log2, k-steps per group
    int nr1, nr2, nc1, nc2;
    int nt1, n1p, ks1;             // P1: n-tiles per i1, rows (i1, j1 padded), k-steps
    int n22, mtb;                  // P2: rows (i2, j2), m-tiles
    int nb, sn;                    // stage-A output: columns (jj, l), row stride
    int nx, mc, mtc2, skc;         // stage-B output: x range, rows (i2, x), m-tiles (even), stride
    int nrow, ncol, ldt;           // output tile [nrow][ldt] (rows i1 + nr1 i2, columns nc1 x + j1)
    int oP1, oP2, oA, oB, oP3, p3sz, oMo, oT, total;
};
constexpr int PANEL_SMEM_2CTA = 112 * 1024;   // dynamic shared memory for two CTAs per SM
DPG_HD inline PanelLayout panel_layout(const BlockDesc &b, int L, int nj) {
    PanelLayout f;
    f.lpad = (L + 7) & ~7; f.lsh = f.lpad == 8 ? 3 : 4; f.ksh = f.lpad >> 3;
    f.nr1 = b.nr[0]; f.nr2 = b.nr[1]; f.nc1 = b.nc[0]; f.nc2 = b.nc[1];
    f.nt1 = (f.nc1 + 7) >> 3; f.n1p = f.nr1 * f.nt1 * 8;
    f.ks1 = b.ng * f.ksh;
    f.n22 = f.nr2 * f.nc2; f.mtb = (f.n22 + 15) >> 4;
    f.nb = nj * f.lpad; f.sn = (f.nb & 15) ? f.nb : f.nb + 8;
    f.nx = f.nc2 * nj; f.mc = f.nr2 * f.nx; f.mtc2 = ((f.mc + 31) >> 5) * 2; f.skc = b.ng * f.lpad + 4;
    f.nrow = f.nr1 * f.nr2; f.ncol = f.nc1 * f.nx; f.ldt = f.ncol | 1;
    f.oP1 = 0;                                                   // [ks][n][tig][4]
    f.oP2 = f.oP1 + f.ks1 * f.n1p * 16;                          // [slot][mt][ks][lane][8]
    f.oA = f.oP2 + b.np2 * f.mtb * f.ksh * 256;                  // [h lpad + m][sn]
    f.oB = f.oA + r4i(b.nh * f.lpad * f.sn);                     // [mtc2 16][skc]
    f.oP3 = f.oB + f.mtc2 * 16 * f.skc;                          // 2 x [t][n][8]
    f.p3sz = b.nterm * L * 8;
    f.oMo = f.oP3 + 2 * f.p3sz;                                  // int [mtc2 16]
    f.oT = f.oMo + f.mtc2 * 16;                                  // [nrow][ldt]
    f.total = f.oT + r4i(f.nrow * f.ldt);
    return f;
}

// Shared-memory and tensor-memory layout of the FP32 tensor-core kernel (tcgen05) for one
// block in the paper's direction order and a chunk of nj stage-A partners.  Stages B and
// C are tcgen05 kind::tf32 products (M = 128 rows per instruction, operands split into
// TF32 high and low parts, three products per operand pair, FP32 accumulation in tensor
// memory):
//   stage B: D_B,g[(i2,j2)][(jj,l)]   = sum_{h in g} sum_m P2_h[(i2,j2)][m] A_h[(jj,l)][m]
//   stage C: D_C[(i2,x)][(i1,j1)]     = sum_{g,l} A_C[(i2,x)][(g,l)] P1[(i1,j1)][(g,l)]
// with x = j2 + nc2 jj and the stage-C columns (i1, j1) at i1 nc1p + j1 (j1 padded to a
// multiple of 8).  Every operand is stored K-major in the canonical no-swizzle layout:
// 8-row x 16-byte core matrices, element (r, k) at byte
//   (r / 8) * sbo + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4,
// sbo = 32 * (row length in k) bytes; one instruction consumes k = 8 (two core-matrix
// columns, 128 bytes apart).  An instruction reads 128 rows of its A operand and N rows of
// its B operand; rows past the stored ones only feed output rows / columns that are never
// read, so stored regions are padded to 8 rows only and the allocation covers the reads.
// The stage-A output A_h is double-buffered (the kernel pipelines consecutive work units).
// The metric fields the block's terms use are staged per element (F), the stage-A factors
// of every unit of the block are resident (P3T: [t][i3][j3][n], signs folded in).  Output
// tile rows start at a shift of 0..3 floats so that each has the 16-byte alignment of its
// destination row (vector write-out).  Byte offsets are from the start of dynamic shared
// memory.
struct TcLayout {
    int lpad, lsh, ksh;            // L rounded up to 8, its log2, k-steps of 8 per group
    int nr1, nr2, nc1, nc2, n22;   // stage-C / stage-B extents, (i2, j2) pairs (<= 128)
    int nc1p;                      // j1 range padded to a multiple of 8
    int NB, NC;                    // N of the stage-B (nj lpad, to 16) / stage-C (nr1 nc1p, to 16) products
    int mc, mt;                    // stage-C rows (i2, x) and 128-row tiles (chunk nj)
    int nrow, ncol, ldt;           // output tile [nrow][ldt]: rows i1 + nr1 i2, columns nc1 x + j1
    int nbB;                       // stage-B accumulators (2: double-buffered when TMEM allows)
    int tcolC, tneed, tcols;       // TMEM: D_B,g of buffer u at column (u ng + g) NB, D_C tile t
                                   // at tcolC + t NC; columns used, allocated (power of two >= 32)
    int sbo2, sboC;                // row-group strides: K = lpad (P2, A_h), K = ng lpad (P1, A_C)
    int nfs;                       // distinct metric fields of the block's terms
    int oP1, p1b;                  // P1 high part at oP1, low part at oP1 + p1b
    int oP2, p2b;                  // slot s: high at oP2 + 2 s p2b, low at + p2b
    int oAh, ahb, ahbuf;           // buffer u, h group: high at oAh + u ahbuf + 2 h ahb, low at + ahb
    int oAC, acb;                  // high at oAC, low at oAC + acb
    int oP3, p3b;                  // stage-A factors of a unit, two buffers [t][n][8] floats
    int oP3T;                      // stage-A factors of every unit [t][i3][j3][n]
    int oF;                        // metric fields of the current element [nfs][L^3]
    int oT;                        // output tile
    int total;                     // dynamic shared memory (bytes)
    int ok;                        // the block fits the tensor-core kernel
};
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_MAXROW = 128;     // output-tile rows (nr1 nr2) of the tensor-core kernel
DPG_HD inline TcLayout tc_layout(const BlockDesc &b, int L, int nj) {
    TcLayout f;
    auto r8 = [](int v) { return (v + 7) & ~7; };
    auto r16 = [](int v) { return (v + 15) & ~15; };
    f.lpad = r8(L); f.lsh = f.lpad == 8 ? 3 : 4; f.ksh = f.lpad >> 3;
    f.nr1 = b.nr[0]; f.nr2 = b.nr[1]; f.nc1 = b.nc[0]; f.nc2 = b.nc[1];
    f.n22 = f.nr2 * f.nc2; f.nc1p = r8(f.nc1);
    f.NB = r16(nj * f.lpad); f.NC = r16(f.nr1 * f.nc1p);
    f.mc = f.nr2 * f.nc2 * nj; f.mt = (f.mc + 127) >> 7;
    f.nrow = f.nr1 * f.nr2; f.ncol = f.nc1 * f.nc2 * nj; f.ldt = (f.ncol + 6) & ~3;
    f.nbB = 2 * b.ng * f.NB + f.mt * f.NC <= TC_TMEM_COLS ? 2 : 1;
    f.tcolC = f.nbB * b.ng * f.NB; f.tneed = f.tcolC + f.mt * f.NC;
    f.tcols = 32;
    while (f.tcols < f.tneed && f.tcols < TC_TMEM_COLS) f.tcols <<= 1;
    f.sbo2 = 32 * f.lpad; f.sboC = 32 * b.ng * f.lpad;
    f.nfs = distinct_fields(b);
    f.oP1 = 0; f.p1b = (f.NC >> 3) * f.sboC;
    f.oP2 = f.oP1 + 2 * f.p1b; f.p2b = (r8(f.n22) >> 3) * f.sbo2;
    f.oAh = f.oP2 + 2 * b.np2 * f.p2b; f.ahb = nj * f.lpad / 8 * f.sbo2; f.ahbuf = 2 * b.nh * f.ahb;
    f.oAC = f.oAh + 2 * f.ahbuf; f.acb = (r8(f.mc) >> 3) * f.sboC;
    f.oP3 = f.oAC + 2 * f.acb; f.p3b = b.nterm * L * 8 * 4;
    f.oP3T = f.oP3 + 2 * f.p3b;
    f.oF = f.oP3T + ((b.nterm * b.nr[2] * b.nc[2] * L * 4 + 15) & ~15);
    f.oT = f.oF + ((f.nfs * L * L * L * 4 + 15) & ~15);
    int end = f.oT + f.nrow * f.ldt * 4;
    // reads past the stored rows: 128 rows of the last P2 slot and of the last A_C tile,
    // NB rows of the last A_h slot
    const int e2 = f.oP2 + (2 * b.np2 - 1) * f.p2b + 16 * f.sbo2;
    const int eh = f.oAh + f.ahbuf + (2 * b.nh - 1) * f.ahb + (f.NB >> 3) * f.sbo2;
    const int ec = f.oAC + f.acb + f.mt * 16 * f.sboC;
    if (e2 > end) end = e2;
    if (eh > end) end = eh;
    if (ec > end) end = ec;
    f.total = (end + 127) & ~127;
    f.ok = f.n22 <= 128 && f.NB <= 256 && f.NC <= 256 && f.tneed <= TC_TMEM_COLS && f.lpad <= 16 &&
           f.nrow <= TC_MAXROW && (b.ng == 0 || (b.nh >= 1 && b.np2 >= 1));   // a block without terms: zeros
    return f;
}

// Shared-memory and tensor-memory layout of the FP32 general kernel with stage C on the
// tensor cores (sf_tcc_kernel) for one block in the paper's direction order.  A work item
// is (element, block, i3) with every partner j3; its output rows (i1, i2) are computed in
// tiles of at most 128 stage-C rows (i2, x), x = j2 + nc2 j3: whole i2 rows of x when
// nx = nc2 nc3 <= 128 (ipt of them per tile), else chunks of 128 x of one i2.
//   stage A (FMA)      A_h[m][j3][l] = sum_{t in h} sum_n M_t(l,m,n) P3_t(n, j3)          (Eq. 2.23)
//   stage B (FMA)      A_C[(i2,x)][(g,l)] = sum_{h in g} sum_m P2_h(m)[i2,j2] A_h[m][j3][l] (Eq. 2.24)
//   stage C (tcgen05)  D[(i2,x)][(i1,j1)] = sum_{g,l} A_C[(i2,x)][(g,l)] P1[(i1,j1)][(g,l)]  (Eq. 2.25)
// Stage-C operands are K-major in the canonical no-swizzle layout (element (r, k) at byte
// (r/8) sbo + (k/4) 128 + (r%8) 16 + (k%4) 4, sbo = 32 K), split into TF32 high and low
// parts (three products per operand pair, FP32 accumulation); K = (g, l) with l padded to
// lpad (a multiple of 4) and the whole K to a multiple of 8; N = (i1, j1) = i1 nc1 + j1,
// padded to a multiple of 16.  Two accumulators of N tensor-memory columns alternate
// between consecutive tiles.  Byte offsets from the start of dynamic shared memory; the
// constant image [0, oC) (P1 high, P1 low, P2) is built on the host (build_tcc_tables).
struct TccLayout {
    int L, lpad, K, ksteps, N;
    int nr1, nr2, nr3, nc1, nc2, nc3, nc3p;
    int n22, n22p, nx, ipt, nxc, ntile;   // (i2,j2) pairs; x range; i2 per tile (0: x chunks); chunks per i2; tiles
    int sbo;                               // 32 K bytes
    int oP1, p1b, oP2, oC;                 // P1 high at oP1, low at oP1 + p1b; P2 [np2][L][n22p] floats
    int oAC, acb;                          // A_C high at oAC, low at oAC + acb (128 rows)
    int oA;                                // stage-A output [nh][L][nc3][lpad] floats
    int oP3;                               // stage-A factors [nterm][L][nc3p] floats
    int npad, oF;                          // element fields of the block's terms [nfs][L][L][npad]
    int total;                             // bytes
    int tcols;                             // tensor-memory columns to allocate
    int ok;
};
constexpr int TCC_NTH = 256;
DPG_HD inline TccLayout tcc_layout(const BlockDesc &b, int L) {
    TccLayout f;
    auto r8 = [](int v) { return (v + 7) & ~7; };
    auto r16 = [](int v) { return (v + 15) & ~15; };
    auto a128 = [](int v) { return (v + 127) & ~127; };
    f.L = L; f.lpad = r4i(L);
    f.K = r8(b.ng * f.lpad); f.ksteps = f.K / 8;
    f.nr1 = b.nr[0]; f.nr2 = b.nr[1]; f.nr3 = b.nr[2];
    f.nc1 = b.nc[0]; f.nc2 = b.nc[1]; f.nc3 = b.nc[2]; f.nc3p = r4i(f.nc3);
    f.N = r16(f.nr1 * f.nc1);
    f.n22 = f.nr2 * f.nc2; f.n22p = r4i(f.n22);
    f.nx = f.nc2 * f.nc3;
    if (f.nx <= 128) { f.ipt = 128 / f.nx; f.nxc = 1; f.ntile = (f.nr2 + f.ipt - 1) / f.ipt; }
    else { f.ipt = 0; f.nxc = (f.nx + 127) / 128; f.ntile = f.nr2 * f.nxc; }
    f.sbo = 32 * f.K;
    f.oP1 = 0; f.p1b = (f.N / 8) * f.sbo;
    f.oP2 = f.oP1 + 2 * f.p1b;
    f.oC = a128(f.oP2 + 4 * b.np2 * L * f.n22p);
    f.oAC = f.oC; f.acb = 16 * f.sbo;
    f.oA = f.oAC + 2 * f.acb;
    f.oP3 = f.oA + 4 * b.nh * L * f.nc3 * f.lpad;
    f.npad = L | 1;
    f.oF = f.oP3 + 4 * b.nterm * L * f.nc3p;
    f.oF = (f.oF + 15) & ~15;
    f.total = a128(f.oF + 4 * distinct_fields(b) * L * L * f.npad);
    f.tcols = 32;
    while (f.tcols < 2 * f.N + 16 && f.tcols < 512) f.tcols <<= 1;
    f.ok = (2 * f.N + 16 <= 512) && f.nc1 <= 16 && f.nc3 <= 16 && f.lpad <= 16 && b.ng >= 1 && b.nh >= 1 &&
           b.np2 >= 1;
    return f;
}

// Device-resident tables of one (q, L).
struct DevTables {
    int q, L;
    const double *zeta, *w;          // Gauss rule, [L]
    const double *pp64;              // [NPAIR][NQ1][NQ1][L]  f_kr(i,l) f_kc(j,l)
    const float *pp32;
    const double *F;                 // [NPAIR][NQ1][NQ1]     int_0^1 f_kr,i f_kc,j
};

// Metric fields per space (per quadrature point, weights and coefficients folded in):
//   H1   : 0: c0 |J| w,  1..6: c1 D_ab |J| w          (ab = 11,22,33,12,13,23)
//   L2   : 0: c0 w / |J|
//   HDIV : 0..5: c0 C_ab w / |J|,  6: c1 w / |J|
//   HCURL: 0..5: c0 D_ab |J| w,  6..11: c1 C_ab w / |J|
//   B    : 0..8: (J^-1)_ac w (index 3a + c),  9..17: J_cd w / |J| (index 9 + 3c + d)
//   AX   : 0: w   (acoustics cross block: the Piola maps cancel, Eq. 3.18)
//   AB   : 0: w,  1..9: (J^-1)_dc w (index 1 + 3d + c),  10: w / |J|,
//          11..19: J_ca w / |J| (index 11 + 3c + a)   (acoustics stiffness, Eq. 3.16)
// with D = J^-1 J^-T (Eq. 2.32) and C = J^T J (Eq. 2.50).
DPG_HD inline int sym_index(int a, int b) {
    if (a == b) return a;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}
inline int nfields_of(int space) {
    switch (space) {
    case S_H1: return 7;
    case S_L2: return 1;
    case S_HDIV: return 7;
    case S_HCURL: return 12;
    case S_B: return 18;
    case S_AX: return 1;
    case S_AB: return 20;
    }
    return 0;
}

}  // namespace dpg
