// dpg_condense.cu -- static condensation of the DPG test variables, per element.
//
// Eq. 3.7 couples the test-space unknowns s to the trial unknowns through the Gram matrix G
// and the enriched stiffness B; eliminating s (G is positive definite) gives the condensed
// system of Eq. 3.8 with K = B^T G^-1 B and F = B^T G^-1 l.  The paper's route: a Cholesky
// factorization G = L L^T, the substitutions W = L^-1 B and y = L^-1 l, then the products
// K = W^T W and F = W^T y.
//
// condense_kernel<EMU>: one CTA per element at a time, persistent over the batch.
//   * Right-looking blocked Cholesky, panels of CD_NB columns, in place in the lower
//     triangle of G.  The diagonal block is factored in shared memory by all threads,
//     which then form L11^-1; the panel rows below it (L21 = A21 L11^-T) and the matching
//     CD_NB rows of [B | l] (W1 = L11^-1 B1) are products with that inverse; the trailing
//     lower triangle of G and the rows of [B | l] below the panel are updated by
//     CD_TM x CD_TM tiles.
//   * The substitution of [B | l] rides along with the factorization (same panel loop),
//     so W and y overwrite B and l in place.
//   * K: the lower tiles of W^T W over all n rows, mirrored; F = W^T y by one dot product
//     per column (the load column is likewise a dot product per row in the updates).
// EMU = false (DPG_CONDENSE_FMA): every product is FP64 FMA work, 16 outputs of a tile per
// thread (TileSpan), three CTAs per SM; the kernel is bound by the FP64 FMA rate (2 per
// clock per SM on GB300), not by memory -- an element's G streams through L2 O(n / CD_NB)
// times against O(n^3) multiply-adds.
// EMU = true (DPG_CONDENSE_TC, the default): the panel products, the tile updates and
// W^T W are exact BF16 digit products on the tensor cores (dpg_digits.cuh), a 16 x 32
// sub-tile per warp, two CTAs per SM; the diagonal blocks and F stay FP64 FMA.
#include "dpg_digits.cuh"
#include "dpg_kernels.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace dpg {

constexpr int CD_NB = 32;          // panel width
constexpr int CD_TM = 64;          // tile edge of the updates
constexpr int CD_NTH = 256;        // 16 outputs of a 64 x 64 tile per thread
constexpr int CD_LDS = CD_TM + 1;  // padded row of the staged operands

__device__ __forceinline__ void report_cd(DevStatus *st, int code, long long elem) {
    atomicCAS(&st->code, 0, code);
    atomicMin(&st->first_bad[code], (unsigned long long)elem);
}

// Column c of the right-hand side [B | l] at row i (c == m: the load vector).
struct Rhs {
    double *B, *l;
    int m;
    __device__ __forceinline__ double &at(int i, int c) const {
        return c < m ? B[(size_t)i * m + c] : l[i];
    }
};

// Outputs of one CD_TM x CD_TM tile owned by a thread: column c = tid % 64 and rows
// rw + 4 k, k < 16, rw = tid / 64 -- the row is the same for a whole warp, so a group of
// four k whose rows are all outside the tile (or, on a diagonal tile, above the first
// column of the warp) is skipped by the warp as a whole: on a part with 2 FP64 FMAs per
// clock per SM the tiles' ragged edges would otherwise cost more than the loads.
struct TileSpan {
    int c, rw, rows_v, cols_v, c0;
    bool lower;
    __device__ __forceinline__ bool ok(int k) const {
        const int r = rw + 4 * k;
        return r < rows_v && c < cols_v && (!lower || c <= r);
    }
    __device__ __forceinline__ bool group(int q4) const {
        const int rlo = rw + 16 * q4, rhi = rlo + 12;                  // rows of k = 4 q4 .. 4 q4 + 3
        return c0 < cols_v && rlo < rows_v && (!lower || c0 <= rhi);
    }
};
__device__ __forceinline__ TileSpan tile_span(int rows_v, int cols_v, bool lower) {
    TileSpan s;
    s.c = threadIdx.x & (CD_TM - 1);
    s.c0 = threadIdx.x & 32;
    s.rw = threadIdx.x >> 6;
    s.rows_v = rows_v < CD_TM ? rows_v : CD_TM;
    s.cols_v = cols_v < CD_TM ? cols_v : CD_TM;
    s.lower = lower;
    return s;
}

// acc[k] += (or -=) sum_{t < tn} sA[t][rw + 4 k] sB[t][c] over a thread's outputs.  The
// active groups of four k form one contiguous range; when it is all four (every tile
// but the ragged and diagonal ones) the sixteen chains advance together, else group by
// group with the inactive groups skipped by the whole warp.
template <bool NEG>
__device__ __forceinline__ void tile_fma(double (&acc)[16], const double (*sA)[CD_LDS],
                                         const double (*sB)[CD_LDS], const TileSpan &sp, int tn) {
    if (sp.group(0) && sp.group(3)) {
        for (int t = 0; t < tn; ++t) {
            const double bv = NEG ? -sB[t][sp.c] : sB[t][sp.c];
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = fma(sA[t][sp.rw + 4 * k], bv, acc[k]);
        }
        return;
    }
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
        if (!sp.group(q4)) continue;                                       // the same for the warp
        for (int t = 0; t < tn; ++t) {
            const double bv = NEG ? -sB[t][sp.c] : sB[t][sp.c];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[4 * q4 + u] = fma(sA[t][sp.rw + 16 * q4 + 4 * u], bv, acc[4 * q4 + u]);
        }
    }
}

// ---- updates on the tensor cores: FP64 products from exact BF16 digits (dpg_digits.cuh) ---
constexpr size_t EM_SIDE = (size_t)EM_S * CD_TM * EM_ROWBYTES;          // one operand side
constexpr size_t EM_SMEM = 2 * EM_SIDE + 2 * CD_TM * sizeof(int);       // + row exponents
constexpr size_t CD_SMEM = 2 * (size_t)CD_NB * CD_LDS * sizeof(double); // FP64 staging
__device__ __forceinline__ bool slice_row(double x, uint16_t *dst, int *e_out, int lane) {
    return slice_row_planes(x, dst, e_out, lane, CD_TM);
}

__device__ __forceinline__ void emu_products(long long (&tot)[16], const unsigned char *si,
                                             const unsigned char *sj, int rb, int cb, int lane) {
    emu_products_g(tot, si, CD_TM, sj, CD_TM, rb, cb, lane);
}

template <bool EMU>
__global__ void __launch_bounds__(CD_NTH, EMU ? 2 : 3) condense_kernel(CondParams p) {
    __shared__ double srd[CD_NB];               // reciprocals of the factor's diagonal
    __shared__ double sIT[CD_NB][CD_NB + 1];    // (L11^-1)^T
    // dynamic arena: staged FP64 operand rows sA, sB (k-major), or, in the tensor-core
    // updates, the digit planes of the two operand sides and their row exponents
    extern __shared__ __align__(16) unsigned char cd_smem[];
    double (*sA)[CD_LDS] = reinterpret_cast<double (*)[CD_LDS]>(cd_smem);
    double (*sB)[CD_LDS] = sA + CD_NB;
    // the diagonal block and its factor share sA's storage: they are last read before the
    // barrier that precedes the first staging into sA of the same panel step
    double (*sD)[CD_NB + 1] = reinterpret_cast<double (*)[CD_NB + 1]>(&sA[0][0]);
    __shared__ int sbad;
    const int n = p.n, m = p.m, mc = m + (p.l ? 1 : 0);
    const int tid = threadIdx.x;
#if defined(DPG_DEBUG_BOUNDS)
    if (!DPG_INB((EMU ? EM_SMEM : CD_SMEM) <= dpg_dyn_smem_bytes(), p.status, p.elem_base)) return;   // uniform
#endif
    const int warp = tid >> 5, lane = tid & 31;   // phase 2: warp -> 4 columns, lane -> 2 rows
    for (int64_t e = blockIdx.x; e < p.n_elem; e += gridDim.x) {
        double *G = p.G + (size_t)e * n * n;
        const Rhs R{ p.B + (size_t)e * n * m, p.l ? p.l + (size_t)e * n : nullptr, m };
        if (tid == 0) sbad = 0;
        for (int kb = 0; kb < n; kb += CD_NB) {
            const int w = n - kb < CD_NB ? n - kb : CD_NB;
            // 1. the diagonal block (lower triangle), factored by warp 0
            for (int idx = tid; idx < w * w; idx += CD_NTH) {
                const int r = idx / w, c = idx - r * w;
                sD[r][c] = c <= r ? G[(size_t)(kb + r) * n + kb + c] : 0.0;
            }
            __syncthreads();
            // right-looking unblocked factorization of the block by all threads: per column
            // j, the pivot, then the rank-1 update of the trailing lower triangle with the
            // column still unscaled (A_rc -= A_rj A_cj / piv^2); the columns are scaled at
            // the end
            for (int j = 0; j < w; ++j) {
                if (tid == 0) {
                    const double d = sD[j][j];
                    if (!(d > 0.0) || !isfinite(d)) sbad = 1;
                    const double piv = sqrt(d);
                    sD[j][j] = piv;
                    srd[j] = 1.0 / piv;
                }
                __syncthreads();
                const int nb = w - j - 1;
                const double rd2 = srd[j] * srd[j];
                for (int idx = tid; idx < nb * nb; idx += CD_NTH) {
                    const int r = j + 1 + idx / nb, c = j + 1 + idx % nb;
                    if (c <= r) sD[r][c] = fma(-sD[r][j] * rd2, sD[c][j], sD[r][c]);
                }
                __syncthreads();
            }
            if (sbad) break;
            for (int idx = tid; idx < w * w; idx += CD_NTH) {
                const int r = idx / w, c = idx - r * w;
                if (c < r) sD[r][c] *= srd[c];
            }
            __syncthreads();
            for (int idx = tid; idx < w * w; idx += CD_NTH) {
                const int r = idx / w, c = idx - r * w;
                if (c <= r) G[(size_t)(kb + r) * n + kb + c] = sD[r][c];
            }
            // 2. the panel rows below the block, L21 = A21 L11^-T, and the block's rows of
            //    [B | l], W1 = L11^-1 B1, as products with X = L11^-1.  X is formed row by
            //    row, X_jj = 1 / L_jj and X_jc = -(sum_{c <= t < j} L_jt X_tc) / L_jj, with 8
            //    threads per column c summing every 8th term (stored transposed:
            //    sIT[c][j] = X_jc).  Each warp then owns 4 columns (rows) of the products, so
            //    the triangular bound t <= j of its sums is the same for all its lanes.
            {
                const int cc = tid >> 3, sl = tid & 7;
                for (int j = 0; j < w; ++j) {
                    double part = 0.0;
                    for (int t = cc + sl; t < j; t += 8) part = fma(sD[j][t], sIT[cc][t], part);
                    part += __shfl_xor_sync(0xffffffffu, part, 1);
                    part += __shfl_xor_sync(0xffffffffu, part, 2);
                    part += __shfl_xor_sync(0xffffffffu, part, 4);
                    if (sl == 0) sIT[cc][j] = cc < j ? -part * srd[j] : (cc == j ? srd[j] : 0.0);
                    __syncthreads();
                }
            }
            const int r0 = kb + w, nr = n - r0;
            if constexpr (EMU) {
                // the same products from digits: X = L11^-1 (rows j, K = t) once per panel,
                // then 64-row tiles of A21 (L21 = A21 X^T, warps 0-3) and 64-column tiles of
                // [B | l]_1 (W1 = X B1, warps 0-3 in 2 x 2 sub-tiles)
                unsigned char *sx = cd_smem, *so = cd_smem + (size_t)EM_S * CD_NB * EM_ROWBYTES;
                int *ex = reinterpret_cast<int *>(cd_smem + 2 * EM_SIDE), *eo = ex + CD_TM;
                bool nonfinite = false;
                for (int jr = warp; jr < CD_NB; jr += CD_NTH / 32) {
                    const double x = (lane < w && jr < w) ? sIT[lane][jr] : 0.0;   // X[jr][lane]
                    unsigned char *base = sx + (size_t)jr * EM_ROWBYTES;
                    nonfinite |= slice_row_planes(x, reinterpret_cast<uint16_t *>(base) + lane, ex + jr, lane, CD_NB);
                }
                for (int gi0 = r0; gi0 < n; gi0 += CD_TM) {
                    constexpr int RPW = CD_TM / (CD_NTH / 32);
                    double xv[RPW];
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const int rr = warp + (CD_NTH / 32) * q;
                        xv[q] = (lane < w && gi0 + rr < n) ? G[(size_t)(gi0 + rr) * n + kb + lane] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const int rr = warp + (CD_NTH / 32) * q;
                        unsigned char *base = so + (size_t)rr * EM_ROWBYTES;
                        nonfinite |= slice_row_planes(xv[q], reinterpret_cast<uint16_t *>(base) + lane, eo + rr, lane, CD_TM);
                    }
                    __syncthreads();
                    if (warp < 4 && 16 * warp < n - gi0) {
                        long long tot[16];
                        emu_products_g(tot, so, CD_TM, sx, CD_NB, 16 * warp, 0, lane);
                        const int g = lane >> 2, tq = lane & 3;
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int r = 16 * warp + g + 8 * (i >> 1), c = 8 * nt + 2 * tq + (i & 1);
                                if (gi0 + r >= n || c >= w) continue;
                                const int se = min(max(eo[r] + ex[c] - 57, -1022), 1023);
                                G[(size_t)(gi0 + r) * n + kb + c] =
                                    (double)tot[4 * nt + i] * __longlong_as_double((long long)(se + 1023) << 52);
                            }
                    }
                    __syncthreads();
                }
                for (int gj0 = 0; gj0 < mc; gj0 += CD_TM) {
                    constexpr int RPW = CD_TM / (CD_NTH / 32);
                    double xv[RPW];
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const int cc = warp + (CD_NTH / 32) * q;
                        xv[q] = (lane < w && gj0 + cc < mc) ? R.at(kb + lane, gj0 + cc) : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const int cc = warp + (CD_NTH / 32) * q;
                        unsigned char *base = so + (size_t)cc * EM_ROWBYTES;
                        nonfinite |= slice_row_planes(xv[q], reinterpret_cast<uint16_t *>(base) + lane, eo + cc, lane, CD_TM);
                    }
                    __syncthreads();
                    const int rb = 16 * (warp & 1), cb = 32 * ((warp >> 1) & 1);
                    if (warp < 4 && rb < w && gj0 + cb < mc) {
                        long long tot[16];
                        emu_products_g(tot, sx, CD_NB, so, CD_TM, rb, cb, lane);
                        const int g = lane >> 2, tq = lane & 3;
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int r = rb + g + 8 * (i >> 1), c = cb + 8 * nt + 2 * tq + (i & 1);
                                if (r >= w || gj0 + c >= mc) continue;
                                const int se = min(max(ex[r] + eo[c] - 57, -1022), 1023);
                                R.at(kb + r, gj0 + c) =
                                    (double)tot[4 * nt + i] * __longlong_as_double((long long)(se + 1023) << 52);
                            }
                    }
                    __syncthreads();
                }
                if (nonfinite && lane == 0) sbad = 1;
            } else {
            const int jw = 4 * warp, tmax = jw + 4 < w ? jw + 4 : w;      // t < tmax
            for (int gi0 = r0; gi0 < n; gi0 += CD_TM) {
                for (int idx = tid; idx < CD_TM * CD_NB; idx += CD_NTH) {
                    const int r = idx / CD_NB, t = idx - r * CD_NB;
                    sA[t][r] = (t < w && gi0 + r < n) ? G[(size_t)(gi0 + r) * n + kb + t] : 0.0;
                }
                __syncthreads();
                double o[2][4] = {};
                for (int t = 0; t < tmax; ++t) {
                    const double a0 = sA[t][2 * lane], a1 = sA[t][2 * lane + 1];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const double li = sIT[t][jw + b];                 // (L11^-1)_{jw+b, t}
                        o[0][b] = fma(a0, li, o[0][b]);
                        o[1][b] = fma(a1, li, o[1][b]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int gi = gi0 + 2 * lane + a, j = jw + b;
                        if (gi < n && j < w) G[(size_t)gi * n + kb + j] = o[a][b];
                    }
                __syncthreads();
            }
            for (int gj0 = 0; gj0 < mc; gj0 += CD_TM) {
                for (int idx = tid; idx < CD_TM * CD_NB; idx += CD_NTH) {
                    const int t = idx / CD_TM, c = idx - t * CD_TM;
                    sB[t][c] = (t < w && gj0 + c < mc) ? R.at(kb + t, gj0 + c) : 0.0;
                }
                __syncthreads();
                double o[4][2] = {};
                for (int t = 0; t < tmax; ++t) {
                    const double b0 = sB[t][2 * lane], b1 = sB[t][2 * lane + 1];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const double li = sIT[t][jw + a];
                        o[a][0] = fma(li, b0, o[a][0]);
                        o[a][1] = fma(li, b1, o[a][1]);
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int j = jw + a, gj = gj0 + 2 * lane + b;
                        if (j < w && gj < mc) R.at(kb + j, gj) = o[a][b];
                    }
                __syncthreads();
            }
            // 3. trailing update: G22 -= L21 L21^T (lower tiles), [B | l]_2 -= L21 W1
            }
            // the load column is a plain dot product per row (no 64-wide tile for one column):
            // l_i -= sum_t L_{i, kb+t} y_{kb+t}, i >= r0
            if (R.l)
                for (int i = r0 + tid; i < n; i += CD_NTH) {
                    const double *Li = G + (size_t)i * n + kb;
                    double s0 = 0.0, s1 = 0.0;
                    int t = 0;
                    for (; t + 1 < w; t += 2) {
                        s0 = fma(Li[t], R.l[kb + t], s0);
                        s1 = fma(Li[t + 1], R.l[kb + t + 1], s1);
                    }
                    if (t < w) s0 = fma(Li[t], R.l[kb + t], s0);
                    R.l[i] -= s0 + s1;
                }
            const int ntr = (nr + CD_TM - 1) / CD_TM, ntc = (m + CD_TM - 1) / CD_TM;
            if constexpr (EMU) {
                // row block by row block: the digits of the 64 I rows (L21 rows) once per block,
                // those of the J rows (L21 rows, or the columns of W1 for a right-hand-side
                // tile) per tile; a warp per row, its loads issued before the digit splits
                unsigned char *si = cd_smem, *sj = cd_smem + EM_SIDE;
                int *ei = reinterpret_cast<int *>(cd_smem + 2 * EM_SIDE), *ej = ei + CD_TM;
                constexpr int RPW = CD_TM / (CD_NTH / 32);                   // rows per warp
                bool nonfinite = false;
                for (int I = 0; I < ntr; ++I) {
                    const int gi0 = r0 + I * CD_TM;
                    {
                        double xv[RPW];
#pragma unroll
                        for (int q = 0; q < RPW; ++q) {
                            const int rr = warp + (CD_NTH / 32) * q;
                            xv[q] = (lane < w && gi0 + rr < n) ? G[(size_t)(gi0 + rr) * n + kb + lane] : 0.0;
                        }
#pragma unroll
                        for (int q = 0; q < RPW; ++q) {
                            const int rr = warp + (CD_NTH / 32) * q;
                            nonfinite |= slice_row(xv[q], reinterpret_cast<uint16_t *>(si + (size_t)rr * EM_ROWBYTES) + lane,
                                                   ei + rr, lane);
                        }
                    }
                    for (int jt = 0; jt < I + 1 + ntc; ++jt) {
                        const bool isA = jt <= I;
                        const int J = isA ? jt : jt - I - 1;
                        const int gj0 = isA ? r0 + J * CD_TM : J * CD_TM;
                        double xv[RPW];
#pragma unroll
                        for (int q = 0; q < RPW; ++q) {
                            const int rr = warp + (CD_NTH / 32) * q;
                            double x = 0.0;
                            if (lane < w) {
                                if (isA) {
                                    if (gj0 + rr < n) x = G[(size_t)(gj0 + rr) * n + kb + lane];
                                } else if (gj0 + rr < m) {
                                    x = R.B[(size_t)(kb + lane) * m + gj0 + rr];
                                }
                            }
                            xv[q] = x;
                        }
#pragma unroll
                        for (int q = 0; q < RPW; ++q) {
                            const int rr = warp + (CD_NTH / 32) * q;
                            nonfinite |= slice_row(xv[q], reinterpret_cast<uint16_t *>(sj + (size_t)rr * EM_ROWBYTES) + lane,
                                                   ej + rr, lane);
                        }
                        __syncthreads();
                        // a 16 x 32 sub-tile per warp; sub-tiles outside the tile or above a
                        // diagonal tile's diagonal are skipped by the whole warp
                        const int rb = 16 * (warp & 3), cb = 32 * (warp >> 2);
                        const int rows_v = n - gi0, cols_v = (isA ? n : m) - gj0;
                        const bool diag = isA && I == J;
                        if (rb < rows_v && cb < cols_v && !(diag && cb >= rb + 16)) {
                            long long tot[16];
                            emu_products(tot, si, sj, rb, cb, lane);
                            const int g = lane >> 2, tq = lane & 3;
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    const int r = rb + g + 8 * (i >> 1), c = cb + 8 * nt + 2 * tq + (i & 1);
                                    if (r >= rows_v || c >= cols_v || (diag && c > r)) continue;
                                    // 2^(e_i + e_j - 57), a normal number for the exponents here
                                    const int se = min(max(ei[r] + ej[c] - 57, -1022), 1023);
                                    const double sc = __longlong_as_double((long long)(se + 1023) << 52);
                                    double *dst = isA ? G + (size_t)(gi0 + r) * n + gj0 + c
                                                      : R.B + (size_t)(gi0 + r) * m + gj0 + c;
                                    *dst = fma(-(double)tot[4 * nt + i], sc, *dst);
                                }
                        }
                        __syncthreads();
                    }
                }
                if (nonfinite && lane == 0) sbad = 1;
            } else {
            const int tilesA = ntr * (ntr + 1) / 2, tiles = tilesA + ntr * ntc;
            for (int tile = 0; tile < tiles; ++tile) {
                int I, J;
                const bool isA = tile < tilesA;
                if (isA) {                                 // lower tiles, row by row
                    I = 0;
                    while ((I + 1) * (I + 2) / 2 <= tile) ++I;
                    J = tile - I * (I + 1) / 2;
                } else {
                    I = (tile - tilesA) / ntc;
                    J = (tile - tilesA) - I * ntc;
                }
                const int gi0 = r0 + I * CD_TM;                           // rows of G / rhs
                const int gj0 = isA ? r0 + J * CD_TM : J * CD_TM;         // columns
                {
                for (int idx = tid; idx < CD_TM * CD_NB; idx += CD_NTH) {
                    const int r = idx / CD_NB, t = idx - r * CD_NB;
                    const bool tv = t < w;
                    sA[t][r] = (tv && gi0 + r < n) ? G[(size_t)(gi0 + r) * n + kb + t] : 0.0;
                    if (isA) sB[t][r] = (tv && gj0 + r < n) ? G[(size_t)(gj0 + r) * n + kb + t] : 0.0;
                }
                if (!isA)
                    for (int idx = tid; idx < CD_TM * CD_NB; idx += CD_NTH) {
                        const int t = idx / CD_TM, c = idx - t * CD_TM;
                        sB[t][c] = (t < w && gj0 + c < m) ? R.B[(size_t)(kb + t) * m + gj0 + c] : 0.0;
                    }
                __syncthreads();
                const TileSpan sp = tile_span(n - gi0, (isA ? n : m) - gj0, isA && I == J);
                double acc[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int gi = gi0 + sp.rw + 4 * k, gj = gj0 + sp.c;
                    acc[k] = sp.ok(k) ? (isA ? G[(size_t)gi * n + gj] : R.B[(size_t)gi * m + gj]) : 0.0;
                }
                tile_fma<true>(acc, sA, sB, sp, w);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if (!sp.ok(k)) continue;
                    const int gi = gi0 + sp.rw + 4 * k, gj = gj0 + sp.c;
                    if (isA) G[(size_t)gi * n + gj] = acc[k];
                    else R.B[(size_t)gi * m + gj] = acc[k];
                }
                __syncthreads();
                }
            }
            }
        }
        double *K = p.K + (size_t)e * m * m;
        double *F = p.F ? p.F + (size_t)e * m : nullptr;
        if (sbad) {
            for (int idx = tid; idx < m * m; idx += CD_NTH) K[idx] = __longlong_as_double(0x7ff8000000000000LL);
            if (F)
                for (int idx = tid; idx < m; idx += CD_NTH) F[idx] = __longlong_as_double(0x7ff8000000000000LL);
            if (tid == 0) report_cd(p.status, 11 /*DPG_ERR_NOT_SPD*/, p.elem_base + e);
            __syncthreads();
            continue;
        }
        // 4. K = W^T W, lower tiles over all n rows, mirrored; F = W^T y, one column of W
        //    per thread
        const int nt = (m + CD_TM - 1) / CD_TM;
        for (int tile = 0; tile < nt * (nt + 1) / 2; ++tile) {
            int I = 0;
            while ((I + 1) * (I + 2) / 2 <= tile) ++I;
            const int J = tile - I * (I + 1) / 2;
            const int ci0 = I * CD_TM, cj0 = J * CD_TM;
            if constexpr (EMU) {
                // the same digit products, the columns of W as the operand rows, in chunks
                // of 32 rows of W (each chunk with its own column exponents)
                unsigned char *si = cd_smem, *sj = cd_smem + EM_SIDE;
                int *ei = reinterpret_cast<int *>(cd_smem + 2 * EM_SIDE), *ej = ei + CD_TM;
                const int rb = 16 * (warp & 3), cb = 32 * (warp >> 2);
                const int rows_v = m - ci0, cols_v = m - cj0;
                const bool diag = I == J;
                const bool active = rb < rows_v && cb < cols_v && !(diag && cb >= rb + 16);
                const int g = lane >> 2, tq = lane & 3;
                double out[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) out[k] = 0.0;
                for (int i0 = 0; i0 < n; i0 += CD_NB) {
                    constexpr int RPW = 2 * CD_TM / (CD_NTH / 32);            // rows per warp
                    double xv[RPW];
#pragma unroll
                    for (int j = 0; j < RPW; ++j) {
                        const int r = warp + (CD_NTH / 32) * j;
                        const bool side_j = r >= CD_TM;
                        const int col = (side_j ? cj0 + r - CD_TM : ci0 + r);
                        xv[j] = (i0 + lane < n && col < m) ? R.B[(size_t)(i0 + lane) * m + col] : 0.0;
                    }
                    bool nonfinite = false;
#pragma unroll
                    for (int j = 0; j < RPW; ++j) {
                        const int r = warp + (CD_NTH / 32) * j;
                        const bool side_j = r >= CD_TM;
                        const int rr = side_j ? r - CD_TM : r;
                        unsigned char *base = (side_j ? sj : si) + (size_t)rr * EM_ROWBYTES;
                        nonfinite |= slice_row(xv[j], reinterpret_cast<uint16_t *>(base) + lane,
                                               (side_j ? ej : ei) + rr, lane);
                    }
                    if (nonfinite && lane == 0) sbad = 1;
                    __syncthreads();
                    if (active) {
                        long long tot[16];
                        emu_products(tot, si, sj, rb, cb, lane);
#pragma unroll
                        for (int nt2 = 0; nt2 < 4; ++nt2)
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int r = rb + g + 8 * (i >> 1), c = cb + 8 * nt2 + 2 * tq + (i & 1);
                                const int se = min(max(ei[r] + ej[c] - 57, -1022), 1023);
                                const double sc = __longlong_as_double((long long)(se + 1023) << 52);
                                out[4 * nt2 + i] = fma((double)tot[4 * nt2 + i], sc, out[4 * nt2 + i]);
                            }
                    }
                    __syncthreads();
                }
                if (active)
#pragma unroll
                    for (int nt2 = 0; nt2 < 4; ++nt2)
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int r = rb + g + 8 * (i >> 1), c = cb + 8 * nt2 + 2 * tq + (i & 1);
                            if (r >= rows_v || c >= cols_v || (diag && c > r)) continue;
                            if (!DPG_INB(ci0 + r < m && cj0 + c < m, p.status, p.elem_base + e)) continue;
                            K[(size_t)(ci0 + r) * m + cj0 + c] = out[4 * nt2 + i];
                            K[(size_t)(cj0 + c) * m + ci0 + r] = out[4 * nt2 + i];
                        }
                continue;
            }
            const TileSpan sp = tile_span(m - ci0, m - cj0, I == J);
            double acc[16] = {};
            for (int i0 = 0; i0 < n; i0 += CD_NB) {
                const int h = n - i0 < CD_NB ? n - i0 : CD_NB;
                for (int idx = tid; idx < CD_TM * CD_NB; idx += CD_NTH) {
                    const int t = idx / CD_TM, c = idx - t * CD_TM;
                    const double *Wr = R.B + (size_t)(i0 + t) * m;
                    sA[t][c] = (t < h && ci0 + c < m) ? Wr[ci0 + c] : 0.0;
                    sB[t][c] = (t < h && cj0 + c < m) ? Wr[cj0 + c] : 0.0;
                }
                __syncthreads();
                tile_fma<false>(acc, sA, sB, sp, h);
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (!sp.ok(k)) continue;
                const int ci = ci0 + sp.rw + 4 * k, cj = cj0 + sp.c;
                if (!DPG_INB(ci < m && cj < m, p.status, p.elem_base + e)) continue;
                K[(size_t)ci * m + cj] = acc[k];
                K[(size_t)cj * m + ci] = acc[k];
            }
        }
        if (F)
            for (int c = tid; c < m; c += CD_NTH) {
                double s0 = 0.0, s1 = 0.0;
                int i = 0;
                for (; i + 1 < n; i += 2) {
                    s0 = fma(R.B[(size_t)i * m + c], R.l[i], s0);
                    s1 = fma(R.B[(size_t)(i + 1) * m + c], R.l[i + 1], s1);
                }
                if (i < n) s0 = fma(R.B[(size_t)i * m + c], R.l[i], s0);
                F[c] = s0 + s1;
            }
        __syncthreads();
        if (EMU && sbad) {          // a value of W that is not finite, met by the digit split
            for (int idx = tid; idx < m * m; idx += CD_NTH) K[idx] = __longlong_as_double(0x7ff8000000000000LL);
            if (F)
                for (int idx = tid; idx < m; idx += CD_NTH) F[idx] = __longlong_as_double(0x7ff8000000000000LL);
            if (tid == 0) report_cd(p.status, 11 /*DPG_ERR_NOT_SPD*/, p.elem_base + e);
            __syncthreads();
        }
    }
}

int condense_ctas_per_sm(bool emu) {
    int per_sm = 0;
    const cudaError_t e = emu ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, condense_kernel<true>, CD_NTH, EM_SMEM)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, condense_kernel<false>, CD_NTH, CD_SMEM);
    if (e != cudaSuccess) return 1;
    return per_sm < 1 ? 1 : per_sm;
}

cudaError_t init_condense_attributes() {
    cudaError_t e = cudaFuncSetAttribute(condense_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EM_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(condense_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CD_SMEM);
    return e;
}

cudaError_t launch_condense(const CondParams &p, int num_sms, bool emu, cudaStream_t s) {
    if (p.n_elem == 0) return cudaSuccess;
    const int64_t cap = (int64_t)condense_ctas_per_sm(emu) * num_sms;
    const unsigned grid = (unsigned)(p.n_elem < cap ? p.n_elem : cap);
    if (emu) condense_kernel<true><<<grid, CD_NTH, EM_SMEM, s>>>(p);
    else condense_kernel<false><<<grid, CD_NTH, CD_SMEM, s>>>(p);
    return cudaGetLastError();
}

}  // namespace dpg
