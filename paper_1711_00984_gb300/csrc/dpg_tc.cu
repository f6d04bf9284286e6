// dpg_tc.cu -- FP32 general path on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// sf_tc_f32_kernel integrates one block (a, b) of the element matrix by sum factorization
// (Eqs. 2.23-2.25 and their H1 / H(div) / H(curl) forms 2.38-2.44, 2.61-2.63, 2.78-2.84)
// in the paper's direction order, every block computed (no mirrored tiles), so that each
// output row of the element matrix leaves as one contiguous run.  A CTA keeps one block
// resident and walks a chunk of elements and every work unit (i3, chunk of j3) of the
// block:
//   stage A (FMA pipe)  A_h[(jj,l)][m]     = sum_{t in h} sum_n M_t(l,m,n) P3_t(jj,n)       (Eq. 2.23)
//   stage B (tcgen05)   D_B,g[(i2,j2)][(jj,l)] = sum_{h in g} sum_m P2_h[(i2,j2)][m] A_h[(jj,l)][m]  (Eq. 2.24)
//   stage C (tcgen05)   D_C[(i2,x)][(i1,j1)]   = sum_{g,l} A_C[(i2,x)][(g,l)] P1[(i1,j1)][(g,l)]    (Eq. 2.25)
// with x = j2 + nc2 jj and A_C the stage-B result rearranged in shared memory.  The
// tensor-core products take TF32 operands: every operand is split into a TF32 high part
// and an FP32 remainder and each product is a_lo b_hi + a_hi b_lo + a_hi b_hi, accumulated
// in FP32 in tensor memory (the a_lo b_lo term, 2^-22 relative, is dropped).  One thread
// issues the MMAs; their completion is signalled through an mbarrier (tcgen05.commit), the
// accumulators are read back with tcgen05.ld.
//
// Warp roles (20 warps), one work unit v at a time each, coupled only through mbarriers:
//   producers (warps 0-7):   stage A(v) -> A_h[v & 1]; stage-B epilogue of v-1 (TMEM -> A_C)
//   consumers (warps 8-15):  stage-C epilogue of v (TMEM -> output tile), tile rows to
//                            global memory as 16-byte vector stores
//   MMA issue (warps 16, 17): stage B(v), even / odd g groups, into D_B[v & 1] (double-
//                            buffered where tensor memory allows);
//             (warps 18, 19): stage C(v), even / odd 128-row tiles
// so that stage A, the two epilogues, the tensor-core products and the output stream of
// neighbouring units overlap.  A thread issues one tcgen05.mma about every 100 cycles, the
// tensor core finishes a 128 x 64 x 8 product in about half that: four issuing warps
// keep it busy.  Every mbarrier wait is bounded (about 2^31 cycles); when one runs out the
// CTA stops, releases its tensor memory and records DPG_ERR_TIMEOUT.
#include <cstdint>

#include "dpg_kernels.h"
#include "dpg_tcgen05.cuh"

namespace dpg {

namespace {
using namespace ::dpg::tc;

constexpr int TC_NP = 8;           // producer warps
constexpr int TC_NC = 8;           // consumer warps
constexpr int TC_NMMA = 4;         // MMA-issuing warps: two for stage B, two for stage C
constexpr int TC_NTH = (TC_NP + TC_NC + TC_NMMA) * 32;
constexpr int TC_BAR_P = 1, TC_BAR_C = 2;   // named barriers of the producer / consumer groups

}  // namespace

__global__ void __launch_bounds__(TC_NTH, 1) sf_tc_f32_kernel(TcParams p) {
    extern __shared__ __align__(1024) unsigned char smb[];
    __shared__ BlockDesc bd;
    __shared__ TcLayout f;
    __shared__ int rsh[2][TC_MAXROW];               // tile row r of unit parity u at float r ldt + shift
    __shared__ uint32_t tslot;
    // mbarriers (the first three per unit parity): A_h written, stage B done, stage-B
    // epilogue done; stage C done, stage-C epilogue done (D_C free)
    __shared__ __align__(8) uint64_t bar_ah[2], bar_b[2], bar_eb[2], bar_c, bar_dc;
    __shared__ int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = blockIdx.x % p.nblock;
    const int64_t e0 = (int64_t)(blockIdx.x / p.nblock) * p.elems_per_cta;
    const int64_t e1 = min(e0 + (int64_t)p.elems_per_cta, p.n_elem_dev ? (int64_t)*p.n_elem_dev : p.n_elem);
    if (e0 >= e1) return;
    // element i of the launch -> its output matrix and its metric fields
    const int estart = p.elist_start ? *p.elist_start : 0;
    auto out_of = [&](int64_t i) -> float * {
        return p.out + (p.elist ? p.out_off[p.elist[estart + i]] : i * p.mat_stride);
    };
    auto fields_of = [&](int64_t i) -> const float * {
        return p.fields + (p.elist ? p.foff[p.elist[estart + i]] : i * (int64_t)p.nfields * p.L * p.L * p.L);
    };
    load_block_tc(p.blocks + k, bd);
    __syncthreads();
    const int ub = p.block_unit_begin[k], ue = p.block_unit_begin[k + 1];
    const int64_t ld = p.ld;

    if (bd.ng == 0) {                              // a block without terms: zero rows
        const int nr = bd.nr[0] * bd.nr[1] * bd.nr[2], nc = bd.nc[0] * bd.nc[1] * bd.nc[2];
        const int nw = TC_NTH / 32;
        for (int64_t e = e0; e < e1; ++e) {
            float *o = out_of(e) + bd.base + (int64_t)bd.row_off * ld + bd.col_off;
            for (int r = warp; r < nr; r += nw)
                for (int c = lane; c < nc; c += 32) o[r * ld + c] = 0.0f;
        }
        return;
    }

    if (tid == 0) {
        f = tc_layout(bd, p.L, p.nj_max);
        fail = 0;
        mbar_init(&bar_ah[0], TC_NP);
        mbar_init(&bar_ah[1], TC_NP);
        mbar_init(&bar_b[0], 2);
        mbar_init(&bar_b[1], 2);
        mbar_init(&bar_eb[0], TC_NP);
        mbar_init(&bar_eb[1], TC_NP);
        mbar_init(&bar_c, 2);
        mbar_init(&bar_dc, TC_NC);
    }
    __syncthreads();
#if defined(DPG_DEBUG_BOUNDS)
    // the layout against the launch's shared memory, the tensor-memory columns against the
    // allocation, the unit chunk against the 8 stage-A partners of P3; uniform, before any
    // tensor memory is held
    if (!DPG_INB(f.ok && (unsigned)f.total <= dpg_dyn_smem_bytes() && f.tneed <= f.tcols && p.nj_max <= 8 &&
                 f.nrow <= TC_MAXROW, p.status, e0))
        return;
#endif
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(&tslot)), "r"(f.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }

    const int L = p.L, L2 = L * L, L3 = L2 * L;
    const int lpad = f.lpad, lsh = f.lsh, ksh = f.ksh;
    const int nr1 = f.nr1, nc1 = f.nc1, nc2 = f.nc2, nr2 = f.nr2, nc1p = f.nc1p;
    const int nterm = bd.nterm, nr3 = bd.nr[2], nc3 = bd.nc[2];

    // constant operands (P1, P2: one image per block); A_h and A_C start at zero: their
    // padded k entries (m >= L, l >= L) are never written and must stay zero.  Stage-A
    // factors of every unit of the block: P3T[t][i3][j3][n] = sign_t f3_t(i3, n) f3'_t(j3, n).
    {
        const float4 *src = reinterpret_cast<const float4 *>(p.ctab + p.ctab_off[k]);
        float4 *dst = reinterpret_cast<float4 *>(smb);
        for (int i = tid; i < (f.oAh >> 4); i += TC_NTH) dst[i] = src[i];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = (f.oAh >> 4) + tid; i < (f.oP3 >> 4); i += TC_NTH) dst[i] = z;
        float *P3T = reinterpret_cast<float *>(smb + f.oP3T);
        const int n3 = nterm * nr3 * nc3 * L;
        const unsigned mL = magic(L), mc3 = magic(nc3), mr3 = magic(nr3);
        for (int i = tid; i < n3; i += TC_NTH) {
            const int n = i - mdiv(i, mL) * L, r1 = mdiv(i, mL);
            const int j3 = r1 - mdiv(r1, mc3) * nc3, r2 = mdiv(r1, mc3);
            const int i3 = r2 - mdiv(r2, mr3) * nr3, t = mdiv(r2, mr3);
            const TermDesc &td = bd.term[t];
            const float v = p.pp[(((size_t)(3 * td.kr[2] + td.kc[2]) * NQ1 + i3) * NQ1 + j3) * L + n];
            P3T[i] = td.sign < 0 ? -v : v;
        }
    }
    __syncthreads();
    // P3[t][n][jj] of unit u into buffer b (jj padded to 8 with zeros), by nth threads of
    // ranks 0 .. nth - 1
    auto fill_p3 = [&](const Unit &u, int b, int rank, int nth) {
        float *P3 = reinterpret_cast<float *>(smb + f.oP3 + b * f.p3b);
        const float *P3T = reinterpret_cast<const float *>(smb + f.oP3T);
        const unsigned mL = magic(L);
        for (int it = rank; it < nterm * L * 8; it += nth) {
            const int jj = it & 7, r = it >> 3;
            const int t = mdiv(r, mL), n = r - t * L;
            P3[it] = jj < u.nj ? P3T[((t * nr3 + u.i3) * nc3 + u.j3b + jj) * L + n] : 0.0f;
        }
    };
    if (warp < TC_NP) fill_p3(p.units[ub], 0, tid, TC_NP * 32);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot, sbase = saddr(smb);
    const int nub = ue - ub;
    const int nv = (int)((e1 - e0) * nub);
    const int sp = warp & 3;                      // TMEM lane quarter of this warp

    if (warp < TC_NP) {
        // ================================ producers ================================
        const int wq = warp >> 2;                 // 0, 1: the two producer warps of a quarter
        const int rB = 32 * sp + lane;            // row (i2, j2) of D_B held by this lane
        const int i2B = rB / nc2, j2B = rB - (rB / nc2) * nc2;
        const bool warpB = 32 * sp < f.n22, rowB = rB < f.n22;
        // producer warps without D_B rows (lane quarters >= ceil(n22 / 32)) fill the stage-A
        // factors during the stage-B epilogue; with n22 > 64 every producer warp holds rows
        const int qB = (f.n22 + 31) >> 5;
        const int nfill = qB >= 4 ? 0 : (4 - qB) * 2 * 32;
        const int fill_rank = warpB ? 0 : (wq * (4 - qB) + (sp - qB)) * 32 + lane;
        float *const ach = reinterpret_cast<float *>(smb + f.oAC);
        float *const acl = reinterpret_cast<float *>(smb + f.oAC + f.acb);
        float *const F = reinterpret_cast<float *>(smb + f.oF);
        const int sgC = f.sboC >> 2, sg2 = f.sbo2 >> 2;
        // stage-B epilogue of unit w with nj partners: D_B (stage B of w) into A_C, once
        // stage C of w - 1 has finished reading A_C
        // warps of the lane quarters that hold D_B rows do the epilogue; the others fill the
        // next unit's stage-A factors (next_unit >= 0) meanwhile
        auto epi_b = [&](int nj, int w, int next_unit, int next_buf) {
            if (!warpB && next_unit >= 0) fill_p3(p.units[next_unit], next_buf, fill_rank, nfill);
            mbar_wait(&bar_b[w & 1], (uint32_t)((w >> 1) & 1), &fail);
            if (w > 0) mbar_wait(&bar_c, (uint32_t)((w - 1) & 1), &fail);
            const int dB = (f.nbB == 2 ? (w & 1) : 0) * bd.ng * f.NB;     // D_B buffer of unit w
            tc_fence_after();
            if (warpB) {
                const int nx = nc2 * nj, nch = (nj * lpad + 15) >> 4, nit = bd.ng * nch;
                const unsigned mnch = magic(nch);
                for (int it = 2 * wq; it < nit; it += 4) {
                    const int it1 = it + 1 < nit ? it + 1 : it;
                    const int g0 = mdiv(it, mnch), c00 = (it - g0 * nch) << 4;
                    const int g1 = mdiv(it1, mnch), c01 = (it1 - g1 * nch) << 4;
                    uint32_t r[32];
                    tmem_ld16x2(tbase + ((uint32_t)(32 * sp) << 16) + (uint32_t)(dB + g0 * f.NB + c00),
                                tbase + ((uint32_t)(32 * sp) << 16) + (uint32_t)(dB + g1 * f.NB + c01), r);
                    if (rowB) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            if (hh == 1 && it1 == it) break;
                            const int g = hh ? g1 : g0, c0 = hh ? c01 : c00;
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const int col = c0 + 4 * q4, jj = col >> lsh, l0 = col & (lpad - 1);
                                if (jj < nj) {
                                    const int R = i2B * nx + j2B + nc2 * jj, K = g * lpad + l0;
                                    const int off = (R >> 3) * sgC + (K >> 2) * 32 + (R & 7) * 4;
                                    float4 hv, lv;
                                    tf32_split(__uint_as_float(r[16 * hh + 4 * q4 + 0]), hv.x, lv.x);
                                    tf32_split(__uint_as_float(r[16 * hh + 4 * q4 + 1]), hv.y, lv.y);
                                    tf32_split(__uint_as_float(r[16 * hh + 4 * q4 + 2]), hv.z, lv.z);
                                    tf32_split(__uint_as_float(r[16 * hh + 4 * q4 + 3]), hv.w, lv.w);
                                    *reinterpret_cast<float4 *>(ach + off) = hv;
                                    *reinterpret_cast<float4 *>(acl + off) = lv;
                                }
                            }
                        }
                    }
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_eb[w & 1]);
        };
        int64_t e = e0, fe_loaded = -1;
        int ui = ub, pnj = 0, pnj_next = 0;
        bool stopped = false;
        for (int v = 0; v < nv; ++v) {
            const Unit u = p.units[ui];
            const int nj = u.nj;
            if (e != fe_loaded) {                  // metric fields of the element's terms
                const float *src = fields_of(e);
                for (int sl = 0; sl < f.nfs; ++sl) {
                    const float *fs = src + (size_t)bd.slot_field[sl] * L3;
                    for (int i = tid; i < L3; i += TC_NP * 32) cp_async4(F + sl * L3 + i, fs + i);
                }
                cp_async_wait_all();
                fe_loaded = e;
                group_sync_or(TC_BAR_P, TC_NP * 32, 0);
            }
            // stage A (FMA pipe) into A_h[v & 1], split into TF32 high / low parts
            {
                const float *P3 = reinterpret_cast<const float *>(smb + f.oP3 + (v & 1) * f.p3b);
                unsigned char *ahv = smb + f.oAh + (v & 1) * f.ahbuf;
                for (int it = tid; it < (bd.nh << (2 * lsh)); it += TC_NP * 32) {
                    const int l = it & (lpad - 1), m = (it >> lsh) & (lpad - 1), h = it >> (2 * lsh);
                    if (l >= L || m >= L) continue;
                    float acc[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0f;
                    const int nt = bd.h_nterm[h];
                    for (int ti = 0; ti < nt; ++ti) {
                        const int t = bd.h_terms[h][ti];
                        const float *M = F + bd.term_slot[t] * L3 + l * L2 + m * L;
                        const float4 *Pt = reinterpret_cast<const float4 *>(P3 + t * L * 8);
#pragma unroll 4
                        for (int n = 0; n < L; ++n) {
                            const float mv = M[n];
                            const float4 q0 = Pt[2 * n], q1 = Pt[2 * n + 1];
                            acc[0] = fmaf(mv, q0.x, acc[0]); acc[1] = fmaf(mv, q0.y, acc[1]);
                            acc[2] = fmaf(mv, q0.z, acc[2]); acc[3] = fmaf(mv, q0.w, acc[3]);
                            acc[4] = fmaf(mv, q1.x, acc[4]); acc[5] = fmaf(mv, q1.y, acc[5]);
                            acc[6] = fmaf(mv, q1.z, acc[6]); acc[7] = fmaf(mv, q1.w, acc[7]);
                        }
                    }
                    float *dh = reinterpret_cast<float *>(ahv + 2 * h * f.ahb) + (m >> 2) * 32 + (m & 3);
                    float *dl = dh + (f.ahb >> 2);
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj)
                        if (jj < nj) {
                            const int r = jj * lpad + l;
                            const int off = (r >> 3) * sg2 + (r & 7) * 4;
                            float hi, lo;
                            tf32_split(acc[jj], hi, lo);
                            dh[off] = hi;
                            dl[off] = lo;
                        }
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_ah[v & 1]);
            // stage-B epilogue of the previous unit (its stage B ran while stage A ran), the
            // next unit's stage-A factors
            pnj_next = nj;
            if (++ui == ue) { ui = ub; ++e; }
            const int nxt = v + 1 < nv ? ui : -1;
            if (v > 0 && nfill > 0) {
                epi_b(pnj, v - 1, nxt, (v + 1) & 1);
            } else {
                if (v > 0) epi_b(pnj, v - 1, -1, 0);
                if (nxt >= 0) fill_p3(p.units[nxt], (v + 1) & 1, tid, TC_NP * 32);
            }
            pnj = pnj_next;
            if (group_sync_or(TC_BAR_P, TC_NP * 32, fail)) { stopped = true; break; }
        }
        if (!stopped) epi_b(pnj, nv - 1, -1, 0);
    } else if (warp < TC_NP + TC_NC) {
        // ================================ consumers ================================
        const int ct = tid - TC_NP * 32, cw = warp - TC_NP, wq = cw >> 2;
        float *const T = reinterpret_cast<float *>(smb + f.oT);
        const int nch = f.NC >> 4;                // 16-column groups of D_C per tile
        const unsigned mnch = magic(nch);
        // destination of tile row r of unit u (element e) and its row shift
        auto out_row = [&](int64_t e, const Unit &u, int r) -> float * {
            return out_of(e) + bd.base + (bd.row_off + (int64_t)u.i3 * f.nrow + r) * ld +
                   bd.col_off + (int64_t)u.j3b * nc1 * nc2;
        };
        auto set_rows = [&](int64_t e, const Unit &u, int b) {
            for (int r = ct; r < f.nrow; r += TC_NC * 32)
                rsh[b][r] = r * f.ldt + (int)((reinterpret_cast<uintptr_t>(out_row(e, u, r)) >> 2) & 3);
        };
        int64_t e = e0;
        int ui = ub;
        set_rows(e, p.units[ui], 0);
        group_sync_or(TC_BAR_C, TC_NC * 32, 0);
        for (int v = 0; v < nv; ++v) {
            const Unit u = p.units[ui];
            const int b = v & 1;
            const int ncol = nc1 * nc2 * u.nj;
            // stage-C epilogue: D_C (rows (i2, x), columns i1 nc1p + j1) into the tile
            mbar_wait(&bar_c, (uint32_t)(v & 1), &fail);
            tc_fence_after();
            {
                const int nx = nc2 * u.nj, mc = nr2 * nx, mt = (mc + 127) >> 7;
                const unsigned mnx = magic(nx);
                const int nit = mt * nch;
                for (int it = 2 * wq; it < nit; it += 4) {
                    // items it and it + 1 (16 columns each) in one round trip
                    const int it1 = it + 1 < nit ? it + 1 : it;
                    const int t0 = mdiv(it, mnch), c00 = (it - t0 * nch) << 4;
                    const int t1 = mdiv(it1, mnch), c01 = (it1 - t1 * nch) << 4;
                    uint32_t r[32];
                    tmem_ld16x2(tbase + ((uint32_t)(32 * sp) << 16) + (uint32_t)(f.tcolC + t0 * f.NC + c00),
                                tbase + ((uint32_t)(32 * sp) << 16) + (uint32_t)(f.tcolC + t1 * f.NC + c01), r);
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        if (hh == 1 && it1 == it) break;
                        const int t = hh ? t1 : t0, c0 = hh ? c01 : c00;
                        const int R = 128 * t + 32 * sp + lane;
                        if (R < mc) {
                            const int i2 = mdiv(R, mnx), x = R - i2 * nx;
                            const int *rs = &rsh[b][nr1 * i2];
#pragma unroll
                            for (int g8 = 0; g8 < 2; ++g8) {       // 8-column groups: one i1 each
                                const int cc = c0 + 8 * g8, i1 = cc / nc1p, j1b = cc - i1 * nc1p;
                                if (i1 < nr1) {
                                    float *trow = T + rs[i1] + nc1 * x + j1b;
#pragma unroll
                                    for (int j = 0; j < 8; ++j)
                                        if (j1b + j < nc1) trow[j] = __uint_as_float(r[16 * hh + 8 * g8 + j]);
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_dc);
            if (group_sync_or(TC_BAR_C, TC_NC * 32, fail)) break;
            // tile rows to global memory: one warp per row, 16-byte vector stores for the
            // aligned middle, plain stores for the ends
            for (int r = cw; r < f.nrow; r += TC_NC) {
                if (!DPG_INB((bd.row_off + (int64_t)u.i3 * f.nrow + r) * ld + bd.col_off +
                             (int64_t)u.j3b * nc1 * nc2 + ncol <= p.mat_stride - bd.base, p.status, e))
                    continue;
                const float *trow = T + rsh[b][r];
                float *orow = out_row(e, u, r);
                const int head = min((4 - (int)((reinterpret_cast<uintptr_t>(orow) >> 2) & 3)) & 3, ncol);
                const int n4 = (ncol - head) >> 2, tail = head + 4 * n4;
                if (lane < head) orow[lane] = trow[lane];
                if (lane < ncol - tail) orow[tail + lane] = trow[tail + lane];
                const float4 *t4 = reinterpret_cast<const float4 *>(trow + head);
                float4 *o4 = reinterpret_cast<float4 *>(orow + head);
                for (int c = lane; c < n4; c += 32) o4[c] = t4[c];
            }
            if (++ui == ue) { ui = ub; ++e; }
            if (v + 1 < nv) set_rows(e, p.units[ui], b ^ 1);
            if (group_sync_or(TC_BAR_C, TC_NC * 32, fail)) break;
        }
    } else if (lane == 0) {
        // ================================ MMA issue ================================
        const int mw = warp - TC_NP - TC_NC;      // 0 / 1: stage B, 2 / 3: stage C
        const int par = mw & 1;                   // g groups (stage B) / tiles (stage C) of this parity
        // descriptor of the operand `off` bytes further (the start-address field, in 16 bytes)
        auto adv = [](uint64_t d, uint32_t off) { return d + (uint64_t)(off >> 4); };
        int ui = ub;
        if (mw < 2) {
            const uint64_t dP2 = sdesc(sbase + f.oP2, f.sbo2), dAh = sdesc(sbase + f.oAh, f.sbo2);
            // test hook (dpg_test_stall_tc_once): the stage-B completion of this CTA never
            // arrives, so its bounded waits run out and the CTA reports DPG_ERR_TIMEOUT
            const int nvB = (int)blockIdx.x == p.stall_cta ? 0 : nv;
            for (int v = 0; v < nvB; ++v) {
                const Unit u = p.units[ui];
                mbar_wait(&bar_ah[v & 1], (uint32_t)((v >> 1) & 1), &fail);
                // the D_B buffer of this unit has been read out (unit v - 2, or v - 1 when
                // single-buffered)
                const int wprev = v - f.nbB;
                if (wprev >= 0) mbar_wait(&bar_eb[wprev & 1], (uint32_t)((wprev >> 1) & 1), &fail);
                if (fail) break;
                tc_fence_after();
                const uint32_t idB = idesc_tf32(128, (u.nj * lpad + 15) & ~15);
                const uint32_t oab = (v & 1) * f.ahbuf;
                const uint32_t dB = (f.nbB == 2 ? (v & 1) : 0) * bd.ng * f.NB;
                for (int g = par; g < bd.ng; g += 2) {
                    uint32_t acc = 0;
                    for (int hi = 0; hi < bd.g_nh[g]; ++hi) {
                        const int h = bd.g_hs[g][hi];
                        const uint32_t oa = 2 * bd.h_p2[h] * f.p2b, ob = oab + 2 * h * f.ahb;
                        for (int ks = 0; ks < ksh; ++ks) {
                            umma3(tbase + dB + g * f.NB, adv(dP2, oa + ks * 256), adv(dP2, oa + f.p2b + ks * 256),
                                  adv(dAh, ob + ks * 256), adv(dAh, ob + f.ahb + ks * 256), idB, acc);
                            acc = 1;
                        }
                    }
                }
                umma_commit(&bar_b[v & 1]);
                if (++ui == ue) ui = ub;
            }
        } else {
            const uint32_t idC = idesc_tf32(128, f.NC);
            const uint64_t dP1h = sdesc(sbase + f.oP1, f.sboC), dP1l = sdesc(sbase + f.oP1 + f.p1b, f.sboC);
            const uint64_t dACh = sdesc(sbase + f.oAC, f.sboC), dACl = sdesc(sbase + f.oAC + f.acb, f.sboC);
            const int nk = bd.ng * ksh;
            for (int v = 0; v < nv; ++v) {
                const Unit u = p.units[ui];
                mbar_wait(&bar_eb[v & 1], (uint32_t)((v >> 1) & 1), &fail);      // A_C of v written
                if (v > 0) mbar_wait(&bar_dc, (uint32_t)((v - 1) & 1), &fail);    // D_C read out
                if (fail) break;
                tc_fence_after();
                const int mt = (nr2 * nc2 * u.nj + 127) >> 7;
                for (int t = par; t < mt; t += 2)
                    for (int kk = 0; kk < nk; ++kk) {
                        const uint32_t oa = t * 16 * f.sboC + kk * 256, ob = kk * 256;
                        umma3(tbase + f.tcolC + t * f.NC, adv(dACh, oa), adv(dACl, oa), adv(dP1h, ob), adv(dP1l, ob),
                              idC, kk > 0 ? 1u : 0u);
                    }
                umma_commit(&bar_c);
                if (++ui == ue) ui = ub;
            }
        }
    }
    tc_fence_before();
    const int failed = __syncthreads_or(fail);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(f.tcols));
    }
    if (failed && tid == 0) report_tc(p.status, 9 /*DPG_ERR_TIMEOUT*/, e0);
}

// --------------------------------------------------------------------------------------
// TF32 tensor-core rate probe (not part of the method): the denominator of the roofline of
// the 3xTF32 stages.  One CTA per SM (its dynamic shared memory admits no second CTA);
// one thread issues `iters` rounds of two kind::tf32 products of 128 x 256 x 8 into two
// accumulators of 256 tensor-memory columns each, completion through one mbarrier (a
// bounded wait: a wait that runs out sets *status and the CTA still releases its tensor
// memory).  Operands are K-major no-swizzle tiles of zeros.
// --------------------------------------------------------------------------------------
constexpr int TCP_SMEM = 160 * 1024;

__global__ void __launch_bounds__(128, 1) tc_tf32_peak_kernel(int iters, int *status) {
    extern __shared__ __align__(1024) unsigned char smb[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int fail;
    float *sA = reinterpret_cast<float *>(smb);            // 128 rows x 8: 4 KB
    float *sB = sA + 128 * 8;                              // 256 rows x 8: 8 KB
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < 384 * 8; i += 128) sA[i] = 0.0f;
    if (tid == 0) {
        fail = 0;
        mbar_init(&bar, 1);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(&tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot;
    if (tid == 0) {
        const uint32_t id = idesc_tf32(128, 256);
        const uint64_t dA = sdesc(saddr(sA), 256), dB = sdesc(saddr(sB), 256);
        for (int i = 0; i < iters; ++i) {
            umma(tbase, dA, dB, id, i > 0 ? 1u : 0u);
            umma(tbase + 256, dA, dB, id, i > 0 ? 1u : 0u);
        }
        umma_commit(&bar);
    }
    __syncwarp();
    mbar_wait(&bar, 0u, &fail);
    tc_fence_before();
    const int failed = __syncthreads_or(fail);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512));
    }
    if (failed && tid == 0) atomicExch(status, 1);
}

cudaError_t launch_tc_tf32_peak(int ctas, int iters, int *status, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute((const void *)tc_tf32_peak_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc_tf32_peak_kernel<<<ctas, 128, TCP_SMEM, s>>>(iters, status);
    return cudaGetLastError();
}

cudaError_t launch_tc_f32(const TcParams &p, size_t smem, cudaStream_t s) {
    if (p.n_elem == 0) return cudaSuccess;
    const int64_t chunks = (p.n_elem + p.elems_per_cta - 1) / p.elems_per_cta;
    const int64_t ctas = chunks * p.nblock;
    sf_tc_f32_kernel<<<(unsigned)ctas, TC_NTH, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t init_tc_attributes(int optin_smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)sf_tc_f32_kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)sf_tc_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin_smem - (int)a.sharedSizeBytes);
}

int tc_static_smem() {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void *)sf_tc_f32_kernel) != cudaSuccess) return -1;
    return (int)a.sharedSizeBytes;
}

}  // namespace dpg
