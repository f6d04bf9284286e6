// dpg_tcc.cu -- FP32 form of the general (trilinear-map) path with stage C on the
// fifth-generation tensor cores, for uniform batches and for mixed-order (hp) batches.
//
// A CTA walks a contiguous range of work items (element, block (a, b), i3) -- block-major,
// so that a block's constant operands are loaded once per run of items and an element's
// metric fields once per run of its i3 -- and computes every partner j3 of an item:
//   stage A (FMA pipe)   A_h[m][j3][l] = sum_{t in h} sum_n M_t(l,m,n) P3_t(n, j3)                (Eq. 2.23)
//   stage B (FMA pipe)   A_C[(i2,x)][(g,l)] = sum_{h in g} sum_m P2_h(m)[i2,j2] A_h[m][j3][l]      (Eq. 2.24)
//   stage C (tcgen05)    D[(i2,x)][(i1,j1)] = sum_{g,l} A_C[(i2,x)][(g,l)] P1[(i1,j1)][(g,l)]       (Eq. 2.25)
// with x = j2 + nc2 j3, in the paper's direction order and with every block of the matrix
// computed (no mirrored tiles).  The stage-C operands are split into TF32 high and low
// parts, D accumulates a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32 in tensor memory (the
// a_lo b_lo term, 2^-22 relative, is dropped).  Stage C runs in tiles of at most 128 rows
// (i2, x); one thread issues a tile's products and commits them to an mbarrier, and the
// CTA computes the next tile's stage B meanwhile, then moves the previous tile's
// accumulator (the other of two) to the output: each warp reads 32 rows of one i1 from
// tensor memory and every lane stores its nc1 consecutive columns of output row
// (i1, i2, i3) (lanes hold consecutive x: a warp's stores cover contiguous runs).  Waits are bounded: a wait that runs out
// stops the CTA, which releases its tensor memory and records DPG_ERR_TIMEOUT.
#include <cstdint>

#include "dpg_kernels.h"
#include "dpg_tcgen05.cuh"

namespace dpg {

namespace {
using namespace ::dpg::tc;

// Row rho of stage-C tile t: (i2, x); false for a padding row.
__device__ __forceinline__ bool tcc_row(const TccLayout &f, int t, int rho, unsigned mnx, int &i2, int &x) {
    if (f.ipt > 0) {
        const int di = mdiv(rho, mnx);
        i2 = t * f.ipt + di;
        x = rho - di * f.nx;
        return di < f.ipt && i2 < f.nr2;
    }
    const int c = t % f.nxc;
    i2 = t / f.nxc;
    x = c * 128 + rho;
    return x < f.nx;
}

// Stage A (Eq. 2.23) of one item: thread = (h, l, m), the NC4 x 4 partners j3 in registers.
template <int NC4>
__device__ __forceinline__ void tcc_stage_a(const TccLayout &f, const BlockDesc &bd, const float *F, const float *P3,
                                            float *A, int L, unsigned mLL, unsigned mL, int tid) {
    const int L2 = L * L, npad = f.npad, nc3 = f.nc3, lpad = f.lpad;
    for (int task = tid; task < bd.nh * L2; task += TCC_NTH) {
        const int h = mdiv(task, mLL), lm = task - h * L2;
        const int l = mdiv(lm, mL), m = lm - l * L;
        float acc[4 * NC4];
#pragma unroll
        for (int j = 0; j < 4 * NC4; ++j) acc[j] = 0.0f;
        for (int ti = 0; ti < bd.h_nterm[h]; ++ti) {
            const int t = bd.h_terms[h][ti];
            const float *Mt = F + (bd.term_slot[t] * L2 + l * L + m) * npad;
            const float4 *Pt = reinterpret_cast<const float4 *>(P3 + t * L * 4 * NC4);
            for (int n = 0; n < L; ++n) {
                const float mv = Mt[n];
#pragma unroll
                for (int c4 = 0; c4 < NC4; ++c4) {
                    const float4 q4 = Pt[n * NC4 + c4];
                    acc[4 * c4 + 0] = fmaf(mv, q4.x, acc[4 * c4 + 0]);
                    acc[4 * c4 + 1] = fmaf(mv, q4.y, acc[4 * c4 + 1]);
                    acc[4 * c4 + 2] = fmaf(mv, q4.z, acc[4 * c4 + 2]);
                    acc[4 * c4 + 3] = fmaf(mv, q4.w, acc[4 * c4 + 3]);
                }
            }
        }
        float *dst = A + ((h * L + m) * nc3) * lpad + l;
#pragma unroll
        for (int j = 0; j < 4 * NC4; ++j)
            if (j < nc3) dst[j * lpad] = acc[j];
    }
}

// Stage B (Eq. 2.24) of tile t: thread = (g, row rho), the LP4 x 4 values l in registers,
// written split into TF32 high and low parts to the stage-C A operand.
template <int LP4>
__device__ __forceinline__ void tcc_stage_b(const TccLayout &f, const BlockDesc &bd, int t, unsigned mnx,
                                            unsigned mnc2, const float *P2s, const float *A, float *ach, float *acl,
                                            int L, int tid) {
    constexpr int lpad = 4 * LP4;
    const int sg = f.sbo >> 2, nc3 = f.nc3;
    for (int task = tid; task < bd.ng * 128; task += TCC_NTH) {
        const int g = task >> 7, rho = task & 127;
        int i2, x;
        if (!tcc_row(f, t, rho, mnx, i2, x)) continue;
        const int j3 = mdiv(x, mnc2), j2 = x - j3 * f.nc2;
        float acc[lpad];
#pragma unroll
        for (int j = 0; j < lpad; ++j) acc[j] = 0.0f;
        for (int hi = 0; hi < bd.g_nh[g]; ++hi) {
            const int h = bd.g_hs[g][hi];
            const float *p2 = P2s + bd.h_p2[h] * L * f.n22p + i2 * f.nc2 + j2;
            const float4 *ah = reinterpret_cast<const float4 *>(A + ((h * L) * nc3 + j3) * lpad);
            for (int m = 0; m < L; ++m) {
                const float pv = p2[m * f.n22p];
                const float4 *a4 = ah + m * nc3 * LP4;
#pragma unroll
                for (int c4 = 0; c4 < LP4; ++c4) {
                    const float4 av = a4[c4];
                    acc[4 * c4 + 0] = fmaf(pv, av.x, acc[4 * c4 + 0]);
                    acc[4 * c4 + 1] = fmaf(pv, av.y, acc[4 * c4 + 1]);
                    acc[4 * c4 + 2] = fmaf(pv, av.z, acc[4 * c4 + 2]);
                    acc[4 * c4 + 3] = fmaf(pv, av.w, acc[4 * c4 + 3]);
                }
            }
        }
#pragma unroll
        for (int c4 = 0; c4 < LP4; ++c4) {
            const int k0 = g * lpad + 4 * c4;
            const int off = (rho >> 3) * sg + (k0 >> 2) * 32 + (rho & 7) * 4;
            float4 hv, lv;
            tf32_split(acc[4 * c4 + 0], hv.x, lv.x);
            tf32_split(acc[4 * c4 + 1], hv.y, lv.y);
            tf32_split(acc[4 * c4 + 2], hv.z, lv.z);
            tf32_split(acc[4 * c4 + 3], hv.w, lv.w);
            *reinterpret_cast<float4 *>(ach + off) = hv;
            *reinterpret_cast<float4 *>(acl + off) = lv;
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(TCC_NTH, 3) sf_tcc_kernel(TccParams p) {
    extern __shared__ __align__(1024) unsigned char smb[];
    __shared__ BlockDesc bd;
    __shared__ TccLayout f;
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ne = p.n_elem_dev ? (int64_t)*p.n_elem_dev : p.n_elem;
    const int estart = p.elist_start ? *p.elist_start : 0;
    const int64_t nitems = p.blk_base[p.nblock];
    const int64_t total = ne * nitems;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per;
    const int64_t it1 = min(total, it0 + per);
    if (it0 >= it1) return;
    if (tid == 0) {
        fail = 0;
        mbar_init(&bar, 1);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(saddr(&tslot)), "r"(p.tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tslot, sbase = saddr(smb);
    const int L = p.L, L2 = L * L, L3 = L2 * L;
    const int64_t ld = p.ld;

    int cur_block = -1;                            // block whose constants are loaded
    int64_t cur_e = -1;                            // element whose fields are staged (for cur_block)
    uint32_t ncommit = 0;                          // committed tiles (uniform over the CTA)
    // the tile whose accumulator awaits its epilogue
    bool pend = false;
    int64_t pend_e = 0;
    int pend_i3 = 0, pend_t = 0;
    unsigned mnx = 0, mnc2 = 0, mLL = 0, mL = 0, mnc3p = 0;
    auto adv = [](uint64_t d, uint32_t off) { return d + (uint64_t)(off >> 4); };

    // ---- epilogue of a finished tile: accumulator buffer dbuf -> output rows
    auto epilogue = [&](int64_t e, int i3, int t, uint32_t dbuf) {
        const int64_t obase = (p.out_off ? p.out_off[e] : e * p.mat_stride) + bd.base;
        float *oe = p.out + obase;
        const int qd = warp & 3, half = warp >> 2;
        const int rho = 32 * qd + lane;
        int i2 = 0, x = 0;
        const bool valid = tcc_row(f, t, rho, mnx, i2, x);
        const int nc1 = f.nc1, nr1 = f.nr1;
        const int64_t rowi = (int64_t)bd.row_off + nr1 * i2 + (int64_t)nr1 * f.nr2 * i3;
        for (int i1 = half; i1 < nr1; i1 += 2) {
            uint32_t r[16];
            tmem_ld16(tbase + ((uint32_t)(32 * qd) << 16) + dbuf * (uint32_t)f.N + (uint32_t)(i1 * nc1), r);
            // the lane's nc1 consecutive columns of output row (i1, i2, i3); the lanes of a
            // warp hold consecutive x, so a warp's stores cover one contiguous run per i2
            const int64_t d0 = (rowi + i1) * ld + bd.col_off + (int64_t)x * nc1;
            if (valid && DPG_INB(d0 + nc1 <= p.mat_stride - bd.base, p.status, e)) {
                float *od = oe + d0;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < nc1) od[j] = __uint_as_float(r[j]);
            }
        }
    };

    for (int64_t it = it0; it < it1; ++it) {
        // ---- decode the item: block k (block-major), element-local index, i3
        int k = 0;
        while (k + 1 < p.nblock && it >= (int64_t)p.blk_base[k + 1] * ne) ++k;
        const int64_t rel = it - (int64_t)p.blk_base[k] * ne;
        const int nr3k = p.blk_base[k + 1] - p.blk_base[k];
        // (32-bit division where the index allows: a 64-bit division costs far more)
        const int64_t le = rel < 0x7fffffffLL ? (int64_t)((unsigned)rel / (unsigned)nr3k) : rel / nr3k;
        const int i3 = (int)(rel - le * nr3k);
        const int64_t e = p.elist ? (int64_t)p.elist[estart + le] : le;

        if (k != cur_block) {
            // the pending tile belongs to the loaded block: finish it first
            if (pend) {
                mbar_wait(&bar, (ncommit - 1) & 1, &fail);
                tc_fence_after();
                epilogue(pend_e, pend_i3, pend_t, (ncommit - 1) & 1);
                pend = false;
                tc_fence_before();
            }
            __syncthreads();
            load_block_tc(p.blocks + k, bd);
            __syncthreads();
            if (tid == 0) f = tcc_layout(bd, L);
            __syncthreads();
#if defined(DPG_DEBUG_BOUNDS)
            if (!DPG_INB(f.ok && f.total <= p.smem_bytes && f.tcols <= p.tcols &&
                         (p.img_off[k + 1] - p.img_off[k]) * 4 <= f.oC, p.status, e)) {
                fail = 2;
                break;                                          // uniform
            }
#endif
            {
                const float4 *src = reinterpret_cast<const float4 *>(p.img + p.img_off[k]);
                float4 *dst = reinterpret_cast<float4 *>(smb);
                const int n4 = (p.img_off[k + 1] - p.img_off[k]) >> 2;
                for (int i = tid; i < n4; i += TCC_NTH) dst[i] = src[i];
                // A_C starts at zero: its padded k columns are never written
                float4 *ac = reinterpret_cast<float4 *>(smb + f.oAC);
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int i = tid; i < (2 * f.acb) >> 4; i += TCC_NTH) ac[i] = z;
            }
            mnx = magic(f.nx); mnc2 = magic(f.nc2); mLL = magic(L2); mL = magic(L); mnc3p = magic(f.nc3p);
            cur_block = k;
            cur_e = -1;
        }
        if (__syncthreads_or(fail)) break;

        // ---- the element's metric fields (once per element and block) and the stage-A
        //      factors of i3: P3[t][n][j3] = sign_t f3_t(i3, n) f3'_t(j3, n)
        float *F = reinterpret_cast<float *>(smb + f.oF);
        float *P3 = reinterpret_cast<float *>(smb + f.oP3);
        float *A = reinterpret_cast<float *>(smb + f.oA);
        const int npad = f.npad, nc3 = f.nc3, nc3p = f.nc3p, lpad = f.lpad;
        if (e != cur_e) {
            const float *fe = p.fields + (p.foff ? p.foff[e] : e * (int64_t)p.nfields * L3);
            for (int sl = 0; sl < bd.nslot; ++sl) {
                const float *fs = fe + (int64_t)bd.slot_field[sl] * L3;
                float *ds = F + sl * L2 * npad;
                for (int i = tid; i < L3; i += TCC_NTH) {
                    const int lm = mdiv(i, mL), n = i - lm * L;
                    ds[lm * npad + n] = fs[i];
                }
            }
            cur_e = e;
        }
        for (int i = tid; i < bd.nterm * L * nc3p; i += TCC_NTH) {
            const int r = mdiv(i, mnc3p), j3 = i - r * nc3p;
            const int t = mdiv(r, mL), n = r - t * L;
            const TermDesc &td = bd.term[t];
            float v = 0.0f;
            if (j3 < nc3) {
                v = p.pp[(((size_t)(3 * td.kr[2] + td.kc[2]) * NQ1 + i3) * NQ1 + j3) * L + n];
                if (td.sign < 0) v = -v;
            }
            P3[i] = v;
        }
        __syncthreads();

        // ---- stage A (Eq. 2.23)
        switch (nc3p >> 2) {
        case 1: tcc_stage_a<1>(f, bd, F, P3, A, L, mLL, mL, tid); break;
        case 2: tcc_stage_a<2>(f, bd, F, P3, A, L, mLL, mL, tid); break;
        case 3: tcc_stage_a<3>(f, bd, F, P3, A, L, mLL, mL, tid); break;
        default: tcc_stage_a<4>(f, bd, F, P3, A, L, mLL, mL, tid); break;
        }
        // padded l entries of A are read by stage B's 16-byte loads: keep them zero
        if (lpad > L)
            for (int i = tid; i < bd.nh * L * nc3 * (lpad - L); i += TCC_NTH) {
                const int r = i / (lpad - L), l = L + (i - r * (lpad - L));
                A[r * lpad + l] = 0.0f;
            }
        __syncthreads();

        // ---- stage C tiles: stage B of tile t, its products, the previous tile's epilogue
        const float *P2s = reinterpret_cast<const float *>(smb + f.oP2);
        float *ach = reinterpret_cast<float *>(smb + f.oAC);
        float *acl = reinterpret_cast<float *>(smb + f.oAC + f.acb);
        for (int t = 0; t < f.ntile; ++t) {
            if (ncommit > 0) mbar_wait(&bar, (ncommit - 1) & 1, &fail);   // A_C is free again
            tc_fence_after();
            switch (lpad >> 2) {
            case 1: tcc_stage_b<1>(f, bd, t, mnx, mnc2, P2s, A, ach, acl, L, tid); break;
            case 2: tcc_stage_b<2>(f, bd, t, mnx, mnc2, P2s, A, ach, acl, L, tid); break;
            case 3: tcc_stage_b<3>(f, bd, t, mnx, mnc2, P2s, A, ach, acl, L, tid); break;
            default: tcc_stage_b<4>(f, bd, t, mnx, mnc2, P2s, A, ach, acl, L, tid); break;
            }
            fence_async_smem();
            tc_fence_before();
            if (__syncthreads_or(fail)) break;
            const uint32_t dbuf = ncommit & 1;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t id = idesc_tf32(128, f.N);
                const uint64_t dAh = sdesc(sbase + f.oAC, f.sbo), dAl = sdesc(sbase + f.oAC + f.acb, f.sbo);
                const uint64_t dBh = sdesc(sbase + f.oP1, f.sbo), dBl = sdesc(sbase + f.oP1 + f.p1b, f.sbo);
                const uint32_t d = tbase + dbuf * (uint32_t)f.N;
                for (int ks = 0; ks < f.ksteps; ++ks)
                    umma3(d, adv(dAh, ks * 256), adv(dAl, ks * 256), adv(dBh, ks * 256), adv(dBl, ks * 256), id,
                          ks > 0 ? 1u : 0u);
                // test hook (dpg_test_stall_tc_once): the completion never arrives, the CTA's
                // bounded wait runs out and it reports DPG_ERR_TIMEOUT
                if ((int)blockIdx.x != p.stall_cta) umma_commit(&bar);
            }
            ++ncommit;
            if (pend) {
                tc_fence_after();
                epilogue(pend_e, pend_i3, pend_t, dbuf ^ 1u);
                tc_fence_before();
            }
            pend = true;
            pend_e = e; pend_i3 = i3; pend_t = t;
        }
        if (__syncthreads_or(fail)) break;
    }
    if (!fail && pend) {
        mbar_wait(&bar, (ncommit - 1) & 1, &fail);
        tc_fence_after();
        if (!fail) epilogue(pend_e, pend_i3, pend_t, (ncommit - 1) & 1);
        tc_fence_before();
    }
    __syncthreads();
    const int failed = fail;                      // 1: a wait ran out; 2: a bounds check failed
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(p.tcols));
    }
    if (failed == 1 && tid == 0) report_tc(p.status, 9 /*DPG_ERR_TIMEOUT*/, p.elist ? 0 : it0 / nitems);
}

cudaError_t launch_tcc(const TccParams &p, int grid, size_t smem, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    sf_tcc_kernel<<<grid, TCC_NTH, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t init_tcc_attributes(int optin_smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)sf_tcc_kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)sf_tcc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin_smem - (int)a.sharedSizeBytes);
}

int tcc_static_smem() {
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, (const void *)sf_tcc_kernel) != cudaSuccess) return -1;
    return (int)a.sharedSizeBytes;
}

}  // namespace dpg
