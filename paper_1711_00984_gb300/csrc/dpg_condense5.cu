// dpg_condense5.cu -- static condensation of the DPG test variables (Eq. 3.8 from Eq. 3.7)
// with the digit products on the fifth-generation tensor cores (tcgen05, BF16 operands,
// FP32 accumulators in tensor memory).
//
// Per element the paper's steps: G = L L^T, W = L^-1 B, y = L^-1 l, K = W^T W, F = W^T y.
// One CTA per element at a time (persistent), one CTA per SM; right-looking blocked
// Cholesky in panels of 64 columns, the load vector carried as column m of the right-hand
// side [B | l], so that F is row m of the extended product [W | y]^T [W | y].  Per panel kb:
//   F-phase (FP64, shared memory): the 64 x 64 diagonal block is factored, L11 is written to
//     G and X = L11^-1 formed by forward substitution.
//   P-phase (panel products, digits): L21 = A21 X^T in 128-row blocks and W1^T = B1^T X^T
//     in 128-column blocks: the rows of A21 (of B1^T) and of X are split into seven BF16
//     digit planes, the products run on the tensor cores, the FP64 results are written back
//     (G below the block, rows kb.. of [B | l]) and split once more into digit planes kept
//     in a per-CTA scratch in global memory (row exponents beside them).
//   T-phase (trailing updates, pipelined): G22 -= L21 L21^T (lower triangle),
//     [B | l]_2 -= L21 W1 and [K | F] += W1^T W1 (lower triangle), as 128 x (<= 64) tiles;
//     warp 8 loads each tile's digit planes with bulk copies (two buffers) and issues its
//     products, the eight other warps drain the accumulators of the previous tile and
//     apply its FP64 update while the tensor core works on the next one.
// Digit products (as in the mma.sync route): every operand row of 64 values is written
// x = 2^e sum_{u<7} d_u 2^-(8u+7) (row exponent e, balanced base-256 digits |d_u| <= 128,
// exact in BF16).  The product of rows i and j is 2^(e_i+e_j-14) sum_D 2^-8D P_D with
// P_D = sum_{u+v=D} d_u(i) . d_v(j); |P_D| <= (D+1) 64 2^14 < 2^23, an integer the FP32
// accumulator holds exactly.  The seven P_D are combined exactly in a 64-bit integer
// (D = 6 floored to 2^-6 of its unit), which enters the FP64 update once per tile and
// panel.  Results agree with FP64 arithmetic normwise, relative to the rows' maxima.
// Tensor memory: accumulator D in columns [64 D, 64 D + 64), 448 of the 512 allocated.
// Every mbarrier wait is bounded; a wait that runs out stops the CTA's element loop, the
// tensor memory is released after the last committed product, DPG_ERR_TIMEOUT is recorded.
#include <cstdint>

#include "dpg_kernels.h"
#include "dpg_tcgen05.cuh"

namespace dpg {

namespace {
using namespace ::dpg::tc;

constexpr int C5_NB = 64;                         // panel width = K of every product
constexpr int C5_BM = 128;                        // rows of an A block (tensor-memory lanes)
constexpr int C5_BN = 64;                         // rows of a B tile (accumulator columns)
constexpr int C5_S = 7;                           // digits per value
constexpr int C5_WORKERS = 256;                   // warps 0-7
constexpr int C5_NTH = C5_WORKERS + 32;           // + warp 8, the issuer
constexpr uint32_t C5_ROWB = C5_NB * 2;           // bytes of one digit row (64 BF16)
constexpr uint32_t C5_APLANE = C5_BM * C5_ROWB;   // 16384
constexpr uint32_t C5_BPLANE = C5_BN * C5_ROWB;   // 8192
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_B = OFF_A + C5_S * C5_APLANE;          // two B buffers
constexpr uint32_t OFF_EA = OFF_B + 2 * C5_S * C5_BPLANE;     // int[2][128] A-row exponents
constexpr uint32_t OFF_EB = OFF_EA + 2 * C5_BM * 4;           // int[4][64] B-row exponents
constexpr uint32_t OFF_BAR = OFF_EB + 4 * C5_BN * 4;          // mbarriers
constexpr uint32_t OFF_MISC = OFF_BAR + 8 * 8;
constexpr uint32_t C5_SMEM = OFF_MISC + 32;
static_assert(C5_SMEM <= 232448, "shared memory");
// F-phase arrays (inside the A region, free then)
constexpr int C5_LD = C5_NB + 1;
constexpr uint32_t OFF_SD = OFF_A;                                      // double[64][65] L11
constexpr uint32_t OFF_SX = OFF_SD + C5_NB * C5_LD * 8;                 // double[64][65] X
constexpr uint32_t OFF_SV = OFF_SX + C5_NB * C5_LD * 8;                 // double[64] 1 / L_jj, then
                                                                        // u16[2080] triangle order
static_assert(OFF_SV + 64 * 8 + C5_NB * (C5_NB + 1) <= C5_S * C5_APLANE, "F-phase arrays");

// Byte offset of the 16-byte chunk `chunk` (digits 8 chunk .. 8 chunk + 7) of row r within a
// plane: K-major with the 128-byte swizzle, a row's 64 digits in one 128-byte line, its
// chunks permuted by chunk ^ (r & 7) within each 1024-byte group of 8 rows (the layout the
// tensor core reads without bank conflicts; planes and tiles start on 1024-byte boundaries).
__device__ __forceinline__ uint32_t c5_off(int r, int chunk) { return (uint32_t)r * 128u + ((uint32_t)(chunk ^ (r & 7)) << 4); }

// Shared-memory descriptor of a K-major operand with the 128-byte swizzle: start address,
// 8-row-group stride 1024 bytes, fixed field 0b001 at bit 46, swizzle mode 2 at bits 61-63.
__device__ __forceinline__ uint64_t c5_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ uint32_t c5_bf16(int d) {      // exact for |d| < 2^22
    return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// The seven digits of x relative to the row's largest biased exponent emax, as BF16 bits.
__device__ __forceinline__ void c5_digits(double x, unsigned emax, uint32_t (&bits)[C5_S]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned eb = (unsigned)(b >> 52) & 0x7ffu;
    unsigned long long f = 0;
    if (eb != 0 && eb != 0x7ffu) {
        const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
        const int sh = (int)eb - (int)emax + 2;                 // <= 2: f < 2^55
        f = sh >= 0 ? mant << sh : (sh > -55 ? mant >> (-sh) : 0ull);
    }
    const unsigned lo = (unsigned)f, hi = (unsigned)(f >> 32);
    int dig[C5_S];
    unsigned carry = 0;
#pragma unroll
    for (int k = 0; k < C5_S - 1; ++k) {
        const unsigned byte = ((k < 4 ? lo >> (8 * k) : hi >> (8 * (k - 4))) & 255u) + carry;
        carry = byte >= 128u;
        dig[C5_S - 1 - k] = (int)byte - (int)(carry << 8);
    }
    dig[0] = (int)((hi >> 16) + carry);
    const bool neg = (b >> 63) != 0;
#pragma unroll
    for (int u = 0; u < C5_S; ++u) bits[u] = c5_bf16(neg ? -dig[u] : dig[u]);
}

__device__ __forceinline__ unsigned c5_ebits(double x) {
    return (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
}

// Digit planes of the eight consecutive values x[O .. O+8) (one 16-byte chunk of a row) ->
// seven 16-byte words.
template <int O, int N>
__device__ __forceinline__ void c5_pack8(const double (&x)[N], unsigned emax, uint4 (&w)[C5_S]) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        uint32_t b0[C5_S], b1[C5_S];
        c5_digits(x[O + k], emax, b0);
        c5_digits(x[O + k + 1], emax, b1);
#pragma unroll
        for (int u = 0; u < C5_S; ++u) {
            const uint32_t pk = b0[u] | (b1[u] << 16);
            if (k == 0) w[u].x = pk;
            else if (k == 2) w[u].y = pk;
            else if (k == 4) w[u].z = pk;
            else w[u].w = pk;
        }
    }
}

// Split 64 * npass rows of 64 values, src(r, t), into digit planes at dst (plane stride
// pstride, shared memory) and row exponents edst[r].  Workers only: a warp takes 8 rows, a
// lane (row r & 7, chunks ch and ch + 4 of 8 values), so that a store phase of 8 lanes
// writes eight rows' chunks on distinct banks.  Returns true when a value is not finite.
template <class Src>
__device__ __forceinline__ bool c5_split_rows(const Src &src, int npass, unsigned char *dst, uint32_t pstride,
                                              int *edst, int warp, int lane) {
    const int rr = lane & 7, ch = lane >> 3;
    bool bad = false;
    for (int pass = 0; pass < npass; ++pass) {
        const int r = 8 * (warp + 8 * pass) + rr;
        double x[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            x[k] = src(r, 8 * ch + k);
            x[8 + k] = src(r, 8 * (ch + 4) + k);
        }
        unsigned em = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) em = max(em, c5_ebits(x[k]));
        em = max(em, __shfl_xor_sync(0xffffffffu, em, 8));
        em = max(em, __shfl_xor_sync(0xffffffffu, em, 16));
        bad |= em == 0x7ffu;
        if (ch == 0) edst[r] = em ? (int)em - 1022 : 0;
        {
            uint4 w[C5_S];
            c5_pack8<0>(x, em, w);
            const uint32_t o = c5_off(r, ch);
#pragma unroll
            for (int u = 0; u < C5_S; ++u) *reinterpret_cast<uint4 *>(dst + u * pstride + o) = w[u];
            c5_pack8<8>(x, em, w);
            const uint32_t o2 = c5_off(r, ch + 4);
#pragma unroll
            for (int u = 0; u < C5_S; ++u) *reinterpret_cast<uint4 *>(dst + u * pstride + o2) = w[u];
        }
    }
    return bad;
}

__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {   // D FP32, A and B BF16, K-major
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}

// The 28 digit products of a tile, accumulator D = u + v at column 64 D; then one commit.
__device__ __forceinline__ void c5_issue(uint32_t tmem, uint32_t a0, uint32_t apl, uint32_t b0, uint32_t bpl, int n,
                                         int ksteps, uint64_t *done) {
    const uint32_t id = idesc_bf16(C5_BM, n);
    // descriptors advance in their 16-byte address field (shared addresses < 2^18: no carry);
    // a K step of 16 digits is 32 bytes along the swizzled line
    const uint64_t da = c5_desc(a0), db = c5_desc(b0);
#pragma unroll 1
    for (int D = 0; D < C5_S; ++D)
#pragma unroll 1
        for (int u = 0; u <= D; ++u) {
            const uint64_t au = da + ((u * apl) >> 4), bv = db + (((D - u) * bpl) >> 4);
            const uint32_t dt = tmem + 64u * D;
            if (ksteps == 4) {
                umma_bf16(dt, au, bv, id, u != 0);
                umma_bf16(dt, au + 2u, bv + 2u, id, 1u);
                umma_bf16(dt, au + 4u, bv + 4u, id, 1u);
                umma_bf16(dt, au + 6u, bv + 6u, id, 1u);
            } else {
                for (int ks = 0; ks < ksteps; ++ks) umma_bf16(dt, au + 2u * ks, bv + 2u * ks, id, (u | ks) != 0);
            }
        }
    umma_commit(done);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(saddr(sdst)), "l"(gsrc), "r"(bytes), "r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void worker_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Wait for the completion of phase `parity` of bar, polling without a suspend-time hint (the
// waits here are short and on the critical path).  Bounded like mbar_wait: after about 2^31
// cycles the CTA's failure flag is raised and the caller goes on.
__device__ __forceinline__ void c5_wait(uint64_t *bar, uint32_t parity, volatile int *fail) {
    if (*fail) return;
    long long t0 = 0;
    for (int spin = 0;; ++spin) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
        if (ok) return;
        if (spin == 0) t0 = clock64();
        else if (clock64() - t0 > (1LL << 31)) { *fail = 1; return; }
    }
}

// t 2^s for a 64-bit integer t, rounded to nearest (ties to even), flushed to zero below the
// normal range, infinite above it: integer operations only.
__device__ __forceinline__ double c5_i2d(long long t, int s) {
    if (t == 0) return 0.0;
    const unsigned long long sg = (unsigned long long)t & (1ull << 63);
    unsigned long long u = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
    const int lz = __clzll((long long)u);
    u <<= lz;                                             // leading one at bit 63
    unsigned long long mant = u >> 11;                    // 53 bits
    const unsigned rem = (unsigned)u & 0x7ffu;
    mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
    const int e = 1086 - lz + s;                          // biased exponent of the leading one
    if (e <= 0) return __longlong_as_double((long long)sg);
    if (e >= 2047) return __longlong_as_double((long long)(sg | 0x7ff0000000000000ull));
    // the implicit bit of mant adds one to the exponent field (a rounding carry, one more)
    return __longlong_as_double((long long)(sg | (((unsigned long long)(e - 1) << 52) + mant)));
}

// t 2^s converted on the FP64 pipe (one conversion, the scale added to the exponent field),
// or by c5_i2d when the result leaves the normal range: the conversion shares the load
// between the FP64 and the integer pipes, the latter busy with the digit combination.
__device__ __forceinline__ double c5_i2d_fp(long long t, int s) {
    const long long b = __double_as_longlong(__ll2double_rn(t));
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex != 0 && ex + s > 0 && ex + s < 2047) return __longlong_as_double(b + ((long long)s << 52));
    return c5_i2d(t, s);
}

// The accumulators of one tile for a worker: its lane's row of the A block, 32 columns
// (half hq of the tile), in two passes of 16 columns.  Adjacent diagonals pair exactly in
// 32 bits (Q = 2^8 P_D + P_{D+1}, |Q| < 2^31 for D <= 4), the pairs into the 64-bit integer
// sum_D P_D 2^(42 - 8 D), which is scaled: dv[c] = 2^(ea + eb[c]) times it.
__device__ __forceinline__ int c5_f2i_small(uint32_t r) {        // |x| <= 2^22
    return __float_as_int(__uint_as_float(r) + 12582912.0f) - 0x4B400000;
}
__device__ __forceinline__ void c5_drain(uint32_t tbase, int wq, int hq, int ea, const int *eb, double (&dv)[32]) {
    const uint32_t t0 = tbase + ((uint32_t)(32 * wq) << 16) + 32u * hq;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
        const uint32_t ta = t0 + 16u * hf;
        int q01[16], q23[16], q45[16];
        {
            uint32_t r[32];
            tmem_ld16x2(ta, ta + 64u, r);                  // P_0, P_1 (|P| <= 2^21)
#pragma unroll
            for (int c = 0; c < 16; ++c) q01[c] = c5_f2i_small(r[c]) * 256 + c5_f2i_small(r[16 + c]);
            tmem_ld16x2(ta + 128u, ta + 192u, r);          // P_2 (<= 3 2^20), P_3 (<= 2^22)
#pragma unroll
            for (int c = 0; c < 16; ++c) q23[c] = c5_f2i_small(r[c]) * 256 + c5_f2i_small(r[16 + c]);
            tmem_ld16x2(ta + 256u, ta + 320u, r);          // P_4, P_5 (< 2^23)
#pragma unroll
            for (int c = 0; c < 16; ++c)
                q45[c] = __float2int_rn(__uint_as_float(r[c])) * 256 + __float2int_rn(__uint_as_float(r[16 + c]));
        }
        uint32_t r6[16];
        tmem_ld16(ta + 384u, r6);                          // P_6, floored to 2^-6 of its unit
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const long long tot = (long long)q01[c] * (1ll << 34) + (long long)q23[c] * (1ll << 18) +
                                  (long long)q45[c] * 4 + (long long)(__float2int_rn(__uint_as_float(r6[c])) >> 6);
            dv[16 * hf + c] = c5_i2d_fp(tot, ea + eb[16 * hf + c]);
        }
    }
}

// Trailing-update jobs of one panel, in the order both roles walk them:
//   ph 0: G tiles, A = L21 rows [128 a, +128) (columns of G), B = L21 rows [b0, +64) (rows);
//   ph 1: right-hand-side tiles, A = W1^T rows [128 a, +128) (columns c), B = L21 rows b0..;
//   ph 2: [K | F] tiles, A = W1^T rows [128 a, +128) (c2), B = W1^T rows b0.. (c1 >= c2).
struct C5Jobs {
    int ph, a, b0, nr, mc;
    __device__ void init(int nr_, int mc_) { nr = nr_; mc = mc_; ph = 0; a = 0; b0 = 0; settle(); }
    __device__ void settle() {
        for (;;) {
            if (ph == 0) {
                if (C5_BM * a >= nr) { ph = 1; a = 0; b0 = 0; continue; }
                if (b0 < C5_BM * a) b0 = C5_BM * a;
                if (b0 >= nr) { ++a; b0 = 0; continue; }
                return;
            }
            if (ph == 1) {
                if (C5_BM * a >= mc || nr == 0) { ph = 2; a = 0; b0 = 0; continue; }
                if (b0 >= nr) { ++a; b0 = 0; continue; }
                return;
            }
            if (ph == 2) {
                if (C5_BM * a >= mc) { ph = 3; return; }
                if (b0 < C5_BM * a) b0 = C5_BM * a;
                if (b0 >= mc) { ++a; b0 = 0; continue; }
                return;
            }
            return;
        }
    }
    __device__ void next() { b0 += C5_BN; settle(); }
    __device__ bool done() const { return ph == 3; }
    __device__ int akey() const { return ph == 0 ? a : 65536 + a; }     // A source and block
    __device__ int brows() const { return min(C5_BN, (ph == 2 ? mc : nr) - b0); }   // valid B rows
};

// A worker's part of one trailing tile: its A row (one column of the destination) and 32 B
// rows, as a strided walk over the destination -- the G column r0 + arow from row
// r0 + brow0 (stride n), the [B | l] column arow from row r0 + brow0 (stride m, or l
// itself), the K column arow from row brow0 (stride m; row m of the extended product is F) --
// over the columns c in [cfirst, clast) of the worker's half of the tile.
struct C5Target {
    double *d;
    int64_t stride;
    int cfirst, clast, ncol, brow0, arow;
    bool live;            // the warp holds outputs (else it skips the accumulators)
    bool any;             // this lane holds outputs
};
__device__ __forceinline__ C5Target c5_target(const C5Jobs &it, int wq, int hq, int lane, int n, int m, int mc, int r0,
                                             double *G, double *Bm, double *lv, double *K) {
    C5Target t;
    const int nvalid = it.brows(), acnt = it.ph == 0 ? it.nr : mc;
    t.arow = C5_BM * it.a + 32 * wq + lane;
    t.brow0 = it.b0 + 32 * hq;
    t.live = 32 * hq < nvalid && C5_BM * it.a + 32 * wq < acnt && !(it.ph != 1 && C5_BM * it.a + 32 * wq > t.brow0 + 31);
    t.ncol = min(32, nvalid - 32 * hq);
    // columns past the B rows or above the diagonal (G and K tiles: A row > B row) hold nothing
    t.cfirst = it.ph == 1 ? 0 : max(0, t.arow - t.brow0);
    t.clast = it.ph == 2 ? min(t.ncol, m - t.brow0) : t.ncol;
    t.any = t.live && t.arow < acnt;
    if (it.ph == 0) { t.d = G + (size_t)(r0 + t.brow0) * n + r0 + t.arow; t.stride = n; }
    else if (it.ph == 1) {
        if (t.arow < m) { t.d = Bm + (size_t)(r0 + t.brow0) * m + t.arow; t.stride = m; }
        else { t.d = lv + r0 + t.brow0; t.stride = 1; }
    } else { t.d = K + (size_t)t.brow0 * m + t.arow; t.stride = m; }
    return t;
}

__device__ __forceinline__ void report5(DevStatus *st, int code, long long elem) {
    atomicCAS(&st->code, 0, code);
    atomicMin(&st->first_bad[code], (unsigned long long)elem);
}

// 288 threads: 9 warps share 4 sub-partitions of 16384 registers, at most 168 a thread
__global__ void __launch_bounds__(C5_NTH, 1) condense5_kernel(Cond5Params p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
    uint64_t *a_full = bar, *b_full = bar + 1, *mma_done = bar + 3, *tmem_free = bar + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC);
    volatile int *fail = reinterpret_cast<volatile int *>(sm + OFF_MISC + 4);
    volatile int *sbad = reinterpret_cast<volatile int *>(sm + OFF_MISC + 8);
    int *eA = reinterpret_cast<int *>(sm + OFF_EA), *eB = reinterpret_cast<int *>(sm + OFF_EB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = warp < 8;
    const int wq = warp & 3, hq = (warp >> 2) & 1;
    const int n = p.n, m = p.m, mc = m + (p.l ? 1 : 0);
#if defined(DPG_DEBUG_BOUNDS)
    if (!DPG_INB(C5_SMEM <= dpg_dyn_smem_bytes(), p.status, p.elem_base)) return;   // uniform
#endif
    if (tid == 0) {
        *fail = 0;
        mbar_init(a_full, 1);
        mbar_init(b_full, 1);
        mbar_init(b_full + 1, 1);
        mbar_init(mma_done, 1);
        mbar_init(tmem_free, 8);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(saddr(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot, sbase = saddr(sm);
    // per-CTA digit scratch: L21 rows then W1^T rows, each plane-major, then the exponents
    const int lrows = p.lrows, wrows = p.wrows;
    unsigned char *scr = p.scratch + (size_t)blockIdx.x * p.scratch_per_cta;
    unsigned char *Ldig = scr, *Wdig = scr + (size_t)C5_S * lrows * C5_ROWB;
    int *eLs = reinterpret_cast<int *>(Wdig + (size_t)C5_S * wrows * C5_ROWB), *eWs = eLs + lrows;
    const uint32_t lpl = (uint32_t)lrows * C5_ROWB, wpl = (uint32_t)wrows * C5_ROWB;
    // running counts (the same on every thread that uses them): products committed, A
    // loads, B loads per buffer, tensor-memory releases
    uint32_t njob = 0, na = 0, nb0 = 0, nb1 = 0, ntf = 0;
    long long last_elem = -1;
    for (int64_t e = blockIdx.x; e < p.n_elem; e += gridDim.x) {
        double *G = p.G + (size_t)e * n * n, *Bm = p.B + (size_t)e * n * m;
        double *lv = p.l ? p.l + (size_t)e * n : nullptr;
        double *K = p.K + (size_t)e * m * m, *F = p.F ? p.F + (size_t)e * m : nullptr;
        auto rhs = [&](int i, int c) -> double & { return c < m ? Bm[(size_t)i * m + c] : lv[i]; };
        last_elem = p.elem_base + e;
        if (tid == 0) *sbad = 0;
        if (worker) {
            for (int idx = tid; idx < m * m; idx += C5_WORKERS) K[idx] = 0.0;
            if (F) for (int idx = tid; idx < m; idx += C5_WORKERS) F[idx] = 0.0;
        }
        __syncthreads();
        for (int kb = 0; kb < n; kb += C5_NB) {
            const int w = min(C5_NB, n - kb), r0 = kb + w, nr = n - r0;
            const int ksteps = (w + 15) >> 4, wn = ksteps * 16;
            // ---- F-phase: the diagonal block (workers) ----
            double (*sD)[C5_LD] = reinterpret_cast<double (*)[C5_LD]>(sm + OFF_SD);
            double (*sX)[C5_LD] = reinterpret_cast<double (*)[C5_LD]>(sm + OFF_SX);    // sX[j][t] = X_jt
            double *srd = reinterpret_cast<double *>(sm + OFF_SV);                      // 1 / L_jj
            unsigned short *stab = reinterpret_cast<unsigned short *>(sm + OFF_SV + 64 * 8);
            if (worker) {
                // The block, padded to 64 x 64 with the identity, in shared memory.  Every loop
                // runs over exactly its active entries (dynamic bounds): a predicated FP64
                // instruction costs the FP64 pipe as much as an active one on this part, so
                // idle warps must not issue.  tab[idx] = (r, c) of the lower triangle in the
                // order column 63, 62, .., 0 (rows ascending): step j updates the columns
                // right of j, exactly the idx below T_j = (63-j)(64-j)/2.
                for (int idx = tid; idx < C5_NB * (C5_NB + 1) / 2; idx += C5_WORKERS) {
                    int k = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
                    if ((k + 1) * (k + 2) / 2 <= idx) ++k;
                    if (k * (k + 1) / 2 > idx) --k;
                    const int c = C5_NB - 1 - k, r = c + idx - k * (k + 1) / 2;
                    stab[idx] = (unsigned short)(r | (c << 8));
                }
                for (int idx = tid; idx < C5_NB * C5_NB; idx += C5_WORKERS) {
                    const int r = idx >> 6, c = idx & 63;
                    sD[r][c] = c > r ? 0.0 : (r < w && c < w) ? G[(size_t)(kb + r) * n + kb + c] : (r == c ? 1.0 : 0.0);
                    sX[r][c] = r == c ? 1.0 : 0.0;
                }
                worker_sync();
                // right-looking Cholesky: the pivot gives L_jj, column j is scaled, the columns
                // right of j are updated
                for (int j = 0; j < w; ++j) {
                    if (tid == 0) {
                        const double d = sD[j][j];
                        if (!(d > 0.0) || !isfinite(d)) *sbad = 1;
                        const double rs = rsqrt(d);
                        srd[j] = rs;
                        sD[j][j] = d * rs;
                    }
                    worker_sync();
                    const double rj = srd[j];
                    for (int r = j + 1 + tid; r < C5_NB; r += C5_WORKERS) sD[r][j] *= rj;
                    worker_sync();
                    const int Tj = (C5_NB - 1 - j) * (C5_NB - j) / 2;
                    for (int idx = tid; idx < Tj; idx += C5_WORKERS) {
                        const int rc = stab[idx], r = rc & 255, c = rc >> 8;
                        sD[r][c] = fma(-sD[r][j], sD[c][j], sD[r][c]);
                    }
                    worker_sync();
                }
                // L11 into G
                for (int idx = tid; idx < w * w; idx += C5_WORKERS) {
                    const int r = idx / w, c = idx - r * w;
                    if (c <= r) G[(size_t)(kb + r) * n + kb + c] = sD[r][c];
                }
                // X = L11^-1 by right-looking forward substitution: row t of X is final at step t
                // (scaled by 1 / L_tt), then X_rc -= L_rt X_tc for c <= t < r < w
                for (int t = 0; t < w; ++t) {
                    const double rt = srd[t];
                    for (int c = tid; c <= t; c += C5_WORKERS) sX[t][c] *= rt;
                    worker_sync();
                    const int nc = t + 1, cnt = (w - 1 - t) * nc;
                    for (int q = tid; q < cnt; q += C5_WORKERS) {
                        const int rr = q / nc, c = q - rr * nc, r = t + 1 + rr;
                        sX[r][c] = fma(-sD[r][t], sX[t][c], sX[r][c]);
                    }
                    worker_sync();
                }
                // digits of X (rows j, K index t) -> B buffer 0, exponents -> eB slot 0
                const bool bad = c5_split_rows([&](int j, int t) { return (j < w && t <= j) ? sX[j][t] : 0.0; }, 1,
                                               sm + OFF_B, C5_BPLANE, eB, warp, lane);
                if (bad) *sbad = 1;
                fence_async_smem();
            }
            __syncthreads();
            if (*sbad) break;
            // ---- P-phase: L21 = A21 X^T (jobs 0 .. nL-1), W1^T = B1^T X^T (nL .. nL+nW-1) ----
            const int nL = (nr + C5_BM - 1) / C5_BM, nW = (mc + C5_BM - 1) / C5_BM;
            int *xch = reinterpret_cast<int *>(sm + OFF_B + C5_S * C5_BPLANE);    // B buffer 1: int[2][128]
            for (int pj = 0; pj < nL + nW; ++pj) {
                const bool isL = pj < nL;
                const int base = C5_BM * (isL ? pj : pj - nL);
                const int cnt = isL ? nr : mc;
                if (worker) {
                    bool bad;
                    if (isL)
                        bad = c5_split_rows([&](int r, int t) {
                            return (base + r < nr && t < w) ? G[(size_t)(r0 + base + r) * n + kb + t] : 0.0;
                        }, 2, sm + OFF_A, C5_APLANE, eA, warp, lane);
                    else
                        bad = c5_split_rows([&](int r, int t) {
                            return (base + r < mc && t < w) ? rhs(kb + t, base + r) : 0.0;
                        }, 2, sm + OFF_A, C5_APLANE, eA, warp, lane);
                    if (bad) *sbad = 1;
                    fence_async_smem();
                }
                __syncthreads();
                if (tid == C5_WORKERS && !*fail) {
                    tc_fence_after();
                    // (test hook: a stalled CTA never issues its first product, so its workers'
                    // bounded wait runs out)
                    if (!((int)blockIdx.x == p.stall_cta && njob == 0))
                        c5_issue(tbase, sbase + OFF_A, C5_APLANE, sbase + OFF_B, C5_BPLANE, wn, ksteps, mma_done);
                }
                if (worker) {
                    c5_wait(mma_done, njob & 1, fail);
                    tc_fence_after();
                    const int row = 32 * wq + lane;                    // row of the A block
                    const bool rv = base + row < cnt;
                    double v[32];
                    c5_drain(tbase, wq, hq, eA[row] - 56, eB + 32 * hq, v);
                    tc_fence_before();
                    unsigned em = 0;
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        if (!(rv && 32 * hq + c < w)) v[c] = 0.0;
                        em = max(em, c5_ebits(v[c]));
                    }
                    // FP64 results: L21 into G, W1 into [B | l] (rows kb..)
                    if (rv) {
                        if (isL) {
                            double *gr = G + (size_t)(r0 + base + row) * n + kb;
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                if (32 * hq + c < w) gr[32 * hq + c] = v[c];
                        } else {
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                if (32 * hq + c < w) rhs(kb + 32 * hq + c, base + row) = v[c];
                        }
                    }
                    // the row's exponent over both halves, then its digits into the scratch
                    xch[hq * C5_BM + row] = (int)em;
                    worker_sync();
                    em = max((unsigned)xch[row], (unsigned)xch[C5_BM + row]);
                    if (em == 0x7ffu) *sbad = 1;
                    unsigned char *dd = isL ? Ldig : Wdig;
                    const uint32_t pl = isL ? lpl : wpl;
                    int grow = base + row;                          // row of the scratch
                    if (!DPG_INB(grow < (isL ? lrows : wrows), p.status, p.elem_base + e)) grow = 0;
                    auto put = [&](const uint4 (&wd)[C5_S], int k) {
                        const uint32_t o = c5_off(grow, 4 * hq + k);
#pragma unroll
                        for (int u = 0; u < C5_S; ++u) *reinterpret_cast<uint4 *>(dd + (size_t)u * pl + o) = wd[u];
                    };
                    {
                        uint4 wd[C5_S];
                        c5_pack8<0>(v, em, wd);
                        put(wd, 0);
                        c5_pack8<8>(v, em, wd);
                        put(wd, 1);
                        c5_pack8<16>(v, em, wd);
                        put(wd, 2);
                        c5_pack8<24>(v, em, wd);
                        put(wd, 3);
                    }
                    if (hq == 0) (isL ? eLs : eWs)[grow] = em ? (int)em - 1022 : 0;
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                ++njob;
                __syncthreads();
            }
            // ---- T-phase: the trailing updates, pipelined ----
            if (tid == C5_WORKERS) {
                C5Jobs it;
                it.init(nr, mc);
                int akey = -1, k = 0;
                auto load_b = [&](const C5Jobs &jb, int buf, int slot) {
                    int rows = (jb.brows() + 15) & ~15;
                    const bool fromL = jb.ph <= 1;
                    if (!DPG_INB(jb.b0 + rows <= (fromL ? lrows : wrows), p.status, p.elem_base + e)) rows = 0;
                    const unsigned char *src = (fromL ? Ldig : Wdig) + (size_t)jb.b0 * C5_ROWB;
                    const uint32_t pl = fromL ? lpl : wpl;
                    const int *es = (fromL ? eLs : eWs) + jb.b0;
                    uint64_t *fb = b_full + buf;
                    mbar_expect_tx(fb, (uint32_t)(C5_S * rows * C5_ROWB + rows * 4));
                    if (rows > 0) {
                        for (int u = 0; u < C5_S; ++u)
                            bulk_g2s(sm + OFF_B + buf * C5_S * C5_BPLANE + u * C5_BPLANE, src + (size_t)u * pl,
                                     (uint32_t)rows * C5_ROWB, fb);
                        bulk_g2s(eB + slot * C5_BN, es, (uint32_t)rows * 4, fb);
                    }
                };
                if (!it.done() && !*fail) load_b(it, 0, 0);
                while (!it.done()) {
                    if (k > 0) { c5_wait(tmem_free, ntf & 1, fail); ++ntf; }
                    if (it.akey() != akey && !*fail) {
                        akey = it.akey();
                        const bool fromL = it.ph == 0;
                        const bool ok = DPG_INB(C5_BM * (it.a + 1) <= (fromL ? lrows : wrows), p.status, p.elem_base + e);
                        const unsigned char *src = (fromL ? Ldig : Wdig) + (size_t)(C5_BM * it.a) * C5_ROWB;
                        const uint32_t pl = fromL ? lpl : wpl;
                        mbar_expect_tx(a_full, ok ? (uint32_t)(C5_S * C5_APLANE + C5_BM * 4) : 0u);
                        if (ok) {
                            for (int u = 0; u < C5_S; ++u)
                                bulk_g2s(sm + OFF_A + u * C5_APLANE, src + (size_t)u * pl, C5_APLANE, a_full);
                            bulk_g2s(eA + (na & 1) * C5_BM, (fromL ? eLs : eWs) + C5_BM * it.a, C5_BM * 4, a_full);
                        }
                        c5_wait(a_full, na & 1, fail);
                        ++na;
                    }
                    const int buf = k & 1;
                    c5_wait(b_full + buf, (buf ? nb1 : nb0) & 1, fail);
                    if (buf) ++nb1; else ++nb0;
                    tc_fence_after();
                    if (!*fail)
                        c5_issue(tbase, sbase + OFF_A, C5_APLANE, sbase + OFF_B + buf * C5_S * C5_BPLANE, C5_BPLANE,
                                 (it.brows() + 15) & ~15, ksteps, mma_done);
                    C5Jobs nx = it;
                    nx.next();
                    if (!nx.done() && !*fail) load_b(nx, (k + 1) & 1, (k + 1) & 3);
                    it = nx;
                    ++k;
                    ++njob;
                }
                if (k > 0) ++ntf;                       // the last tile's release, awaited below
            } else if (worker) {
                C5Jobs it;
                it.init(nr, mc);
                int akey = -1, k = 0;
                while (!it.done()) {
                    if (it.akey() != akey) { akey = it.akey(); ++na; }
                    const int aslot = (na - 1) & 1, slot = k & 3;
                    const C5Target tg = c5_target(it, wq, hq, lane, n, m, mc, r0, G, Bm, lv, K);
                    c5_wait(mma_done, njob & 1, fail);
                    tc_fence_after();
                    double dv[32];
                    if (tg.live) c5_drain(tbase, wq, hq, eA[aslot * C5_BM + 32 * wq + lane] - 56, eB + slot * C5_BN + 32 * hq, dv);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tmem_free);
                    {
                        // the next tile's destination lines into L2 while this one is applied
                        C5Jobs nx = it;
                        nx.next();
                        if (!nx.done()) {
                            const C5Target tn = c5_target(nx, wq, hq, lane, n, m, mc, r0, G, Bm, lv, K);
                            if (tn.any)
#pragma unroll 4
                                for (int c = tn.cfirst; c < tn.clast; ++c)
                                    asm volatile("prefetch.global.L2 [%0];" :: "l"(tn.d + c * tn.stride));
                        }
                    }
                    if (tg.any && DPG_INB(it.b0 + it.brows() <= (it.ph == 2 ? mc : nr), p.status, p.elem_base + e)) {
                        const int cfirst = tg.cfirst, clast = tg.clast, ncol = tg.ncol, brow0 = tg.brow0, arow = tg.arow;
                        double *d = tg.d;
                        const int64_t stride = tg.stride;
                        const bool add = it.ph == 2;
                        // sixteen loads issued before their stores
#pragma unroll
                        for (int g = 0; g < 2; ++g) {
                            double old[16];
#pragma unroll
                            for (int c16 = 0; c16 < 16; ++c16) {
                                const int c = 16 * g + c16;
                                old[c16] = (c >= cfirst && c < clast) ? d[c * stride] : 0.0;
                            }
#pragma unroll
                            for (int c16 = 0; c16 < 16; ++c16) {
                                const int c = 16 * g + c16;
                                if (c >= cfirst && c < clast) d[c * stride] = add ? old[c16] + dv[c] : old[c16] - dv[c];
                            }
                        }
                        if (it.ph == 2 && arow < m && m - brow0 >= cfirst && m - brow0 < ncol) {
                            double fv = 0.0;                     // the column of row m: F
#pragma unroll
                            for (int c = 0; c < 32; ++c)
                                if (brow0 + c == m) fv = dv[c];
                            F[arow] += fv;
                        }
                    }
                    it.next();
                    ++k;
                    ++njob;
                }
            } else {
                // lanes 1-31 of the issuing warp: keep the job count in step
                C5Jobs it;
                it.init(nr, mc);
                while (!it.done()) { it.next(); ++njob; }
            }
            __syncthreads();
            if (*fail) break;
        }
        // K: mirror the lower triangle; a failed element gets NaN in K and F
        __syncthreads();
        if (worker) {
            if (*sbad) {
                for (int idx = tid; idx < m * m; idx += C5_WORKERS) K[idx] = __longlong_as_double(0x7ff8000000000000LL);
                if (F) for (int idx = tid; idx < m; idx += C5_WORKERS) F[idx] = __longlong_as_double(0x7ff8000000000000LL);
                if (tid == 0) report5(p.status, 11 /*DPG_ERR_NOT_SPD*/, p.elem_base + e);
            } else {
                for (int idx = tid; idx < m * m; idx += C5_WORKERS) {
                    const int r = idx / m, c = idx - r * m;
                    if (c > r) K[idx] = K[(size_t)c * m + r];
                }
            }
        }
        __syncthreads();
        if (*fail) break;
    }
    // no product in flight when the tensor memory is released
    __syncthreads();
    if (tid == C5_WORKERS && njob > 0) {
        volatile int local = 0;
        c5_wait(mma_done, (njob - 1) & 1, &local);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512));
    }
    if (*fail && tid == 0) report5(p.status, 9 /*DPG_ERR_TIMEOUT*/, last_elem < 0 ? 0 : last_elem);
}

}  // namespace

size_t condense5_scratch_per_cta(int n, int m, bool with_l, int *lrows, int *wrows) {
    const int mc = m + (with_l ? 1 : 0);
    const int lr = (n + C5_BM - 1) / C5_BM * C5_BM, wr = (mc + C5_BM - 1) / C5_BM * C5_BM;
    if (lrows) *lrows = lr;
    if (wrows) *wrows = wr;
    const size_t bytes = (size_t)C5_S * (lr + wr) * C5_ROWB + (size_t)(lr + wr) * 4;
    return (bytes + 1023) / 1024 * 1024;
}

cudaError_t init_condense5_attributes() {
    cudaError_t e = cudaFuncSetAttribute(condense5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C5_SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, condense5_kernel, C5_NTH, C5_SMEM);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorLaunchOutOfResources;    // one CTA must fit an SM
    return e;
}

cudaError_t launch_condense5(const Cond5Params &p, int grid, cudaStream_t s) {
    if (p.n_elem == 0 || grid <= 0) return cudaSuccess;
    condense5_kernel<<<grid, C5_NTH, C5_SMEM, s>>>(p);
    return cudaGetLastError();
}

}  // namespace dpg
