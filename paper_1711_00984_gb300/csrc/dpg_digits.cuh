// dpg_digits.cuh -- FP64 products from exact BF16 digits on the tensor cores (internal;
// used by the condensation kernel).
//
// Every operand row of a product (its <= 32 values along the summed index) is written as
// x = 2^e sum_{u<7} d_u 2^-(8u+7) with the row exponent e (|x| < 2^e over the row) and
// balanced base-256 digits |d_u| <= 128 (exact in BF16), from the FP64 bits with integer
// operations only; what lies below 2^-55 of the row maximum is dropped.  A product of two
// rows is then 2^(e_i+e_j) sum_D 2^-(8D+14) P_D with P_D = sum_{u+v=D} d_u(i) . d_v(j),
// and every P_D is a sum of at most 7 x 32 integer products of at most 2^14, below 2^22
// in all: the BF16 tensor-core products accumulate it exactly in FP32.  The diagonals
// D <= 6 (28 digit products) are combined exactly in a 64-bit integer (the D = 6 term
// floored to 2^-5 of its unit) and enter the FP64 output once, so the FP64 pipe sees two
// operations per output and panel instead of 32 FMAs.  Accuracy is normwise, relative to
// the row maxima: a product of rows i and j is exact to about 2^-53 max_k|x_ik| max_k|y_jk|
// (the dropped digit planes and the floor of D = 6, the latter a one-signed offset per
// panel), where FP64 FMAs err by about 2^-53 sum_k |x_ik y_jk|; an entry far below its
// row's maximum keeps fewer correct bits than under FP64 arithmetic (about 55 - log2 of
// the ratio).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace dpg {

constexpr int EM_S = 7;                  // digits per value
constexpr int EM_SK = 40;                // BF16 per digit row (32 used; 80-byte rows keep the
                                         // fragment loads free of bank conflicts)
constexpr int EM_ROWBYTES = EM_SK * 2;

// Digits of one row held by a warp (lane t: value t of the row, zero beyond w).  Writes the
// digits to dst[u * plane_rows * EM_SK + t] (BF16 bits) and, from lane 0, the row exponent;
// returns true when a value of the row is not finite.
__device__ __forceinline__ bool slice_row_planes(double x, uint16_t *dst, int *e_out, int lane, int plane_rows) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned eb = (unsigned)(bits >> 52) & 0x7ffu;
    const unsigned emax = __reduce_max_sync(0xffffffffu, eb);
    if (lane == 0) *e_out = emax ? (int)emax - 1022 : 0;
    unsigned long long f = 0;
    if (eb != 0 && eb != 0x7ffu) {
        const unsigned long long mant = (bits & 0xfffffffffffffull) | (1ull << 52);
        const int sh = (int)eb - (int)emax + 2;                 // <= 2: f < 2^55
        f = sh >= 0 ? mant << sh : (sh > -55 ? mant >> (-sh) : 0ull);
    }
    // balanced base-256 digits from the low end (a byte >= 128 becomes byte - 256 with a
    // carry into the next); the top digit is below 2^7 plus the carry, so |d| <= 128
    const unsigned lo = (unsigned)f, hi = (unsigned)(f >> 32);
    int dig[EM_S];
    unsigned carry = 0;
#pragma unroll
    for (int k = 0; k < EM_S - 1; ++k) {
        const unsigned byte = ((k < 4 ? lo >> (8 * k) : hi >> (8 * (k - 4))) & 255u) + carry;
        carry = byte >= 128u;
        dig[EM_S - 1 - k] = (int)byte - (int)(carry << 8);
    }
    dig[0] = (int)((hi >> 16) + carry);
    const bool neg = (bits >> 63) != 0;
#pragma unroll
    for (int u = 0; u < EM_S; ++u) {
        const float fd = (float)(neg ? -dig[u] : dig[u]);
        dst[(size_t)u * plane_rows * EM_SK] = (uint16_t)(__float_as_uint(fd) >> 16);
    }
    return __any_sync(0xffffffffu, eb == 0x7ffu);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}

// tot[4 nt + i] (the warp's 16 x 32 sub-tile, mma accumulator order) = sum_D P_D 2^(43-8D)
// (D = 6: 2^-5, floor), from the digit planes of the I rows (rows rb ..) and J rows (cb ..).
// Fragments come in with ldmatrix: lane L addresses row (L & 7) + 8 ((L >> 3) & 1) of the A
// block at column 8 (L >> 4), and J row (L & 7) + 8 (L >> 4) at column 8 ((L >> 3) & 1)
// (two n-tiles per load); 80-byte rows keep the eight rows of a phase on distinct banks.
__device__ __forceinline__ void emu_products_g(long long (&tot)[16], const unsigned char *si, int rows_i,
                                               const unsigned char *sj, int rows_j, int rb, int cb, int lane) {
    const int arow = rb + (lane & 7) + 8 * ((lane >> 3) & 1), acol = 16 * (lane >> 4);       // bytes
    const int brow = cb + (lane & 7) + 8 * (lane >> 4), bcol = 16 * ((lane >> 3) & 1);
#pragma unroll
    for (int k = 0; k < 16; ++k) tot[k] = 0;
#pragma unroll 1
    for (int D = 0; D < EM_S; ++D) {
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll 1
        for (int u = 0; u <= D; ++u) {
            const unsigned char *pa = si + (size_t)u * rows_i * EM_ROWBYTES + arow * EM_ROWBYTES + acol;
            const unsigned char *pb = sj + (size_t)(D - u) * rows_j * EM_ROWBYTES + brow * EM_ROWBYTES + bcol;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t a[4], b01[4], b23[4];
                ldsm_x4(a, pa + 32 * ks);
                ldsm_x4(b01, pb + 32 * ks);                          // n-tiles 0, 1
                ldsm_x4(b23, pb + 16 * EM_ROWBYTES + 32 * ks);       // n-tiles 2, 3
                mma_bf16(acc[0], a, b01[0], b01[1]);
                mma_bf16(acc[1], a, b01[2], b01[3]);
                mma_bf16(acc[2], a, b23[0], b23[1]);
                mma_bf16(acc[3], a, b23[2], b23[3]);
            }
        }
        // the exact integer sums into the 64-bit total (|P_D| < 2^22: the 1.5 2^23 shift
        // puts the integer in the low mantissa bits; |total| < 2^62)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long long iv = (long long)(__float_as_int(acc[nt][i] + 12582912.0f) - 0x4B400000);
                tot[4 * nt + i] += D < EM_S - 1 ? iv * (1ll << (43 - 8 * D)) : (iv >> 5);   // floor
            }
    }
}

}  // namespace dpg
