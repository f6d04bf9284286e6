// dpg_kernels.h -- kernel parameter blocks and launchers (internal).
#pragma once
#include <cuda_runtime.h>

#include "dpg_internal.h"

namespace dpg {

// Device status word: the first error code recorded (0 = none) and, per code, the
// smallest offending element index.
struct DevStatus {
    int code;
    int pad;
    unsigned long long first_bad[16];
};

// Bounds-checked build (nvcc -DDPG_DEBUG_BOUNDS, libdpg_debug.so): every kernel checks its
// global-memory store indices against the extents of the buffer it writes, its metric-field
// reads against the element's fields, and its shared-memory layout (and tensor-memory
// columns) against what the launch provides; a failed check records DPG_ERR_BOUNDS (12)
// with the element index in the status word and skips the access (or the work unit) --
// nothing traps.  In the normal build every check is the constant `true`.
constexpr int DPG_STATUS_BOUNDS = 12;
#if defined(__CUDACC__)
#if defined(DPG_DEBUG_BOUNDS)
__device__ __forceinline__ bool dpg_in_bounds(bool ok, DevStatus *st, long long elem) {
    if (!ok && st) {
        atomicCAS(&st->code, 0, DPG_STATUS_BOUNDS);
        atomicMin(&st->first_bad[DPG_STATUS_BOUNDS], (unsigned long long)(elem < 0 ? 0 : elem));
    }
    return ok;
}
#define DPG_INB(cond, st, elem) ::dpg::dpg_in_bounds((cond), (st), (long long)(elem))
#else
#define DPG_INB(cond, st, elem) true
#endif
// bytes of dynamic shared memory of the running launch
__device__ __forceinline__ unsigned dpg_dyn_smem_bytes() {
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
#endif

struct GeomParams {
    int space, L, nfields;
    int64_t n_elem;            // elements of this chunk
    int64_t elem_base;         // index of the chunk's first element in the call
    const double *verts;       // chunk start, [n_elem][8][3]
    const double *coeffs;      // chunk start, [n_elem][2] or NULL
    const double *zeta, *w;    // Gauss rule
    void *fields;              // [n_elem][nfields][L^3] of the stage type
    DevStatus *status;
};

template <typename T>
struct SfParams {
    const BlockDesc *blocks;
    const Unit *units;
    int nunits;
    int L, nfields;
    const T *pp;               // pair products [NPAIR][NQ1][NQ1][L]
    const T *fields;           // [n_elem][nfields][L^3]
    T *out;                    // chunk start
    int64_t mat_stride;        // values per element (parts * rows * cols)
    int64_t ld;                // columns
    int64_t n_elem;
    DevStatus *status;         // bounds-checked build only
};

// Per-element constants of the affine path: up to MAXFIELDS metric fields and the
// element's status code in the last slot.
constexpr int AFF_CONST_STRIDE = 24;

struct AffConstParams {
    int space;
    int64_t n_elem, elem_base;
    const double *verts, *coeffs;
    double *consts;            // [n_elem][AFF_CONST_STRIDE]
    DevStatus *status;
};

// FP32 general kernel: one CTA per (block, chunk of elements).
struct SfParams32 {
    const BlockDesc *blocks;
    const Unit *units;
    const int *block_unit_begin;   // [nblock + 1]: units of block k are [begin[k], begin[k+1])
    int nblock, nj_max, elems_per_cta;
    int L, nfields;
    const float *pp;               // pair products [NPAIR][NQ1][NQ1][L]
    const float *fields;           // [n_elem][nfields][L^3]
    float *out;
    int64_t mat_stride, ld, n_elem;
    DevStatus *status;             // bounds-checked build only
};

// FP32 row-panel kernel: one CTA per (block, chunk of elements).
struct PanelParams {
    const BlockDesc *blocks;
    const Unit *units;
    const int *block_unit_begin;   // [nblock + 1]
    const float *ctab;             // constant operands of every block (build_panel_tables)
    const int *ctab_off;           // [nblock]
    int nblock, nj_max, elems_per_cta;
    int L, nfields;
    const float *pp;               // pair products [NPAIR][NQ1][NQ1][L]
    const float *fields;           // [n_elem][nfields][L^3]
    float *out;
    int64_t mat_stride, ld, n_elem;
    DevStatus *status;             // bounds-checked build only
};

// FP32 tensor-core kernel (tcgen05): one CTA per (block, chunk of elements).
struct TcParams {
    const BlockDesc *blocks;
    const Unit *units;
    const int *block_unit_begin;   // [nblock + 1]
    const float *ctab;             // constant operands of every block (build_tc_tables)
    const int *ctab_off;           // [nblock], in floats
    int nblock, nj_max, elems_per_cta;
    int L, nfields;
    const float *pp;               // pair products [NPAIR][NQ1][NQ1][L]
    const float *fields;           // [n_elem][nfields][L^3]
    float *out;
    int64_t mat_stride, ld, n_elem;
    DevStatus *status;
    int stall_cta;                 // test hook: this CTA issues no stage-B MMA (-1: none)
    // the elements of one order of an hp batch (all NULL for a uniform batch): element i of
    // the launch is elist[*elist_start + i], *n_elem_dev of them (n_elem: their maximum),
    // its fields at fields + foff[e], its matrix at out + out_off[e]
    const int *elist = nullptr, *elist_start = nullptr, *n_elem_dev = nullptr;
    const int64_t *foff = nullptr, *out_off = nullptr;
};

// FP32 general kernel with stage C on the tensor cores (sf_tcc_kernel): a persistent grid
// over the work items (block, element, i3) of one program, block-major; uniform batches
// (elist = NULL: element index = item's element) or the elements of one order of an hp
// batch (elist[*elist_start + i], *n_elem_dev of them, per-element offsets foff / out_off).
struct TccParams {
    const BlockDesc *blocks;
    int nblock;
    const int *blk_base;           // [nblock + 1]: prefix sums of nr3 (items per element)
    const float *img;              // constant images of the blocks (build_tcc_tables)
    const int *img_off;            // [nblock + 1], in floats
    int L, nfields, tcols;         // tcols: tensor-memory columns every CTA allocates
    const float *pp;               // FP32 pair products [NPAIR][NQ1][NQ1][L]
    const float *fields;           // [n_elem][nfields][L^3] (foff == NULL) or the base of foff
    const int64_t *foff;
    float *out;                    // [n_elem][mat_stride] (out_off == NULL) or the base of out_off
    const int64_t *out_off;
    int64_t mat_stride, ld;        // values of one element matrix (all parts), its leading dimension
    int64_t n_elem;
    const int *n_elem_dev, *elist, *elist_start;
    DevStatus *status;
    int smem_bytes;                // dynamic shared memory of the launch
    int stall_cta;                 // test hook: this CTA commits no product (-1: none)
};

template <typename T>
struct AffParams {
    const BlockDesc *blocks;
    const Unit *units;
    const int *block_unit_begin;   // [nblock + 1]
    int nblock, nj_max;
    int nsplit;                    // CTAs per (element chunk, block): each takes every nsplit-th unit
    int elems_per_cta;             // elements of a CTA's chunk
    const T *F;                // exact 1D integrals [NPAIR][NQ1][NQ1]
    const void *img;           // constant shared-memory images of the blocks (build_aff_image)
    const int *img_off16;      // [nblock + 1], in 16-byte units
    const unsigned *qlist;     // structural stage-B lists of the units (affine; build_aff_qlists)
    const int *qoff;           // [nunits + 1] list starts (affine)
    const double *consts;      // [n_elem][AFF_CONST_STRIDE] from affine_const_kernel (affine)
    // extruded maps: 2D metric fields [n_elem][nfields][L][L] (xi2, xi3) from geom2d_kernel,
    // per-element status, pair products at the Gauss points [NPAIR][NQ1][NQ1][L]
    const T *xfields;
    const int *estatus;
    const T *pp;
    int L, nfields;
    T *out;
    int64_t mat_stride, ld, n_elem;
    DevStatus *status;         // bounds-checked build only
};

// Affine elements whose matrix is diagonal for every element (one square block, every term
// with diagonal exact 1D integrals): zeros, and on the diagonal
// G_rr = sum_t sign_t c_t D_t(r), D_t(r) = F_t1(i1, i1) F_t2(i2, i2) F_t3(i3, i3),
// r = i1 + nr1 (i2 + nr2 i3).  A CTA writes a span of one element.
constexpr int AFF_DIAG_MAXT = 4;            // terms
constexpr int AFF_DIAG_SPAN_BYTES = 65536;  // output bytes per CTA
constexpr int AFF_DIAG_MAXR = 192;          // diagonal entries per CTA (shared-memory table)
template <typename T>
struct AffDiagParams {
    int64_t n_elem;
    const double *consts;                   // [n_elem][AFF_CONST_STRIDE] from affine_const_kernel
    const double *D;                        // [nterm][n]
    int nterm, field[AFF_DIAG_MAXT], sign[AFF_DIAG_MAXT];
    T *out;                                 // [n_elem][n][n]
    int n, spans;                           // CTAs per element
    int64_t span;                           // values per CTA
    DevStatus *status;
};

// Geometry of extruded elements: metric fields at the (xi2, xi3) Gauss points.
struct Geom2dParams {
    int space, L, nfields;
    int64_t n_elem, elem_base;
    const double *verts, *coeffs;
    const double *zeta, *w;
    void *fields;              // [n_elem][nfields][L][L] of the stage type
    int *estatus;              // [n_elem], zeroed by the caller; set to the element's error
    DevStatus *status;
};

// Load vector of a test space (dpg_integrate_load): one CTA per element at a time.
struct LoadParams {
    int space, q, L;
    int64_t n_elem, elem_base;
    const double *verts;       // chunk start, [n_elem][8][3]
    const double *coef;        // source coefficients: [10 ncomp] shared, or per element
    int64_t coef_stride;       // 0: one source for every element; else values per element
    const double *zeta, *w;    // Gauss rule
    const void *pp;            // pair products of the stage type [NPAIR][NQ1][NQ1][L]
    void *out;                 // chunk start, [n_elem][rows] of the stage type
    DevStatus *status;
};

// Static condensation (dpg_condense), FP64, in place on G, B and l.
struct CondParams {
    int64_t n_elem, elem_base;
    int n, m;
    double *G;                 // [n_elem][n][n], lower triangle -> Cholesky factor
    double *B;                 // [n_elem][n][m] -> L^-1 B
    double *l;                 // [n_elem][n] -> L^-1 l, or NULL
    double *K;                 // [n_elem][m][m]
    double *F;                 // [n_elem][m], NULL when l is NULL
    DevStatus *status;
};

// Static condensation with the digit products on tcgen05 (dpg_condense5.cu): as CondParams,
// plus a per-CTA digit scratch in global memory (scratch_per_cta bytes per CTA of the grid,
// zeroed before the first launch that uses it; lrows / wrows digit rows of L21 / W1^T).
struct Cond5Params {
    int64_t n_elem, elem_base;
    int n, m;
    double *G, *B, *l, *K, *F;
    unsigned char *scratch;
    size_t scratch_per_cta;
    int lrows, wrows;
    int stall_cta;             // test hook: this CTA issues no product for its first panel product (-1: none)
    DevStatus *status;
};

// hp batching: per-q programs in device memory, indexed by q (entry 0 unused).
struct HpProg {
    const BlockDesc *blocks;
    const Unit *units;
    const void *pp;            // pair products of the stage type (double or float)
    const double *zeta, *w;    // Gauss rule
    int nunits, L, nfields, cols, valid;
};

struct HpParams {
    int space;                 // base space id
    int64_t n_elem;
    const double *verts, *coeffs;
    const int *q_elem;
    const int64_t *out_offset;
    void *out;
    const HpProg *tab;         // [MAXQ + 1]
    DevStatus *status;
    // workspace (stream-ordered, per call)
    int *hist, *bstart, *bfill;      // [16] each
    int *order;                      // [n_elem]: elements sorted by descending q
    int64_t *ucnt, *uoff;            // [n_elem]: units of order[k] and their exclusive prefix
    int64_t *fcnt, *foff;            // [n_elem]: field values of element e and their prefix
    int *item_k;                     // [max_items]: position k of each work item
    int64_t *counters;               // [4]: 0 work counter, 1 total items, 2 valid elements
    int64_t *scan_tmp;               // block sums of the scans
    void *fields;
};

// The hp sequence; contract = false stops after the geometry (the caller launches the
// contraction itself).
cudaError_t launch_hp(const HpParams &p, bool fp32, size_t smem, int persistent_ctas, cudaStream_t s,
                      bool contract = true);
int hp_ctas_per_sm(bool fp32, size_t smem);

template <typename TF> cudaError_t launch_geom(const GeomParams &p, cudaStream_t s);
template <typename T> cudaError_t launch_general(const SfParams<T> &p, size_t smem, cudaStream_t s);
cudaError_t launch_general_f32(const SfParams32 &p, size_t smem, int max_nc1, cudaStream_t s);
cudaError_t launch_panel_f32(const PanelParams &p, size_t smem, cudaStream_t s);
cudaError_t launch_tc_f32(const TcParams &p, size_t smem, cudaStream_t s);
cudaError_t launch_tcc(const TccParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t init_tcc_attributes(int optin_smem);
int tcc_static_smem();
cudaError_t init_tc_attributes(int optin_smem);
int tc_static_smem();
cudaError_t launch_affine_const(const AffConstParams &p, cudaStream_t s);
template <typename T> cudaError_t launch_affine(const AffParams<T> &p, size_t smem, cudaStream_t s);
template <typename T> cudaError_t launch_affine_diag(const AffDiagParams<T> &p, cudaStream_t s);
template <typename T> cudaError_t launch_extruded(const AffParams<T> &p, size_t smem, cudaStream_t s);
template <typename TF> cudaError_t launch_geom2d(const Geom2dParams &p, cudaStream_t s);
// Vector-valued Gram matrices (DPG_VEC3): the scalar Gram matrix of each element sits in the
// (0, 0) block of its [3n][3n] matrix; copy it to the (1, 1) and (2, 2) blocks and zero the
// off-diagonal blocks.
template <typename T> cudaError_t launch_vec3_fill(T *out, int64_t n_elem, int n, cudaStream_t s);
size_t extruded_smem_values(const BlockDesc &b, int L, int nj);
template <typename T> cudaError_t launch_load(const LoadParams &p, int num_sms, cudaStream_t s);
// emu: trailing updates as exact BF16-digit products on the tensor cores (else FP64 FMA)
cudaError_t launch_condense(const CondParams &p, int num_sms, bool emu, cudaStream_t s);
int condense_ctas_per_sm(bool emu);
cudaError_t init_condense_attributes();
size_t condense5_scratch_per_cta(int n, int m, bool with_l, int *lrows, int *wrows);
cudaError_t init_condense5_attributes();
cudaError_t launch_condense5(const Cond5Params &p, int grid, cudaStream_t s);
template <typename T> cudaError_t launch_fma_peak(T *out, int blocks, int iters, cudaStream_t s);
cudaError_t init_kernel_attributes(int optin_smem);
cudaError_t launch_dmma_peak(double *out, int blocks, int iters, cudaStream_t s);
// TF32 tensor-core (tcgen05 kind::tf32) rate probe: `ctas` CTAs (one per SM), each 2 iters
// products of 128 x 256 x 8; *status (device) is set to 1 if a bounded wait ran out.
cudaError_t launch_tc_tf32_peak(int ctas, int iters, int *status, cudaStream_t s);
size_t affine_smem_values(const BlockDesc &b, int nj);
int max_dynamic_smem(int optin_smem);

}  // namespace dpg
