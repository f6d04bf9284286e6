/*
 * dpg.h -- C ABI of the GB300 element-matrix library for
 * Mora & Demkowicz, "Fast integration of DPG matrices based on tensorization"
 * (arXiv 1711.00984).
 *
 * The library integrates, for a batch of hexahedral elements, the element Gram matrices
 * of the 3D exact sequence H1 -> H(curl) -> H(div) -> L2 (Eq. 2.1) with integrated
 * Legendre / Legendre tensor-product shape functions (Eqs. 2.33, 2.51-2.57, 2.69-2.74,
 * Sec. 2.8.2), by sum factorization (Eqs. 2.20-2.25 and their H1 / H(div) / H(curl)
 * forms, Eqs. 2.38-2.44, 2.61-2.63, 2.78-2.84), and one mixed stiffness matrix B
 * (pattern of Eqs. 3.15-3.16).  Elements with a constant Jacobian use the O(p^6)
 * variant of Sec. 2.8.1 (Algorithm 10, generalised to a full constant Jacobian).
 *
 * Conventions shared by every entry point:
 *   - Element map: trilinear from 8 vertices; vertex v = v1 + 2 v2 + 4 v3 is the image of
 *     the master-cube corner (v1, v2, v3), master cube (0,1)^3 (Sec. 2.2).
 *   - Quadrature: L-point Gauss-Legendre rule on (0,1) per direction (Eq. 2.23).
 *   - Degrees of freedom: the index maps of the paper, i1 fastest (H1: after Eq. 2.33;
 *     L2: after Eq. 2.17; H(div): Eq. 2.53; H(curl): Eq. 2.71).
 *   - Output: one dense matrix per element, row-major, both triangles, element-major.
 *   - Memory: every pointer argument is DEVICE memory owned by the caller, except in
 *     dpg_integrate_host.  The library owns only its tables and a small status word per
 *     device; they live until dpg_tables_free or process exit.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work is stream-ordered; no entry point synchronises the host except
 *     dpg_sync_status and dpg_integrate_host.
 *   - Errors: every entry point returns a dpg_status.  Argument and set-up errors are
 *     detected on the host before anything is launched.  Errors found on the device
 *     (a non-positive Jacobian determinant, a non-affine element on the affine path) are
 *     recorded in the device status word: the offending element's matrix is filled with
 *     NaN, the call still returns DPG_OK, and dpg_sync_status reports the error and the
 *     first offending element.  Nothing traps the device.
 *   - Threading: table set-up (dpg_tables_init*, dpg_tables_free) must not race with
 *     itself or with integration calls; integration calls on different streams may run
 *     concurrently.
 */
#ifndef DPG_H
#define DPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- spaces (low byte of `space`) ---- */
#define DPG_H1             1   /* (u,v) + (grad u, grad v), Eq. 2.28 / 2.31              */
#define DPG_HCURL          2   /* (E,F) + (curl E, curl F), Eq. 2.65 / 2.68              */
#define DPG_HDIV           3   /* (V,W) + (div V, div W),   Eq. 2.46 / 2.49              */
#define DPG_L2             4   /* (p,q),                    Eq. 2.14 / 2.16              */
#define DPG_B_L2VEC_HCURL  5   /* B_IK = (u_K, psi_I) + (u_K, curl psi_I), vector-L2
                                  trial u of order p, H(curl) test psi of order q
                                  (real, unit-coefficient analogue of Eqs. 3.15-3.16)   */
/* Ultraweak acoustics (Sec. 3.3), real arithmetic with the i*omega factors kept apart.
 * The Gram matrix of the adjoint graph norm (Eq. 3.17) of the test space H1 x H(div) is
 *   [[ G_H1(c0 = omega^2 + alpha, c1 = 1),  -i omega X^T                           ],
 *    [ i omega X,                            G_HDIV(c0 = omega^2 + alpha, c1 = 1)  ]]
 * with the two diagonal blocks from DPG_H1 / DPG_HDIV with coefficients and X below. */
#define DPG_ACOUSTIC_CROSS 6   /* X_IJ = -(div v_I, q_J) + (v_I, grad q_J) (Eq. 3.18, the
                                  coefficient of i omega): rows the H(div) test functions,
                                  columns the H1 test functions, both of order q      */
#define DPG_ACOUSTIC_B     7   /* stiffness of Eq. 3.16, test (q, v) in H1 x H(div) of order
                                  q (rows: H1 then H(div)), trial (p, u) in L2 x (L2)^3 of
                                  order p_trial (columns: scalar then three components);
                                  output [2][rows][cols]: part 0 = -(p, div v) - (u, grad q),
                                  part 1 = (p, q) + (u, v), the coefficient of i omega;
                                  the blocks a part does not contain are written as
                                  zeros (also for an element reported degenerate) */
/* ---- flags ORed into `space` ---- */
/* DPG_FP32: geometry and metric fields computed in FP64, then rounded to FP32; the
 * contraction stages run in FP32 (stage A on the FMA pipe; stages B and C of the general
 * path as tensor-core TF32 products of high/low operand splits, three products per pair,
 * FP32 accumulation); FP32 output.  Target: relative Frobenius error <= 1e-5 per element
 * matrix against the FP64 form.  General-path FP32 Gram matrices are computed block by
 * block without mirroring, so they are symmetric to rounding, not bit for bit. */
#define DPG_FP32        0x100  /* FP32 form (above) */
/* DPG_MAP_AFFINE: the elements are parallelepipeds (constant Jacobian, Sec. 2.8.1): the
 * O(p^6) path of Algorithm 10 with the exact 1D integrals F of Eq. 2.90.  An element whose
 * vertices 3, 5, 6 or 7 deviate from the parallelepiped spanned at vertex 0 by the edges to
 * vertices 1, 2 and 4 by more than 1e-10 times the largest |J_ab| (or by a non-finite amount)
 * is reported as DPG_ERR_NOT_AFFINE and NaN-filled. */
#define DPG_MAP_AFFINE  0x200
#define DPG_B_SPLIT     0x400  /* B only: write [2][rows][cols] = (mass part, curl part) */
/* DPG_MAP_EXTRUDED: the elements are extrusions along x1 of a bilinear quadrilateral in
 * (x2, x3), the second map of Eq. 2.89: x1 = x1(v0) + lambda1 xi1 with lambda1 the same on
 * all four xi1-edges, and (x2, x3) independent of xi1, so J(xi2, xi3) =
 * [[lambda1, 0, 0], [0, eta(xi2, xi3)]].  The metric fields then do not depend on xi1: the
 * xi1 integrals are taken exactly from the 1D integrals F (Eq. 2.90) and the quadrature
 * runs in (xi2, xi3) only (Algorithm 11, O(p^6)).  On such elements the result is the
 * general path's discrete sum (a Gauss rule with L >= q + 1 points is exact in xi1).
 * Elements that are not of this form are reported as DPG_ERR_NOT_EXTRUDED (relative
 * tolerance 1e-10 on the vertices) and NaN-filled.  Not combinable with DPG_MAP_AFFINE. */
#define DPG_MAP_EXTRUDED 0x800
/* DPG_VEC3: the vector- / matrix-valued version V^3 of a Gram space V (H1, H(curl),
 * H(div), L2; Sec. 2.7): test functions e_a (x) v_i with the physical unit vectors e_a,
 * a = 1..3, numbered I = (a - 1) n + i (component-major, n = dim V).  Their inner product
 * is delta_ab (v_i, v_j)_V (Eqs. 2.86, 2.88), so the element matrix is [3n][3n] with the
 * Gram matrix of V in the three diagonal blocks and zeros elsewhere; dpg_matrix_rows /
 * cols return 3n.  Combinable with DPG_FP32 and either map flag; not with the mixed
 * stiffness, the acoustics blocks, dpg_integrate_hp or dpg_integrate_noalloc. */
#define DPG_VEC3 0x1000

/* ---- status codes ---- */
typedef enum {
    DPG_OK = 0,
    DPG_ERR_ARG = 1,         /* bad argument (NULL pointer, bad space/flags, p > q ...) */
    DPG_ERR_NOT_INIT = 2,    /* no tables for (space, q): call dpg_tables_init first    */
    DPG_ERR_RANGE = 3,       /* q or L outside the supported range                      */
    DPG_ERR_CUDA = 4,        /* a CUDA runtime call failed                              */
    DPG_ERR_DEGENERATE = 5,  /* device: |J| <= 0 or not finite at a quadrature point    */
    DPG_ERR_NOT_AFFINE = 6,  /* device: element is not a parallelepiped (affine path)   */
    DPG_ERR_NOMEM = 7,       /* device or host allocation failed                        */
    DPG_ERR_SCRATCH = 8,     /* dpg_integrate_noalloc: the call needs more metric-field
                                scratch than DPG_NOALLOC_SCRATCH_BYTES                  */
    DPG_ERR_TIMEOUT = 9,     /* device: a bounded wait of the FP32 tensor-core kernel for
                                its own MMAs ran out; the CTA stopped, the matrices of the
                                call are not valid (first_bad = first element of the CTA) */
    DPG_ERR_NOT_EXTRUDED = 10, /* device: element is not an extrusion along x1
                                (DPG_MAP_EXTRUDED)                                       */
    DPG_ERR_NOT_SPD = 11,    /* device: dpg_condense met a Gram matrix that is not positive
                                definite (a pivot <= 0 or not finite)                    */
    DPG_ERR_BOUNDS = 12      /* device, bounds-checked build (libdpg_debug.so) only: a
                                kernel's shared- or global-memory index, metric-field
                                index or tensor-memory column left the extent it was
                                given; the access was skipped (first_bad = the element) */
} dpg_status;

#define DPG_MAX_Q 12           /* supported test orders: 1 <= q <= DPG_MAX_Q           */
#define DPG_MAX_L 14           /* supported points per direction: 1 <= L <= DPG_MAX_L  */

/* Build and upload the tables for test order q of `space` (flags ignored) with the
 * default rule L = q + 2: Gauss nodes and weights on (0,1) (Eq. 2.23), the 1D families
 * chi_i = L_i, chi'_i, nu_i = P_i at the nodes (Eqs. 2.91-2.101, 2.54), products of pairs
 * of them (the 1D factors of Eqs. 2.23-2.25), the exact 1D integrals F^{rs} (Eq. 2.90),
 * and the term programs of each space.  Synchronous (host work and cudaMemcpy); call it
 * before capturing integration calls in a CUDA graph.  Re-initialising (space, q) with a
 * different L makes that L the active rule for (space, q).
 * Errors: DPG_ERR_ARG (unknown space), DPG_ERR_RANGE (q), DPG_ERR_CUDA, DPG_ERR_NOMEM. */
int dpg_tables_init(int q, int space);

/* Same with an explicit number of Gauss points L per direction (1 <= L <= DPG_MAX_L). */
int dpg_tables_init_L(int q, int L, int space);

/* Release every table and program on every device.  Not stream-ordered: the caller must
 * make sure no integration call is in flight. */
int dpg_tables_free(void);

/* Number of rows of the element matrix: dim of the test space at order q
 * ((q+1)^3, 3q(q+1)^2, 3(q+1)q^2, q^3 for H1, H(curl), H(div), L2; H(curl) for B;
 * H(div) for DPG_ACOUSTIC_CROSS; H1 + H(div) for DPG_ACOUSTIC_B).
 * Returns -1 for a bad space or q. */
int64_t dpg_matrix_rows(int space, int q);

/* Number of columns: equal to rows for Gram matrices; 3 p^3 for DPG_B_L2VEC_HCURL;
 * (q+1)^3 for DPG_ACOUSTIC_CROSS; 4 p^3 for DPG_ACOUSTIC_B.  Returns -1 for bad arguments. */
int64_t dpg_matrix_cols(int space, int p_trial, int q);

/* Integrate the element matrices of n_elem elements (the paper's per-element routine
 * PROC(mid, G) of Algorithms 2-11, batched; problem statement Eq. 2.13).
 *   space    : DPG_H1 .. DPG_ACOUSTIC_B, ORed with DPG_FP32 / DPG_MAP_AFFINE or
 *              DPG_MAP_EXTRUDED / DPG_B_SPLIT (B only) / DPG_VEC3 (Gram spaces).
 *   p_trial  : trial order for DPG_B_L2VEC_HCURL and DPG_ACOUSTIC_B
 *              (1 <= p_trial <= q_test); ignored (pass 0) otherwise.
 *   q_test   : test order; tables for (space, q_test) must be initialised.
 *   n_elem   : number of elements (0 is allowed and does nothing).
 *   vertices : device, double[n_elem][8][3].
 *   coeffs   : device, double[n_elem][2] = (mass weight c0, derivative weight c1), or
 *              NULL for (1, 1).  G = c0 (mass term) + c1 (derivative term); L2 uses c0.
 *              Ignored for the non-Gram spaces (B, acoustics cross block and stiffness).
 *   out      : device, double (FP64 form) or float (DPG_FP32) array of
 *              n_elem * parts * rows * cols values, parts = 2 with DPG_B_SPLIT and for
 *              DPG_ACOUSTIC_B, else 1.
 *   stream   : cudaStream_t.
 * The call allocates a stream-ordered workspace for the per-point metric fields from a
 * library memory pool and frees it in stream order.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOT_INIT, DPG_ERR_RANGE, DPG_ERR_CUDA, DPG_ERR_NOMEM;
 * device-detected errors through dpg_sync_status. */
int dpg_integrate(int space, int p_trial, int q_test, int64_t n_elem,
                  const double *vertices, const double *coeffs, void *out, void *stream);

/* hp-mixed batch (elements of different test orders q in one call), general map: the
 * per-element routine of the paper (Algorithms 5, 7, 9 and their L2 form) for every
 * element at its own order q_elem[e] with its own rule L(q) (the active rule of
 * dpg_tables_init for (space, q)).  One device-driven sequence: the elements are sorted by
 * descending q on the device, the work units of all elements are handed out by one
 * persistent kernel from an atomic counter, and the whole sequence is captured into a
 * CUDA graph on the first call with a given argument set and replayed afterwards (the
 * cache is cleared by dpg_tables_init* and dpg_tables_free).
 *   space      : DPG_H1, DPG_HCURL, DPG_HDIV or DPG_L2, optionally | DPG_FP32.
 *   q_elem     : device, int[n_elem], each in [1, DPG_MAX_Q] with tables initialised.
 *   out_offset : device, int64[n_elem]: element e's rows(q_e) x cols(q_e) matrix starts
 *                at out + out_offset[e] (counted in values of the output type).
 *   vertices, coeffs, out : as for dpg_integrate (out is the packed batch).
 * Elements with an order outside the range or without tables are skipped and reported
 * through dpg_sync_status (DPG_ERR_RANGE / DPG_ERR_NOT_INIT with the first such element).
 * Workspace: stream-ordered from the library pool, about n_elem * (max nfields L^3) values.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOT_INIT (no order of `space` initialised), DPG_ERR_CUDA. */
int dpg_integrate_hp(int space, int64_t n_elem, const double *vertices, const double *coeffs,
                     const int *q_elem, const int64_t *out_offset, void *out, void *stream);

/* Autotuner (not in the paper): for the general path of (space, q) with its active rule,
 * time every stage-A chunk width nj (the number of partner indices j_A one work unit
 * produces: tile shape and stage schedule of the contraction kernels) on a synthetic batch
 * of up to 512 elements (fewer where their output would pass 2 GB, at least 8; median of
 * five runs) on `stream`, and install the fastest for dpg_integrate and
 * dpg_integrate_hp; for FP64 programs that hold both diagonal blocks of the symmetric
 * matrix (their work units run from j_A = i_A up, so they are uneven) and full blocks
 * (H(curl), H(div)), a second pass picks a smaller width for the diagonal blocks alone.
 * space = DPG_H1 .. DPG_L2, optionally | DPG_FP32 (tunes the FP32 form: besides the widths
 * of the earlier FP32 kernels it times the kernel with stage C on the tensor cores and
 * stages A and B on the FMA pipe, reported as nj = 0; dpg_integrate_hp uses that kernel
 * for every order that has it).  If the environment variable DPG_AUTOTUNE_CACHE names a file, a choice stored
 * there for (space, q, L, precision) is installed without timing, and new choices are
 * appended as JSON lines ({"space", "q", "L", "fp32", "nj", "ms", "nj_sym"}; nj_sym = 0:
 * the diagonal blocks use nj too).  Synchronous; allocates temporary device buffers; call it at
 * set-up, not inside stream capture.  *best_nj (if not NULL) receives the chosen width.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOT_INIT, DPG_ERR_RANGE, DPG_ERR_CUDA. */
int dpg_autotune(int q, int space, void *stream, int *best_nj);

/* Allocation-free variant of dpg_integrate for the general (trilinear-map) path.  The
 * paper has no counterpart: this is a service for callers that must not allocate device
 * memory while they integrate -- a solver whose device memory is carved up once at start
 * and may not grow, code that runs inside another framework's allocator or memory
 * budget, or a call issued where an allocation would stall the stream or the device.
 * dpg_integrate takes its metric-field workspace from a memory pool; this entry point
 * instead uses one file-scope device array of DPG_NOALLOC_SCRATCH_BYTES (32 MiB).  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   Arguments, layouts and results are those of dpg_integrate for the general map, FP64
 *   and FP32 forms (the same programs and kernels); DPG_MAP_AFFINE, DPG_MAP_EXTRUDED and
 *   DPG_VEC3 are rejected (DPG_ERR_ARG).
 *   Limit: n_elem * nfields * L^3 * (8 or 4 bytes) must fit the array (nfields = 7, 12,
 *   7, 1, 18 for H1, H(curl), H(div), L2, B; 4 bytes with DPG_FP32), else the call
 *   returns DPG_ERR_SCRATCH before launching anything.  Example: H(curl), q = 5, L = 7,
 *   FP64 fits 1019 elements per call, FP32 2038.
 *   Set-up and memory: the array belongs to a module that CUDA loads lazily (by default),
 *   so its 32 MiB are reserved on a device by the first call on that device -- the call
 *   that looks up the array's device address (cudaGetSymbolAddress, with that device
 *   current) -- and stay reserved until the process exits.  Make that first call at
 *   set-up, within the caller's memory budget, and before any stream capture; later
 *   calls reserve nothing.  Tables must be initialised with dpg_tables_init beforehand.
 *   Sharing: all calls use the same array and it keeps the last call's contents (every
 *   value a call reads is written by that call first, so nothing needs clearing); calls
 *   that overlap on the GPU, e.g. on two streams, race on it and must be serialised by
 *   the caller.  On the host, a call holds the library's lock from its program look-up to
 *   its last launch, like dpg_integrate. */
#define DPG_NOALLOC_SCRATCH_BYTES (32u << 20)
int dpg_integrate_noalloc(int space, int p_trial, int q_test, int64_t n_elem,
                          const double *vertices, const double *coeffs, void *out, void *stream);

/* Same as dpg_integrate, but vertices, coeffs and out are HOST buffers (page-locked for
 * full copy speed).  Copies the inputs to the device, then streams the batch: chunks of
 * about 64 MB of output are integrated on `stream` while earlier chunks are copied back
 * on library-owned copy streams, so compute and device-to-host traffic overlap.  The call
 * synchronises `stream` before returning; device buffers come from the library memory
 * pool.  Device-detected errors are returned directly (the call reads the status word). */
int dpg_integrate_host(int space, int p_trial, int q_test, int64_t n_elem,
                       const double *vertices, const double *coeffs, void *out, void *stream);

/* Load vector of a test space: l_I = (f, v_I)_K for every test function v_I of order q_test
 * (the right-hand side ell(v_I) of the DPG system, Sec. 3, e.g. the (f, q) of Eq. 3.13 with
 * v = q), by conventional Gauss quadrature on the active rule of (space, q_test) evaluated by
 * sum factorization (Eqs. 2.23-2.25 with a single test index).  The source is a polynomial
 * of total degree <= 2 in the physical coordinates x:
 *   f_c(x) = sum_k src_coef[10 c + k] m_k(x),  m = (1, x1, x2, x3, x1^2, x2^2, x3^2,
 *   x1 x2, x1 x3, x2 x3),
 * scalar (c = 0) for H1 and L2, a vector (c = 0, 1, 2) for H(curl) and H(div); test
 * functions are mapped by Eqs. 2.3-2.6, so the integrand is w |J| f v^ (H1), w f q^ (L2),
 * w |J| (J^-1 f) . psi^ (H(curl)), w (J^T f) . theta^ (H(div)).
 *   space       : DPG_H1 .. DPG_L2, optionally | DPG_FP32 (geometry and source in FP64,
 *                 contractions and output in FP32).  Tables for (space, q_test) must be
 *                 initialised (DPG_ERR_NOT_INIT).
 *   vertices    : device, double[n_elem][8][3].
 *   src_coef    : device, double: 10 (H1, L2) or 30 (H(curl), H(div)) values shared by all
 *                 elements when coef_stride = 0, else element e reads
 *                 src_coef + e * coef_stride (coef_stride >= 10 or 30).
 *   out         : device, double or float [n_elem][dpg_matrix_rows(space, q_test)].
 * An element with |J| <= 0 at a point is NaN-filled and reported as DPG_ERR_DEGENERATE
 * through dpg_sync_status.  No workspace is allocated.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOT_INIT, DPG_ERR_RANGE, DPG_ERR_CUDA. */
int dpg_integrate_load(int space, int q_test, int64_t n_elem, const double *vertices,
                       const double *src_coef, int64_t coef_stride, void *out, void *stream);

/* Static condensation of the test variables, element by element (Eq. 3.8 from Eq. 3.7):
 *   K = B^T G^-1 B   and   F = B^T G^-1 l,
 * with G the Gram matrix of the test space (n x n, symmetric positive definite), B the
 * enriched stiffness (n x m; the skeleton block B~ of Eq. 3.8 is handled by passing the
 * columns [B | B~] as one matrix) and l the load vector.  Steps as the paper names them:
 * Cholesky factorization G = L L^T, the substitutions W = L^-1 B and y = L^-1 l, and the
 * products K = W^T W, F = W^T y.  FP64 results; the O(n^3) updates and W^T W run on the
 * tensor cores as exact digit products unless dpg_condense_set_method selects FP64 FMA
 * (with the default method the load vector rides along as one more column of B, so that
 * y and F come out of the same products).
 *   n_elem   : number of elements (0 does nothing).
 *   n, m     : 1 <= n <= 8192, 1 <= m <= 8192.
 *   G        : device, double[n_elem][n][n] row-major.  Only the lower triangle is read;
 *              it is OVERWRITTEN with the Cholesky factor L (the strict upper triangle is
 *              left as it was).
 *   B        : device, double[n_elem][n][m] row-major (rows: test functions, e.g. the
 *              output of DPG_B_L2VEC_HCURL); OVERWRITTEN with W = L^-1 B.
 *   l        : device, double[n_elem][n], or NULL; OVERWRITTEN with y = L^-1 l.
 *   K        : device, double[n_elem][m][m], both triangles written.
 *   F        : device, double[n_elem][m]; must be NULL exactly when l is NULL.
 *   stream   : cudaStream_t.
 * An element whose G is not positive definite gets NaN in K (and F) and is reported as
 * DPG_ERR_NOT_SPD through dpg_sync_status; its G, B, l are left partially factored.  With
 * the digit-product methods, a value of B or l that is not finite is reported the same way
 * (the FMA route lets it propagate as NaN into K and F without a status).
 * Workspace: none for DPG_CONDENSE_FMA and DPG_CONDENSE_TC (everything happens in place);
 * DPG_CONDENSE_TCGEN05 takes a digit scratch of about 0.9 (ceil(n / 128) + ceil((m + 1) /
 * 128)) 128 kB per SM from the library pool, stream-ordered (1.1 MB per SM at n = 882,
 * m = 192), released before the call returns to the stream.
 * Errors: DPG_ERR_ARG, DPG_ERR_RANGE (n or m), DPG_ERR_CUDA. */
int dpg_condense(int64_t n_elem, int n, int m, double *G, double *B, double *l, double *K, double *F,
                 void *stream);

/* Arithmetic of the condensation's trailing updates (the O(n^3) and O(n^2 m) part of
 * dpg_condense and dpg_condensed_system) and of K = W^T W, for every later call in the
 * process:
 *   DPG_CONDENSE_FMA    : FP64 fused multiply-adds (panels of 32 columns).
 *   DPG_CONDENSE_TC     : the same FP64 products from exact BF16 digits on the tensor cores
 *                         (mma.sync, panels of 32) -- each operand row split as
 *                         2^e sum_{u<7} d_u 2^-(8u+7) with balanced digits |d_u| <= 128, the
 *                         digit products summed exactly in FP32 and combined in a 64-bit
 *                         integer, entering the FP64 result once per product; what is dropped
 *                         lies below about 2^-53 of the product of the two rows' maxima, so
 *                         the results agree with the FMA route normwise (relative to the row
 *                         maxima), not entry by entry: an entry far below its row's maximum
 *                         keeps fewer correct bits.
 *   DPG_CONDENSE_TCGEN05: (the default) the same digit scheme on the fifth-generation tensor
 *                         cores (tcgen05, accumulators in tensor memory), panels of 64, the
 *                         digits of each panel's rows split once and reused by every tile,
 *                         the load vector carried as a column of B (F = the last row of the
 *                         extended W^T W); one CTA per SM and a digit scratch (dpg_condense).
 * The factorization of the diagonal blocks stays FP64 in every method (the panel products
 * with the inverse diagonal blocks follow the method; F = W^T y is FP64 FMA in the first
 * two).  Errors: DPG_ERR_ARG. */
#define DPG_CONDENSE_FMA     0
#define DPG_CONDENSE_TC      1
#define DPG_CONDENSE_TCGEN05 2
int dpg_condense_set_method(int method);

/* The DPG element routine of the mixed-stiffness pair in one call (Sec. 3, Eqs. 3.7-3.8):
 * per element, the Gram matrix G of the H(curl) test space of order q_test (coefficients as
 * in dpg_integrate), the enriched stiffness B of DPG_B_L2VEC_HCURL with trial order p_trial,
 * the load vector l of dpg_integrate_load (optional), then K = B^T G^-1 B and F = B^T G^-1 l
 * as in dpg_condense.  G, B and l live only in a library workspace (stream-ordered, from the
 * library pool, processed in chunks of at most 8 GB): the caller receives K and F.
 *   q_test, p_trial : tables for (DPG_HCURL, q_test) and (DPG_B_L2VEC_HCURL, q_test) must be
 *                     initialised with the same rule L; 1 <= p_trial <= q_test.
 *   vertices        : device, double[n_elem][8][3].
 *   coeffs          : device, double[n_elem][2] (G's mass and curl weights) or NULL.
 *   src_coef        : device, the source of dpg_integrate_load for H(curl) (30 values, or
 *                     per element with coef_stride >= 30), or NULL for no load vector.
 *   K               : device, double[n_elem][m][m], m = 3 p_trial^3.
 *   F               : device, double[n_elem][m]; NULL exactly when src_coef is NULL.
 * Device-detected errors (a degenerate element: DPG_ERR_DEGENERATE; G not positive definite:
 * DPG_ERR_NOT_SPD) through dpg_sync_status, element indices relative to the call.
 * Errors: DPG_ERR_ARG, DPG_ERR_NOT_INIT, DPG_ERR_RANGE, DPG_ERR_CUDA, DPG_ERR_NOMEM. */
int dpg_condensed_system(int q_test, int p_trial, int64_t n_elem, const double *vertices,
                         const double *coeffs, const double *src_coef, int64_t coef_stride, double *K,
                         double *F, void *stream);

/* Test hook (not part of the method): the next launch of a tcgen05 kernel -- the FP32
 * contraction of the general map (DPG_FP32 through dpg_integrate) or the condensation
 * (DPG_CONDENSE_TCGEN05 through dpg_condense / dpg_condensed_system) -- runs with its first
 * CTA never completing its tensor-core products (no stage-B product, no commit of the
 * stage-C products, or no first panel product), so that CTA's bounded mbarrier waits run out
 * (after about a second), the CTA releases its tensor memory and records DPG_ERR_TIMEOUT
 * (first_bad = its first element); the other CTAs and later calls are unaffected.  Exercises
 * the kernels' failure path without a GPU fault.  Returns DPG_OK. */
int dpg_test_stall_tc_once(void);

/* Test hook (not part of the method): caps the metric-field workspace of one chunk of the
 * general and extruded-map paths (dpg_integrate, dpg_integrate_host, dpg_autotune) at
 * `bytes` (at least one element per chunk) instead of the library's 512 MB, so that a
 * small call runs through several chunks; 0 restores the default.  Applies to every later
 * call in the process.  Returns DPG_OK, or DPG_ERR_ARG for bytes < 0. */
int dpg_test_set_workspace_limit(int64_t bytes);

/* Synchronise `stream`, read and clear the device status word of the current device.
 * Returns DPG_OK or the first device-detected error; *first_bad_elem (if not NULL)
 * receives the smallest offending element index of that error, or -1. */
int dpg_sync_status(void *stream, int64_t *first_bad_elem);

/* Static English description of a status code. */
const char *dpg_strerror(int code);

/* Diagnostic text of the last CUDA runtime failure seen by the library (the failing call
 * and the CUDA error name), or "" if none.  Not thread-safe; for error messages only. */
const char *dpg_last_cuda_error(void);

/* Algorithmic floating-point operations of one element (multiply and add counted
 * separately) of the sum-factorization path (stages of Eqs. 2.23-2.25 per block of
 * terms, symmetric tiles counted once), or of the affine path (non-zero products of the
 * Kronecker sums of Sec. 2.8.1) with DPG_MAP_AFFINE.  The count is the same for the FP64
 * and FP32 forms (cheapest direction order per block).  Tables must be initialised.
 * Returns -1 on error.  Used to report the ALU roofline. */
double dpg_flops_per_element(int space, int p_trial, int q_test);

/* Not part of the paper's method: measure the device's peak fused multiply-add rate in
 * FP64 (precision = 64) or FP32 (precision = 32) with a register-resident FMA loop, the
 * FP64 tensor-core rate (precision = 65, mma.sync m8n8k4 FP64), or the TF32 rate of the
 * fifth-generation tensor cores (precision = 19: tcgen05 kind::tf32, 128 x 256 x 8
 * products, one CTA per SM), on `stream`; writes the flop rate (2 flops per multiply-add)
 * in flop/s to *flops.  Synchronous.  Used only to give the ALU and tensor rooflines a
 * measured denominator.  DPG_ERR_TIMEOUT if the tensor-core probe's bounded wait ran out. */
int dpg_measure_fma_peak(int precision, void *stream, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* DPG_H */
