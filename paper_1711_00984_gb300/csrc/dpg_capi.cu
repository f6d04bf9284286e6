// dpg_capi.cu -- the C ABI (include/dpg.h): argument checks, table registry, workspace,
// launches.  No per-element host work.
#include "../../include/dpg.h"

#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <algorithm>
#include <tuple>
#include <vector>

#include "dpg_kernels.h"
#include "dpg_registry.h"
#include "dpg_setup.h"
#include "dpg_trace.h"

using namespace dpg;

namespace {

constexpr size_t kWorkspaceLimit = size_t(512) << 20;   // metric fields per launch chunk
enum { K32_MIRROR = 0, K32_PANEL = 1, K32_TC = 2, K32_TCC = 3 };   // FP32 general-path kernels
int g_max_dyn_smem = 0;                                  // per launch, set at device set-up
int g_max_dyn_smem_tc = 0;                               // the same for the tensor-core kernel
int g_max_dyn_smem_tcc = 0;                              // and for the stage-C tensor-core kernel
int g_smem_per_sm = 0;                                   // shared memory of an SM
int g_tc_stall_once = 0;                                 // test hook, see dpg_test_stall_tc_once
int g_num_sms = 152;                                     // set at device set-up
int g_condense_method = DPG_CONDENSE_TCGEN05;                 // see dpg_condense_set_method
size_t g_ws_limit_test = 0;                              // see dpg_test_set_workspace_limit

struct TableEntry {
    HostTables host;
    double *zeta = nullptr, *w = nullptr, *pp64 = nullptr, *F64 = nullptr;
    float *pp32 = nullptr, *F32 = nullptr;
};

struct AffProg {
    Program prog;
    BlockDesc *d_blocks = nullptr;
    Unit *d_units = nullptr;
    int *d_block_units = nullptr;   // [nblock + 1] unit ranges
    unsigned char *d_img = nullptr; // constant shared-memory images of the blocks
    int *d_img_off = nullptr;       // [nblock + 1], 16-byte units
    size_t smem_values = 0;         // values of the kernel's shared memory
    unsigned *d_qlist = nullptr;    // structural stage-B lists of the units (affine only)
    int *d_qoff = nullptr;          // [nunits + 1]
    // the matrix is diagonal whatever the element (affine only): its terms and the products
    // D_t(r) of their diagonal exact 1D integrals, [nterm][rows]
    bool diag = false;
    double *d_diag = nullptr;
    int diag_nterm = 0, diag_field[AFF_DIAG_MAXT] = {}, diag_sign[AFF_DIAG_MAXT] = {};
};

// Program of the FP32 general kernel with stage C on the tensor cores (sf_tcc_kernel).
struct TccProg {
    bool ok = false;
    Program prog;
    BlockDesc *d_blocks = nullptr;
    float *d_img = nullptr;         // constant images of the blocks
    int *d_off = nullptr, *d_base = nullptr;
    int tcols = 0, cps = 1;         // tensor-memory columns per CTA, CTAs per SM
    size_t smem = 0;                // dynamic shared memory of the launch
};

struct ProgEntry {
    Program prog;                   // general path: per-block contraction order
    BlockDesc *d_blocks = nullptr;
    Unit *d_units = nullptr;
    // affine path, the paper's direction order: [0] FP64 kernel (a chunk for three CTAs per
    // SM), [1] FP32 kernel (the larger chunk that fits two)
    AffProg aff[2];
    double flops_aff = 0.0;         // algorithmic flops of the affine path
    AffProg ext[2];                 // extruded-map path, [0] FP64, [1] FP32
    double flops_ext = 0.0;         // algorithmic flops of the extruded-map path
    Program prog32;                 // FP32 general path: tensor-core program (kind32 = K32_TC),
                                    // row-panel program (K32_PANEL) or the mirrored-tile
                                    // program with stage A on xi_3 (K32_MIRROR)
    int kind32 = 0;
    float *d_ctab32 = nullptr;      // K32_TC / K32_PANEL: constant operands of every block
    int *d_ctab_off32 = nullptr;    // [nblock] offsets into d_ctab32
    BlockDesc *d_blocks32 = nullptr;
    Unit *d_units32 = nullptr;
    int max_nc1_32 = 0;             // largest stage-C column extent of prog32
    int *d_block_units32 = nullptr; // [nblock + 1] unit ranges of prog32
    TccProg tcc;                    // the stage-C tensor-core program (uniform when kind32 ==
                                    // K32_TCC; the FP32 hp contraction whenever it exists)
};

using ProgKey = std::tuple<int, int, int, int, int>;   // space, q, L, p, split

// Key of a captured hp graph: every argument that the captured launches bake in.
struct HpKey {
    int space;
    int64_t n_elem;
    const void *verts, *coeffs, *q_elem, *out_offset, *out;
    bool operator<(const HpKey &o) const {
        return std::tie(space, n_elem, verts, coeffs, q_elem, out_offset, out) <
               std::tie(o.space, o.n_elem, o.verts, o.coeffs, o.q_elem, o.out_offset, o.out);
    }
};

struct DeviceState {
    DevStatus *status = nullptr;
    cudaMemPool_t pool = nullptr;
    // hp batching: per (precision, space) the device table of per-q programs
    HpProg h_hp[2][6][MAXQ + 1] = {};
    HpProg *d_hp[2][6] = {};
    size_t hp_smem[2][6] = {};       // dynamic shared memory of the persistent kernel
    int hp_max_units[6] = {};        // most work units of an initialised q
    int64_t hp_max_fields[6] = {};   // most metric-field values of an initialised q
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_streams[4] = {};   // device-to-host drains of dpg_integrate_host
    std::map<HpKey, cudaGraphExec_t> hp_graphs;
    std::map<std::pair<int, int>, std::unique_ptr<TableEntry>> tables;   // (q, L)
    std::map<ProgKey, std::unique_ptr<ProgEntry>> progs;
    std::map<std::pair<int, int>, int> active_L;                         // (space, q) -> L
};

std::mutex g_mu;
std::map<int, std::unique_ptr<DeviceState>> g_dev;

char g_last_error[512] = "";

int cuda_fail(cudaError_t e, const char *what, int line) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s (line %d): %s: %s", what, line,
                  cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DPG_ERR_NOMEM : DPG_ERR_CUDA;
}

#define CK(x)                                                               \
    do {                                                                    \
        cudaError_t e_ = (x);                                               \
        if (e_ != cudaSuccess) { return cuda_fail(e_, #x, __LINE__); }      \
    } while (0)

template <typename T>
int upload(const T *src, size_t n, T **dst) {
    CK(cudaMalloc(dst, n * sizeof(T)));
    CK(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return DPG_OK;
}

// Device copy of the constant images of an affine / extruded program in precision prec.
int upload_aff_image(AffProg &ap, const HostTables &tab, bool extruded, int prec) {
    std::vector<unsigned char> img;
    std::vector<int> off;
    if (prec) build_aff_image<float>(ap.prog, tab, extruded, img, off);
    else build_aff_image<double>(ap.prog, tab, extruded, img, off);
    int r;
    if ((r = upload(img.data(), img.size(), &ap.d_img))) return r;
    if ((r = upload(off.data(), off.size(), &ap.d_img_off))) return r;
    return DPG_OK;
}

void reset_host_status(DevStatus &s) {
    std::memset(&s, 0, sizeof(s));
    for (int i = 0; i < 16; ++i) s.first_bad[i] = ULLONG_MAX;
}

int device_state(DeviceState **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) { *out = it->second.get(); return DPG_OK; }
    auto st = std::make_unique<DeviceState>();
    CK(cudaMalloc(&st->status, sizeof(DevStatus)));
    DevStatus h;
    reset_host_status(h);
    CK(cudaMemcpy(st->status, &h, sizeof(h), cudaMemcpyHostToDevice));
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    CK(cudaMemPoolCreate(&st->pool, &props));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(st->pool, cudaMemPoolAttrReleaseThreshold, &thr));
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(init_kernel_attributes(optin));
    CK(init_condense_attributes());
    CK(init_condense5_attributes());
    g_max_dyn_smem = max_dynamic_smem(optin);
    CK(init_tc_attributes(optin));
    g_max_dyn_smem_tc = optin - tc_static_smem();
    CK(init_tcc_attributes(optin));
    g_max_dyn_smem_tcc = optin - tcc_static_smem();
    CK(cudaDeviceGetAttribute(&g_smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CK(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking));
    for (auto &cs : st->copy_streams) CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    *out = st.get();
    g_dev[dev] = std::move(st);
    return DPG_OK;
}

int get_tables(DeviceState *ds, int q, int L, TableEntry **out) {
    auto key = std::make_pair(q, L);
    auto it = ds->tables.find(key);
    if (it != ds->tables.end()) { *out = it->second.get(); return DPG_OK; }
    auto te = std::make_unique<TableEntry>();
    te->host = make_tables(q, L);
    const HostTables &h = te->host;
    std::vector<float> pp32(h.pp.begin(), h.pp.end()), F32(h.F.begin(), h.F.end());
    int r;
    if ((r = upload(h.zeta.data(), h.zeta.size(), &te->zeta))) return r;
    if ((r = upload(h.w.data(), h.w.size(), &te->w))) return r;
    if ((r = upload(h.pp.data(), h.pp.size(), &te->pp64))) return r;
    if ((r = upload(pp32.data(), pp32.size(), &te->pp32))) return r;
    if ((r = upload(h.F.data(), h.F.size(), &te->F64))) return r;
    if ((r = upload(F32.data(), F32.size(), &te->F32))) return r;
    *out = te.get();
    ds->tables[key] = std::move(te);
    return DPG_OK;
}

// Build and upload the FP32 general-path program of pe with stage-A chunk nj (0: largest
// that fits): the tensor-core program where every block fits the tcgen05 kernel, else the
// row-panel program where its shared memory fits a CTA, else the mirrored-tile program.
// The previous device copies are freed (the caller synchronises).
// Build and upload the stage-C tensor-core program of pe where every block fits the kernel.
int setup_tcc(ProgEntry *pe, int space, int q, int L, int p, bool split, const HostTables &tab) {
    TccProg &t = pe->tcc;
    Program tp = make_program(space, q, L, p, split, tab, ORDER_TCC, 1, (size_t)g_max_dyn_smem_tcc);
    if (tp.smem_bytes > (size_t)g_max_dyn_smem_tcc) { t.ok = false; return DPG_OK; }
    std::vector<float> img;
    std::vector<int> off, base(tp.nblock + 1, 0);
    build_tcc_tables(tp, tab, img, off);
    int tcols = 32;
    for (int k = 0; k < tp.nblock; ++k) {
        base[k + 1] = base[k] + tp.blocks[k].nr[2];
        tcols = std::max(tcols, tcc_layout(tp.blocks[k], L).tcols);
    }
    int r;
    if ((r = upload(tp.blocks, (size_t)tp.nblock, &t.d_blocks))) return r;
    if ((r = upload(img.data(), img.size(), &t.d_img))) return r;
    if ((r = upload(off.data(), off.size(), &t.d_off))) return r;
    if ((r = upload(base.data(), base.size(), &t.d_base))) return r;
    t.tcols = tcols;
    // CTAs per SM: at most three (the kernel's register budget), as many as the tensor memory
    // (each CTA holds tcols columns for its whole life) and the shared memory allow; below
    // three, the shared-memory request is raised so that no further CTA is placed on the SM
    // (it would wait for tensor memory)
    const size_t st = (size_t)(tcc_static_smem() + 1024);
    int cps = std::min(3, 512 / tcols);
    cps = std::min(cps, (int)((size_t)g_smem_per_sm / (tp.smem_bytes + st)));
    cps = std::max(cps, 1);
    size_t req = tp.smem_bytes;
    if (cps < 3) req = std::max(req, (size_t)g_smem_per_sm / (cps + 1) - st + 16);
    t.cps = cps;
    t.smem = std::min(req, (size_t)g_max_dyn_smem_tcc);
    t.prog = tp;
    t.ok = true;
    return DPG_OK;
}

int setup_prog32(ProgEntry *pe, int space, int q, int L, int p, bool split, const HostTables &tab, int nj) {
    // nj == 0: stage C on the tensor cores (stages A and B on the FMA pipe) where the
    // program exists; nj > 0 (autotuner): the earlier FP32 kernels with stage-A chunk nj
    if (nj == 0 && pe->tcc.ok) {
        cudaFree(pe->d_blocks32); cudaFree(pe->d_units32); cudaFree(pe->d_block_units32);
        cudaFree(pe->d_ctab32); cudaFree(pe->d_ctab_off32);
        pe->d_blocks32 = nullptr; pe->d_units32 = nullptr; pe->d_block_units32 = nullptr;
        pe->d_ctab32 = nullptr; pe->d_ctab_off32 = nullptr;
        pe->kind32 = K32_TCC;
        pe->prog32 = pe->tcc.prog;
        pe->max_nc1_32 = 0;
        return DPG_OK;
    }
    int kind = K32_TC;
    Program np = make_program(space, q, L, p, split, tab, ORDER_TC, nj, (size_t)g_max_dyn_smem_tc);
    if (np.smem_bytes > (size_t)g_max_dyn_smem_tc) {
        kind = K32_PANEL;
        np = make_program(space, q, L, p, split, tab, ORDER_PANEL, nj);
        if (np.smem_bytes > (size_t)g_max_dyn_smem) {
            kind = K32_MIRROR;
            np = make_program(space, q, L, p, split, tab, ORDER_A3, nj);
        }
    }
    if (np.smem_bytes > (size_t)g_max_dyn_smem) return DPG_ERR_RANGE;
    BlockDesc *db = nullptr;
    Unit *du = nullptr;
    int *dbu = nullptr, *doff = nullptr;
    float *dct = nullptr;
    int r;
    if ((r = upload(np.blocks, (size_t)np.nblock, &db))) return r;
    if ((r = upload(np.units.data(), np.units.size(), &du))) return r;
    std::vector<int> ub(np.nblock + 1, 0);
    for (const Unit &u : np.units) ub[u.block + 1]++;
    for (int k = 0; k < np.nblock; ++k) ub[k + 1] += ub[k];
    if ((r = upload(ub.data(), ub.size(), &dbu))) return r;
    if (kind != K32_MIRROR) {
        std::vector<float> ct;
        std::vector<int> off;
        if (kind == K32_TC) build_tc_tables(np, tab, ct, off);
        else build_panel_tables(np, tab, ct, off);
        if ((r = upload(ct.data(), ct.size(), &dct))) return r;
        if ((r = upload(off.data(), off.size(), &doff))) return r;
    }
    cudaFree(pe->d_blocks32); cudaFree(pe->d_units32); cudaFree(pe->d_block_units32);
    cudaFree(pe->d_ctab32); cudaFree(pe->d_ctab_off32);
    pe->d_blocks32 = db; pe->d_units32 = du; pe->d_block_units32 = dbu;
    pe->d_ctab32 = dct; pe->d_ctab_off32 = doff;
    pe->kind32 = kind;
    pe->prog32 = np;
    pe->max_nc1_32 = 0;
    for (int k = 0; k < np.nblock; ++k) pe->max_nc1_32 = std::max(pe->max_nc1_32, np.blocks[k].nc[np.blocks[k].dir[0]]);
    return DPG_OK;
}

int get_program(DeviceState *ds, int space, int q, int L, int p, int split, const HostTables &tab, ProgEntry **out) {
    ProgKey key{ space, q, L, p, split };
    auto it = ds->progs.find(key);
    if (it != ds->progs.end()) { *out = it->second.get(); return DPG_OK; }
    auto pe = std::make_unique<ProgEntry>();
    pe->prog = make_program(space, q, L, p, split != 0, tab);
    const Program &pr = pe->prog;
    if (pr.smem_values * sizeof(double) > (size_t)g_max_dyn_smem) return DPG_ERR_RANGE;
    int r;
    if ((r = upload(pr.blocks, (size_t)pr.nblock, &pe->d_blocks))) return r;
    if ((r = upload(pr.units.data(), pr.units.size(), &pe->d_units))) return r;
    for (int prec = 0; prec < 2; ++prec) {
        AffProg &ap = pe->aff[prec];
        ap.prog = make_program(space, q, L, p, split != 0, tab, ORDER_NATURAL, 0, prec == 0 ? 72 * 1024 : 0);
        const Program &pa = ap.prog;
        if ((r = upload(pa.blocks, (size_t)pa.nblock, &ap.d_blocks))) return r;
        if ((r = upload(pa.units.data(), pa.units.size(), &ap.d_units))) return r;
        size_t m = 0;
        for (int k = 0; k < pa.nblock; ++k) m = std::max(m, affine_smem_values(pa.blocks[k], pa.nj));
        if ((r = upload_aff_image(ap, tab, false, prec))) return r;
        {
            std::vector<unsigned> ql;
            std::vector<int> qo;
            if (!build_aff_qlists(pa, tab, ql, qo)) return DPG_ERR_RANGE;
            if ((r = upload(ql.data(), ql.size(), &ap.d_qlist))) return r;
            if ((r = upload(qo.data(), qo.size(), &ap.d_qoff))) return r;
        }
        std::vector<int> ub(pa.nblock + 1, 0);
        for (const Unit &u : pa.units) ub[u.block + 1]++;
        for (int k = 0; k < pa.nblock; ++k) ub[k + 1] += ub[k];
        if ((r = upload(ub.data(), ub.size(), &ap.d_block_units))) return r;
        if (m * (prec ? sizeof(float) : sizeof(double)) > (size_t)g_max_dyn_smem) return DPG_ERR_RANGE;
        ap.smem_values = m;
        // a matrix diagonal for every element (the L2 Gram matrix, Eq. 2.95) is written by a
        // fill kernel from the products of the diagonal 1D integrals
        std::vector<double> D;
        ap.diag = affine_diagonal(pa, tab, AFF_DIAG_MAXT, D);
        if (ap.diag) {
            const BlockDesc &b0 = pa.blocks[0];
            for (int t = 0; t < b0.nterm; ++t) {
                ap.diag_field[t] = b0.term[t].field;
                ap.diag_sign[t] = b0.term[t].sign;
            }
            ap.diag_nterm = b0.nterm;
            if ((r = upload(D.data(), D.size(), &ap.d_diag))) return r;
        }
    }
    pe->flops_aff = pe->aff[0].prog.flops_affine;
    for (int prec = 0; prec < 2; ++prec) {
        AffProg &ap = pe->ext[prec];
        const size_t esz = prec ? sizeof(float) : sizeof(double);
        // the largest chunk whose shared memory fits three CTAs per SM, else the largest that fits
        size_t budget = (size_t)72 * 1024 * sizeof(double) / esz;
        ap.prog = make_program(space, q, L, p, split != 0, tab, ORDER_EXTRUDED, 0, budget);
        if (ap.prog.smem_bytes > budget)
            ap.prog = make_program(space, q, L, p, split != 0, tab, ORDER_EXTRUDED, 0,
                                   (size_t)g_max_dyn_smem * sizeof(double) / esz);
        const Program &pa = ap.prog;
        if ((r = upload(pa.blocks, (size_t)pa.nblock, &ap.d_blocks))) return r;
        if ((r = upload(pa.units.data(), pa.units.size(), &ap.d_units))) return r;
        size_t m = 0;
        for (int k = 0; k < pa.nblock; ++k) m = std::max(m, extruded_smem_values(pa.blocks[k], L, pa.nj));
        if ((r = upload_aff_image(ap, tab, true, prec))) return r;
        std::vector<int> ub(pa.nblock + 1, 0);
        for (const Unit &u : pa.units) ub[u.block + 1]++;
        for (int k = 0; k < pa.nblock; ++k) ub[k + 1] += ub[k];
        if ((r = upload(ub.data(), ub.size(), &ap.d_block_units))) return r;
        if (m * esz > (size_t)g_max_dyn_smem) return DPG_ERR_RANGE;
        ap.smem_values = m;
    }
    pe->flops_ext = pe->ext[0].prog.flops_extruded;
    if ((r = setup_tcc(pe.get(), space, q, L, p, split != 0, tab))) return r;
    if ((r = setup_prog32(pe.get(), space, q, L, p, split != 0, tab, 0))) return r;
    *out = pe.get();
    ds->progs[key] = std::move(pe);
    return DPG_OK;
}

// Make (space, q) with its active program the hp entry of that q, for both precisions.
int update_hp_table(DeviceState *ds, int space, int q, ProgEntry *pe, TableEntry *te) {
    if (space < S_H1 || space > S_L2) return DPG_OK;
    const Program &pr = pe->prog;
    for (int prec = 0; prec < 2; ++prec) {
        HpProg g;
        g.blocks = pe->d_blocks; g.units = pe->d_units;
        g.pp = prec ? (const void *)te->pp32 : (const void *)te->pp64;
        g.zeta = te->zeta; g.w = te->w;
        g.nunits = (int)pr.units.size(); g.L = pr.L; g.nfields = pr.nfields; g.cols = pr.cols; g.valid = 1;
        ds->h_hp[prec][space][q] = g;
        if (!ds->d_hp[prec][space]) CK(cudaMalloc(&ds->d_hp[prec][space], sizeof(HpProg) * (MAXQ + 1)));
        CK(cudaMemcpy(ds->d_hp[prec][space], ds->h_hp[prec][space], sizeof(HpProg) * (MAXQ + 1), cudaMemcpyHostToDevice));
    }
    // maxima over the initialised orders of this space
    size_t sm64 = 0, sm32 = 0;
    int mu = 0;
    int64_t mf = 0;
    for (int qq = 1; qq <= MAXQ; ++qq) {
        if (!ds->h_hp[0][space][qq].valid) continue;
        auto it = ds->active_L.find(std::make_pair(space, qq));
        const int L = (qq == q) ? pr.L : (it == ds->active_L.end() ? 0 : it->second);
        auto pt = ds->progs.find(ProgKey{ space, qq, L, 0, 0 });
        const Program &pp = (qq == q || pt == ds->progs.end()) ? pr : pt->second->prog;
        sm64 = std::max(sm64, pp.smem_values * sizeof(double));
        sm32 = std::max(sm32, pp.smem_values * sizeof(float));
        mu = std::max(mu, (int)pp.units.size());
        mf = std::max<int64_t>(mf, (int64_t)pp.nfields * pp.L * pp.L * pp.L);
    }
    ds->hp_smem[0][space] = sm64; ds->hp_smem[1][space] = sm32;
    ds->hp_max_units[space] = mu; ds->hp_max_fields[space] = mf;
    for (auto &kv : ds->hp_graphs) cudaGraphExecDestroy(kv.second);   // launches bake smem sizes in
    ds->hp_graphs.clear();
    return DPG_OK;
}

void free_device_state(DeviceState &ds) {
    for (auto &kv : ds.tables) {
        TableEntry &t = *kv.second;
        cudaFree(t.zeta); cudaFree(t.w); cudaFree(t.pp64); cudaFree(t.pp32); cudaFree(t.F64); cudaFree(t.F32);
    }
    for (auto &kv : ds.progs) {
        cudaFree(kv.second->d_blocks); cudaFree(kv.second->d_units);
        for (AffProg *aps : { kv.second->aff, kv.second->ext })
            for (int i = 0; i < 2; ++i) {
                AffProg &ap = aps[i];
                cudaFree(ap.d_blocks); cudaFree(ap.d_units); cudaFree(ap.d_block_units);
                cudaFree(ap.d_img); cudaFree(ap.d_img_off); cudaFree(ap.d_diag);
                cudaFree(ap.d_qlist); cudaFree(ap.d_qoff);
            }
        cudaFree(kv.second->d_blocks32); cudaFree(kv.second->d_units32); cudaFree(kv.second->d_block_units32);
        cudaFree(kv.second->d_ctab32); cudaFree(kv.second->d_ctab_off32);
        cudaFree(kv.second->tcc.d_blocks); cudaFree(kv.second->tcc.d_img); cudaFree(kv.second->tcc.d_off);
        cudaFree(kv.second->tcc.d_base);
    }
    for (auto &kv : ds.hp_graphs) cudaGraphExecDestroy(kv.second);
    ds.hp_graphs.clear();
    for (int pr = 0; pr < 2; ++pr)
        for (int sp = 0; sp < 6; ++sp) {
            cudaFree(ds.d_hp[pr][sp]);
            ds.d_hp[pr][sp] = nullptr;
            for (int q = 0; q <= MAXQ; ++q) ds.h_hp[pr][sp][q] = HpProg{};
            ds.hp_smem[pr][sp] = 0;
        }
    for (int sp = 0; sp < 6; ++sp) { ds.hp_max_units[sp] = 0; ds.hp_max_fields[sp] = 0; }
    ds.tables.clear(); ds.progs.clear(); ds.active_L.clear();
}

bool valid_space(int space) {
    const int base = space & 0xff;
    const int flags = space & ~0xff;
    if (base < S_H1 || base > S_AB) return false;
    if (flags & ~(DPG_FP32 | DPG_MAP_AFFINE | DPG_MAP_EXTRUDED | DPG_B_SPLIT | DPG_VEC3)) return false;
    if ((flags & DPG_VEC3) && base > S_L2) return false;
    if ((flags & DPG_MAP_AFFINE) && (flags & DPG_MAP_EXTRUDED)) return false;
    if ((flags & DPG_B_SPLIT) && base != S_B) return false;
    return true;
}

// Resolve the program of a call; fills *pe and *te.
int resolve(int space, int p_trial, int q, ProgEntry **pe, TableEntry **te, DeviceState **dso) {
    if (!valid_space(space)) return DPG_ERR_ARG;
    if (q < 1 || q > DPG_MAX_Q) return DPG_ERR_RANGE;
    const int base = space & 0xff;
    int p = 0, split = 0;
    if (base == S_B || base == S_AB) {
        if (p_trial < 1 || p_trial > q) return DPG_ERR_ARG;
        p = p_trial;
        split = (space & DPG_B_SPLIT) ? 1 : 0;
    }
    DeviceState *ds = nullptr;
    int r = device_state(&ds);
    if (r) return r;
    auto it = ds->active_L.find(std::make_pair(base, q));
    if (it == ds->active_L.end()) return DPG_ERR_NOT_INIT;
    const int L = it->second;
    auto tt = ds->tables.find(std::make_pair(q, L));
    if (tt == ds->tables.end()) return DPG_ERR_NOT_INIT;
    auto pt = ds->progs.find(ProgKey{ base, q, L, p, split });
    if (pt == ds->progs.end()) return DPG_ERR_NOT_INIT;
    *pe = pt->second.get();
    *te = tt->second.get();
    *dso = ds;
    return DPG_OK;
}

// Leading dimension and per-element stride of the output a call writes (the program's own,
// or those of the (0, 0) block of a DPG_VEC3 matrix).
struct OutGeom {
    int64_t ld, mat;
};

// Metric-field bytes per element of the general-path program of the form T.
template <typename T>
size_t general_field_bytes(const ProgEntry *pe) {
    const Program &pr = sizeof(T) == 4 ? pe->prog32 : pe->prog;
    return (size_t)pr.nfields * pr.L * pr.L * pr.L * sizeof(T);
}

// Elements per chunk of the general path: the workspace bound, the CTA-count bound of the
// FP64 grid (one CTA per element and unit) and n_elem.
template <typename T>
int64_t general_chunk(const ProgEntry *pe, int64_t n_elem, size_t ws_limit) {
    const Program &pr = sizeof(T) == 4 ? pe->prog32 : pe->prog;
    int64_t chunk = (int64_t)(ws_limit / general_field_bytes<T>(pe));
    if (chunk < 1) chunk = 1;
    const int64_t max_ctas = INT_MAX / (int64_t)pr.units.size();
    if (chunk > max_ctas) chunk = max_ctas;
    if (chunk > n_elem) chunk = n_elem;
    return chunk;
}

// The general path over n_elem elements in chunks of `chunk` elements, the metric fields
// of a chunk in ws (at least chunk * general_field_bytes<T> bytes, reused by every chunk:
// the launches are stream-ordered).
template <typename T>
int run_general_in(DeviceState *ds, ProgEntry *pe, TableEntry *te, int64_t n_elem, const double *verts,
                   const double *coeffs, T *out, cudaStream_t s, OutGeom og, int64_t base, void *ws,
                   int64_t chunk) {
    constexpr bool f32 = sizeof(T) == 4;
    const Program &pr = f32 ? pe->prog32 : pe->prog;
    const int L = pr.L;
    const int64_t mat = og.mat;
    int rc = DPG_OK;
    for (int64_t e0 = 0; e0 < n_elem && rc == DPG_OK; e0 += chunk) {
        const int64_t ne = std::min(chunk, n_elem - e0);
        GeomParams g;
        g.space = pr.space; g.L = L; g.nfields = pr.nfields;
        g.n_elem = ne; g.elem_base = base + e0;
        g.verts = verts + 24 * e0;
        g.coeffs = coeffs ? coeffs + 2 * e0 : nullptr;
        g.zeta = te->zeta; g.w = te->w;
        g.fields = ws; g.status = ds->status;
        cudaError_t le;
        {
            TraceRange tr("dpg geometry");
            le = launch_geom<T>(g, s);
        }
        if (le != cudaSuccess) { rc = cuda_fail(le, "geom_kernel launch", __LINE__); break; }
        if constexpr (f32) if (pe->kind32 == K32_TCC) {
            TccParams tp;
            tp.blocks = pe->tcc.d_blocks; tp.nblock = pr.nblock; tp.blk_base = pe->tcc.d_base;
            tp.img = pe->tcc.d_img; tp.img_off = pe->tcc.d_off;
            tp.L = L; tp.nfields = pr.nfields; tp.tcols = pe->tcc.tcols;
            tp.pp = te->pp32;
            tp.fields = reinterpret_cast<const float *>(ws); tp.foff = nullptr;
            tp.out = reinterpret_cast<float *>(out + e0 * mat); tp.out_off = nullptr;
            tp.mat_stride = mat; tp.ld = og.ld; tp.n_elem = ne;
            tp.n_elem_dev = nullptr; tp.elist = nullptr; tp.elist_start = nullptr;
            tp.status = ds->status; tp.smem_bytes = (int)pe->tcc.smem;
            tp.stall_cta = g_tc_stall_once ? 0 : -1;
            g_tc_stall_once = 0;
            {
                TraceRange tr("dpg contraction: general, FP32, stage C on tcgen05");
                le = launch_tcc(tp, g_num_sms * pe->tcc.cps, pe->tcc.smem, s);
            }
            if (le != cudaSuccess) { rc = cuda_fail(le, "contraction kernel launch", __LINE__); break; }
            continue;
        }
        if constexpr (f32) if (pe->kind32 == K32_TC) {
            TcParams tp;
            tp.blocks = pe->d_blocks32; tp.units = pe->d_units32; tp.block_unit_begin = pe->d_block_units32;
            tp.ctab = pe->d_ctab32; tp.ctab_off = pe->d_ctab_off32;
            tp.nblock = pr.nblock; tp.nj_max = pr.nj;
            // about four waves of one CTA per SM, each CTA a chunk of elements of one block
            const int64_t target = (int64_t)g_num_sms * 4;
            int64_t epc = (ne * pr.nblock + target - 1) / target;
            tp.elems_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(epc, 1 << 20));
            tp.L = L; tp.nfields = pr.nfields;
            tp.pp = te->pp32;
            tp.fields = reinterpret_cast<const float *>(ws);
            tp.out = reinterpret_cast<float *>(out + e0 * mat);
            tp.mat_stride = mat; tp.ld = og.ld; tp.n_elem = ne;
            tp.status = ds->status;
            tp.stall_cta = g_tc_stall_once ? 0 : -1;
            g_tc_stall_once = 0;
            {
                TraceRange tr("dpg contraction: general, FP32, tcgen05");
                le = launch_tc_f32(tp, pr.smem_bytes, s);
            }
            if (le != cudaSuccess) { rc = cuda_fail(le, "contraction kernel launch", __LINE__); break; }
            continue;
        }
        if constexpr (f32) if (pe->kind32 == K32_PANEL) {
            PanelParams pp;
            pp.blocks = pe->d_blocks32; pp.units = pe->d_units32; pp.block_unit_begin = pe->d_block_units32;
            pp.ctab = pe->d_ctab32; pp.ctab_off = pe->d_ctab_off32;
            pp.nblock = pr.nblock; pp.nj_max = pr.nj;
            // about four waves of two CTAs per SM, each CTA a chunk of elements of one block
            const int64_t target = (int64_t)g_num_sms * 2 * 4;
            int64_t epc = (ne * pr.nblock + target - 1) / target;
            pp.elems_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(epc, 1 << 20));
            pp.L = L; pp.nfields = pr.nfields;
            pp.pp = te->pp32;
            pp.fields = reinterpret_cast<const float *>(ws);
            pp.out = reinterpret_cast<float *>(out + e0 * mat);
            pp.mat_stride = mat; pp.ld = og.ld; pp.n_elem = ne; pp.status = ds->status;
            {
                TraceRange tr("dpg contraction: general, FP32, row panels");
                le = launch_panel_f32(pp, pr.smem_bytes, s);
            }
            if (le != cudaSuccess) { rc = cuda_fail(le, "contraction kernel launch", __LINE__); break; }
            continue;
        }
        if constexpr (f32) {
            SfParams32 sp;
            sp.blocks = pe->d_blocks32; sp.units = pe->d_units32; sp.block_unit_begin = pe->d_block_units32;
            sp.nblock = pr.nblock; sp.nj_max = pr.nj;
            // about four waves of two CTAs per SM, each CTA a chunk of elements of one block
            const int64_t target = (int64_t)g_num_sms * 2 * 4;
            int64_t epc = (ne * pr.nblock + target - 1) / target;
            sp.elems_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(epc, 1 << 20));
            sp.L = L; sp.nfields = pr.nfields;
            sp.pp = te->pp32;
            sp.fields = reinterpret_cast<const float *>(ws);
            sp.out = reinterpret_cast<float *>(out + e0 * mat);
            sp.mat_stride = mat; sp.ld = og.ld; sp.n_elem = ne; sp.status = ds->status;
            TraceRange tr("dpg contraction: general, FP32, mirrored tiles");
            le = launch_general_f32(sp, pr.smem_bytes, pe->max_nc1_32, s);
        } else {
            SfParams<T> sp;
            sp.blocks = pe->d_blocks; sp.units = pe->d_units;
            sp.nunits = (int)pr.units.size();
            sp.L = L; sp.nfields = pr.nfields;
            sp.pp = te->pp64;
            sp.fields = reinterpret_cast<const T *>(ws);
            sp.out = out + e0 * mat;
            sp.mat_stride = mat; sp.ld = og.ld; sp.n_elem = ne; sp.status = ds->status;
            TraceRange tr("dpg contraction: general, FP64");
            le = launch_general<T>(sp, pr.smem_values * sizeof(T), s);
        }
        if (le != cudaSuccess) { rc = cuda_fail(le, "contraction kernel launch", __LINE__); break; }
    }
    return rc;
}

// The general path with its workspace from the library pool (chunks of at most
// kWorkspaceLimit bytes of metric fields, or g_ws_limit_test when a test sets it).
template <typename T>
int run_general(DeviceState *ds, ProgEntry *pe, TableEntry *te, int64_t n_elem, const double *verts,
                const double *coeffs, T *out, cudaStream_t s, OutGeom og, int64_t base = 0) {
    const int64_t chunk = general_chunk<T>(pe, n_elem, g_ws_limit_test ? g_ws_limit_test : kWorkspaceLimit);
    void *ws = nullptr;
    CK(cudaMallocFromPoolAsync(&ws, (size_t)chunk * general_field_bytes<T>(pe), ds->pool, s));
    int rc = run_general_in<T>(ds, pe, te, n_elem, verts, coeffs, out, s, og, base, ws, chunk);
    cudaError_t fe = cudaFreeAsync(ws, s);
    if (fe != cudaSuccess && rc == DPG_OK) rc = cuda_fail(fe, "cudaFreeAsync", __LINE__);
    return rc;
}

// Elements per CTA of the affine / extruded kernels.  A CTA that would hold a single small
// work unit (the block split over several CTAs, under 8000 output values per unit) takes
// a chunk of up to four elements so that its block set-up is amortised, as long as about
// four waves of three CTAs per SM remain; otherwise one element (longer CTAs would only
// lengthen the tail).
int aff_elems_per_cta(const Program &pr, int64_t n_elem, int nsplit) {
    const double values_per_unit = (double)pr.parts * pr.rows * pr.cols / std::max<size_t>(pr.units.size(), 1);
    if (nsplit == 1 || values_per_unit >= 8000.0) return 1;
    const int64_t ctas_wanted = (int64_t)g_num_sms * 3 * 4;
    const int64_t work = n_elem * pr.nblock * nsplit;
    return (int)std::max<int64_t>(1, std::min<int64_t>(work / ctas_wanted, 4));
}

template <typename T>
int run_affine(DeviceState *ds, ProgEntry *pe, TableEntry *te, int64_t n_elem, const double *verts,
               const double *coeffs, T *out, cudaStream_t s, OutGeom og) {
    const AffProg &aprog = pe->aff[sizeof(T) == 4 ? 1 : 0];
    const Program &pr = aprog.prog;
    const int64_t mat = og.mat;
    // CTAs per (element, block): enough for about six waves of the SMs, at most one per unit
    int max_units_block = 1;
    for (int k = 0; k < pr.nblock; ++k) {
        int c = 0;
        for (const Unit &u : pr.units) c += u.block == k;
        max_units_block = std::max(max_units_block, c);
    }
    const int64_t target = (int64_t)g_num_sms * 6 * 4;
    const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(max_units_block,
                                              (target + n_elem * pr.nblock - 1) / (n_elem * pr.nblock)));
    // elements per CTA: about four waves of three CTAs per SM, the block set-up amortised
    const int epc = aff_elems_per_cta(pr, n_elem, nsplit);
    const int64_t per_launch = (int64_t)epc * (INT_MAX / ((int64_t)pr.nblock * nsplit));
    void *consts = nullptr;
    CK(cudaMallocFromPoolAsync(&consts, (size_t)n_elem * AFF_CONST_STRIDE * sizeof(double), ds->pool, s));
    AffConstParams cp;
    cp.space = pr.space; cp.n_elem = n_elem; cp.elem_base = 0;
    cp.verts = verts; cp.coeffs = coeffs; cp.consts = (double *)consts; cp.status = ds->status;
    int rc = DPG_OK;
    cudaError_t le;
    {
        TraceRange tr("dpg geometry: affine constants");
        le = launch_affine_const(cp, s);
    }
    if (le != cudaSuccess) rc = cuda_fail(le, "affine_const_kernel launch", __LINE__);
    // a matrix diagonal for every element (L2, by Eq. 2.95): one store-bound kernel, its zeros
    // written while the constants are computed
    const int64_t span = AFF_DIAG_SPAN_BYTES / (int64_t)sizeof(T), spans = (mat + span - 1) / span;
    const bool diag = aprog.diag && og.ld == pr.cols && mat == (int64_t)pr.rows * pr.cols &&
                      (span - 1) / (pr.rows + 1) + 1 <= AFF_DIAG_MAXR && n_elem * spans <= INT_MAX;
    if (diag && rc == DPG_OK) {
        AffDiagParams<T> dp;
        dp.n_elem = n_elem; dp.consts = (const double *)consts;
        dp.D = aprog.d_diag; dp.nterm = aprog.diag_nterm;
        for (int t = 0; t < AFF_DIAG_MAXT; ++t) { dp.field[t] = aprog.diag_field[t]; dp.sign[t] = aprog.diag_sign[t]; }
        dp.out = out; dp.n = pr.rows; dp.span = span;
        dp.spans = (int)spans; dp.status = ds->status;
        {
            TraceRange tr("dpg contraction: affine, diagonal matrix");
            le = launch_affine_diag<T>(dp, s);
        }
        if (le != cudaSuccess) rc = cuda_fail(le, "affine_diag_kernel launch", __LINE__);
    }
    for (int64_t e0 = 0; e0 < n_elem && rc == DPG_OK && !diag; e0 += per_launch) {
        const int64_t ne = std::min(per_launch, n_elem - e0);
        AffParams<T> ap;
        ap.blocks = aprog.d_blocks; ap.units = aprog.d_units; ap.block_unit_begin = aprog.d_block_units;
        ap.nblock = pr.nblock; ap.nj_max = pr.nj; ap.nsplit = nsplit; ap.elems_per_cta = epc;
        ap.img = aprog.d_img; ap.img_off16 = aprog.d_img_off; ap.qlist = aprog.d_qlist; ap.qoff = aprog.d_qoff;
        ap.xfields = nullptr; ap.estatus = nullptr; ap.pp = nullptr; ap.L = pr.L; ap.nfields = pr.nfields;
        if constexpr (sizeof(T) == 8) ap.F = te->F64; else ap.F = te->F32;
        ap.consts = (const double *)consts + AFF_CONST_STRIDE * e0;
        ap.out = out + e0 * mat;
        ap.mat_stride = mat; ap.ld = og.ld; ap.n_elem = ne; ap.status = ds->status;
        {
            TraceRange tr("dpg contraction: affine");
            le = launch_affine<T>(ap, aprog.smem_values * sizeof(T), s);
        }
        if (le != cudaSuccess) rc = cuda_fail(le, "sf_affine_kernel launch", __LINE__);
    }
    cudaError_t fe = cudaFreeAsync(consts, s);
    if (fe != cudaSuccess && rc == DPG_OK) rc = cuda_fail(fe, "cudaFreeAsync", __LINE__);
    return rc;
}

// Extruded maps (Eq. 2.89, right; Algorithm 11): 2D geometry and metric fields per element,
// then the extruded-mode contraction, chunked like the general path.
template <typename T>
int run_extruded(DeviceState *ds, ProgEntry *pe, TableEntry *te, int64_t n_elem, const double *verts,
                 const double *coeffs, T *out, cudaStream_t s, OutGeom og) {
    const AffProg &aprog = pe->ext[sizeof(T) == 4 ? 1 : 0];
    const Program &pr = aprog.prog;
    const int L = pr.L, L2 = L * L;
    const int64_t mat = og.mat;
    int max_units_block = 1;
    for (int k = 0; k < pr.nblock; ++k) {
        int c = 0;
        for (const Unit &u : pr.units) c += u.block == k;
        max_units_block = std::max(max_units_block, c);
    }
    const size_t per_elem = (size_t)pr.nfields * L2 * sizeof(T) + sizeof(int);
    const size_t ws_limit = g_ws_limit_test ? g_ws_limit_test : kWorkspaceLimit;
    int64_t chunk = std::max<int64_t>(1, (int64_t)(ws_limit / per_elem));
    const int64_t target = (int64_t)g_num_sms * 6 * 4;
    const int64_t ne_all = std::min(chunk, n_elem);
    const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(max_units_block,
                                              (target + ne_all * pr.nblock - 1) / (ne_all * pr.nblock)));
    const int epc = aff_elems_per_cta(pr, ne_all, nsplit);
    chunk = std::min<int64_t>(chunk, (int64_t)epc * (INT_MAX / ((int64_t)pr.nblock * nsplit)));
    if (chunk > n_elem) chunk = n_elem;
    void *ws = nullptr;
    CK(cudaMallocFromPoolAsync(&ws, (size_t)chunk * per_elem + 16, ds->pool, s));
    T *fields = reinterpret_cast<T *>(ws);
    int *est = reinterpret_cast<int *>(reinterpret_cast<char *>(ws) + (((size_t)chunk * pr.nfields * L2 * sizeof(T) + 15) & ~size_t(15)));
    int rc = DPG_OK;
    for (int64_t e0 = 0; e0 < n_elem && rc == DPG_OK; e0 += chunk) {
        const int64_t ne = std::min(chunk, n_elem - e0);
        cudaError_t le = cudaMemsetAsync(est, 0, (size_t)ne * sizeof(int), s);
        if (le != cudaSuccess) { rc = cuda_fail(le, "cudaMemsetAsync", __LINE__); break; }
        Geom2dParams g;
        g.space = pr.space; g.L = L; g.nfields = pr.nfields;
        g.n_elem = ne; g.elem_base = e0;
        g.verts = verts + 24 * e0;
        g.coeffs = coeffs ? coeffs + 2 * e0 : nullptr;
        g.zeta = te->zeta; g.w = te->w;
        g.fields = fields; g.estatus = est; g.status = ds->status;
        {
            TraceRange tr("dpg geometry: extruded");
            le = launch_geom2d<T>(g, s);
        }
        if (le != cudaSuccess) { rc = cuda_fail(le, "geom2d_kernel launch", __LINE__); break; }
        AffParams<T> ap;
        ap.blocks = aprog.d_blocks; ap.units = aprog.d_units; ap.block_unit_begin = aprog.d_block_units;
        ap.nblock = pr.nblock; ap.nj_max = pr.nj; ap.nsplit = nsplit; ap.elems_per_cta = epc;
        ap.img = aprog.d_img; ap.img_off16 = aprog.d_img_off; ap.qlist = nullptr; ap.qoff = nullptr;
        if constexpr (sizeof(T) == 8) { ap.F = te->F64; ap.pp = te->pp64; } else { ap.F = te->F32; ap.pp = te->pp32; }
        ap.consts = nullptr;
        ap.xfields = fields; ap.estatus = est;
        ap.L = L; ap.nfields = pr.nfields;
        ap.out = out + e0 * mat;
        ap.mat_stride = mat; ap.ld = og.ld; ap.n_elem = ne; ap.status = ds->status;
        {
            TraceRange tr("dpg contraction: extruded");
            le = launch_extruded<T>(ap, aprog.smem_values * sizeof(T), s);
        }
        if (le != cudaSuccess) { rc = cuda_fail(le, "extruded contraction launch", __LINE__); break; }
    }
    cudaError_t fe = cudaFreeAsync(ws, s);
    if (fe != cudaSuccess && rc == DPG_OK) rc = cuda_fail(fe, "cudaFreeAsync", __LINE__);
    return rc;
}

int integrate_locked(int space, int p_trial, int q_test, int64_t n_elem, const double *vertices,
                     const double *coeffs, void *out, cudaStream_t s) {
    ProgEntry *pe; TableEntry *te; DeviceState *ds;
    int r = resolve(space, p_trial, q_test, &pe, &te, &ds);
    if (r) return r;
    if (n_elem < 0) return DPG_ERR_ARG;
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !out) return DPG_ERR_ARG;
    const bool fp32 = (space & DPG_FP32) != 0, affine = (space & DPG_MAP_AFFINE) != 0;
    const bool use_coeffs = (space & 0xff) <= S_L2;            // Gram matrices only
    const double *c = use_coeffs ? coeffs : nullptr;
    const Program &pr = pe->prog;
    const bool vec3 = (space & DPG_VEC3) != 0;
    // DPG_VEC3: the scalar Gram matrix goes to the (0, 0) block of the [3n][3n] matrix,
    // then it is replicated on the diagonal (Eqs. 2.86, 2.88)
    const OutGeom og = vec3 ? OutGeom{ 3 * (int64_t)pr.cols, 9 * (int64_t)pr.rows * pr.cols }
                            : OutGeom{ pr.cols, (int64_t)pr.parts * pr.rows * pr.cols };
    if (affine)
        r = fp32 ? run_affine<float>(ds, pe, te, n_elem, vertices, c, (float *)out, s, og)
                 : run_affine<double>(ds, pe, te, n_elem, vertices, c, (double *)out, s, og);
    else if (space & DPG_MAP_EXTRUDED)
        r = fp32 ? run_extruded<float>(ds, pe, te, n_elem, vertices, c, (float *)out, s, og)
                 : run_extruded<double>(ds, pe, te, n_elem, vertices, c, (double *)out, s, og);
    else
        r = fp32 ? run_general<float>(ds, pe, te, n_elem, vertices, c, (float *)out, s, og)
                 : run_general<double>(ds, pe, te, n_elem, vertices, c, (double *)out, s, og);
    if (r == DPG_OK && vec3) {
        TraceRange tr("dpg vec3 replication");
        const cudaError_t le = fp32 ? launch_vec3_fill<float>((float *)out, n_elem, pr.rows, s)
                                    : launch_vec3_fill<double>((double *)out, n_elem, pr.rows, s);
        if (le != cudaSuccess) r = cuda_fail(le, "vec3_fill_kernel launch", __LINE__);
    }
    return r;
}

// The hp sequence (workspace, work generation, geometry, persistent contraction) on s.
int enqueue_hp(DeviceState *ds, int space, int64_t n, const double *verts, const double *coeffs,
               const int *q_elem, const int64_t *out_offset, void *out, cudaStream_t s) {
    const int base = space & 0xff;
    const bool fp32 = (space & DPG_FP32) != 0;
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    const int64_t nb = (n + 1023) / 1024;
    const int64_t max_items = n * (int64_t)ds->hp_max_units[base];
    const size_t small = 64 * sizeof(int) + 8 * sizeof(int64_t);
    HpParams p;
    p.space = base; p.n_elem = n; p.verts = verts; p.coeffs = coeffs; p.q_elem = q_elem;
    p.out_offset = out_offset; p.out = out; p.tab = ds->d_hp[fp32 ? 1 : 0][base]; p.status = ds->status;
    void *wsmall = nullptr, *word = nullptr, *wu = nullptr, *wf = nullptr, *wit = nullptr, *wtmp = nullptr, *wfield = nullptr;
    CK(cudaMallocFromPoolAsync(&wsmall, small, ds->pool, s));
    CK(cudaMallocFromPoolAsync(&word, n * sizeof(int), ds->pool, s));
    CK(cudaMallocFromPoolAsync(&wu, 2 * n * sizeof(int64_t), ds->pool, s));
    CK(cudaMallocFromPoolAsync(&wf, 2 * n * sizeof(int64_t), ds->pool, s));
    CK(cudaMallocFromPoolAsync(&wit, std::max<int64_t>(max_items, 1) * sizeof(int), ds->pool, s));
    CK(cudaMallocFromPoolAsync(&wtmp, std::max<int64_t>(nb, 1) * sizeof(int64_t), ds->pool, s));
    CK(cudaMallocFromPoolAsync(&wfield, (size_t)n * ds->hp_max_fields[base] * esz, ds->pool, s));
    int *si = (int *)wsmall;
    p.hist = si; p.bstart = si + 16; p.bfill = si + 32;
    p.counters = (int64_t *)(si + 64);
    p.order = (int *)word;
    p.ucnt = (int64_t *)wu; p.uoff = (int64_t *)wu + n;
    p.fcnt = (int64_t *)wf; p.foff = (int64_t *)wf + n;
    p.item_k = (int *)wit; p.scan_tmp = (int64_t *)wtmp; p.fields = wfield;
    const size_t smem = ds->hp_smem[fp32 ? 1 : 0][base];
    const int ctas = g_num_sms * hp_ctas_per_sm(fp32, smem);
    // FP32: when every initialised order has a program of a tcgen05 kernel, the contraction is
    // one launch per order of the kernel the order's program uses (the stage-C kernel, or the
    // stages-B-and-C kernel where the autotuner chose it), over the elements of the order from
    // the device-side sort; else the persistent kernel over every work item
    std::vector<std::pair<ProgEntry *, TableEntry *>> tcc(MAXQ + 1, { nullptr, nullptr });
    bool use_tcc = fp32;
    int nvalid = 0;
    for (int q = 1; q <= MAXQ && use_tcc; ++q) {
        if (!ds->h_hp[1][base][q].valid) continue;
        auto ai = ds->active_L.find(std::make_pair(base, q));
        if (ai == ds->active_L.end()) { use_tcc = false; break; }
        auto pt = ds->progs.find(ProgKey{ base, q, ai->second, 0, 0 });
        auto tt = ds->tables.find(std::make_pair(q, ai->second));
        if (pt == ds->progs.end() || tt == ds->tables.end() ||
            !(pt->second->tcc.ok || pt->second->kind32 == K32_TC)) { use_tcc = false; break; }
        tcc[q] = { pt->second.get(), tt->second.get() };
        ++nvalid;
    }
    int rc = DPG_OK;
    cudaError_t le;
    {
        TraceRange tr("dpg hp: work generation, geometry, persistent contraction");
        le = launch_hp(p, fp32, smem, ctas, s, !use_tcc);
    }
    for (int q = MAXQ; q >= 1 && use_tcc && le == cudaSuccess; --q) {
        if (!tcc[q].first) continue;
        ProgEntry *pq = tcc[q].first;
        if (pq->kind32 == K32_TC) {
            const Program &pr = pq->prog32;
            TcParams tp;
            tp.blocks = pq->d_blocks32; tp.units = pq->d_units32; tp.block_unit_begin = pq->d_block_units32;
            tp.ctab = pq->d_ctab32; tp.ctab_off = pq->d_ctab_off32;
            tp.nblock = pr.nblock; tp.nj_max = pr.nj;
            // about four waves of one CTA per SM for the order's share of the elements (its
            // count is known on the device only: the batch spread evenly over its orders)
            const int64_t nest = std::max<int64_t>(1, n / std::max(nvalid, 1));
            const int64_t target = (int64_t)g_num_sms * 4;
            const int64_t epc = (nest * pr.nblock + target - 1) / target;
            tp.elems_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(epc, 1 << 20));
            tp.L = pr.L; tp.nfields = pr.nfields;
            tp.pp = tcc[q].second->pp32;
            tp.fields = reinterpret_cast<const float *>(p.fields); tp.foff = p.foff;
            tp.out = reinterpret_cast<float *>(out); tp.out_off = out_offset;
            tp.mat_stride = (int64_t)pr.parts * pr.rows * pr.cols; tp.ld = pr.cols; tp.n_elem = n;
            tp.n_elem_dev = p.hist + q; tp.elist = p.order; tp.elist_start = p.bstart + q;
            tp.status = ds->status; tp.stall_cta = -1;
            TraceRange tr("dpg hp: contraction of one order, FP32, stages B and C on tcgen05");
            le = launch_tc_f32(tp, pr.smem_bytes, s);
            continue;
        }
        const TccProg &tg = pq->tcc;
        const Program &pr = tg.prog;
        TccParams tp;
        tp.blocks = tg.d_blocks; tp.nblock = pr.nblock; tp.blk_base = tg.d_base;
        tp.img = tg.d_img; tp.img_off = tg.d_off;
        tp.L = pr.L; tp.nfields = pr.nfields; tp.tcols = tg.tcols;
        tp.pp = tcc[q].second->pp32;
        tp.fields = reinterpret_cast<const float *>(p.fields); tp.foff = p.foff;
        tp.out = reinterpret_cast<float *>(out); tp.out_off = out_offset;
        tp.mat_stride = (int64_t)pr.parts * pr.rows * pr.cols; tp.ld = pr.cols; tp.n_elem = 0;
        tp.n_elem_dev = p.hist + q; tp.elist = p.order; tp.elist_start = p.bstart + q;
        tp.status = ds->status; tp.smem_bytes = (int)tg.smem; tp.stall_cta = -1;
        TraceRange tr("dpg hp: contraction of one order, FP32, stage C on tcgen05");
        le = launch_tcc(tp, g_num_sms * tg.cps, tg.smem, s);
    }
    if (le != cudaSuccess) rc = cuda_fail(le, "hp launch sequence", __LINE__);
    for (void *w : { wfield, wtmp, wit, wf, wu, word, wsmall }) cudaFreeAsync(w, s);
    return rc;
}

// Replace the general-path program of pe (FP32 kernel's or FP64 kernel's) by one built
// with stage-A chunk nj.  Synchronises the device (the old descriptors are freed).
int install_program(ProgEntry *pe, TableEntry *te, int space, int q, int L, bool fp32, int nj, int nj_sym = 0) {
    if (fp32) {
        CK(cudaDeviceSynchronize());
        return setup_prog32(pe, space, q, L, 0, false, te->host, nj);
    }
    Program np = make_program(space, q, L, 0, false, te->host, ORDER_BEST, nj, 0, nj_sym);
    if (np.smem_values * sizeof(double) > (size_t)g_max_dyn_smem) return DPG_ERR_RANGE;
    BlockDesc *db = nullptr;
    Unit *du = nullptr;
    int r;
    if ((r = upload(np.blocks, (size_t)np.nblock, &db))) return r;
    if ((r = upload(np.units.data(), np.units.size(), &du))) return r;
    CK(cudaDeviceSynchronize());
    cudaFree(pe->d_blocks); cudaFree(pe->d_units);
    pe->d_blocks = db; pe->d_units = du;
    pe->prog = np;
    return DPG_OK;
}

int read_status(DeviceState *ds, int64_t *first_bad) {
    DevStatus h;
    CK(cudaMemcpy(&h, ds->status, sizeof(h), cudaMemcpyDeviceToHost));
    DevStatus z;
    reset_host_status(z);
    CK(cudaMemcpy(ds->status, &z, sizeof(z), cudaMemcpyHostToDevice));
    if (first_bad) *first_bad = -1;
    if (h.code != 0) {
        if (first_bad && h.code > 0 && h.code < 16 && h.first_bad[h.code] != ULLONG_MAX)
            *first_bad = (int64_t)h.first_bad[h.code];
        return h.code;
    }
    return DPG_OK;
}

}  // namespace

int dpg::integrate_in_scratch(int space, int p_trial, int q_test, int64_t n_elem, const double *vertices,
                              const double *coeffs, void *out, void *scratch, size_t scratch_bytes, void *stream) {
    if (space & (DPG_MAP_AFFINE | DPG_MAP_EXTRUDED | DPG_VEC3)) return DPG_ERR_ARG;
    if (!valid_space(space)) return DPG_ERR_ARG;
    if (q_test < 1 || q_test > DPG_MAX_Q) return DPG_ERR_RANGE;
    const int base = space & 0xff;
    int p = 0, split = 0;
    if (base == S_B || base == S_AB) {
        if (p_trial < 1 || p_trial > q_test) return DPG_ERR_ARG;
        p = p_trial;
        split = (space & DPG_B_SPLIT) ? 1 : 0;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // the lock is held from the look-up to the last launch, so that no dpg_tables_init,
    // dpg_tables_free or dpg_autotune on another thread replaces the program meanwhile;
    // only existing state is looked up (nothing is created, nothing allocated)
    std::lock_guard<std::mutex> lk(g_mu);
    auto di = g_dev.find(dev);
    if (di == g_dev.end()) return DPG_ERR_NOT_INIT;
    DeviceState *ds = di->second.get();
    auto it = ds->active_L.find(std::make_pair(base, q_test));
    if (it == ds->active_L.end()) return DPG_ERR_NOT_INIT;
    const int L = it->second;
    auto tt = ds->tables.find(std::make_pair(q_test, L));
    auto pt = ds->progs.find(ProgKey{ base, q_test, L, p, split });
    if (tt == ds->tables.end() || pt == ds->progs.end()) return DPG_ERR_NOT_INIT;
    ProgEntry *pe = pt->second.get();
    TableEntry *te = tt->second.get();
    if (n_elem < 0) return DPG_ERR_ARG;
    const bool fp32 = (space & DPG_FP32) != 0;
    // the whole call in one chunk: its metric fields must fit the scratch, and the FP64
    // grid (one CTA per element and unit) must stay below 2^31 CTAs
    const size_t per_elem = fp32 ? general_field_bytes<float>(pe) : general_field_bytes<double>(pe);
    const Program &pr = fp32 ? pe->prog32 : pe->prog;
    if ((size_t)n_elem > scratch_bytes / per_elem) return DPG_ERR_SCRATCH;
    if ((int64_t)pr.units.size() * n_elem > INT_MAX) return DPG_ERR_SCRATCH;
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !out || !scratch) return DPG_ERR_ARG;
    const double *c = base <= S_L2 ? coeffs : nullptr;                 // Gram matrices only
    const OutGeom og{ pe->prog.cols, (int64_t)pe->prog.parts * pe->prog.rows * pe->prog.cols };
    cudaStream_t s = (cudaStream_t)stream;
    return fp32 ? run_general_in<float>(ds, pe, te, n_elem, vertices, c, (float *)out, s, og, 0, scratch, n_elem)
                : run_general_in<double>(ds, pe, te, n_elem, vertices, c, (double *)out, s, og, 0, scratch, n_elem);
}

extern "C" {

int dpg_tables_init_L(int q, int L, int space) {
    const int base = space & 0xff;
    if (base < S_H1 || base > S_AB) return DPG_ERR_ARG;
    if (q < 1 || q > DPG_MAX_Q || L < 1 || L > DPG_MAX_L) return DPG_ERR_RANGE;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *ds = nullptr;
    int r = device_state(&ds);
    if (r) return r;
    TableEntry *te = nullptr;
    if ((r = get_tables(ds, q, L, &te))) return r;
    ProgEntry *pe = nullptr;
    if (base == S_B || base == S_AB) {
        for (int p = 1; p <= q; ++p)
            for (int split = 0; split < (base == S_B ? 2 : 1); ++split)
                if ((r = get_program(ds, base, q, L, p, split, te->host, &pe))) return r;
    } else {
        if ((r = get_program(ds, base, q, L, 0, 0, te->host, &pe))) return r;
    }
    ds->active_L[std::make_pair(base, q)] = L;
    if (base <= S_L2 && (r = update_hp_table(ds, base, q, pe, te))) return r;
    return DPG_OK;
}

int dpg_tables_init(int q, int space) { return dpg_tables_init_L(q, q + 2 > DPG_MAX_L ? DPG_MAX_L : q + 2, space); }

int dpg_tables_free(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_dev) {
        cudaSetDevice(kv.first);
        free_device_state(*kv.second);
    }
    cudaSetDevice(cur);
    return DPG_OK;
}

int64_t dpg_matrix_rows(int space, int q) {
    const int64_t r = rows_of(space & 0xff, q);
    return (r > 0 && (space & DPG_VEC3)) ? 3 * r : r;
}

int64_t dpg_matrix_cols(int space, int p_trial, int q) {
    const int base = space & 0xff;
    if (rows_of(base, q) < 0) return -1;
    const int64_t c = cols_of(base, p_trial, q);
    return (c > 0 && (space & DPG_VEC3)) ? 3 * c : c;
}

int dpg_integrate(int space, int p_trial, int q_test, int64_t n_elem, const double *vertices,
                  const double *coeffs, void *out, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    return integrate_locked(space, p_trial, q_test, n_elem, vertices, coeffs, out, (cudaStream_t)stream);
}

int dpg_integrate_hp(int space, int64_t n_elem, const double *vertices, const double *coeffs,
                     const int *q_elem, const int64_t *out_offset, void *out, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int base = space & 0xff;
    if (base < S_H1 || base > S_L2 || (space & ~(0xff | DPG_FP32))) return DPG_ERR_ARG;
    if (n_elem < 0) return DPG_ERR_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    auto di = g_dev.find(dev);
    if (di == g_dev.end() || di->second->hp_max_units[base] == 0) return DPG_ERR_NOT_INIT;
    DeviceState *ds = di->second.get();
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !q_elem || !out_offset || !out) return DPG_ERR_ARG;
    if (n_elem > INT_MAX) return DPG_ERR_RANGE;
    cudaStream_t s = (cudaStream_t)stream;
    HpKey key{ space, n_elem, vertices, coeffs, q_elem, out_offset, out };
    auto it = ds->hp_graphs.find(key);
    if (it == ds->hp_graphs.end()) {
        // capture the whole sequence once on the library's capture stream
        CK(cudaStreamBeginCapture(ds->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int r = enqueue_hp(ds, space, n_elem, vertices, coeffs, q_elem, out_offset, out, ds->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(ds->cap_stream, &graph);
        if (r != DPG_OK) { if (graph) cudaGraphDestroy(graph); return r; }
        if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture", __LINE__);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate", __LINE__);
        it = ds->hp_graphs.emplace(key, exec).first;
    }
    CK(cudaGraphLaunch(it->second, s));
    return DPG_OK;
}

int dpg_integrate_host(int space, int p_trial, int q_test, int64_t n_elem, const double *vertices,
                       const double *coeffs, void *out, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    ProgEntry *pe; TableEntry *te; DeviceState *ds;
    int r = resolve(space, p_trial, q_test, &pe, &te, &ds);
    if (r) return r;
    if (n_elem < 0) return DPG_ERR_ARG;
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !out) return DPG_ERR_ARG;
    const Program &pr = pe->prog;
    const size_t esz = (space & DPG_FP32) ? sizeof(float) : sizeof(double);
    const size_t per_out = (size_t)pr.parts * pr.rows * pr.cols * esz * ((space & DPG_VEC3) ? 9 : 1);
    const size_t out_bytes = (size_t)n_elem * per_out;
    const size_t v_bytes = (size_t)n_elem * 24 * sizeof(double);
    const size_t c_bytes = coeffs ? (size_t)n_elem * 2 * sizeof(double) : 0;
    void *dv = nullptr, *dc = nullptr, *dout = nullptr;
    CK(cudaMallocFromPoolAsync(&dv, v_bytes, ds->pool, s));
    if (c_bytes) CK(cudaMallocFromPoolAsync(&dc, c_bytes, ds->pool, s));
    CK(cudaMallocFromPoolAsync(&dout, out_bytes, ds->pool, s));
    {
        TraceRange tr("dpg host-to-device inputs");
        CK(cudaMemcpyAsync(dv, vertices, v_bytes, cudaMemcpyHostToDevice, s));
        if (c_bytes) CK(cudaMemcpyAsync(dc, coeffs, c_bytes, cudaMemcpyHostToDevice, s));
    }
    // stream the batch: chunk k is integrated on `s` while earlier chunks drain to the
    // host on the copy streams (about 64 MB per chunk, at most 64 chunks)
    const int64_t by_bytes = (int64_t)((out_bytes + (size_t(64) << 20) - 1) / (size_t(64) << 20));
    const int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>({ n_elem, by_bytes, 64 }));
    const int64_t per = (n_elem + nchunk - 1) / nchunk;
    std::vector<cudaEvent_t> evs;
    for (int64_t e0 = 0, c = 0; e0 < n_elem && r == DPG_OK; e0 += per, ++c) {
        const int64_t ne = std::min(per, n_elem - e0);
        r = integrate_locked(space, p_trial, q_test, ne, (const double *)dv + 24 * e0,
                             dc ? (const double *)dc + 2 * e0 : nullptr, (char *)dout + e0 * per_out, s);
        if (r) break;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        evs.push_back(ev);
        CK(cudaEventRecord(ev, s));
        cudaStream_t cs = ds->copy_streams[c % 4];
        TraceRange tr("dpg device-to-host chunk");
        CK(cudaStreamWaitEvent(cs, ev, 0));
        CK(cudaMemcpyAsync((char *)out + e0 * per_out, (char *)dout + e0 * per_out, ne * per_out,
                           cudaMemcpyDeviceToHost, cs));
    }
    // join the copy streams back into `s` before the buffers are released
    for (auto cs : ds->copy_streams) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        evs.push_back(ev);
        CK(cudaEventRecord(ev, cs));
        CK(cudaStreamWaitEvent(s, ev, 0));
    }
    cudaFreeAsync(dv, s);
    if (dc) cudaFreeAsync(dc, s);
    cudaFreeAsync(dout, s);
    CK(cudaStreamSynchronize(s));
    for (auto ev : evs) cudaEventDestroy(ev);
    if (r) return r;
    return read_status(ds, nullptr);
}

int dpg_integrate_load(int space, int q_test, int64_t n_elem, const double *vertices,
                       const double *src_coef, int64_t coef_stride, void *out, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int base = space & 0xff;
    if (base < S_H1 || base > S_L2 || (space & ~(0xff | DPG_FP32))) return DPG_ERR_ARG;
    ProgEntry *pe; TableEntry *te; DeviceState *ds;
    int r = resolve(base, 0, q_test, &pe, &te, &ds);
    if (r) return r;
    const int nc = (base == S_HCURL || base == S_HDIV) ? 3 : 1;
    if (n_elem < 0 || (coef_stride != 0 && coef_stride < 10 * nc)) return DPG_ERR_ARG;
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !src_coef || !out) return DPG_ERR_ARG;
    LoadParams p;
    p.space = base; p.q = q_test; p.L = te->host.L;
    p.n_elem = n_elem; p.elem_base = 0;
    p.verts = vertices; p.coef = src_coef; p.coef_stride = coef_stride;
    p.zeta = te->zeta; p.w = te->w;
    p.out = out; p.status = ds->status;
    cudaError_t le;
    TraceRange tr("dpg load vector");
    if (space & DPG_FP32) { p.pp = te->pp32; le = launch_load<float>(p, g_num_sms, (cudaStream_t)stream); }
    else { p.pp = te->pp64; le = launch_load<double>(p, g_num_sms, (cudaStream_t)stream); }
    if (le != cudaSuccess) return cuda_fail(le, "load_kernel launch", __LINE__);
    return DPG_OK;
}

// CTAs per SM of the condensation kernel of the current method (chunk sizes are whole waves)
int condense_wave_per_sm() {
    if (g_condense_method == DPG_CONDENSE_TCGEN05) return 1;
    return condense_ctas_per_sm(g_condense_method == DPG_CONDENSE_TC);
}

// The condensation of p.n_elem elements with the current method; the tcgen05 kernel's digit
// scratch (about 1 MB per SM at n = 882) comes from the pool, stream-ordered.
int run_condense(DeviceState *ds, const CondParams &p, cudaStream_t s) {
    TraceRange tr(g_condense_method == DPG_CONDENSE_TCGEN05 ? "dpg condensation (tcgen05)" : "dpg condensation");
    if (g_condense_method != DPG_CONDENSE_TCGEN05) {
        const cudaError_t le = launch_condense(p, g_num_sms, g_condense_method == DPG_CONDENSE_TC, s);
        if (le != cudaSuccess) return cuda_fail(le, "condense_kernel launch", __LINE__);
        return DPG_OK;
    }
    Cond5Params q;
    q.n_elem = p.n_elem; q.elem_base = p.elem_base; q.n = p.n; q.m = p.m;
    q.G = p.G; q.B = p.B; q.l = p.l; q.K = p.K; q.F = p.F; q.status = p.status;
    q.stall_cta = g_tc_stall_once ? 0 : -1;
    g_tc_stall_once = 0;
    q.scratch_per_cta = condense5_scratch_per_cta(p.n, p.m, p.l != nullptr, &q.lrows, &q.wrows);
    const int grid = (int)std::min<int64_t>(p.n_elem, g_num_sms);
    void *scr = nullptr;
    CK(cudaMallocFromPoolAsync(&scr, (size_t)grid * q.scratch_per_cta, ds->pool, s));
    q.scratch = static_cast<unsigned char *>(scr);
    cudaError_t le = cudaMemsetAsync(scr, 0, (size_t)grid * q.scratch_per_cta, s);
    if (le == cudaSuccess) le = launch_condense5(q, grid, s);
    const cudaError_t fe = cudaFreeAsync(scr, s);
    if (le != cudaSuccess) return cuda_fail(le, "condense5_kernel launch", __LINE__);
    if (fe != cudaSuccess) return cuda_fail(fe, "cudaFreeAsync", __LINE__);
    return DPG_OK;
}

int dpg_condense(int64_t n_elem, int n, int m, double *G, double *B, double *l, double *K, double *F,
                 void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (n_elem < 0) return DPG_ERR_ARG;
    if (n < 1 || n > 8192 || m < 1 || m > 8192) return DPG_ERR_RANGE;
    if ((l == nullptr) != (F == nullptr)) return DPG_ERR_ARG;
    if (n_elem == 0) return DPG_OK;
    if (!G || !B || !K) return DPG_ERR_ARG;
    DeviceState *ds = nullptr;
    int r = device_state(&ds);
    if (r) return r;
    CondParams p;
    p.n_elem = n_elem; p.elem_base = 0; p.n = n; p.m = m;
    p.G = G; p.B = B; p.l = l; p.K = K; p.F = F;
    p.status = ds->status;
    return run_condense(ds, p, (cudaStream_t)stream);
}

int dpg_condensed_system(int q_test, int p_trial, int64_t n_elem, const double *vertices,
                         const double *coeffs, const double *src_coef, int64_t coef_stride, double *K,
                         double *F, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    const cudaStream_t s = (cudaStream_t)stream;
    if (n_elem < 0 || (coef_stride != 0 && coef_stride < 30)) return DPG_ERR_ARG;
    if ((src_coef == nullptr) != (F == nullptr)) return DPG_ERR_ARG;
    ProgEntry *pg, *pb; TableEntry *tg, *tb; DeviceState *ds;
    int r = resolve(S_HCURL, 0, q_test, &pg, &tg, &ds);
    if (r) return r;
    if ((r = resolve(S_B, p_trial, q_test, &pb, &tb, &ds))) return r;
    if (tg != tb) return DPG_ERR_NOT_INIT;          // G and B must use the same rule
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !K) return DPG_ERR_ARG;
    const int n = pg->prog.rows, m = pb->prog.cols;
    const bool with_l = src_coef != nullptr;
    // per element: G, B and l in a pool workspace; chunks of whole waves of the
    // condensation kernel within about 8 GB, so that only the last chunk has a partial wave
    const size_t per_elem = ((size_t)n * n + (size_t)n * m + (with_l ? n : 0)) * sizeof(double);
    int64_t chunk = (int64_t)((size_t(8) << 30) / per_elem);
    const int64_t wave = (int64_t)condense_wave_per_sm() * g_num_sms;
    if (chunk >= wave) chunk -= chunk % wave;
    if (chunk < 1) chunk = 1;
    if (chunk > n_elem) chunk = n_elem;
    void *ws = nullptr;
    CK(cudaMallocFromPoolAsync(&ws, (size_t)chunk * per_elem, ds->pool, s));
    double *G = static_cast<double *>(ws);
    double *B = G + (size_t)chunk * n * n;
    double *l = with_l ? B + (size_t)chunk * n * m : nullptr;
    int rc = DPG_OK;
    for (int64_t e0 = 0; e0 < n_elem && rc == DPG_OK; e0 += chunk) {
        const int64_t ne = n_elem - e0 < chunk ? n_elem - e0 : chunk;
        const double *v = vertices + 24 * e0;
        rc = run_general<double>(ds, pg, tg, ne, v, coeffs ? coeffs + 2 * e0 : nullptr, G, s,
                                 OutGeom{ n, (int64_t)n * n }, e0);
        if (rc) break;
        rc = run_general<double>(ds, pb, tb, ne, v, nullptr, B, s, OutGeom{ m, (int64_t)n * m }, e0);
        if (rc) break;
        if (with_l) {
            LoadParams lp;
            lp.space = S_HCURL; lp.q = q_test; lp.L = tg->host.L;
            lp.n_elem = ne; lp.elem_base = e0;
            lp.verts = v; lp.coef = coef_stride ? src_coef + e0 * coef_stride : src_coef;
            lp.coef_stride = coef_stride;
            lp.zeta = tg->zeta; lp.w = tg->w; lp.pp = tg->pp64;
            lp.out = l; lp.status = ds->status;
            TraceRange tr("dpg load vector");
            const cudaError_t le = launch_load<double>(lp, g_num_sms, s);
            if (le != cudaSuccess) { rc = cuda_fail(le, "load_kernel launch", __LINE__); break; }
        }
        CondParams cp;
        cp.n_elem = ne; cp.elem_base = e0; cp.n = n; cp.m = m;
        cp.G = G; cp.B = B; cp.l = l;
        cp.K = K + (size_t)e0 * m * m; cp.F = with_l ? F + (size_t)e0 * m : nullptr;
        cp.status = ds->status;
        rc = run_condense(ds, cp, s);
    }
    const cudaError_t fe = cudaFreeAsync(ws, s);
    if (fe != cudaSuccess && rc == DPG_OK) rc = cuda_fail(fe, "cudaFreeAsync", __LINE__);
    return rc;
}

int dpg_condense_set_method(int method) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (method != DPG_CONDENSE_FMA && method != DPG_CONDENSE_TC && method != DPG_CONDENSE_TCGEN05) return DPG_ERR_ARG;
    g_condense_method = method;
    return DPG_OK;
}

int dpg_test_stall_tc_once(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tc_stall_once = 1;
    return DPG_OK;
}

int dpg_test_set_workspace_limit(int64_t bytes) {
    if (bytes < 0) return DPG_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_ws_limit_test = (size_t)bytes;
    return DPG_OK;
}

int dpg_sync_status(void *stream, int64_t *first_bad_elem) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (first_bad_elem) *first_bad_elem = -1;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    DeviceState *ds = nullptr;
    int r = device_state(&ds);
    if (r) return r;
    return read_status(ds, first_bad_elem);
}

const char *dpg_last_cuda_error(void) { return g_last_error; }

int dpg_autotune(int q, int space, void *stream, int *best_nj) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int base = space & 0xff;
    const bool fp32 = (space & DPG_FP32) != 0;
    if (base < S_H1 || base > S_L2 || (space & ~(0xff | DPG_FP32))) return DPG_ERR_ARG;
    ProgEntry *pe; TableEntry *te; DeviceState *ds;
    int r = resolve(space & ~DPG_FP32, 0, q, &pe, &te, &ds);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = pe->prog.L;
    const char *cache = std::getenv("DPG_AUTOTUNE_CACHE");
    // cached choice
    if (cache) {
        if (FILE *f = std::fopen(cache, "r")) {
            char line[256];
            int found = -1, found_sym = 0;
            while (std::fgets(line, sizeof(line), f)) {
                int cs, cq, cl, cf, cn, cy = 0;
                double cms;
                // {"space", "q", "L", "fp32", "nj", "ms"} and, in newer lines, "nj_sym"
                const int got = std::sscanf(line,
                    "{\"space\": %d, \"q\": %d, \"L\": %d, \"fp32\": %d, \"nj\": %d, \"ms\": %lf, \"nj_sym\": %d}",
                    &cs, &cq, &cl, &cf, &cn, &cms, &cy);
                if (got >= 6 && cs == base && cq == q && cl == L && cf == (int)fp32) {
                    found = cn;
                    found_sym = got == 7 ? cy : 0;
                }
            }
            std::fclose(f);
            if ((found > 0 || (fp32 && found == 0 && pe->tcc.ok)) &&
                install_program(pe, te, base, q, L, fp32, found, found_sym) == DPG_OK) {
                if ((r = update_hp_table(ds, base, q, pe, te))) return r;
                if (best_nj) *best_nj = found;
                return DPG_OK;
            }
        }
    }
    // synthetic batch: unit cubes (timing does not depend on the geometry values); up to
    // 512 elements, fewer where their output would pass 2 GB (at least 8)
    const Program &pz = (space & DPG_FP32) ? pe->prog32 : pe->prog;
    const size_t out_elem = (size_t)pz.parts * pz.rows * pz.cols * ((space & DPG_FP32) ? sizeof(float) : sizeof(double));
    const int ne = (int)std::max<size_t>(8, std::min<size_t>(512, (size_t(2) << 30) / out_elem));
    std::vector<double> hv(24 * (size_t)ne);
    for (int e = 0; e < ne; ++e)
        for (int v = 0; v < 8; ++v)
            for (int d = 0; d < 3; ++d) hv[24 * e + 3 * v + d] = ((v >> d) & 1) + (d == 0 ? e : 0);
    double *dv = nullptr;
    void *dout = nullptr;
    const Program &p0 = fp32 ? pe->prog32 : pe->prog;
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&dv, hv.size() * sizeof(double)));
    CK(cudaMemcpy(dv, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&dout, (size_t)ne * p0.rows * p0.cols * esz));
    int maxnA = 1;
    for (int k = 0; k < p0.nblock; ++k) maxnA = std::max(maxnA, p0.blocks[k].nc[p0.blocks[k].dir[2]]);
    const int orig = p0.nj;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    int best = orig;
    float best_ms = 1e30f;
    // FP32: nj = 0 is the stage-C tensor-core kernel, nj > 0 the earlier kernels
    for (int nj = (fp32 && pe->tcc.ok) ? 0 : 1; nj <= std::min(NJMAX, maxnA); ++nj) {
        if (install_program(pe, te, base, q, L, fp32, nj) != DPG_OK) continue;
        float ts[6];
        int nt = 0;
        bool ok = true;
        for (int rep = 0; rep < 6 && ok; ++rep) {
            cudaEventRecord(a, s);
            const OutGeom og{ pe->prog.cols, (int64_t)pe->prog.parts * pe->prog.rows * pe->prog.cols };
            const int rr = fp32 ? run_general<float>(ds, pe, te, ne, dv, nullptr, (float *)dout, s, og)
                                : run_general<double>(ds, pe, te, ne, dv, nullptr, (double *)dout, s, og);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ok = rr == DPG_OK;
            if (rep > 0) ts[nt++] = ms;                   // the first run warms up
        }
        if (!ok) continue;
        std::sort(ts, ts + nt);
        const float med = ts[nt / 2];                     // median of five
        if (med < best_ms) { best_ms = med; best = nj; }
    }
    // FP64 programs that mix diagonal blocks of the symmetric matrix (units from i_A up:
    // uneven) with full blocks: a second pass over the diagonal blocks' own chunk
    int best_sym = 0;
    bool has_sym = false, has_full = false;
    for (int k = 0; k < p0.nblock; ++k) (p0.blocks[k].sym == 1 ? has_sym : has_full) = true;
    if (!fp32 && has_sym && has_full && best > 1) {
        for (int nj_sym = 1; nj_sym < best; ++nj_sym) {
            if (install_program(pe, te, base, q, L, fp32, best, nj_sym) != DPG_OK) continue;
            float ts[6];
            int nt = 0;
            bool ok = true;
            for (int rep = 0; rep < 6 && ok; ++rep) {
                cudaEventRecord(a, s);
                const OutGeom og{ pe->prog.cols, (int64_t)pe->prog.parts * pe->prog.rows * pe->prog.cols };
                ok = run_general<double>(ds, pe, te, ne, dv, nullptr, (double *)dout, s, og) == DPG_OK;
                cudaEventRecord(b, s);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) ts[nt++] = ms;
            }
            if (!ok) continue;
            std::sort(ts, ts + nt);
            if (ts[nt / 2] < best_ms) { best_ms = ts[nt / 2]; best_sym = nj_sym; }
        }
    }
    cudaEventDestroy(a); cudaEventDestroy(b);
    cudaFree(dv); cudaFree(dout);
    if ((r = install_program(pe, te, base, q, L, fp32, best, best_sym))) return r;
    if ((r = update_hp_table(ds, base, q, pe, te))) return r;
    read_status(ds, nullptr);                             // the synthetic runs report nothing
    if (cache) {
        if (FILE *f = std::fopen(cache, "a")) {
            std::fprintf(f, "{\"space\": %d, \"q\": %d, \"L\": %d, \"fp32\": %d, \"nj\": %d, \"ms\": %.6f, \"nj_sym\": %d}\n",
                         base, q, L, (int)fp32, best, (double)best_ms, best_sym);
            std::fclose(f);
        }
    }
    if (best_nj) *best_nj = best;
    return DPG_OK;
}

const char *dpg_strerror(int code) {
    switch (code) {
    case DPG_OK: return "ok";
    case DPG_ERR_ARG: return "invalid argument";
    case DPG_ERR_NOT_INIT: return "tables not initialised for this (space, q)";
    case DPG_ERR_RANGE: return "order or quadrature size out of range";
    case DPG_ERR_CUDA: return "CUDA runtime error";
    case DPG_ERR_DEGENERATE: return "non-positive or non-finite Jacobian determinant";
    case DPG_ERR_NOT_AFFINE: return "element is not a parallelepiped";
    case DPG_ERR_NOMEM: return "out of memory";
    case DPG_ERR_SCRATCH: return "request larger than the fixed scratch of dpg_integrate_noalloc";
    case DPG_ERR_TIMEOUT: return "a bounded tensor-core wait ran out (the call's matrices are not valid)";
    case DPG_ERR_NOT_EXTRUDED: return "element is not an extrusion along x1";
    case DPG_ERR_NOT_SPD: return "Gram matrix is not positive definite";
    case DPG_ERR_BOUNDS: return "a kernel index left its extent (bounds-checked build)";
    }
    return "unknown status";
}

double dpg_flops_per_element(int space, int p_trial, int q_test) {
    std::lock_guard<std::mutex> lk(g_mu);
    ProgEntry *pe; TableEntry *te; DeviceState *ds;
    if (resolve(space, p_trial, q_test, &pe, &te, &ds) != DPG_OK) return -1.0;
    if (space & DPG_MAP_AFFINE) return pe->flops_aff;
    if (space & DPG_MAP_EXTRUDED) return pe->flops_ext;
    // the same algorithmic count for both forms (the FP32 row-panel kernel also computes
    // the mirrored blocks; that extra work is not counted)
    return pe->prog.flops;
}

int dpg_measure_fma_peak(int precision, void *stream, double *flops) {
    if (!flops || (precision != 32 && precision != 64 && precision != 65 && precision != 19)) return DPG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool tc = precision == 19;
    const int blocks = tc ? sms : sms * 8;
    void *buf = nullptr;
    CK(cudaMalloc(&buf, 256 * sizeof(double)));
    CK(cudaMemset(buf, 0, 256 * sizeof(double)));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto run = [&](int iters, float *ms) -> int {
        CK(cudaEventRecord(a, s));
        cudaError_t e = precision == 64 ? launch_fma_peak<double>((double *)buf, blocks, iters, s)
                      : precision == 65 ? launch_dmma_peak((double *)buf, blocks, iters, s)
                      : tc             ? launch_tc_tf32_peak(blocks, iters, (int *)buf, s)
                                        : launch_fma_peak<float>((float *)buf, blocks, iters, s);
        if (e != cudaSuccess) return cuda_fail(e, "peak probe launch", __LINE__);
        CK(cudaEventRecord(b, s));
        CK(cudaEventSynchronize(b));
        CK(cudaEventElapsedTime(ms, a, b));
        return DPG_OK;
    };
    float ms = 0.f;
    int iters = 16;
    int r = run(iters, &ms);                           // warm-up and calibration
    while (r == DPG_OK && ms < 20.f && iters < (1 << 24)) { iters *= 4; r = run(iters, &ms); }
    double best = 0.0;
    for (int rep = 0; rep < 5 && r == DPG_OK; ++rep) {
        r = run(iters, &ms);
        // flops per CTA-thread and iteration: 8 chains x 16 FMAs x 2, or 8 mma x 512 / 32
        // lanes; the tensor-core probe: 2 products of 2 x 128 x 256 x 8 per CTA
        const double f = tc ? 2.0 * 2.0 * 128 * 256 * 8 * (double)iters * blocks / (ms * 1e-3)
                            : (precision == 65 ? 128.0 : 256.0) * (double)iters * 256.0 * blocks / (ms * 1e-3);
        if (f > best) best = f;
    }
    int st = 0;
    if (r == DPG_OK && tc) {
        cudaError_t e = cudaMemcpy(&st, buf, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) r = cuda_fail(e, "cudaMemcpy", __LINE__);
        else if (st) r = DPG_ERR_TIMEOUT;
    }
    cudaEventDestroy(a); cudaEventDestroy(b); cudaFree(buf);
    if (r) return r;
    *flops = best;
    return DPG_OK;
}

}  // extern "C"
