// dpg_noalloc.cu -- dpg_integrate_noalloc: the general path with its metric-field
// scratch in a fixed file-scope device array instead of a pool allocation, for callers
// that may not allocate device memory during integration (see include/dpg.h).
#include "../../include/dpg.h"

#include <cuda_runtime.h>

#include <climits>
#include <map>
#include <mutex>

#include "dpg_kernels.h"
#include "dpg_registry.h"

namespace {

// Scratch of every dpg_integrate_noalloc call on a device.  In host code this name is
// only a stand-in for the device object; kernels receive its device address, looked up
// once per device by scratch_address().
static __device__ __align__(256) unsigned char g_noalloc_scratch[DPG_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
std::map<int, void *> g_na_addr;   // device ordinal -> device address of g_noalloc_scratch

// Set-up, once per device, with that device current.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DPG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_addr.find(dev);
    if (it == g_na_addr.end()) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DPG_ERR_CUDA;
        it = g_na_addr.emplace(dev, p).first;
    }
    *out = it->second;
    return DPG_OK;
}

template <typename T>
int run(const dpg::ProgramView &v, int64_t n_elem, const double *verts, const double *coeffs, T *out,
        void *ws, cudaStream_t s) {
    const dpg::Program &pr = *v.prog;
    const int L = pr.L;
    dpg::GeomParams g;
    g.space = pr.space; g.L = L; g.nfields = pr.nfields;
    g.n_elem = n_elem; g.elem_base = 0;
    g.verts = verts; g.coeffs = coeffs;
    g.zeta = v.zeta; g.w = v.w;
    g.fields = ws; g.status = v.status;
    if (dpg::launch_geom<T>(g, s) != cudaSuccess) return DPG_ERR_CUDA;
    dpg::SfParams<T> sp;
    sp.blocks = v.d_blocks; sp.units = v.d_units; sp.nunits = (int)pr.units.size();
    sp.L = L; sp.nfields = pr.nfields;
    if constexpr (sizeof(T) == 8) sp.pp = v.pp64; else sp.pp = v.pp32;
    sp.fields = reinterpret_cast<const T *>(ws);
    sp.out = out;
    sp.mat_stride = (int64_t)pr.parts * pr.rows * pr.cols;
    sp.ld = pr.cols; sp.n_elem = n_elem;
    if (dpg::launch_general<T>(sp, pr.smem_values * sizeof(T), s) != cudaSuccess) return DPG_ERR_CUDA;
    return DPG_OK;
}

}  // namespace

extern "C" int dpg_integrate_noalloc(int space, int p_trial, int q_test, int64_t n_elem,
                                     const double *vertices, const double *coeffs, void *out, void *stream) {
    if (space & (DPG_MAP_AFFINE | DPG_MAP_EXTRUDED | DPG_VEC3)) return DPG_ERR_ARG;
    dpg::ProgramView v;
    int r = dpg::lookup_program_view(space, p_trial, q_test, &v);
    if (r) return r;
    if (n_elem < 0) return DPG_ERR_ARG;
    if (n_elem == 0) return DPG_OK;
    if (!vertices || !out) return DPG_ERR_ARG;
    const bool fp32 = (space & DPG_FP32) != 0;
    const int L = v.prog->L;
    const size_t per_elem = (size_t)v.prog->nfields * L * L * L * (fp32 ? sizeof(float) : sizeof(double));
    if ((size_t)n_elem > DPG_NOALLOC_SCRATCH_BYTES / per_elem) return DPG_ERR_SCRATCH;
    if ((int64_t)v.prog->units.size() * n_elem > INT_MAX) return DPG_ERR_SCRATCH;
    void *ws = nullptr;
    if ((r = scratch_address(&ws))) return r;
    const double *c = (space & 0xff) > DPG_L2 ? nullptr : coeffs;          // Gram matrices only
    cudaStream_t s = (cudaStream_t)stream;
    return fp32 ? run<float>(v, n_elem, vertices, c, (float *)out, ws, s)
                : run<double>(v, n_elem, vertices, c, (double *)out, ws, s);
}
