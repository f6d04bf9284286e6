// dpg_noalloc.cu -- dpg_integrate_noalloc: the general path with its metric-field
// scratch in a fixed file-scope device array instead of a pool allocation, for callers
// that may not allocate device memory during integration (see include/dpg.h).
#include "../../include/dpg.h"

#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "dpg_registry.h"

namespace {

// Scratch of every dpg_integrate_noalloc call on a device.  In host code this name is
// only a stand-in for the device object; kernels receive its device address, looked up
// once per device by scratch_address().
static __device__ __align__(256) unsigned char g_noalloc_scratch[DPG_NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
std::map<int, void *> g_na_addr;   // device ordinal -> device address of g_noalloc_scratch

// Set-up, once per device, with that device current.  Under CUDA's lazy module loading
// this is also where the module holding the array is loaded, i.e. where the device
// memory of the array is reserved.
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

}  // namespace

extern "C" int dpg_integrate_noalloc(int space, int p_trial, int q_test, int64_t n_elem,
                                     const double *vertices, const double *coeffs, void *out, void *stream) {
    if (space & (DPG_MAP_AFFINE | DPG_MAP_EXTRUDED | DPG_VEC3)) return DPG_ERR_ARG;
    void *ws = nullptr;
    const int r = scratch_address(&ws);
    if (r) return r;
    // the same programs and kernels as dpg_integrate (FP64 and FP32 forms), the metric
    // fields in the array; the size check comes before any launch or pointer use
    return dpg::integrate_in_scratch(space, p_trial, q_test, n_elem, vertices, coeffs, out, ws,
                                     DPG_NOALLOC_SCRATCH_BYTES, stream);
}
