"""GB300 element-matrix library for arXiv 1711.00984 (sum-factorized DPG Gram matrices).

A thin ctypes binding of the C ABI in ``include/dpg.h``: the functions below carry the
same names and only marshal arguments (tensor pointers, the current CUDA stream).  Every
step of the integration runs in the CUDA kernels of ``csrc/``; there is no CPU path, and
calling anything without the built library raises.

Submodules: ``meshgen`` (seeded synthetic meshes, no method arithmetic), ``build``
(nvcc build of ``_build/libdpg.so``).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdpg.so")

# spaces and flags (include/dpg.h)
DPG_H1, DPG_HCURL, DPG_HDIV, DPG_L2, DPG_B_L2VEC_HCURL = 1, 2, 3, 4, 5
DPG_ACOUSTIC_CROSS, DPG_ACOUSTIC_B = 6, 7
DPG_FP32, DPG_MAP_AFFINE, DPG_B_SPLIT, DPG_MAP_EXTRUDED, DPG_VEC3 = 0x100, 0x200, 0x400, 0x800, 0x1000
SPACE_IDS = {"H1": DPG_H1, "HCURL": DPG_HCURL, "HDIV": DPG_HDIV, "L2": DPG_L2, "B": DPG_B_L2VEC_HCURL,
             "ACOUSTIC_CROSS": DPG_ACOUSTIC_CROSS, "ACOUSTIC_B": DPG_ACOUSTIC_B}
STATUS = {0: "DPG_OK", 1: "DPG_ERR_ARG", 2: "DPG_ERR_NOT_INIT", 3: "DPG_ERR_RANGE", 4: "DPG_ERR_CUDA",
          5: "DPG_ERR_DEGENERATE", 6: "DPG_ERR_NOT_AFFINE", 7: "DPG_ERR_NOMEM", 8: "DPG_ERR_SCRATCH",
          9: "DPG_ERR_TIMEOUT", 10: "DPG_ERR_NOT_EXTRUDED",
          11: "DPG_ERR_NOT_SPD", 12: "DPG_ERR_BOUNDS"}

EXPORTS = ["dpg_tables_init", "dpg_tables_init_L", "dpg_tables_free", "dpg_matrix_rows",
           "dpg_matrix_cols", "dpg_integrate", "dpg_integrate_noalloc", "dpg_integrate_hp", "dpg_integrate_host", "dpg_sync_status",
           "dpg_strerror", "dpg_last_cuda_error", "dpg_autotune", "dpg_flops_per_element", "dpg_measure_fma_peak",
           "dpg_test_stall_tc_once", "dpg_test_set_workspace_limit", "dpg_integrate_load", "dpg_condense",
           "dpg_condensed_system", "dpg_condense_set_method"]

_lib = None
_lock = threading.Lock()


class DpgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = dpg_strerror(code) if _lib else ""
        if code in (4, 7) and _lib:
            detail += "; " + dpg_last_cuda_error()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({detail})")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libdpg.so (built by ``build.py``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run paper_1711_00984_gb300.build)")
        lib = ctypes.CDLL(p)
        i64, vp, dp = ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        lib.dpg_tables_init.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.dpg_tables_init_L.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.dpg_tables_free.argtypes = []
        lib.dpg_matrix_rows.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.dpg_matrix_rows.restype = i64
        lib.dpg_matrix_cols.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.dpg_matrix_cols.restype = i64
        lib.dpg_integrate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, vp]
        lib.dpg_integrate_host.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, vp]
        lib.dpg_integrate_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, vp]
        lib.dpg_integrate_hp.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, vp]
        lib.dpg_autotune.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int)]
        lib.dpg_autotune.restype = ctypes.c_int
        lib.dpg_sync_status.argtypes = [vp, ctypes.POINTER(i64)]
        lib.dpg_strerror.argtypes = [ctypes.c_int]
        lib.dpg_strerror.restype = ctypes.c_char_p
        lib.dpg_last_cuda_error.argtypes = []
        lib.dpg_last_cuda_error.restype = ctypes.c_char_p
        lib.dpg_flops_per_element.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.dpg_flops_per_element.restype = ctypes.c_double
        lib.dpg_measure_fma_peak.argtypes = [ctypes.c_int, vp, dp]
        lib.dpg_integrate_load.argtypes = [ctypes.c_int, ctypes.c_int, i64, vp, vp, i64, vp, vp]
        lib.dpg_condense.argtypes = [i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        lib.dpg_condensed_system.argtypes = [ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, i64, vp, vp, vp]
        lib.dpg_condense_set_method.argtypes = [ctypes.c_int]
        lib.dpg_test_stall_tc_once.argtypes = []
        lib.dpg_test_stall_tc_once.restype = ctypes.c_int
        lib.dpg_test_set_workspace_limit.argtypes = [i64]
        lib.dpg_test_set_workspace_limit.restype = ctypes.c_int
        for name in ["dpg_tables_init", "dpg_tables_init_L", "dpg_tables_free", "dpg_integrate", "dpg_integrate_noalloc", "dpg_integrate_hp",
                     "dpg_integrate_host", "dpg_sync_status", "dpg_measure_fma_peak", "dpg_integrate_load",
                     "dpg_condense", "dpg_condensed_system", "dpg_condense_set_method"]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _L():
    return _lib if _lib is not None else load()


def _check(code: int, where: str) -> int:
    if code != 0:
        raise DpgError(code, where)
    return code


def space_id(space, fp32: bool = False, affine: bool = False, split: bool = False, extruded: bool = False,
             vec3: bool = False) -> int:
    s = SPACE_IDS[space] if isinstance(space, str) else int(space)
    return (s | (DPG_FP32 if fp32 else 0) | (DPG_MAP_AFFINE if affine else 0) | (DPG_B_SPLIT if split else 0)
            | (DPG_MAP_EXTRUDED if extruded else 0) | (DPG_VEC3 if vec3 else 0))


# ---- the C ABI, name for name ---------------------------------------------------------

def dpg_tables_init(q: int, space) -> int:
    return _check(_L().dpg_tables_init(q, space_id(space)), "dpg_tables_init")


def dpg_tables_init_L(q: int, L: int, space) -> int:
    return _check(_L().dpg_tables_init_L(q, L, space_id(space)), "dpg_tables_init_L")


def dpg_tables_free() -> int:
    return _check(_L().dpg_tables_free(), "dpg_tables_free")


def dpg_matrix_rows(space, q: int) -> int:
    return int(_L().dpg_matrix_rows(space_id(space), q))


def dpg_matrix_cols(space, p_trial: int, q: int) -> int:
    return int(_L().dpg_matrix_cols(space_id(space), p_trial, q))


def dpg_integrate(space: int, p_trial: int, q_test: int, n_elem: int, vertices: int, coeffs: int,
                  out: int, stream: int) -> int:
    """Raw call with integer device pointers and a raw cudaStream_t handle."""
    return _L().dpg_integrate(space, p_trial, q_test, n_elem, vertices or None, coeffs or None, out, stream or None)


def dpg_integrate_noalloc(space: int, p_trial: int, q_test: int, n_elem: int, vertices: int, coeffs: int,
                          out: int, stream: int) -> int:
    """Raw call of the allocation-free variant (fixed device scratch, no allocation)."""
    return _L().dpg_integrate_noalloc(space, p_trial, q_test, n_elem, vertices or None, coeffs or None, out,
                                      stream or None)


def dpg_integrate_hp(space: int, n_elem: int, vertices: int, coeffs: int, q_elem: int, out_offset: int,
                     out: int, stream: int) -> int:
    """Raw call of the hp-mixed batch entry point (device pointers)."""
    return _L().dpg_integrate_hp(space, n_elem, vertices or None, coeffs or None, q_elem or None,
                                 out_offset or None, out, stream or None)


def integrate_hp(space, verts, q_elem, coeffs=None, *, fp32: bool = False, out=None, stream=None):
    """hp batch of device tensors: verts[n, 8, 3] float64, q_elem[n] int32 (CUDA).

    Returns (out, offsets): the packed 1-D output and the int64 element offsets into it.
    Tables for every q present must have been initialised.
    """
    import torch
    n = verts.shape[0]
    qs = q_elem.to(torch.int64)
    if space in ("H1", DPG_H1):
        dims = (qs + 1) ** 3
    elif space in ("L2", DPG_L2):
        dims = qs ** 3
    elif space in ("HDIV", DPG_HDIV):
        dims = 3 * (qs + 1) * qs * qs
    else:
        dims = 3 * qs * (qs + 1) ** 2
    sizes = dims * dims
    offsets = torch.zeros(n, dtype=torch.int64, device=verts.device)
    if n > 1:
        offsets[1:] = torch.cumsum(sizes, 0)[:-1]
    total = int(sizes.sum().item()) if n else 0
    dt = torch.float32 if fp32 else torch.float64
    if out is None:
        out = torch.empty(total, dtype=dt, device=verts.device)
    sid = space_id(space, fp32)
    code = dpg_integrate_hp(sid, n, verts.data_ptr(), coeffs.data_ptr() if coeffs is not None else 0,
                            q_elem.data_ptr(), offsets.data_ptr(), out.data_ptr(), _stream_handle(stream))
    _check(code, "dpg_integrate_hp")
    return out, offsets


def dpg_integrate_host(space: int, p_trial: int, q_test: int, n_elem: int, vertices: int, coeffs: int,
                       out: int, stream: int) -> int:
    return _L().dpg_integrate_host(space, p_trial, q_test, n_elem, vertices or None, coeffs or None, out, stream or None)


def dpg_sync_status(stream: int = 0) -> tuple[int, int]:
    bad = ctypes.c_int64(-1)
    code = _L().dpg_sync_status(stream or None, ctypes.byref(bad))
    return int(code), int(bad.value)


def dpg_test_stall_tc_once() -> int:
    """Test hook: the next FP32 tensor-core launch stalls its first CTA (see include/dpg.h)."""
    return _check(_L().dpg_test_stall_tc_once(), "dpg_test_stall_tc_once")


def dpg_test_set_workspace_limit(nbytes: int) -> int:
    """Test hook: cap the per-chunk metric-field workspace of the general and extruded
    paths at nbytes (0 restores the default; see include/dpg.h)."""
    return _check(_L().dpg_test_set_workspace_limit(int(nbytes)), "dpg_test_set_workspace_limit")


def dpg_strerror(code: int) -> str:
    return _L().dpg_strerror(code).decode()


def dpg_autotune(q: int, space, fp32: bool = False, stream: int = 0) -> int:
    """Tune the stage-A chunk of (space, q); returns the chosen width."""
    nj = ctypes.c_int(0)
    _check(_L().dpg_autotune(q, space_id(space, fp32), stream or None, ctypes.byref(nj)), "dpg_autotune")
    return nj.value


def dpg_last_cuda_error() -> str:
    return _L().dpg_last_cuda_error().decode()


def dpg_flops_per_element(space, p_trial: int, q_test: int) -> float:
    return float(_L().dpg_flops_per_element(space if isinstance(space, int) else space_id(space), p_trial, q_test))


def dpg_measure_fma_peak(precision: int, stream: int = 0) -> float:
    out = ctypes.c_double(0.0)
    _check(_L().dpg_measure_fma_peak(precision, stream or None, ctypes.byref(out)), "dpg_measure_fma_peak")
    return out.value


# ---- torch marshalling -----------------------------------------------------------------

def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def matrix_shape(space, q: int, p: int = 0, split: bool = False, vec3: bool = False) -> tuple[int, ...]:
    """Per-element output shape: (rows, cols), or (2, rows, cols) for split B and for the
    acoustics stiffness (part 0 and the coefficient of i*omega); (3n, 3n) with vec3."""
    sid = space_id(space, vec3=vec3)
    r = dpg_matrix_rows(sid, q)
    c = dpg_matrix_cols(sid, p, q)
    two = split or (space_id(space) & 0xff) == DPG_ACOUSTIC_B
    return (2, r, c) if two else (r, c)


def integrate(space, q: int, verts, coeffs=None, *, p: int = 0, fp32: bool = False, affine: bool = False,
              split: bool = False, extruded: bool = False, vec3: bool = False, out=None, stream=None):
    """Integrate element matrices of device tensors ``verts[n, 8, 3]`` (float64, CUDA).

    Returns ``out[n, rows, cols]`` (``[n, 2, rows, cols]`` with ``split``) in float64, or
    float32 with ``fp32``.  Tables for (space, q) must have been initialised.
    """
    import torch
    if not verts.is_cuda or verts.dtype != torch.float64 or not verts.is_contiguous():
        raise ValueError("verts must be a contiguous float64 CUDA tensor [n, 8, 3]")
    n = verts.shape[0]
    if coeffs is not None and (not coeffs.is_cuda or coeffs.dtype != torch.float64 or not coeffs.is_contiguous()):
        raise ValueError("coeffs must be a contiguous float64 CUDA tensor [n, 2]")
    shape = (n,) + matrix_shape(space, q, p, split, vec3)
    dt = torch.float32 if fp32 else torch.float64
    if out is None:
        out = torch.empty(shape, dtype=dt, device=verts.device)
    elif out.dtype != dt or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {dt} tensor of shape {shape}")
    sid = space_id(space, fp32, affine, split, extruded, vec3)
    code = dpg_integrate(sid, p, q, n, verts.data_ptr(), coeffs.data_ptr() if coeffs is not None else 0,
                         out.data_ptr(), _stream_handle(stream))
    _check(code, "dpg_integrate")
    return out


def dpg_integrate_load(space: int, q_test: int, n_elem: int, vertices: int, src_coef: int, coef_stride: int,
                       out: int, stream: int) -> int:
    """Raw call of the load-vector entry point (integer device pointers)."""
    return _L().dpg_integrate_load(space, q_test, n_elem, vertices or None, src_coef or None, coef_stride,
                                   out or None, stream or None)


def integrate_load(space, q: int, verts, src_coef, *, fp32: bool = False, out=None, stream=None):
    """Load vectors ``out[n, rows]`` of device tensors ``verts[n, 8, 3]`` (float64, CUDA).

    ``src_coef``: float64 CUDA tensor of the degree-2 source's coefficients, ``[10 nc]``
    (one source for all elements) or ``[n, 10 nc]`` (one per element), nc = 1 for H1 and
    L2, 3 for H(curl) and H(div).  Tables for (space, q) must have been initialised.
    """
    import torch
    if not verts.is_cuda or verts.dtype != torch.float64 or not verts.is_contiguous():
        raise ValueError("verts must be a contiguous float64 CUDA tensor [n, 8, 3]")
    if not src_coef.is_cuda or src_coef.dtype != torch.float64 or not src_coef.is_contiguous():
        raise ValueError("src_coef must be a contiguous float64 CUDA tensor")
    n = verts.shape[0]
    nc = 3 if (SPACE_IDS[space] if isinstance(space, str) else int(space) & 0xFF) in (2, 3) else 1
    if src_coef.dim() == 1:
        if src_coef.numel() != 10 * nc:
            raise ValueError(f"src_coef must hold {10 * nc} values")
        stride = 0
    else:
        if tuple(src_coef.shape) != (n, 10 * nc):
            raise ValueError(f"src_coef must have shape [{n}, {10 * nc}]")
        stride = 10 * nc
    shape = (n, dpg_matrix_rows(space, q))
    dt = torch.float32 if fp32 else torch.float64
    if out is None:
        out = torch.empty(shape, dtype=dt, device=verts.device)
    elif out.dtype != dt or tuple(out.shape) != shape or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {dt} tensor of shape {shape}")
    code = dpg_integrate_load(space_id(space, fp32), q, n, verts.data_ptr(), src_coef.data_ptr(), stride,
                              out.data_ptr(), _stream_handle(stream))
    _check(code, "dpg_integrate_load")
    return out


def dpg_condense(n_elem: int, n: int, m: int, G: int, B: int, l: int, K: int, F: int, stream: int) -> int:
    """Raw call of the static condensation (integer device pointers, in place on G, B, l)."""
    return _L().dpg_condense(n_elem, n, m, G or None, B or None, l or None, K or None, F or None,
                             stream or None)


DPG_CONDENSE_FMA, DPG_CONDENSE_TC, DPG_CONDENSE_TCGEN05 = 0, 1, 2


def dpg_condense_set_method(method) -> int:
    """Arithmetic of the condensation's updates: "fma" / DPG_CONDENSE_FMA (FP64 FMA),
    "tc" / DPG_CONDENSE_TC (FP64 products from exact BF16 digits, mma.sync) or "tcgen05" /
    DPG_CONDENSE_TCGEN05 (the same digits on tcgen05 with tensor-memory accumulators)."""
    m = {"fma": DPG_CONDENSE_FMA, "tc": DPG_CONDENSE_TC, "tcgen05": DPG_CONDENSE_TCGEN05}.get(method, method)
    return _check(_L().dpg_condense_set_method(int(m)), "dpg_condense_set_method")


def condense(G, B, l=None, *, K=None, F=None, stream=None):
    """K = B^T G^-1 B (and F = B^T G^-1 l) per element; G, B, l are overwritten in place.

    ``G[ne, n, n]``, ``B[ne, n, m]``, ``l[ne, n]`` contiguous float64 CUDA tensors.
    Returns ``(K[ne, m, m], F[ne, m] or None)``.
    """
    import torch
    for name, t in (("G", G), ("B", B), ("l", l)):
        if t is not None and (not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    ne, n, m = B.shape
    if tuple(G.shape) != (ne, n, n) or (l is not None and tuple(l.shape) != (ne, n)):
        raise ValueError("shapes: G[ne, n, n], B[ne, n, m], l[ne, n]")
    if K is None:
        K = torch.empty((ne, m, m), dtype=torch.float64, device=B.device)
    if l is not None and F is None:
        F = torch.empty((ne, m), dtype=torch.float64, device=B.device)
    code = dpg_condense(ne, n, m, G.data_ptr(), B.data_ptr(), l.data_ptr() if l is not None else 0,
                        K.data_ptr(), F.data_ptr() if l is not None else 0, _stream_handle(stream))
    _check(code, "dpg_condense")
    return K, (F if l is not None else None)


def dpg_condensed_system(q_test: int, p_trial: int, n_elem: int, vertices: int, coeffs: int, src_coef: int,
                         coef_stride: int, K: int, F: int, stream: int) -> int:
    """Raw call of the one-call DPG element routine (integer device pointers)."""
    return _L().dpg_condensed_system(q_test, p_trial, n_elem, vertices or None, coeffs or None, src_coef or None,
                                     coef_stride, K or None, F or None, stream or None)


def condensed_system(q: int, p: int, verts, coeffs=None, src_coef=None, *, K=None, F=None, stream=None):
    """K[n, m, m] = B^T G^-1 B and F[n, m] = B^T G^-1 l of the H(curl) q / vector-L2 p pair.

    ``src_coef``: None, a float64 CUDA tensor of 30 values, or ``[n, 30]`` (per element).
    Tables for ("HCURL", q) and ("B", q) must have been initialised with the same rule.
    """
    import torch
    if not verts.is_cuda or verts.dtype != torch.float64 or not verts.is_contiguous():
        raise ValueError("verts must be a contiguous float64 CUDA tensor [n, 8, 3]")
    n = verts.shape[0]
    m = 3 * p ** 3
    stride = 0
    if src_coef is not None:
        if not src_coef.is_cuda or src_coef.dtype != torch.float64 or not src_coef.is_contiguous():
            raise ValueError("src_coef must be a contiguous float64 CUDA tensor")
        stride = 0 if src_coef.dim() == 1 else 30
    if K is None:
        K = torch.empty((n, m, m), dtype=torch.float64, device=verts.device)
    if src_coef is not None and F is None:
        F = torch.empty((n, m), dtype=torch.float64, device=verts.device)
    code = dpg_condensed_system(q, p, n, verts.data_ptr(), coeffs.data_ptr() if coeffs is not None else 0,
                                src_coef.data_ptr() if src_coef is not None else 0, stride, K.data_ptr(),
                                F.data_ptr() if src_coef is not None else 0, _stream_handle(stream))
    _check(code, "dpg_condensed_system")
    return K, (F if src_coef is not None else None)


def sync_status(stream=None) -> tuple[int, int]:
    """(status code, first offending element or -1) after synchronising the stream."""
    return dpg_sync_status(_stream_handle(stream))
