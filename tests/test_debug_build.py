"""The bounds-checked build (build(debug=True) -> libdpg_debug.so, -DDPG_DEBUG_BOUNDS).

In that build every kernel checks its global store indices, metric-field indices,
shared-memory layout and tensor-memory columns against the extents it was given and
records DPG_ERR_BOUNDS (12) instead of making an out-of-range access; nothing traps.
CPU: the variant compiles (nvcc cross-compiles for sm_103a) and exports every function of
include/dpg.h.  GPU: the small orders q = 1..3 of every path (general FP64 / FP32, affine,
extruded, hp batch, mixed B, load vectors, condensation) run on the debug library in a
fresh process with status DPG_OK and the parity tolerances of the release tests.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_1711_00984_gb300 import build as dbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dpg.h")) as f:
        txt = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(dpg_[a-z_0-9]+)\s*\(", txt)))


def test_debug_variant_builds_and_exports_every_symbol():
    so = dbuild.build(debug=True)
    assert so.endswith("libdpg_debug.so") and os.path.exists(so)
    raw = ctypes.CDLL(so)
    for n in _declared():
        assert hasattr(raw, n), n


_CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle
import paper_1711_00984_gb300 as dpg
from paper_1711_00984_gb300 import build as dbuild, meshgen
dpg.load(dbuild.build(debug=True))
torch.cuda.set_device(0)

def rel(a, b):
    return max(np.linalg.norm(a[e] - b[e]) / np.linalg.norm(b[e]) for e in range(b.shape[0]))

def check(tag, got, ref, tol):
    code, bad = dpg.sync_status()
    assert code == 0, (tag, dpg.STATUS.get(code), bad)
    got = got.double().cpu().numpy() if torch.is_tensor(got) else got
    err = rel(got.reshape(ref.shape), ref)
    assert err <= tol, (tag, err)

rng = np.random.default_rng(7)
vj = meshgen.jittered_grid(2, seed=70, jitter=0.2)[:5].copy()
va = meshgen.affine_parallelepipeds(2, seed=71)[:5].copy()
vx = meshgen.extruded_prisms(2, seed=72, jitter=0.2)[:5].copy()
c = np.stack([rng.uniform(0.5, 2, 5), rng.uniform(0.5, 2, 5)], 1)
ct = torch.from_numpy(c).cuda()
for q in (1, 2, 3):
    for s in ("H1", "HCURL", "HDIV", "L2"):
        dpg.dpg_tables_init(q, s)
        for v, kw in ((vj, {}), (va, {"affine": True}), (vx, {"extruded": True})):
            ref, _ = oracle.gram(s, q, q + 2, v, c)
            vt = torch.from_numpy(v).cuda()
            for f32 in (False, True):
                out = dpg.integrate(s, q, vt, ct, fp32=f32, **kw)
                check((s, q, kw, f32), out, ref, 1e-5 if f32 else 1e-12)
        # load vectors
        src = rng.uniform(-1, 1, 30 if s in ("HCURL", "HDIV") else 10)
        lg = dpg.integrate_load(s, q, torch.from_numpy(vj).cuda(), torch.from_numpy(src).cuda())
        lr, _ = oracle.load(s, q, q + 2, vj, src)
        check(("load", s, q), lg, lr, 1e-12)
    # mixed stiffness B (p = 1..q)
    dpg.dpg_tables_init(q, "B")
    for p in range(1, q + 1):
        Br, _ = oracle.mixed_b(q, p, q + 2, vj)
        check(("B", q, p), dpg.integrate("B", q, torch.from_numpy(vj).cuda(), p=p), Br, 1e-12)
# hp batch of mixed orders, every space, both forms
qe = np.array([1, 3, 2, 2, 1], dtype=np.int32)
for s in ("H1", "HCURL", "HDIV", "L2"):
    for f32 in (False, True):
        dims = np.array([dpg.dpg_matrix_rows(s, int(q)) for q in qe], dtype=np.int64)
        off = np.zeros(5, dtype=np.int64); off[1:] = np.cumsum(dims * dims)[:-1]
        out = torch.empty(int((dims * dims).sum()), dtype=torch.float32 if f32 else torch.float64, device="cuda")
        sh = int(torch.cuda.current_stream().cuda_stream)
        vt, qt, ot = torch.from_numpy(vj).cuda(), torch.from_numpy(qe).cuda(), torch.from_numpy(off).cuda()
        code = dpg.dpg_integrate_hp(dpg.space_id(s, fp32=f32), 5, vt.data_ptr(), 0, qt.data_ptr(), ot.data_ptr(),
                                    out.data_ptr(), sh)
        assert code == 0
        torch.cuda.synchronize()                 # the inputs stay referenced until the graph ran
        for e in range(5):
            q = int(qe[e]); n = int(dims[e])
            ref, _ = oracle.gram(s, q, q + 2, vj[e:e + 1])
            check(("hp", s, q, f32), out[off[e]:off[e] + n * n].reshape(1, n, n), ref, 1e-5 if f32 else 1e-12)
# condensation on an SPD batch, both arithmetics
G = meshgen.spd_batch(3, 70, 1e3, seed=73)
B = rng.uniform(-1, 1, (3, 70, 20)); l = rng.uniform(-1, 1, (3, 70))
Kr, Fr, _ = oracle.condense(G, B, l)
for method in ("tc", "fma", "tcgen05"):
    dpg.dpg_condense_set_method(method)
    K, F = dpg.condense(torch.from_numpy(G.copy()).cuda(), torch.from_numpy(B.copy()).cuda(),
                        torch.from_numpy(l.copy()).cuda())
    tol = 8 * 70 * 2.220446049250313e-16 * 1e3       # 8 n eps cond(G), as in the release tests
    check(("condense K", method), K, Kr, tol)
    check(("condense F", method), F, Fr, tol)
dpg.dpg_condense_set_method("tcgen05")
print("debug build ok")
'''


@pytest.mark.gpu
def test_debug_variant_runs_small_orders_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + _CHILD], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout
