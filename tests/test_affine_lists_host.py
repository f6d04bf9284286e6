"""Host-only check of the affine path's structural stage-B lists (no GPU needed).

The lists that drive the affine kernel's FP64 products (one entry per structurally non-zero
Q_g(i2, j2, jj) of a work unit, with the mask of its contributing terms) are built on the
host.  `affine_lists_check.cu` links the library's set-up object and recounts, from the
lists, the stage-B and stage-C products of every unit; their sum must equal the affine flop
count that the term program computes by its own loops over (i3, j3) pairs (Sec. 2.8.1), for
every space (the four Gram spaces, B, and the acoustics cross block and B of Eqs. 3.16-3.18),
q = 1..7 and both forms.  It also checks the list format the kernel relies on
(whole 32-entry chunks of one group, indices inside the block), and that the affine matrix is
detected as diagonal for L2 alone, with the table of the fill kernel equal to the Legendre
norms of Eq. 2.95.
"""
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_affine_structural_lists_match_flop_count(tmp_path):
    from paper_1711_00984_gb300 import build as B
    B.build()
    exe = tmp_path / "affine_lists_check"
    cmd = [B.nvcc()] + B._flags() + ["-I", B.CSRC, os.path.join(HERE, "affine_lists_check.cu"),
                                     os.path.join(B.BUILD, "dpg_setup.o"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert not [x for x in lines if "fail" in x]
    # H1, H(curl), H(div), L2 and the acoustics cross block at q = 1..7, B and the acoustic B
    # at p = 1..q, each in both forms
    assert len(lines) == 2 * (5 * 7 + 2 * sum(range(1, 8)))
    assert all(x["entries"] > 0 and x["stage_b"] >= x["entries"] for x in lines)
    assert [x["space"] for x in lines if x["diagonal"]] == [4] * 14       # L2, q = 1..7, both forms
