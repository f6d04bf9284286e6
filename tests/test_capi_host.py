"""Host-side checks of the C ABI (no GPU): the library loads, exports every function that
include/dpg.h declares, and its pure host queries (matrix sizes) follow the paper's
dimension formulas (H1 after Eq. 2.33; L2 after Eq. 2.17; H(div) and H(curl) dims in
Secs. 2.5-2.6)."""
import ctypes
import os
import re

import pytest

import oracle
import paper_1711_00984_gb300 as dpg
from paper_1711_00984_gb300 import build as dbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "dpg.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dpg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    dbuild.build()
    return dpg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dpg_integrate" in names and "dpg_tables_init" in names
    raw = ctypes.CDLL(dpg.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert set(names) <= set(dpg.EXPORTS)


@pytest.mark.parametrize("q", [1, 2, 5, 9, 12])
def test_matrix_sizes(lib, q):
    assert dpg.dpg_matrix_rows("H1", q) == (q + 1) ** 3
    assert dpg.dpg_matrix_rows("L2", q) == q ** 3
    assert dpg.dpg_matrix_rows("HDIV", q) == 3 * (q + 1) * q * q
    assert dpg.dpg_matrix_rows("HCURL", q) == 3 * q * (q + 1) ** 2
    for s in ["H1", "L2", "HDIV", "HCURL"]:
        assert dpg.dpg_matrix_cols(s, 0, q) == dpg.dpg_matrix_rows(s, q) == oracle.dim(s, q)
        assert dpg.dpg_matrix_rows(s, q) == oracle.dim(s, q)
    for p in range(1, q + 1):
        assert dpg.dpg_matrix_cols("B", p, q) == 3 * p ** 3
    assert dpg.dpg_matrix_cols("B", q + 1, q) == -1
    assert dpg.dpg_matrix_rows("B", q) == 3 * q * (q + 1) ** 2
    # ultraweak acoustics: cross block H(div) x H1, stiffness (H1 + H(div)) x 4 p^3
    assert dpg.dpg_matrix_rows("ACOUSTIC_CROSS", q) == oracle.dim("HDIV", q)
    assert dpg.dpg_matrix_cols("ACOUSTIC_CROSS", 0, q) == oracle.dim("H1", q)
    assert dpg.dpg_matrix_rows("ACOUSTIC_B", q) == oracle.dim("H1", q) + oracle.dim("HDIV", q)
    for p in range(1, q + 1):
        assert dpg.dpg_matrix_cols("ACOUSTIC_B", p, q) == 4 * p ** 3
    assert dpg.dpg_matrix_cols("ACOUSTIC_B", q + 1, q) == -1


def test_bad_arguments_rejected_on_host(lib):
    assert dpg.dpg_matrix_rows("H1", 0) == -1
    assert dpg.dpg_matrix_rows("H1", 13) == -1
    assert dpg.dpg_matrix_rows(9, 3) == -1
    assert dpg.dpg_strerror(0) == "ok"
    assert "Jacobian" in dpg.dpg_strerror(5)
