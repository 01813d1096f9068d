"""CPU tests of the C ABI library: it builds for sm_103a, loads, exports every
entry point include/cbfm.h declares, and its host-side mesh logic (canonical
RWG edges, octant / RCB cells) matches the oracle's independent code."""
import re
import os

import numpy as np
import pytest

import workloads as W
from oracle import mesh as OM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2111_11058_gb300 import build as B
    B.build()
    import paper_2111_11058_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "cbfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cbfm_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(P):
    lib = P.cbfm.lib()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.cbfm.exported_symbols()) == names


def _enum_values():
    """name -> value of every enumerator in include/cbfm.h."""
    src = open(os.path.join(ROOT, "include", "cbfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body in re.findall(r"typedef enum \{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(CBFM_[A-Z_0-9]+)\s*=\s*(\d+)", body):
            out[name] = int(val)
    return out


def test_binding_constants_match_header(P):
    e = _enum_values()
    C = P.cbfm
    assert (e["CBFM_FP64"], e["CBFM_MIXED"], e["CBFM_MIXED_SIMT"], e["CBFM_MIXED_UNFUSED"], e["CBFM_MIXED_FUSED"]) == (
        C.FP64, C.MIXED, C.MIXED_SIMT, C.MIXED_UNFUSED, C.MIXED_FUSED)
    assert (e["CBFM_PC_NONE"], e["CBFM_PC_CMP"], e["CBFM_PC_TDIAG"], e["CBFM_PC_CMP_INEXACT"]) == \
        (C.PC_NONE, C.PC_CMP, C.PC_TDIAG, C.PC_CMP_INEXACT)
    for name, val in e.items():
        if name in ("CBFM_OK",) or name.startswith("CBFM_E"):
            assert C.STATUS[val] == name


@pytest.mark.parametrize("case", ["sphere_octant", "cube_rcb", "cylinder_rcb7", "array_rcb"])
def test_host_mesh_tables_match_oracle(P, case):
    g, nc, part = {
        "sphere_octant": (W.icosphere(2, 0.3), 8, "octant"),
        "cube_rcb": (W.cube(16), 32, "rcb"),
        "cylinder_rcb7": (W.cylinder(0.3, 0.6, 16, 5, 2), 7, "rcb"),
        "array_rcb": (W.sphere_array(2, 2, 1, 0.5, level=1), 5, "rcb"),
    }[case]
    e, c = P.mesh_edges(g.verts, g.tris, nc, part)
    m = OM.build_rwg(g.verts, g.tris)
    oc = OM.cells_octant(m) if part == "octant" else OM.cells_rcb(m, nc)
    assert np.array_equal(e, m.edges)
    assert np.array_equal(c, oc)
    assert np.bincount(c).min() > 0


def test_rejects_open_and_inconsistent_meshes(P):
    g = W.icosphere(1, 0.5)
    with pytest.raises(P.CbfmError) as ei:
        P.mesh_edges(g.verts, g.tris[:-1], 8, "octant")
    assert ei.value.status == 1
    bad = g.tris.copy()
    bad[0] = bad[0][[0, 2, 1]]
    with pytest.raises(P.CbfmError):
        P.mesh_edges(g.verts, bad, 8, "octant")
    with pytest.raises(P.CbfmError):
        P.mesh_edges(g.verts, g.tris, 7, "octant")


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2111_11058_gb300.cbfm as C
    monkeypatch.setattr(C, "_lib", None)
    monkeypatch.setattr(C, "_LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(C.CbfmError):
        C.lib()


def test_tuning_query_is_host_only(P):
    """cbfm_tuning needs no device: an empty JSON object before any tuned launch."""
    t = P.cbfm.tuning()
    assert isinstance(t, dict)
    assert all(isinstance(v, int) for v in t.values())
