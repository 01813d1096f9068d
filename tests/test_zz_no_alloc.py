"""cbfm_red_export_noalloc: the reduced-matrix export for callers that cannot
allocate device memory (for example a serving process whose HBM is full of
cached matrices).  Called through the C ABI, its output must equal that of
cbfm_red_export on two calls in a row (into host memory and into a device
tensor), free device memory must not change across a call, and sizes beyond
its fixed scratch, or a conventional-MoM handle, must be refused.  Kept in its
own file so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_2111_11058_gb300 import build as B
    B.build()
    import paper_2111_11058_gb300 as pkg
    return pkg


def _abi_export(P, red, fn_name):
    A = np.zeros((red.n, red.n), np.complex128)
    st = getattr(P.cbfm.lib(), fn_name)(red.handle, ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(0))
    assert st == 0, P.cbfm.lib().cbfm_last_error().decode()
    return A


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_export_matches_export(P, prec):
    g = W.icosphere(2, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    Ns = np.bincount(cell)
    CM, CJ = W.random_cbfs(Ns, [12] * 8, seed=3)
    gm = P.mesh(g.verts, g.tris, 8, 4.0, partition="octant")
    red = P.assemble_reduced(gm, P.cbf_import(gm, CM, CJ), prec)
    assert red.n == 192
    ref1 = _abi_export(P, red, "cbfm_red_export")
    got1 = _abi_export(P, red, "cbfm_red_export_noalloc")
    got2 = _abi_export(P, red, "cbfm_red_export_noalloc")
    ref2 = _abi_export(P, red, "cbfm_red_export")
    np.testing.assert_allclose(got1, ref1, rtol=1e-12, atol=0)
    np.testing.assert_allclose(got2, ref2, rtol=1e-12, atol=0)
    assert np.abs(ref1).max() > 0
    # a device destination, and no change of free device memory across the call
    import torch
    Ad = torch.zeros((red.n, red.n, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = P.cbfm.lib().cbfm_red_export_noalloc(red.handle, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(0))
    free1 = torch.cuda.mem_get_info()[0]
    assert st == 0, P.cbfm.lib().cbfm_last_error().decode()
    assert free1 == free0
    got3 = Ad.cpu().numpy()
    np.testing.assert_allclose(got3[..., 0] + 1j * got3[..., 1], ref1, rtol=1e-12, atol=0)


def test_noalloc_export_rejects_oversize(P):
    g = W.icosphere(2, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    Ns = np.bincount(cell)
    CM, CJ = W.random_cbfs(Ns, [40] * 8, seed=4)     # n_cbf = 640 > 512
    gm = P.mesh(g.verts, g.tris, 8, 4.0, partition="octant")
    red = P.assemble_reduced(gm, P.cbf_import(gm, CM, CJ), 1)
    A = np.zeros((red.n, red.n), np.complex128)
    st = P.cbfm.lib().cbfm_red_export_noalloc(red.handle, ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(0))
    assert st == 1
    assert "512" in P.cbfm.lib().cbfm_last_error().decode()


def test_noalloc_export_rejects_mom_handle(P):
    g = W.icosphere(1, 0.3)
    gm = P.mesh(g.verts, g.tris, 8, 4.0, partition="octant")
    mo = P.assemble_mom(gm, 0)
    A = np.zeros((mo.n, mo.n), np.complex128)
    st = P.cbfm.lib().cbfm_red_export_noalloc(mo.handle, ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(0))
    assert st == 1
    assert "cbfm_red_export" in P.cbfm.lib().cbfm_last_error().decode()
