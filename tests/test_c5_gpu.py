"""The 90 000-unknown lossy prolate spheroid (semi-axes 2 and 0.5, eps_r 3 - 0.1j,
T = 30000, 256 RCB cells, 256 Fibonacci directions x 2 polarisations) at full
size on the GPU path, checked where the oracle can follow it:

  * the cells equal the oracle's RCB division;
  * primary CBFs (Sec. III-A, Eq. (pcbf); dual SVD, Sec. III-B) of sampled
    cells: the same L_m and normalised singular values as the oracle's, whose
    Z_mm, LU and SVD are computed from the cell alone;
  * reduced matrix A = (C^JM)^H Z C^MJ (Eq. (CBFM_outer)) from the fused
    assembly-projection kernel (the form CBFM_MIXED takes here: the unfused
    scratch would be ~340 GB), sampled cell-pair blocks -- a cell with itself
    (self and near pairs, lossy interior medium), neighbours and a far pair --
    against oracle.cbfm.reduced_block with the GPU's CBFs injected: within 5e-5
    of the largest entry of A for every block (the matrix bound), and of each
    block's own largest entry 5e-5 for a cell with itself or a neighbour, 1e-4
    for the far pair (cells ~4 wavelengths apart: its entries are oscillatory
    sums with cancellation and the FP32 phase k R reaches ~25 rad, so the error
    relative to the block grows with distance);
  * CMP-preconditioned block GMRES over all 512 excitations reaches tol 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cbfm as OC, mesh as OM, mom as OMo

pytestmark = pytest.mark.gpu

TOL_MATRIX = 5e-5
TOL_BLOCK_NEAR, TOL_BLOCK_FAR = 5e-5, 1e-4


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


@pytest.fixture(scope="module")
def c5(P):
    d = W.spheroid_c5()
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, d["ncell"])
    eps = complex(*d["eps"])
    gm = P.mesh(g.verts, g.tris, d["ncell"], eps, partition=d["partition"])
    cb = P.build_cbfs(gm, d["gen"], 1e-3)
    return dict(d=d, m=m, cell=cell, eps=eps, gm=gm, cb=cb)


def test_c5_cells_equal_oracle(c5):
    assert np.array_equal(c5["gm"].cells(), c5["cell"])


def test_c5_cbfs_sampled_cells_equal_oracle(c5):
    m, cell, eps, d = c5["m"], c5["cell"], c5["eps"], c5["d"]
    v = OMo.rhs(m, d["gen"])
    import scipy.linalg as sla
    for c in (3, 130):
        lam = np.nonzero(cell == c)[0]
        Ks, Ta, Tb = OMo.pmchwt_blocks(m, eps, 1.0, rows=lam, cols=lam)
        Jm = sla.lu_solve(sla.lu_factor(np.block([[Ks, Ta], [Tb, Ks]])), np.vstack([v[lam], v[m.ne + lam]]))
        ref = OC.cell_dual_cbfs(m, lam, Jm[:len(lam)], Jm[len(lam):], 1e-3)
        assert int(c5["cb"].L[c]) == ref.L
        sg = c5["cb"].sigma[c][:ref.L + 2]
        so = (ref.sigma / ref.sigma[0])[:ref.L + 2]
        assert np.abs(sg - so).max() < 1e-9


def test_c5_reduced_blocks_fused_vs_oracle(P, c5):
    m, cell, eps, gm, cb = c5["m"], c5["cell"], c5["eps"], c5["gm"], c5["cb"]
    red = P.assemble_reduced(gm, cb, P.MIXED)
    A = red.export()
    CM, CJ = cb.export()
    Ls = [int(x) for x in cb.L]
    cbfs = [OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), Ls[c]) for c in range(len(Ls))]
    offs = np.cumsum([0] + Ls)
    nh = offs[-1]
    # a cell with its nearest other cell (by edge-midpoint centroid), with itself, and with the farthest one
    mid = 0.5 * (m.verts[m.edges[:, 0]] + m.verts[m.edges[:, 1]])
    cen = np.array([mid[cell == c].mean(0) for c in range(len(Ls))])
    a = 17
    dist = np.linalg.norm(cen - cen[a], axis=1)
    near_c = int(np.argsort(dist)[1])
    far_c = int(np.argmax(dist))
    amax = float(np.abs(A).max())
    for (mi, ni) in [(a, a), (a, near_c), (near_c, a), (a, far_c)]:
        blocks = OC.reduced_block(m, cbfs, eps, mi, ni)
        rm, rn = slice(offs[mi], offs[mi + 1]), slice(offs[ni], offs[ni + 1])
        rm2, rn2 = slice(nh + offs[mi], nh + offs[mi + 1]), slice(nh + offs[ni], nh + offs[ni + 1])
        got = [A[rm, rn], A[rm, rn2], A[rm2, rn], A[rm2, rn2]]
        tol = TOL_BLOCK_FAR if ni == far_c else TOL_BLOCK_NEAR
        for gb, ob in zip(got, blocks):
            err = float(np.abs(gb - ob).max() / np.abs(ob).max())
            print(f"c5 block ({mi}, {ni}): {err:.2e} of the block, {float(np.abs(gb - ob).max()) / amax:.2e} of A")
            assert err < tol, (mi, ni, err)
            assert float(np.abs(gb - ob).max()) < TOL_MATRIX * amax, (mi, ni)


def test_c5_block_gmres_converges(P, c5):
    red = P.assemble_reduced(c5["gm"], c5["cb"], P.MIXED)
    P.cmp_setup(red)
    res = P.solve(red, c5["d"]["exc"], tol=1e-6, maxit=200, restart=red.n + 256, monostatic=True, want_j=False,
                  solver=P.BLOCK)
    assert res.status == 0
    assert (res.resid <= 1e-6).all()
    assert np.isfinite(res.rcs).all() and res.rcs.max() > 0
