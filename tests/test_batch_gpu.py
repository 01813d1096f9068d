"""Batched reduced-matrix assembly (one fused launch over the cell pairs of
all scatterers that fit the fused kernel, one launch per unfused stage for the
rest): every reduced system equals the one assembled on its own, for a seeded
mix of spheres, cubes and cylinders of uneven size with injected seeded CBFs
(one scatterer with cells beyond the fused kernel's limit of 256 RWG functions),
and batched systems solve to the same RCS as single ones.  The fused kernel adds
triangle-pair contributions with FP32 atomics, so two assemblies of the same
system agree to rounding (1e-6 of the largest entry), not bit for bit."""
import numpy as np
import pytest

import workloads as W

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


def _mix(P, count, seed):
    meshes, cbfs = [], []
    for k, d in enumerate(W.scatterer_mix(count, seed=seed)):
        g = d["mesh"]
        ne = 3 * g.tris.shape[0] // 2
        ncell = max(2, ne // 200)                       # cells of about 200 RWGs (uneven across scatterers)
        gm = P.mesh(g.verts, g.tris, ncell, complex(*d["eps"]), partition="rcb")
        Ns = np.bincount(gm.cells(), minlength=ncell)
        CM, CJ = W.random_cbfs(Ns, [int(min(3 + (k + c) % 14, n)) for c, n in enumerate(Ns)], seed=seed + k)
        meshes.append(gm)
        cbfs.append(P.cbf_import(gm, CM, CJ))
    return meshes, cbfs


@pytest.mark.parametrize("prec", [1, 4])
def test_batch_equals_single_on_uneven_mix(P, prec):
    meshes, cbfs = _mix(P, 10, seed=3)
    # one scatterer whose cells (about 430 RWG functions) exceed the fused kernel's tile
    g = W.cube(12, 0.9)
    big = P.mesh(g.verts, g.tris, 6, 3.0)
    Ns = np.bincount(big.cells(), minlength=6)
    CM, CJ = W.random_cbfs(Ns, [9] * 6, seed=11)
    meshes.append(big)
    cbfs.append(P.cbf_import(big, CM, CJ))
    reds = P.assemble_reduced_batch(meshes, cbfs, prec)
    assert len(reds) == 11
    for gm, c, rb in zip(meshes, cbfs, reds):
        rs = P.assemble_reduced(gm, c, prec)
        a, b = rs.export(), rb.export()
        assert a.shape == b.shape and rb.n == rs.n
        assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    tuned = P.tuning()
    assert any(k.startswith("far_strip_f32") and v in (32, 64, 128) for k, v in tuned.items()), tuned


@pytest.mark.parametrize("prec", [1, 4])
def test_batch_solves_like_single(P, prec):
    sph = W.icosphere(2, 0.3)
    cub = W.cube(6, 0.6)
    gen = W.plane_wave_set(W.fibonacci_dirs(12))
    exc = W.plane_wave_set(W.fibonacci_dirs(8))
    ms = [P.mesh(sph.verts, sph.tris, 8, 4.0, partition="octant"), P.mesh(cub.verts, cub.tris, 6, 2.5 - 0.1j)]
    cs = [P.build_cbfs(m, gen, 1e-3) for m in ms]
    reds = P.assemble_reduced_batch(ms, cs, prec)
    for m, c, rb in zip(ms, cs, reds):
        rs = P.assemble_reduced(m, c, prec)
        for r in (rs, rb):
            P.cmp_setup(r)
        a = P.solve(rs, exc, tol=1e-8, monostatic=True, want_j=False, solver=P.BLOCK).rcs.sum(-1)
        b = P.solve(rb, exc, tol=1e-8, monostatic=True, want_j=False, solver=P.BLOCK).rcs.sum(-1)
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_batch_rejects_other_precisions_and_empty(P):
    meshes, cbfs = _mix(P, 2, seed=5)
    with pytest.raises(P.CbfmError):
        P.assemble_reduced_batch(meshes, cbfs, P.FP64)
    assert P.assemble_reduced_batch([], [], P.MIXED) == []


def test_batch_member_with_real_cbfs_vs_oracle(P):
    """One scatterer of the seeded uneven mix, assembled in the same batched
    launches as the nine others, with real primary CBFs (generated on the GPU
    from 12 directions x 2 polarisations, delta_SVD = 1e-3): sampled cell-pair
    blocks of its A against oracle.cbfm.reduced_block with those CBFs injected
    (Eq. (CBFM_outer)), within the mixed-path bound of 5e-5 of each block."""
    from oracle import cbfm as OC, mesh as OM
    gen = W.plane_wave_set(W.fibonacci_dirs(12))
    mix = W.scatterer_mix(10, seed=3)
    meshes, cbfs, geo = [], [], []
    for d in mix:
        g = d["mesh"]
        ne = 3 * g.tris.shape[0] // 2
        ncell = max(2, ne // 200)
        gm = P.mesh(g.verts, g.tris, ncell, complex(*d["eps"]), partition="rcb")
        meshes.append(gm)
        cbfs.append(P.build_cbfs(gm, gen, 1e-3))
        geo.append((g, complex(*d["eps"]), ncell, ne))
    reds = P.assemble_reduced_batch(meshes, cbfs, P.MIXED)
    # the first member small enough for the oracle's dense blocks, with at least three cells
    k = next(i for i, (g, eps, nc, ne) in enumerate(geo) if nc >= 3 and ne <= 2400)
    g, eps, ncell, ne = geo[k]
    m = OM.build_rwg(g.verts, g.tris)
    cell = meshes[k].cells()
    CM, CJ = cbfs[k].export()
    Ls = [int(x) for x in cbfs[k].L]
    ocb = [OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), Ls[c]) for c in range(ncell)]
    A = reds[k].export()
    offs = np.cumsum([0] + Ls)
    nh = offs[-1]
    mid = 0.5 * (m.verts[m.edges[:, 0]] + m.verts[m.edges[:, 1]])
    cen = np.array([mid[cell == c].mean(0) for c in range(ncell)])
    dist = np.linalg.norm(cen - cen[0], axis=1)
    pairs = [(0, 0), (0, int(np.argsort(dist)[1])), (int(np.argmax(dist)), 0)]
    for mi, ni in pairs:
        ref = OC.reduced_block(m, ocb, eps, mi, ni)
        rm, rn = slice(offs[mi], offs[mi + 1]), slice(offs[ni], offs[ni + 1])
        rm2, rn2 = slice(nh + offs[mi], nh + offs[mi + 1]), slice(nh + offs[ni], nh + offs[ni + 1])
        got = [A[rm, rn], A[rm, rn2], A[rm2, rn], A[rm2, rn2]]
        for gb, ob in zip(got, ref):
            err = float(np.abs(gb - ob).max() / np.abs(ob).max())
            print(f"batch member {k} block ({mi}, {ni}): {err:.2e}")
            assert err < 5e-5, (mi, ni, err)
