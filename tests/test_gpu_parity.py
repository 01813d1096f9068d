"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative, max-abs normalised unless stated):
  * FP64 path: reduced matrix and CBF Gram <= 1e-11; currents <= 1e-7 and
    RCS <= 1e-8 with both sides solved to tol 1e-10 (solver tolerance times
    the conditioning of A dominates);
  * mixed path: reduced matrix <= 1e-4 (FP32 quadrature, relative error
    ~1e-7 per point pair; split-TF32 products, ~2^-21 each; FP32 accumulation
    over a few hundred terms), peak-normalised RCS <= 1e-4, currents (relative
    L2 over all right-hand sides, GMRES tol 1e-6) <= J_MIXED.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cbfm as OC, mesh as OM, mom as OMo

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10
# Mixed-path bound on the currents: ~1e-6 relative error of the reduced matrix
# (its largest entry) times the conditioning of the CMP-preconditioned system,
# plus the GMRES tolerance 1e-6.
J_MIXED = 1e-4


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


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _peak_rcs_err(g, o):
    return float(np.abs(g - o).max() / np.abs(o).max())


@pytest.fixture(scope="module")
def c1():
    """The 320-triangle sphere workload with its oracle pipeline."""
    d = W.sphere_c1()
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    exc = np.array([[0.0, 0.0, 0.0], [1.2, 0.7, 0.4], [2.5, 4.0, math.pi / 2]])
    ref = OC.run(m, cell, 8, 4.0, d["gen"], exc, 1e-3, TOL_SOLVE, restart=1000)
    obs = W.bistatic_cut(2.0)
    st, sp = OMo.rcs(*OMo.farfield(m, ref["sol"].j, obs))
    return dict(d=d, g=g, m=m, cell=cell, exc=exc, ref=ref, obs=obs, rcs=np.stack([st, sp], -1))


def _gpu_mesh(P, c1):
    return P.mesh(c1["g"].verts, c1["g"].tris, 8, 4.0, partition="octant")


def _inject(P, gm, cbfs):
    return P.cbf_import(gm, [c.CM for c in cbfs], [c.CJ for c in cbfs])


def test_mesh_cells(P, c1):
    gm = _gpu_mesh(P, c1)
    assert gm.n_edges == 480
    assert np.array_equal(gm.cells(), c1["cell"])


def test_reduced_fp64_c1(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    assert red.n == c1["ref"]["A"].shape[0]
    assert _relmax(red.export(), c1["ref"]["A"]) < 1e-11


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
def test_reduced_mixed_c1(P, c1, prec):
    """Mixed paths: FP32 far-pair quadrature, projections as split-TF32 tensor-core
    products after the assembly (prec 3; what prec 1 picks when memory allows)
    or fused with it (prec 4), or FP32 CUDA-core products (prec 2).  Stated bound on the
    reduced matrix: 2e-5 of its largest entry (FP32 quadrature ~1e-7, split TF32
    ~2^-21 per product, FP32 accumulation over a few hundred terms)."""
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), prec)
    err = _relmax(red.export(), c1["ref"]["A"])
    print(f"mixed ({prec}) reduced-matrix error {err:.2e}")
    assert err < 2e-5


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5), (2, 2e-5), (3, 2e-5), (4, 2e-5)])
def test_reduced_lossy_random_cbfs(P, prec, tol):
    g = W.icosphere(1, 0.4)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, 3)
    Ns = np.bincount(cell)
    CM, CJ = W.random_cbfs(Ns, [min(5, n) for n in Ns], seed=11)
    cbfs = [OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), CM[c].shape[1]) for c in range(3)]
    A, _, _ = OC.reduced_system(m, cbfs, 3.0 - 0.1j)
    gm = P.mesh(g.verts, g.tris, 3, 3.0 - 0.1j, partition="rcb")
    red = P.assemble_reduced(gm, P.cbf_import(gm, CM, CJ), prec)
    assert _relmax(red.export(), A) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 5e-5), (2, 5e-5), (3, 5e-5), (4, 5e-5)])
def test_reduced_cube_full_size_sampled(P, prec, tol):
    """Full-size cube (T = 3072, 32 cells) with seeded injected CBFs; blocks
    the oracle can compute on their own (Z restricted to two cells)."""
    d = W.cube_c2()
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, 32)
    Ns = np.bincount(cell)
    Ls = [14 if c % 3 else 13 for c in range(32)]
    CM, CJ = W.random_cbfs(Ns, Ls, seed=5)
    cbfs = [OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), Ls[c]) for c in range(32)]
    gm = P.mesh(g.verts, g.tris, 32, 2.5, partition="rcb")
    red = P.assemble_reduced(gm, P.cbf_import(gm, CM, CJ), prec)
    A = red.export()
    offs = np.cumsum([0] + Ls)
    nh = offs[-1]
    for (mi, ni) in [(0, 0), (3, 17), (31, 5)]:
        blocks = OC.reduced_block(m, cbfs, 2.5, mi, ni)
        rm, rn = slice(offs[mi], offs[mi + 1]), slice(offs[ni], offs[ni + 1])
        rm2, rn2 = slice(nh + offs[mi], nh + offs[mi + 1]), slice(nh + offs[ni], nh + offs[ni + 1])
        got = [A[rm, rn], A[rm, rn2], A[rm2, rn], A[rm2, rn2]]
        for gb, ob in zip(got, blocks):
            assert _relmax(gb, ob) < tol, (mi, ni)


def test_fused_equals_unfused_cube(P):
    """The fused assembly-projection kernel and the unfused path (RWG matrices in
    memory, then the tensor-core GEMMs) compute the same A: both sum the same FP32
    local entries, in different orders, and the unfused path rounds Y to split
    TF32 once more for its second GEMM where the fused kernel forms C_m^H Y in
    FP32; each lies ~2e-6 of the largest entry from the exact A, so they agree to
    5e-6.  Every entry of A is written by the fused kernel (all finite)."""
    g = W.cube(10, 0.8)
    gm = P.mesh(g.verts, g.tris, 12, 2.5 - 0.05j, partition="rcb")
    Ns = np.bincount(gm.cells(), minlength=12)
    CM, CJ = W.random_cbfs(Ns, [5 + (c * 7) % 23 for c in range(12)], seed=21)
    cb = P.cbf_import(gm, CM, CJ)
    Af = P.assemble_reduced(gm, cb, P.MIXED_FUSED).export()
    Au = P.assemble_reduced(gm, cb, P.MIXED_UNFUSED).export()
    assert np.isfinite(Af).all()
    err = _relmax(Af, Au)
    print(f"fused vs unfused: {err:.2e}")
    assert err < 5e-6


def test_build_cbfs_c1(P, c1):
    gm = _gpu_mesh(P, c1)
    cb = P.build_cbfs(gm, c1["d"]["gen"], 1e-3)
    ref = c1["ref"]["cbfs"]
    assert cb.L.tolist() == [c.L for c in ref]
    CMg, CJg = cb.export()
    for c in range(8):
        L = ref[c].L
        so = ref[c].sigma / ref[c].sigma[0]
        assert np.abs(cb.sigma[c, :L + 2] - so[:L + 2]).max() < 1e-9
        lam = ref[c].edges
        Gm = OC.rwg_gram(c1["m"], lam, lam)
        D = CMg[c].conj().T @ Gm @ CJg[c]
        sig = ref[c].sigma[:L]
        assert np.abs(D - np.diag(sig)).max() < 1e-9 * sig[0]
        # same subspaces as the oracle's CBFs (singular vectors are unique only up to unitary mixing)
        for Cg, Co in ((CMg[c], ref[c].CM), (CJg[c], ref[c].CJ)):
            Qg, _ = np.linalg.qr(Cg)
            Qo, _ = np.linalg.qr(Co)
            cosines = np.linalg.svd(Qg.conj().T @ Qo, compute_uv=False)
            assert cosines.min() > 1 - 1e-8


def test_cmp_gram_c1(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    G = red.gram()
    Go = c1["ref"]["G"]
    assert _relmax(G, Go) < 1e-12


def test_solve_fp64_c1(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    res = P.solve(red, c1["exc"], tol=TOL_SOLVE, obs=c1["obs"])
    jo = c1["ref"]["sol"].j
    assert np.linalg.norm(res.j - jo) / np.linalg.norm(jo) < 1e-7
    assert _peak_rcs_err(res.rcs.sum(-1), c1["rcs"].sum(-1)) < 1e-8
    for a, b in zip(res.iters, c1["ref"]["sol"].iters):
        assert abs(int(a) - int(b)) <= 3
    assert (res.resid <= TOL_SOLVE).all()


@pytest.mark.parametrize("prec", [1, 2, 4])
def test_solve_mixed_c1_rcs_within_1e4(P, c1, prec):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), prec)
    P.cmp_setup(red)
    res = P.solve(red, c1["exc"], tol=1e-6, obs=c1["obs"])
    err = _peak_rcs_err(res.rcs.sum(-1), c1["rcs"].sum(-1))
    jo = c1["ref"]["sol"].j
    errj = float(np.linalg.norm(res.j - jo) / np.linalg.norm(jo))
    print(f"mixed RCS error {err:.2e}, current error {errj:.2e}, iterations {res.iters.tolist()}")
    assert err < 1e-4
    assert errj < J_MIXED


def test_end_to_end_gpu_cbfs_c1(P, c1):
    """Whole GPU pipeline (own CBFs): same subspaces, so the same currents."""
    gm = _gpu_mesh(P, c1)
    cb = P.build_cbfs(gm, c1["d"]["gen"], 1e-3)
    red = P.assemble_reduced(gm, cb, P.FP64)
    P.cmp_setup(red)
    res = P.solve(red, c1["exc"], tol=TOL_SOLVE, obs=c1["obs"])
    assert _peak_rcs_err(res.rcs.sum(-1), c1["rcs"].sum(-1)) < 1e-6


def test_monostatic_matches_bistatic(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    exc = c1["exc"]
    mono = P.solve(red, exc, tol=1e-8, monostatic=True)
    bi = P.solve(red, exc, tol=1e-8, obs=exc[:, :2])
    for r in range(len(exc)):
        assert np.allclose(mono.rcs[r, 0], bi.rcs[r, r], rtol=1e-12, atol=0)


def test_no_cmp_and_noconv_status(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    res = P.solve(red, c1["exc"][:1], tol=1e-12, maxit=3, restart=3, use_cmp=False, allow_noconv=True)
    assert res.status == 5
    with pytest.raises(P.CbfmError) as ei:
        P.solve(red, c1["exc"][:1], tol=1e-6, use_cmp=True)     # cmp_setup not called
    assert ei.value.status == 1


def test_invalid_arguments(P):
    g = W.icosphere(1, 0.3)
    with pytest.raises(P.CbfmError) as ei:
        P.mesh(g.verts, g.tris, 8, 2.0 + 0.1j, partition="octant")   # active medium
    assert ei.value.status == 1
    with pytest.raises(P.CbfmError):
        P.mesh(g.verts, g.tris[:-2], 8, 2.0, partition="octant")    # open mesh


def test_device_buffers_match_host(P, c1):
    import torch
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.MIXED)
    P.cmp_setup(red)
    host = P.solve(red, c1["exc"], tol=1e-6, obs=c1["obs"])
    exc_d = torch.tensor(c1["exc"], dtype=torch.float64, device="cuda")
    obs_d = torch.tensor(c1["obs"], dtype=torch.float64, device="cuda")
    j_d = torch.zeros((2 * gm.n_edges, 3), dtype=torch.complex128, device="cuda")
    rcs_d = torch.zeros((3, len(c1["obs"]), 2), dtype=torch.float64, device="cuda")
    P.solve(red, exc_d, tol=1e-6, obs=obs_d, out_j=j_d, out_rcs=rcs_d)
    torch.cuda.synchronize()
    assert np.array_equal(j_d.cpu().numpy(), host.j)
    assert np.array_equal(rcs_d.cpu().numpy(), host.rcs)


def test_degenerate_eps1_matches_oracle(P):
    """eps_r = 1 (interior = exterior medium), the method's degenerate case:
    GPU-built CBFs end to end against the oracle pipeline."""
    g = W.icosphere(2, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    gen = W.plane_wave_set(W.fibonacci_dirs(12))
    exc = np.array([[0.4, 0.7, 0.3]])
    obs = W.bistatic_cut(10.0)
    ref = OC.run(m, cell, 8, 1.0, gen, exc, 1e-3, TOL_SOLVE, restart=1000)
    st, sp = OMo.rcs(*OMo.farfield(m, ref["sol"].j, obs))
    gm = P.mesh(g.verts, g.tris, 8, 1.0, partition="octant")
    cb = P.build_cbfs(gm, gen, 1e-3)
    red = P.assemble_reduced(gm, cb, P.FP64)
    P.cmp_setup(red)
    res = P.solve(red, exc, tol=TOL_SOLVE, obs=obs)
    assert _peak_rcs_err(res.rcs.sum(-1), st + sp) < 1e-6


# ------------------------------------------------ (G^CBF)^{-1} routine paths
def _inv_path(P, A):
    P.profile(True)
    P.profile_read(reset=True)
    X = P.gram_inverse(A)
    prof = P.profile_read(reset=True)
    P.profile(False)
    return X, prof


def test_gram_inverse_blocked_path(P):
    """Two 70 x 70 matrices (three block steps, the last of 6 columns) whose
    diagonal blocks need row exchanges inside the block (zero diagonal): the
    blocked Gauss-Jordan is kept and matches numpy's inverse."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((2, 70, 70)) + 1j * rng.standard_normal((2, 70, 70))
    for t in range(2):
        np.fill_diagonal(A[t], 0.0)
    X, prof = _inv_path(P, A)
    # the blocked form: all block steps in one cooperative launch, or one launch per step
    assert ("k_gjb_persistent" in prof or "k_gjb_inv" in prof) and "k_gj_sweep" not in prof
    for t in range(2):
        ref = np.linalg.inv(A[t])
        assert np.abs(X[t] - ref).max() < 1e-11 * np.abs(ref).max()


def test_gram_inverse_pivoted_fallback(P):
    """A leading 32 x 32 block that is singular (zero) in an invertible matrix:
    the block check fails and Gauss-Jordan with partial pivoting gives the
    inverse."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((1, 64, 64)) + 1j * rng.standard_normal((1, 64, 64))
    A[0, :32, :32] = 0.0
    assert np.linalg.cond(A[0]) < 1e6
    X, prof = _inv_path(P, A)
    assert "k_gj_sweep" in prof
    ref = np.linalg.inv(A[0])
    assert np.abs(X[0] - ref).max() < 1e-10 * np.abs(ref).max()


def test_gram_inverse_singular(P):
    A = np.zeros((1, 40, 40), np.complex128)
    A[0, :39, :39] = np.eye(39)
    with pytest.raises(P.CbfmError):
        P.gram_inverse(A)


# ------------------------------------------------------------ block GMRES
@pytest.mark.parametrize("prec,tol_rcs", [(0, 1e-8), (1, 1e-4)])
def test_block_gmres_c1(P, c1, prec, tol_rcs):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), prec)
    P.cmp_setup(red)
    res = P.solve(red, c1["exc"], tol=TOL_SOLVE if prec == 0 else 1e-6, obs=c1["obs"], solver=P.BLOCK)
    assert _peak_rcs_err(res.rcs.sum(-1), c1["rcs"].sum(-1)) < tol_rcs
    jo = c1["ref"]["sol"].j
    errj = float(np.linalg.norm(res.j - jo) / np.linalg.norm(jo))
    print(f"block GMRES prec {prec}: current error {errj:.2e}")
    assert errj < (1e-7 if prec == 0 else J_MIXED)
    assert (res.iters >= 1).all()


def test_block_matches_per_rhs_many_and_dependent(P, c1):
    """40 right-hand sides, two of them repeated (the first block is rank deficient):
    block and per-right-hand-side GMRES reach the same solutions."""
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    exc = W.plane_wave_set(W.fibonacci_dirs(19))
    exc = np.vstack([exc, exc[:2]])
    a = P.solve(red, exc, tol=1e-10, solver=P.PER_RHS)
    b = P.solve(red, exc, tol=1e-10, solver=P.BLOCK)
    err = np.linalg.norm(a.j - b.j, axis=0) / np.linalg.norm(a.j, axis=0)
    assert err.max() < 1e-7
    assert np.allclose(b.j[:, -2:], b.j[:, :2], rtol=0, atol=1e-9 * np.abs(b.j).max())


def test_block_nearly_dependent_rhs(P, c1):
    """Plane waves 1e-4 rad apart give a right-hand-side block of condition
    ~5e4: one Cholesky QR pass leaves it about u kappa^2 ~ 1e-7 away from
    orthonormal, far above the 1e-12 under which the second pass is skipped,
    so both passes run (while the smallest pivot, ~3e-10 of the scaled Gram
    diagonal, stays far above the 1e-14 drop).  Block and per-right-hand-side
    GMRES reach the same solutions."""
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    exc = W.plane_wave_set(W.fibonacci_dirs(6))
    near = exc.copy()
    near[:, 0] += 1e-4
    exc = np.vstack([exc, near])
    v = OMo.rhs(c1["m"], exc)
    s = np.linalg.svd(v / np.linalg.norm(v, axis=0), compute_uv=False)
    assert 1e4 < s[0] / s[-1] < 1e6
    a = P.solve(red, exc, tol=1e-10, solver=P.PER_RHS)
    b = P.solve(red, exc, tol=1e-10, solver=P.BLOCK)
    err = np.linalg.norm(a.j - b.j, axis=0) / np.linalg.norm(a.j, axis=0)
    assert err.max() < 1e-7


def test_block_single_rhs_is_gmres(P, c1):
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    a = P.solve(red, c1["exc"][:1], tol=1e-10, solver=P.PER_RHS)
    b = P.solve(red, c1["exc"][:1], tol=1e-10, solver=P.BLOCK)
    assert np.linalg.norm(a.j - b.j) / np.linalg.norm(a.j) < 1e-7
    assert abs(int(a.iters[0]) - int(b.iters[0])) <= 2


def test_block_restart_small_basis(P, c1):
    """A basis cap far below the saturation size forces restarts; the result is unchanged."""
    gm = _gpu_mesh(P, c1)
    red = P.assemble_reduced(gm, _inject(P, gm, c1["ref"]["cbfs"]), P.FP64)
    P.cmp_setup(red)
    a = P.solve(red, c1["exc"], tol=1e-9, solver=P.PER_RHS)
    b = P.solve(red, c1["exc"], tol=1e-9, solver=P.BLOCK, restart=180, maxit=2000)
    assert np.linalg.norm(a.j - b.j) / np.linalg.norm(a.j) < 1e-6


@pytest.mark.parametrize("solver", [0, 1])
def test_solve_odd_half_order_injected_cbfs(P, solver):
    """A reduced system whose halves have odd order (n_h = 15) runs the
    Gauss-Jordan inverse of G^CBF over an odd number of ping-pong sweeps;
    both GMRES variants must reach the oracle's solution (GMRES with the
    Gram matrix applied by an LU solve) on a lossy medium."""
    g = W.icosphere(1, 0.4)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, 3)
    Ns = np.bincount(cell)
    Ls = [5, 4, 6]
    CM, CJ = W.random_cbfs(Ns, Ls, seed=21)
    cbfs = [OC.CellCBF(np.nonzero(cell == c)[0], CM[c], CJ[c], np.ones(1), Ls[c]) for c in range(3)]
    eps = 3.0 - 0.1j
    A, CJM, CMJ = OC.reduced_system(m, cbfs, eps)
    G = OC.cbf_gram(m, cbfs)
    exc = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 0.5], [2.2, 5.0, 1.3]])
    b = CJM.conj().T @ OMo.rhs(m, exc)
    ref = OC.solve_reduced(A, G, CMJ, b, 1e-12, restart=200, maxit=400)
    gm = P.mesh(g.verts, g.tris, 3, eps, partition="rcb")
    red = P.assemble_reduced(gm, P.cbf_import(gm, CM, CJ), P.FP64)
    assert red.n == 30
    P.cmp_setup(red)
    res = P.solve(red, exc, tol=1e-12, maxit=400, solver=solver)
    assert np.linalg.norm(res.j - ref.j) / np.linalg.norm(ref.j) < 1e-8
