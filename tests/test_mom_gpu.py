"""GPU parity of the comparison arrangements of Sec. IV against the FP64 oracle:
the conventional MoM (PMCHWT matrix of Eq. (Z) over all RWG functions, T-diagonal
arrangement with the diagonal preconditioner, Eq. (MoM_T)) and the T-diagonal
CBFM of Eq. (cbfm_Tdiag).

Tolerances: the RWG matrix per block (Ks, Ta, Tb, each normalised by its own
largest entry, since Ta and Tb differ in scale by eta^2) <= 1e-11 on the FP64
path and <= 2e-5 on the mixed path (FP32 far-pair quadrature).  Currents against
a dense solve, with GMRES stopped at a relative residual of 1e-10: the oracle's
own GMRES lands at 2.6e-8 (MoM, T-diagonal + D) and 2.5e-7 (T-diagonal CBFM,
whose reduced matrix has condition number ~1e7 without the CMP), so the bounds
are 3e-7 and 2e-6; peak-normalised RCS <= 1e-7; mixed MoM RCS <= 1e-4.  The
iteration counts of the GPU GMRES (CGS2 Arnoldi) and the oracle's (MGS) agree
within 2 at 1e-6 on the FP64 path.
"""
import math

import numpy as np
import pytest

import workloads as W
from conftest import golden
from oracle import cbfm as OC, mesh as OM, mom as OMo

pytestmark = pytest.mark.gpu

EPS = 3.0 - 0.1j
TOL = 1e-10
EXC = np.array([[0.0, 0.0, 0.0], [1.2, 0.7, 0.4], [2.5, 4.0, math.pi / 2]])


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
def sph():
    """The 320-triangle sphere (N = 960) with the oracle's MoM matrix and solution."""
    g = W.icosphere(2, 1.0 / 6.0)
    m = OM.build_rwg(g.verts, g.tris)
    Z = OMo.pmchwt_matrix(m, EPS)
    v = OMo.rhs(m, EXC)
    j = np.linalg.solve(Z, v)
    obs = W.bistatic_cut(2.0)
    st, sp = OMo.rcs(*OMo.farfield(m, j, obs))
    _, its = OC.solve_tdiag(Z, v, 1e-6, restart=1000, maxit=5000, jacobi=True)
    return dict(g=g, m=m, Z=Z, v=v, j=j, obs=obs, rcs=st + sp, its6=its)


def _blocks_err(G, Z, ne):
    out = []
    for rs, cs in ((slice(0, ne), slice(0, ne)), (slice(0, ne), slice(ne, None)), (slice(ne, None), slice(0, ne)),
                   (slice(ne, None), slice(ne, None))):
        out.append(float(np.abs(G[rs, cs] - Z[rs, cs]).max() / np.abs(Z[rs, cs]).max()))
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_mom_matrix_parity(P, sph, prec, tol):
    gm = P.mesh(sph["g"].verts, sph["g"].tris, 1, EPS)
    red = P.assemble_mom(gm, prec)
    assert red.n == 2 * sph["m"].ne == 960
    errs = _blocks_err(red.export(), sph["Z"], sph["m"].ne)
    print(f"MoM matrix ({prec}) block errors {['%.1e' % e for e in errs]}")
    assert max(errs) < tol


@pytest.mark.parametrize("solver", [0, 1])
def test_mom_tdiag_jacobi_solve(P, sph, solver):
    gm = P.mesh(sph["g"].verts, sph["g"].tris, 1, EPS)
    red = P.assemble_mom(gm, P.FP64)
    P.tdiag_setup(red, jacobi=True)
    res = P.solve(red, EXC, tol=TOL, maxit=5000, restart=1000, precond=P.PC_TDIAG, obs=sph["obs"], solver=solver)
    assert np.linalg.norm(res.j - sph["j"]) / np.linalg.norm(sph["j"]) < 3e-7
    assert float(np.abs(res.rcs.sum(-1) - sph["rcs"]).max() / sph["rcs"].max()) < 1e-7
    if solver == 0:
        r6 = P.solve(red, EXC, tol=1e-6, maxit=5000, restart=1000, precond=P.PC_TDIAG, want_j=False)
        print("MoM T-diag + D iterations (GPU, oracle):", r6.iters.tolist(), sph["its6"])
        for a, b in zip(r6.iters, sph["its6"]):
            assert abs(int(a) - int(b)) <= 2


def test_mom_mixed_rcs(P, sph):
    gm = P.mesh(sph["g"].verts, sph["g"].tris, 1, EPS)
    red = P.assemble_mom(gm, P.MIXED)
    P.tdiag_setup(red, jacobi=True)
    res = P.solve(red, EXC, tol=1e-6, maxit=5000, restart=1000, precond=P.PC_TDIAG, obs=sph["obs"])
    err = float(np.abs(res.rcs.sum(-1) - sph["rcs"]).max() / sph["rcs"].max())
    print(f"mixed MoM RCS error {err:.2e}")
    assert err < 1e-4


def test_mom_kdiag_unpreconditioned(P, sph):
    """The MoM handle also runs the K-diagonal order of Eq. (Z) without a preconditioner."""
    gm = P.mesh(sph["g"].verts, sph["g"].tris, 1, EPS)
    red = P.assemble_mom(gm, P.FP64)
    res = P.solve(red, EXC[:1], tol=TOL, maxit=5000, restart=1000, precond=P.PC_NONE)
    jo = sph["j"][:, :1]
    assert np.linalg.norm(res.j - jo) / np.linalg.norm(jo) < 3e-7


def test_mom_refusals(P, sph):
    gm = P.mesh(sph["g"].verts, sph["g"].tris, 1, EPS)
    red = P.assemble_mom(gm, P.FP64)
    with pytest.raises(P.CbfmError) as ei:
        P.solve(red, EXC[:1], precond=P.PC_TDIAG)      # tdiag_setup not called
    assert ei.value.status == 1
    with pytest.raises(P.CbfmError) as ei:
        P.cmp_setup(red)                               # RWG-only CMP is singular
    assert ei.value.status == 1
    with pytest.raises(P.CbfmError) as ei:
        P.solve(red, EXC[:1], precond=7)
    assert ei.value.status == 1


def _table1_waves():
    t = golden("sphere_table1_waves")
    th = np.deg2rad(t["theta_start_deg"] + np.arange(t["n_theta"]) * t["theta_step_deg"])
    ph = np.deg2rad(t["phi_start_deg"] + np.arange(t["n_phi"]) * t["phi_step_deg"])
    return W.plane_wave_set(np.array([(a, b) for a in th for b in ph]))


@pytest.fixture(scope="module")
def pair():
    """Two disjoint lambda/3 spheres (Sec. IV-A), one cell each, Table I waves,
    L = 70 kept per sphere (N^CBF = 280), eps_r = 1: GMRES stops well below the
    dimension, so the iteration counts tell the arrangements apart."""
    g = W.sphere_array(2, 1, 1, 0.5, level=2, radius=1.0 / 6.0)
    m = OM.build_rwg(g.verts, g.tris)
    cell = (m.edges[:, 0] >= g.nv // 2).astype(np.int32)
    exc = np.array([[0.0, 0.0, 0.0], [1.1, 0.4, math.pi / 2]])
    L = golden("sphere_singular_value_groups")["kept_singular_values"]
    ref = OC.run(m, cell, 2, 1.0, _table1_waves(), exc, 1e-12, TOL, restart=1000, Lmax=L)
    jd = ref["CMJ"] @ np.linalg.solve(ref["A"], ref["b"])
    _, its6 = OC.solve_tdiag(ref["A"], ref["b"], 1e-6, restart=1000, maxit=5000, jacobi=False)
    _, its4 = OC.solve_tdiag(ref["A"], ref["b"], 1e-4, restart=1000, maxit=5000, jacobi=False)
    return dict(g=g, m=m, cell=cell, exc=exc, ref=ref, jd=jd, its6=its6, its4=its4)


@pytest.mark.parametrize("prec", [0, 1])
def test_tdiag_cbfm(P, pair, prec):
    """Eq. (cbfm_Tdiag): the reduced matrix with its column halves exchanged, no
    preconditioner; the same currents as the K-diagonal CBFM."""
    gm = P.mesh(pair["g"].verts, pair["g"].tris, 2, 1.0, edge_cell=pair["cell"])
    cbfs = pair["ref"]["cbfs"]
    cb = P.cbf_import(gm, [c.CM for c in cbfs], [c.CJ for c in cbfs])
    red = P.assemble_reduced(gm, cb, prec)
    assert red.n == 280
    P.tdiag_setup(red, jacobi=False)
    exc = pair["exc"]
    if prec == 0:
        jd = pair["jd"]
        res = P.solve(red, exc, tol=TOL, maxit=5000, restart=1000, precond=P.PC_TDIAG)
        assert np.linalg.norm(res.j - jd) / np.linalg.norm(jd) < 2e-6
        r6 = P.solve(red, exc, tol=1e-6, maxit=5000, restart=1000, precond=P.PC_TDIAG, want_j=False)
        print("T-diagonal CBFM iterations to 1e-6 (GPU, oracle):", r6.iters.tolist(), pair["its6"])
        for a, b in zip(r6.iters, pair["its6"]):
            assert abs(int(a) - int(b)) <= 2
    else:
        # complex64 operator without the CMP (condition number ~1e7): the residual curve
        # leaves the FP64 one before 1e-4 (measured 29 vs 20 and 54 vs 54 iterations), so
        # the mixed path is held to convergence and a bound, not to the FP64 count
        r4 = P.solve(red, exc, tol=1e-4, maxit=5000, restart=1000, precond=P.PC_TDIAG, want_j=False)
        print("mixed T-diagonal CBFM iterations to 1e-4 (GPU, oracle):", r4.iters.tolist(), pair["its4"])
        assert r4.status == 0 and (r4.resid <= 1e-4).all()
        for a, b in zip(r4.iters, pair["its4"]):
            assert int(a) <= 2 * int(b) + 2
