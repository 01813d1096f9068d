"""The paper's 4 x 4 x 2 sphere array at full size (Sec. IV-A-2): 32 identical
disjoint spheres of radius lambda/6 (960 unknowns each, N = 30 720), one cell
per sphere, Table I generating waves with the 70 singular values of the groups
l = 1..5 kept (N^CBF = 4480), FP64 path, excitation from theta = 0,
theta-polarised.

* At eps_r = 3 GMRES with the CMP reaches 1e-6 while the two arrangements
  without it (K-diagonal CBFM, T-diagonal CBFM) do not within 1000 iterations
  (the paper's statement for this array), in fewer than 40 iterations as the
  paper reports (measured 34 with the spheres' centres lambda/2 apart, the
  figures' "15 mm space" read as the centre spacing of spheres of radius 5 mm
  at lambda = 30 mm; 24 when those 15 mm are read as the gap).
* The CMP-vs-K-diagonal table over eps_r = 1, 3, 6: iterations to 1e-4 with
  the CMP against the K-diagonal CBFM without it (the paper: 1/70 at eps_r = 1
  to 1/5 at eps_r = 6) and against the T-diagonal CBFM of Eq. (cbfm_Tdiag);
  each at least four times the CMP's.
* The RMSE of Eq. (RMSE) between the CBFM and the conventional GPU MoM
  (Eq. (MoM_T), same quadrature) bistatic RCS at eps_r = 3 (the paper:
  -39.98 dB) below -30 dB on the phi = 0 and 90 degree cuts.
"""
import math

import numpy as np
import pytest

import workloads as W
from conftest import golden

pytestmark = pytest.mark.gpu

L_KEPT = golden("sphere_singular_value_groups")["kept_singular_values"]   # 70
SPACING = 0.5
EXC_MINUS_Z = np.array([[0.0, 0.0, 0.0]])


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


def _table1_waves():
    t = golden("sphere_table1_waves")
    th = np.deg2rad(t["theta_start_deg"] + np.arange(t["n_theta"]) * t["theta_step_deg"])
    ph = np.deg2rad(t["phi_start_deg"] + np.arange(t["n_phi"]) * t["phi_step_deg"])
    return W.plane_wave_set(np.array([(a, b) for a in th for b in ph]))


def _gpu_array(P, g, nbody, eps):
    edges, _ = P.mesh_edges(g.verts, g.tris, 1)
    nvb = g.nv // nbody
    cell = (edges[:, 0] // nvb).astype(np.int32)
    assert np.array_equal(cell, edges[:, 1] // nvb)
    return P.mesh(g.verts, g.tris, nbody, eps, edge_cell=cell)


def _rmse_db(sc, sm):
    return 10.0 * math.log10(math.sqrt(float(np.mean((sc - sm) ** 2))) / float(sm.max() - sm.min()))


@pytest.fixture(scope="module")
def full_array(P):
    g = W.sphere_array(4, 4, 2, SPACING, level=2, radius=1.0 / 6.0)
    obs = W.bistatic_cut(1.0)
    iters, rcs3 = {}, None
    for eps in (1.0, 3.0, 6.0):
        gm = _gpu_array(P, g, 32, eps)
        cb = P.build_cbfs(gm, _table1_waves(), 1e-12, lmax=L_KEPT)
        assert cb.L.tolist() == [L_KEPT] * 32
        red = P.assemble_reduced(gm, cb, P.FP64)
        assert red.n == 4480
        P.cmp_setup(red)
        c6 = P.solve(red, EXC_MINUS_Z, tol=1e-6, maxit=1000, restart=1000, obs=obs if eps == 3.0 else None,
                     want_j=False)
        if eps == 3.0:   # without the CMP, to 1e-6 (K-diagonal here, T-diagonal below)
            n6 = P.solve(red, EXC_MINUS_Z, tol=1e-6, maxit=1000, restart=1000, use_cmp=False, want_j=False,
                         allow_noconv=True)
        c4 = P.solve(red, EXC_MINUS_Z, tol=1e-4, maxit=1000, restart=1000, want_j=False)
        n4 = P.solve(red, EXC_MINUS_Z, tol=1e-4, maxit=2000, restart=1000, use_cmp=False, want_j=False,
                     allow_noconv=True)
        P.tdiag_setup(red, jacobi=False)
        t4 = P.solve(red, EXC_MINUS_Z, tol=1e-4, maxit=2000, restart=1000, precond=P.PC_TDIAG, want_j=False,
                     allow_noconv=True)
        iters[eps] = (int(c6.iters[0]), int(c4.iters[0]), int(n4.iters[0]), int(t4.iters[0]))
        if eps == 3.0:
            rcs3 = c6.rcs[0].sum(-1)
            t6 = P.solve(red, EXC_MINUS_Z, tol=1e-6, maxit=1000, restart=1000, precond=P.PC_TDIAG, want_j=False,
                         allow_noconv=True)
            no_cmp_1e6 = (int(n6.status), int(t6.status))
        red.free()
        cb.free()
    gm = _gpu_array(P, g, 32, 3.0)
    mo = P.assemble_mom(gm, P.FP64)
    assert mo.n == 30720
    P.tdiag_setup(mo, jacobi=True)
    rm = P.solve(mo, EXC_MINUS_Z, tol=1e-6, maxit=5000, restart=1000, precond=P.PC_TDIAG, obs=obs, want_j=False)
    mo.free()
    nth = len(obs) // 2
    sm = rm.rcs[0].sum(-1)
    rmse = [_rmse_db(rcs3[k * nth:(k + 1) * nth], sm[k * nth:(k + 1) * nth]) for k in range(2)]
    print("array 4x4x2 GMRES iterations (CMP 1e-6, CMP 1e-4, K-diagonal 1e-4, T-diagonal 1e-4):", iters)
    print(f"array 4x4x2 eps 3: CBFM vs MoM RCS RMSE {rmse[0]:.2f} dB (phi 0), {rmse[1]:.2f} dB (phi 90); "
          f"MoM T-diagonal+D GMRES iterations {int(rm.iters[0])}")
    print("array 4x4x2 eps 3 without CMP to 1e-6 (status K-diagonal, T-diagonal; 5 = not reached in 1000):",
          no_cmp_1e6)
    return iters, rmse, no_cmp_1e6


def test_full_array_cmp_reaches_1e6_at_eps3_and_the_others_do_not(full_array):
    iters, _, no_cmp = full_array
    assert iters[3.0][0] < 40
    assert no_cmp == (5, 5)       # CBFM_ENOCONV: 1e-6 not reached in 1000 iterations without the CMP


@pytest.mark.parametrize("eps", [1.0, 3.0, 6.0])
def test_full_array_cmp_vs_kdiag_and_tdiag(full_array, eps):
    c6, c4, n4, t4 = full_array[0][eps]
    assert c4 >= 1
    assert n4 < 0 or n4 >= 4 * c4
    assert t4 < 0 or t4 >= 4 * c4


def test_full_array_rmse_vs_mom(full_array):
    assert max(full_array[1]) < -30.0
