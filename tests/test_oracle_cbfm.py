"""Pins for the oracle's CBF generation, reduced system, CMP and GMRES.

Paper-given facts used as pins:
* duality (C^M)^H G_m C^J = Sigma_L, diagonal and positive (Eq. (CBF_sv));
* one cell covering the lambda/3 sphere with the Table I waves: normalised
  singular values of G'_m fall in groups of 2(2l+1) = 6, 10, 14, 18, 22
  (Sec. IV-A-1), whatever eps_r;
* N = 960 unknowns for that 320-triangle sphere (Sec. IV-A-1);
* identical cells have identical singular values (Sec. IV-B);
* G^CBF is diagonal when no connected boundary is divided (Sec. III-C);
* CMP needs far fewer GMRES iterations than the unpreconditioned system;
* the single-cell CBFM with L = 70 reproduces the MoM RCS closely (Sec. IV-A).

The printed values (Table I's wave grid; the group sizes, L = 70, N^CBF = 140 and
N = 960 of Sec. IV-A-1) live in tests/golden/ with their citations.
"""
import math

import numpy as np
import pytest

import workloads as W
from conftest import golden
from oracle import cbfm, mesh as OM, mom


def _table1_waves():
    t = golden("sphere_table1_waves")
    th = np.deg2rad(t["theta_start_deg"] + np.arange(t["n_theta"]) * t["theta_step_deg"])
    ph = np.deg2rad(t["phi_start_deg"] + np.arange(t["n_phi"]) * t["phi_step_deg"])
    assert t["polarisations"] == ["theta", "phi"]
    return W.plane_wave_set(np.array([(a, b) for a in th for b in ph]))


@pytest.fixture(scope="module")
def small_sphere():
    g = W.icosphere(2, 1.0 / 6.0)
    return OM.build_rwg(g.verts, g.tris)


def test_unknown_count(small_sphere):
    assert 2 * small_sphere.ne == golden("sphere_singular_value_groups")["unknowns"]


@pytest.mark.parametrize("eps", [1.0, 4.0])
def test_singular_value_groups(small_sphere, eps):
    m = small_sphere
    gv = golden("sphere_singular_value_groups")
    assert gv["group_ends"] == np.cumsum(gv["group_sizes"]).tolist()
    assert gv["group_sizes"] == [2 * (2 * l + 1) for l in range(1, 6)]
    assert gv["n_cbf"] == 2 * gv["kept_singular_values"]
    kept = gv["kept_singular_values"]
    cb = cbfm.primary_cbfs(m, np.zeros(m.ne, np.int32), 1, eps, _table1_waves(), 1e-3, Lmax=kept)
    s = cb[0].sigma / cb[0].sigma[0]
    gaps = s[:kept + 1] / s[1:kept + 2]
    top5 = sorted((np.argsort(-gaps)[:5] + 1).tolist())
    assert top5 == gv["group_ends"]


def test_duality_and_single_cell_accuracy(small_sphere):
    m = small_sphere
    exc = np.array([[0.0, 0.0, 0.0], [0.7, 0.3, 0.5]])
    R = cbfm.run(m, np.zeros(m.ne, np.int32), 1, 3.0, _table1_waves(), exc, 1e-3, 1e-8,
                  Lmax=golden("sphere_singular_value_groups")["kept_singular_values"])
    c = R["cbfs"][0]
    Gm = cbfm.rwg_gram(m, c.edges, c.edges)
    D = c.CM.conj().T @ Gm @ c.CJ
    assert np.abs(D - np.diag(c.sigma[:c.L])).max() < 1e-12 * c.sigma[0]
    jm = mom.solve_mom(m, 3.0, exc)
    obs = W.bistatic_cut(2.0)
    st, sp = mom.rcs(*mom.farfield(m, R["sol"].j, obs))
    mt, mp = mom.rcs(*mom.farfield(m, jm, obs))
    for i in range(2):
        assert mom.rmse_db((st + sp)[i], (mt + mp)[i]) < -35.0
    # the reduced-system residual is met
    for i in range(2):
        x = R["sol"].jcbf[:, i]
        assert np.linalg.norm(R["A"] @ x - R["b"][:, i]) <= 1.01e-8 * np.linalg.norm(R["b"][:, i])


def test_disjoint_cells_diagonal_gram_and_identical_sigma():
    g = W.sphere_array(2, 1, 1, 0.5, level=1, radius=1.0 / 6.0)
    m = OM.build_rwg(g.verts, g.tris)
    # one cell per sphere: vertices of body 0 come first
    nv_body = g.nv // 2
    cell = (m.edges[:, 0] >= nv_body).astype(np.int32)
    gen = W.plane_wave_set(W.fibonacci_dirs(20))
    cb = cbfm.primary_cbfs(m, cell, 2, 3.0, gen, 1e-4)
    assert cb[0].L == cb[1].L
    assert np.abs(cb[0].sigma - cb[1].sigma).max() < 1e-10 * cb[0].sigma[0]
    G = cbfm.cbf_gram(m, cb)
    L0, L1 = cb[0].L, cb[1].L
    n = L0 + L1
    # J-tested half: -Sigma_L; M-tested half: +Sigma_L; cross-cell blocks exactly 0
    assert np.abs(G[:L0, L0:n]).max() == 0.0 and np.abs(G[n:n + L0, n + L0:]).max() == 0.0
    assert np.abs(G[:n, n:]).max() == 0.0
    assert np.abs(G[:L0, :L0] + np.diag(cb[0].sigma[:L0])).max() < 1e-12 * cb[0].sigma[0]
    assert np.abs(G[n:n + L0, n:n + L0] - np.diag(cb[0].sigma[:L0])).max() < 1e-12 * cb[0].sigma[0]


@pytest.mark.parametrize("eps", [1.0, 4.0])
def test_cmp_reduces_iterations(small_sphere, eps):
    m = small_sphere
    R = cbfm.run(m, np.zeros(m.ne, np.int32), 1, eps, _table1_waves(), np.array([[0.0, 0.0, 0.0]]),
                 1e-3, 1e-6, restart=1000,
                 Lmax=golden("sphere_singular_value_groups")["kept_singular_values"])
    nocmp = cbfm.solve_reduced(R["A"], R["G"], R["CMJ"], R["b"], 1e-6, restart=1000, use_cmp=False)
    assert R["sol"].iters[0] <= 0.6 * nocmp.iters[0]
    # both reach the same solution of A x = b
    assert np.linalg.norm(R["sol"].jcbf - nocmp.jcbf) < 2e-3 * np.linalg.norm(nocmp.jcbf)


def test_cmp_on_divided_sphere():
    g = W.icosphere(2, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    R = cbfm.run(m, cell, 8, 4.0, W.plane_wave_set(W.fibonacci_dirs(12)), np.array([[0.0, 0.0, 0.0]]),
                 1e-3, 1e-6, restart=1000)
    nocmp = cbfm.solve_reduced(R["A"], R["G"], R["CMJ"], R["b"], 1e-6, restart=1000, use_cmp=False)
    assert R["sol"].iters[0] < nocmp.iters[0]
    G = R["G"]
    assert np.abs(G - np.diag(np.diag(G))).max() > 1e-3 * np.abs(np.diag(G)).max()   # not diagonal


def test_cbf_gram_halves_are_negative_adjoints():
    # Gf = <n x f_i, f_j> is real and antisymmetric, so (C^M)^H Gf C^J = -((C^J)^H Gf C^M)^H
    # (Eq. (CBF_Gram_matrix)); the GPU path inverts one half of G^CBF and takes the other's
    # inverse as minus the adjoint.  Checked on an octant-divided sphere with coupled cells.
    g = W.icosphere(2, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    cb = cbfm.primary_cbfs(m, cell, 8, 4.0, W.plane_wave_set(W.fibonacci_dirs(12)), 1e-3)
    G = cbfm.cbf_gram(m, cb)
    nh = G.shape[0] // 2
    g1, g2 = G[:nh, :nh], G[nh:, nh:]
    assert np.abs(g1).max() > 0 and np.abs(G[:nh, nh:]).max() == 0.0 and np.abs(G[nh:, :nh]).max() == 0.0
    assert np.abs(g1 - np.diag(np.diag(g1))).max() > 1e-3 * np.abs(g1).max()   # cells coupled
    assert np.abs(g2 + g1.conj().T).max() < 1e-13 * np.abs(g1).max()
    assert np.abs(np.linalg.inv(g2) + np.linalg.inv(g1).conj().T).max() < 1e-9 * np.abs(np.linalg.inv(g1)).max()


def test_gmres_against_direct_solve():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    P = np.diag(1.0 / (1.0 + rng.random(n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = cbfm.gmres(lambda z: A @ z, b, 1e-12, 1000, 1000, lambda z: P @ z)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
    assert it <= n
    # restarted: still converges, monotone residual
    A2 = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2 * n)
    x2, it2, h2 = cbfm.gmres(lambda z: A2 @ z, b, 1e-10, 10, 2000)
    assert np.linalg.norm(x2 - np.linalg.solve(A2, b)) < 1e-8 * np.linalg.norm(x2)
    assert it2 > 10                                  # it really restarted
    assert all(h2[i + 1] <= h2[i] * (1 + 1e-12) for i in range(len(h2) - 1) if (i + 1) % 11 != 0)


def test_reduced_block_matches_dense_definition():
    g = W.icosphere(1, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    cb = cbfm.primary_cbfs(m, cell, 8, 2.0, W.plane_wave_set(W.fibonacci_dirs(8)), 1e-3)
    A, _, _ = cbfm.reduced_system(m, cb, 2.0)
    offs = np.cumsum([0] + [c.L for c in cb])
    n = offs[-1]
    for (mi, ni) in [(0, 0), (2, 5), (7, 1)]:
        a11, a12, a21, a22 = cbfm.reduced_block(m, cb, 2.0, mi, ni)
        rm, rn = slice(offs[mi], offs[mi + 1]), slice(offs[ni], offs[ni + 1])
        rm2, rn2 = slice(n + offs[mi], n + offs[mi + 1]), slice(n + offs[ni], n + offs[ni + 1])
        sc = np.abs(A).max()
        assert np.abs(A[rm, rn] - a11).max() < 1e-12 * sc
        assert np.abs(A[rm, rn2] - a12).max() < 1e-12 * sc
        assert np.abs(A[rm2, rn] - a21).max() < 1e-12 * sc
        assert np.abs(A[rm2, rn2] - a22).max() < 1e-12 * sc
