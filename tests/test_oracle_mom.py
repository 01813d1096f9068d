"""Physics pins for the oracle's PMCHWT MoM (operators, RHS, far field).

* Mie series self-checks (optical theorem, Rayleigh limit, m -> 1);
* MoM vs Mie for the eps_r = 4, radius 0.3 sphere: error falls under mesh
  refinement (discretisation pin for operator signs and both media);
* eps_r = 1 transparency: no scattered field (sign convention of J, M, T);
* Galerkin symmetry of Ks, Ta, Tb (paper Eqs. (K), (T) with test = trial);
* discrete bistatic reciprocity of the conventional MoM;
* RWG Gram matrix: centroid closed form, antisymmetry, singular on a closed
  surface (paper Sec. II-C).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cbfm, mesh as OM, mie, mom


def _rwg(g):
    return OM.build_rwg(g.verts, g.tris)


def test_mie_optical_theorem_and_limits():
    x = 1.885
    a, b = mie.mie_coefficients(x, 2.0)
    qe, qs = mie.efficiencies(x, a, b)
    assert abs(qe - qs) < 1e-12 * qs                       # lossless: Q_ext = Q_sca
    S1, S2 = mie.amplitudes(a, b, np.array([0.0]))
    assert abs(4.0 / x ** 2 * S1[0].real - qe) < 1e-12    # optical theorem
    # integrated scattered power equals Q_sca
    th, w = np.polynomial.legendre.leggauss(200)
    th = 0.5 * math.pi * (th + 1)
    w = 0.5 * math.pi * w
    S1, S2 = mie.amplitudes(a, b, th)
    qint = 1.0 / x ** 2 * np.sum(w * (np.abs(S1) ** 2 + np.abs(S2) ** 2) * np.sin(th))
    assert abs(qint - qs) < 1e-10 * qs
    # Rayleigh limit of the backscatter cross-section
    r = 0.002
    sb = mie.sphere_rcs(r, 4.0, np.array([[0.0, 0.0]]))[0][0]
    k = 2 * math.pi
    ray = 4 * math.pi * k ** 4 * r ** 6 * abs((4 - 1) / (4 + 2)) ** 2
    assert abs(sb - ray) < 1e-3 * ray
    # m = 1: nothing scatters
    a1, b1 = mie.mie_coefficients(1.0, 1.0)
    assert np.abs(a1).max() < 1e-14 and np.abs(b1).max() < 1e-14


@pytest.mark.slow
def test_mom_converges_to_mie():
    obs = W.bistatic_cut(2.0)
    mt, mp = mie.sphere_rcs(0.3, 4.0, obs)
    errs = []
    for lvl in (2, 3):
        m = _rwg(W.icosphere(lvl, 0.3))
        j = mom.solve_mom(m, 4.0, np.array([[0.0, 0.0, 0.0]]))
        st, sp = mom.rcs(*mom.farfield(m, j, obs))
        errs.append(mom.rmse_db((st + sp)[0], mt + mp))
    assert errs[0] < -13.0
    assert errs[1] < -19.0
    assert errs[1] < errs[0] - 4.0


def test_mom_small_sphere_vs_mie():
    """Electrically small sphere: MoM backscatter within the polyhedron's
    volume deficit of the Mie value."""
    g = W.icosphere(2, 0.1)
    m = _rwg(g)
    obs = np.array([[0.0, 0.0], [math.pi / 2, 0.0], [math.pi / 2, math.pi / 2]])
    j = mom.solve_mom(m, 4.0, np.array([[0.0, 0.0, 0.0]]))
    st, sp = mom.rcs(*mom.farfield(m, j, obs))
    mt, mp = mie.sphere_rcs(0.1, 4.0, obs)
    assert abs(st[0, 0] - mt[0]) < 0.08 * mt[0]
    assert abs(sp[0, 2] - mp[2]) < 0.08 * mp[2]
    assert sp[0, 0] < 1e-12 * st[0, 0]                      # no cross-pol in the x-z plane


def test_transparency_eps1():
    m = _rwg(W.icosphere(2, 0.3))
    j = mom.solve_mom(m, 1.0, np.array([[0.4, 0.7, 0.3]]))
    obs = W.bistatic_cut(10.0)
    st, sp = mom.rcs(*mom.farfield(m, j, obs))
    # compare with the same currents radiating with the wrong sign of T
    k1, eta1, k2, eta2 = mom.media(4.0)
    Ks, Ta, Tb = mom.pmchwt_blocks(m, 1.0)
    Zbad = np.block([[Ks, -Ta], [-Tb, Ks]])
    jb = np.linalg.solve(Zbad, mom.rhs(m, np.array([[0.4, 0.7, 0.3]])))
    sb, spb = mom.rcs(*mom.farfield(m, jb, obs))
    assert (st + sp).max() < 1e-5 * (sb + spb).max()
    assert (st + sp).max() < 1e-5


def test_galerkin_symmetry():
    m = _rwg(W.icosphere(2, 0.3))
    Ks, Ta, Tb = mom.pmchwt_blocks(m, 3.0 - 0.1j)
    for X in (Ks, Ta, Tb):
        assert np.abs(X - X.T).max() < 1e-13 * np.abs(X).max()


def test_reciprocity():
    m = _rwg(W.icosphere(2, 0.3))
    Z = mom.pmchwt_matrix(m, 4.0)
    waves = np.array([[0.3, 0.2, 0.4], [2.1, 4.0, 1.1]])
    j = np.linalg.solve(Z, mom.rhs(m, waves))

    def pol(th, ph, psi):
        thh = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
        phh = np.array([-math.sin(ph), math.cos(ph), 0.0])
        return math.cos(psi) * thh, math.sin(psi) * phh

    # p_s . F(observe at d_s; wave from d_i, p_i) == p_i . F(observe at d_i; wave from d_s, p_s)
    (ti, pi_, qi), (ts, ps, qs) = waves
    Fth, Fph = mom.farfield(m, j, np.array([[ts, ps], [ti, pi_]]))
    a1 = math.cos(qs) * Fth[0, 0] + math.sin(qs) * Fph[0, 0]
    a2 = math.cos(qi) * Fth[1, 1] + math.sin(qi) * Fph[1, 1]
    assert abs(a1 - a2) < 1e-10 * abs(a1)


def test_rwg_gram():
    m = _rwg(W.icosphere(1, 0.5))
    G = cbfm.rwg_gram(m)
    assert np.abs(G + G.T).max() < 1e-15
    assert np.abs(np.diag(G)).max() < 1e-16
    # closed form on each triangle: c_a c_b A n.((c - p_a) x (c - p_b))
    ref = np.zeros_like(G)
    for t in range(m.nt):
        V = m.verts[m.tris[t]]
        c = V.mean(axis=0)
        for a in range(3):
            for b in range(3):
                ea, eb = m.tri_edge[t, a], m.tri_edge[t, b]
                ca = m.tri_sign[t, a] * m.edge_len[ea] / (2 * m.area[t])
                cb = m.tri_sign[t, b] * m.edge_len[eb] / (2 * m.area[t])
                ref[ea, eb] += ca * cb * m.area[t] * np.dot(m.normal[t], np.cross(c - V[a], c - V[b]))
    assert np.abs(G - ref).max() < 1e-14 * np.abs(ref).max()
    # singular on a closed surface (paper Sec. II-C)
    s = np.linalg.svd(G, compute_uv=False)
    assert s[-1] < 1e-12 * s[0]
