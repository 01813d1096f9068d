"""Pins for the oracle's comparison arrangements of Sec. IV: the T-diagonal
system Z_t with the diagonal preconditioner D (the paper's conventional MoM,
Eq. (MoM_T)) and the T-diagonal CBFM (Eq. (cbfm_Tdiag)).

What fixes them:
* Z_t written out from Eq. (MoM_T) with the blocks of Eq. (Z): rows as in Z,
  unknowns [alpha^J; alpha^M];
* Eq. (cbfm_Tdiag) evaluated literally, (C^JM)^H Z_t C^JM, is the K-diagonal
  reduced matrix with its column halves exchanged (so the T-diagonal CBFM needs
  no second assembly);
* the T operators carry the larger diagonal entries (Sec. IV, the reason given
  for the arrangement): |Z_t[i,i]| > |Z[i,i]| for every row;
* the solution of Z j = v does not depend on the arrangement or on D: the
  GMRES answer equals a dense solve;
* Jacobi scaling cuts the iteration count of the T-diagonal arrangement.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cbfm, mesh as OM, mom


@pytest.fixture(scope="module")
def sphere1():
    g = W.icosphere(1, 1.0 / 6.0)
    return OM.build_rwg(g.verts, g.tris)


def test_tdiag_is_eq_mom_t(sphere1):
    m = sphere1
    Z = mom.pmchwt_matrix(m, 3.0)
    Ks, Ta, Tb = mom.pmchwt_blocks(m, 3.0)
    # Eq. (MoM_T): first row block -eta_i T_i (J columns) and K_i (M columns),
    # second row block K_i (J columns) and T_i / eta_i (M columns)
    assert np.array_equal(cbfm.tdiag(Z), np.block([[Ta, Ks], [Ks, Tb]]))
    # the arrangement exchanges column halves only: applying it twice is the identity
    assert np.array_equal(cbfm.tdiag(cbfm.tdiag(Z)), Z)


@pytest.mark.parametrize("eps", [1.0, 3.0])
def test_t_blocks_dominate_the_diagonal(eps):
    g = W.icosphere(2, 1.0 / 6.0)
    m = OM.build_rwg(g.verts, g.tris)
    Z = mom.pmchwt_matrix(m, eps)
    assert (np.abs(np.diag(cbfm.tdiag(Z))) > np.abs(np.diag(Z))).all()


def test_tdiag_cbfm_is_column_swapped_reduced_matrix():
    g = W.icosphere(1, 0.3)
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    cb = cbfm.primary_cbfs(m, cell, 8, 2.0, W.plane_wave_set(W.fibonacci_dirs(8)), 1e-3)
    Z = mom.pmchwt_matrix(m, 2.0)
    A, CJM, _ = cbfm.reduced_system(m, cb, 2.0, Z=Z)
    At = CJM.conj().T @ cbfm.tdiag(Z) @ CJM          # Eq. (cbfm_Tdiag), as written
    assert np.abs(At - cbfm.tdiag(A)).max() < 1e-12 * np.abs(A).max()


def test_conventional_mom_matches_dense_solve():
    g = W.icosphere(2, 1.0 / 6.0)
    m = OM.build_rwg(g.verts, g.tris)
    exc = np.array([[0.0, 0.0, 0.0], [0.7, 0.3, 0.5]])
    j, its = cbfm.conventional_mom(m, 3.0, exc, 1e-10)
    jd = mom.solve_mom(m, 3.0, exc)
    assert np.linalg.norm(j - jd) / np.linalg.norm(jd) < 1e-7
    assert all(0 < it < 2 * m.ne for it in its)


def test_jacobi_cuts_iterations_and_keeps_the_solution(sphere1):
    m = sphere1
    Z = mom.pmchwt_matrix(m, 3.0)
    v = mom.rhs(m, np.array([[0.0, 0.0, 0.0]]))
    xj, ij = cbfm.solve_tdiag(Z, v, 1e-8, jacobi=True)
    xn, inn = cbfm.solve_tdiag(Z, v, 1e-8, jacobi=False)
    jd = np.linalg.solve(Z, v)
    for x in (xj, xn):
        assert np.linalg.norm(x - jd) / np.linalg.norm(jd) < 1e-5
    assert 2 * ij[0] < inn[0]


def test_zero_excitation_and_two_unknowns():
    # degenerate inputs: a zero right-hand side stops at once with x = 0; the smallest
    # system with two halves is arranged and solved like any other
    rng = np.random.default_rng(5)
    A = np.array([[0.3 + 0.1j, 2.0 - 1.0j], [1.5 + 0.5j, -0.2j]])
    assert np.array_equal(cbfm.tdiag(A), A[:, ::-1])
    b = np.stack([np.zeros(2, complex), rng.standard_normal(2) + 0j], axis=1)
    x, its = cbfm.solve_tdiag(A, b, 1e-12)
    assert its[0] == 0 and not x[:, 0].any()
    assert np.linalg.norm(A @ x[:, 1] - b[:, 1]) < 1e-12 * np.linalg.norm(b[:, 1])
