"""Pins for the oracle's inexact CMP: (G^CBF)^{-1} applied by an inner GMRES with
the diagonal preconditioner D^CBF (Sec. III-C, Sec. IV: tolerance 1e-5).

* Special case: with an inner tolerance at rounding level it is the exact CMP
  (LU): the same outer iterations and the same currents.
* At the paper's 1e-5 the outer GMRES takes the exact CMP's iterations (within
  1) and the currents stay within 1e-4 of the exact-CMP solution at 1e-10.
* The paper's claim that the inner solve is cheap with D^CBF even when G^CBF is
  not diagonal (a connected sphere cut into octants, off-diagonal entries up to
  150 times the smallest diagonal one): at most 30 inner iterations (measured 22).
"""

import numpy as np
import pytest

import workloads as W
from oracle import cbfm, mesh as OM


@pytest.fixture(scope="module")
def c1():
    d = W.sphere_c1()
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_octant(m)
    exc = np.array([[0.0, 0.0, 0.0], [1.2, 0.7, 0.4]])
    return cbfm.run(m, cell, 8, 4.0, d["gen"], exc, 1e-3, 1e-10, restart=1000)


def test_inexact_cmp_reduces_to_exact(c1):
    R = c1
    ex = cbfm.solve_reduced(R["A"], R["G"], R["CMJ"], R["b"], 1e-6, restart=1000)
    ie = cbfm.solve_reduced(R["A"], R["G"], R["CMJ"], R["b"], 1e-6, restart=1000, inner_tol=1e-14)
    assert ie.iters == ex.iters
    assert np.linalg.norm(ie.j - ex.j) / np.linalg.norm(ex.j) < 1e-9


def test_inexact_cmp_at_1e5(c1):
    R = c1
    G = R["G"]
    dg = np.abs(np.diag(G))
    assert np.abs(G - np.diag(np.diag(G))).max() > 10 * dg.min()      # not diagonal
    ex = cbfm.solve_reduced(R["A"], G, R["CMJ"], R["b"], 1e-6, restart=1000)
    its = []
    P = cbfm.cmp_inexact(G, 1e-5, its=its)
    X, outer = [], []
    for c in range(R["b"].shape[1]):
        x, it, _ = cbfm.gmres(lambda z: R["A"] @ z, R["b"][:, c], 1e-6, 1000, 1000, P)
        X.append(x)
        outer.append(it)
    j = R["CMJ"] @ np.stack(X, axis=1)
    for a, b in zip(outer, ex.iters):
        assert abs(a - b) <= 1
    jo = R["sol"].j
    assert np.linalg.norm(j - jo) / np.linalg.norm(jo) < 1e-4
    assert max(its) <= 30
