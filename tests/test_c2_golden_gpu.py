"""The benchmark workload end to end against the oracle.

The 9216-unknown cube (side 1, eps_r 2.5, 32 RCB cells, s = 128 generating
waves, 128 monostatic excitations) runs through exactly the benchmark's path:
CBFs built on the GPU (delta_SVD = 1e-3), the mixed-precision reduced matrix
(FP32 quadrature, tensor-core projection), the CMP and block GMRES over all
128 right-hand sides at tol 1e-6, currents and monostatic RCS.  The plain FP64
GPU path runs the same with tol 1e-10.  Both are compared with the oracle's
answer stored in tests/golden/cube_c2.json (written by make_cube_c2.py from
oracle/ alone: primary CBFs, dense Z, A = (C^JM)^H Z C^MJ, A j^CBF = b solved
exactly, j = C^MJ j^CBF; paper Eqs. (CBFM_outer), (CBFM_inner),
(trans_current)).

Bounds (peak-normalised RCS error, relative L2 current error on the stored
unknowns of excitations 0 and 1):
  * the CBF counts L_m equal the oracle's (the smallest gap of a normalised
    singular value to delta_SVD is 1e-2 relative, far above rounding);
  * MIXED, tol 1e-6:  RCS <= 1e-4, currents <= J_MIXED;
  * FP64, tol 1e-10:  RCS <= 1e-6, currents <= 1e-6.
The CBFs themselves are unique only up to unitary mixing inside degenerate
singular-value groups; the currents and the RCS do not depend on that choice.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# Mixed-path bound on the currents: the reduced matrix carries ~1e-6 relative
# error of its largest entry (FP32 quadrature, split-TF32 products), amplified by
# the conditioning of the CMP-preconditioned system, plus the 1e-6 GMRES tolerance.
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


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "golden", "cube_c2.json")) as f:
        g = json.load(f)
    g["rcs"] = np.asarray(g["rcs"])
    g["j_rows"] = np.asarray(g["j_rows"])
    for k in ("j0", "j1"):
        a = np.asarray(g[k])
        g[k] = a[:, 0] + 1j * a[:, 1]
    return g


@pytest.fixture(scope="module")
def cube(P):
    d = W.cube_c2(128)
    g = d["mesh"]
    mesh = P.mesh(g.verts, g.tris, d["ncell"], complex(*d["eps"]), partition=d["partition"])
    cbf = P.build_cbfs(mesh, d["gen"], 1e-3)
    return dict(d=d, mesh=mesh, cbf=cbf)


def _errors(res, gold):
    rcs = res.rcs[:, 0, :].sum(-1)
    ro = gold["rcs"].sum(-1)
    e_rcs = float(np.abs(rcs - ro).max() / np.abs(ro).max())
    rows = gold["j_rows"]
    e_j = max(float(np.linalg.norm(res.j[rows, c] - gold[k]) / np.linalg.norm(gold[k]))
              for c, k in ((0, "j0"), (1, "j1")))
    e_norm = float(np.abs(np.linalg.norm(res.j, axis=0) - gold["j_norm"]).max() / max(gold["j_norm"]))
    return e_rcs, e_j, e_norm


def test_c2_cbf_counts_equal_oracle(cube, gold):
    assert gold["min_rel_gap_to_delta"] > 1e-6
    assert cube["cbf"].L.tolist() == gold["L_per_cell"]


@pytest.mark.parametrize("prec", [1, 4])
def test_c2_bench_path_mixed_block_gmres(P, cube, gold, prec):
    """prec 1: the form CBFM_MIXED picks (the benchmark's); prec 4: the fused assembly-projection kernel."""
    red = P.assemble_reduced(cube["mesh"], cube["cbf"], prec)
    assert red.n == gold["n_cbf"]
    P.cmp_setup(red)
    res = P.solve(red, cube["d"]["exc"], tol=1e-6, maxit=2000, restart=1000, monostatic=True, solver=P.BLOCK)
    e_rcs, e_j, e_norm = _errors(res, gold)
    print(f"c2 mixed ({prec}) block GMRES vs oracle: RCS {e_rcs:.2e}, currents {e_j:.2e}, norms {e_norm:.2e}, "
          f"block iterations {int(res.iters.max())}")
    assert e_rcs <= 1e-4
    assert e_j <= J_MIXED
    assert e_norm <= J_MIXED


def test_c2_fp64_path(P, cube, gold):
    red = P.assemble_reduced(cube["mesh"], cube["cbf"], P.FP64)
    P.cmp_setup(red)
    res = P.solve(red, cube["d"]["exc"], tol=1e-10, maxit=2000, restart=1000, monostatic=True, solver=P.BLOCK)
    e_rcs, e_j, e_norm = _errors(res, gold)
    print(f"c2 FP64 block GMRES vs oracle: RCS {e_rcs:.2e}, currents {e_j:.2e}, norms {e_norm:.2e}")
    assert e_rcs <= 1e-6
    assert e_j <= 1e-6
    assert e_norm <= 1e-6
