"""Writes tests/golden/cube_c2.json: the oracle's end-to-end answer for the
9216-unknown cube (the benchmark workload), computed by `oracle/` alone.

Workload (workloads.cube_c2): cube of side 1 lambda0, eps_r 2.5, 16 x 16
squares per face (T = 3072, E = 4608, N = 9216), 32 RCB cells, 64 Fibonacci
directions x 2 polarisations (s = 128) as generating waves, 128 monostatic
excitations.

Steps, in the order of the paper's Sec. III (all FP64, oracle functions):
  primary CBFs per cell with delta_SVD = 1e-3 (Eq. (pcbf), Eqs. (gram_CBF),
  (gram_CBF_SVD), (CBF)); the dense PMCHWT matrix Z (Eq. (Z)); the reduced
  matrix A = (C^JM)^H Z C^MJ and b = (C^JM)^H v (Eq. (CBFM_outer)); the reduced
  system solved exactly, A j^CBF = b (the limit of the CMP-preconditioned GMRES
  of Eqs. (CBFM_outer), (CBFM_inner) as its tolerance goes to zero); currents
  j = C^MJ j^CBF (Eq. (trans_current)); monostatic partial RCS (Sec. I).

Stored: L_m per cell, the smallest relative gap |sigma_i/sigma_1 - delta_SVD|
/ delta_SVD over all cells (so a test knows L_m is not decided by rounding),
the monostatic RCS (sigma_theta, sigma_phi) of every excitation, ||j|| of
every excitation, and j of excitations 0 and 1 on every fourth unknown.

Run:  python tests/golden/make_cube_c2.py      (a few minutes on 8 cores)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import cbfm as OC, mesh as OM, mom as OMo  # noqa: E402

DELTA_SVD = 1e-3
OUT = os.path.join(HERE, "cube_c2.json")


def main():
    t0 = time.time()
    d = W.cube_c2(128)
    g = d["mesh"]
    m = OM.build_rwg(g.verts, g.tris)
    cell = OM.cells_rcb(m, d["ncell"])
    eps = complex(*d["eps"])
    cbfs = OC.primary_cbfs(m, cell, d["ncell"], eps, d["gen"], DELTA_SVD)
    gaps = [float(np.min(np.abs(c.sigma / c.sigma[0] - DELTA_SVD)) / DELTA_SVD) for c in cbfs]
    print(f"CBFs: N^CBF = {2 * sum(c.L for c in cbfs)}, min gap {min(gaps):.3e} ({time.time() - t0:.0f} s)", flush=True)
    Z = OMo.pmchwt_matrix(m, eps)
    print(f"Z assembled ({time.time() - t0:.0f} s)", flush=True)
    A, CJM, CMJ = OC.reduced_system(m, cbfs, eps, Z=Z)
    del Z
    v = OMo.rhs(m, d["exc"])
    b = CJM.conj().T @ v
    jcbf = np.linalg.solve(A, b)
    j = CMJ @ jcbf
    res = np.linalg.norm(A @ jcbf - b, axis=0) / np.linalg.norm(b, axis=0)
    rcs = np.zeros((j.shape[1], 2))
    for r in range(j.shape[1]):
        Fth, Fph = OMo.farfield(m, j[:, r:r + 1], d["obs"][r:r + 1])
        st, sp = OMo.rcs(Fth, Fph)
        rcs[r] = (st[0, 0], sp[0, 0])
    sub = np.arange(0, j.shape[0], 4)
    out = {
        "workload": "cube side 1, eps_r 2.5, 16x16 squares per face, 32 RCB cells, s = 128, 128 monostatic RHS",
        "delta_svd": DELTA_SVD,
        "L_per_cell": [int(c.L) for c in cbfs],
        "min_rel_gap_to_delta": min(gaps),
        "n_cbf": int(2 * sum(c.L for c in cbfs)),
        "max_reduced_residual": float(res.max()),
        "rcs": rcs.tolist(),
        "j_norm": np.linalg.norm(j, axis=0).tolist(),
        "j_rows": sub.tolist(),
        "j0": [[float(x.real), float(x.imag)] for x in j[sub, 0]],
        "j1": [[float(x.real), float(x.imag)] for x in j[sub, 1]],
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
