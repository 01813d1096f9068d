"""CBFM with the Calderon multiplicative preconditioner -- plain FP64 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows paper Sec. III in its own order:
  1. primary CBF currents per cell:  Z_mm J_m = V_m  (Eq. (pcbf), LU solve);
  2. RWG Gram matrix of the cell G_m (Eq. (gram_RWG)), CBF Gram
     G'_m = (J_m^M)^H G_m J_m^J  (Eq. (gram_CBF));
  3. SVD of G'_m, keep sigma_i / sigma_1 >= delta_SVD  (Eq. (gram_CBF_SVD));
  4. dual CBFs  C^M = J^M U_L,  C^J = J^J V_L  (Eq. (CBF)); duality
     (C^M)^H G_m C^J = Sigma_L  (Eq. (CBF_sv));
  5. C^JM, C^MJ block matrices (Eqs. (CBF_matrix_JM/MJ)); reduced matrix
     A = (C^JM)^H Z C^MJ and b = (C^JM)^H v  (Eq. (CBFM_outer));
  6. G^CBF = (C^JM)^H G_ffff C^MJ  (Eq. (CBF_Gram_matrix));
  7. GMRES on A (G^CBF)^{-1} y = b, then G^CBF j^CBF = y (Eq. (CBFM_inner))
     and j = C^MJ j^CBF  (Eq. (trans_current)); (G^CBF)^{-1} exact (LU) or, as
     the paper does, by an inner GMRES with the diagonal preconditioner D^CBF.

Readings where the paper is silent: GMRES with x0 = 0, modified Gram-Schmidt
Arnoldi, restart length `restart`, stopping on ||b - A P y|| / ||b|| <= tol;
(G^CBF)^{-1} applied exactly by an LU factorisation.

The comparison arrangements of Sec. IV: the T-diagonal system Z_t of Eq.
(MoM_T) (unknowns [alpha^J; alpha^M]) with the diagonal preconditioner D, the
paper's conventional MoM, and the T-diagonal CBFM of Eq. (cbfm_Tdiag) without
a preconditioner.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import mom
from .mesh import RWGMesh


def rwg_gram(m: RWGMesh, rows=None, cols=None) -> np.ndarray:
    """[G]_ij = int (n x f_i) . f_j  (Eq. (gram_RWG) / (Gffff) block), by the
    7-point rule on every triangle of the common support (the integrand is
    linear, so the rule is exact)."""
    from . import lib  # noqa: F401  (keeps the oracle self-contained)
    ne = m.ne
    rows = np.arange(ne) if rows is None else np.asarray(rows)
    cols = np.arange(ne) if cols is None else np.asarray(cols)
    rpos = {int(e): i for i, e in enumerate(rows)}
    cpos = {int(e): i for i, e in enumerate(cols)}
    G = np.zeros((len(rows), len(cols)))
    s15 = np.sqrt(15.0)
    b1, b2 = (6 - s15) / 21, (6 + s15) / 21
    bary = np.array([[1 / 3, 1 / 3, 1 / 3], [1 - 2 * b1, b1, b1], [b1, 1 - 2 * b1, b1], [b1, b1, 1 - 2 * b1],
                     [1 - 2 * b2, b2, b2], [b2, 1 - 2 * b2, b2], [b2, b2, 1 - 2 * b2]])
    w = np.array([9 / 40] + [(155 - s15) / 1200] * 3 + [(155 + s15) / 1200] * 3)
    for t in range(m.nt):
        V = m.verts[m.tris[t]]
        q = bary @ V
        n = m.normal[t]
        A = m.area[t]
        for a in range(3):
            ea = int(m.tri_edge[t, a])
            if ea not in rpos:
                continue
            ca = m.tri_sign[t, a] * m.edge_len[ea] / (2 * A)
            fa = ca * (q - V[a])
            nfa = np.cross(n, fa)
            for b in range(3):
                eb = int(m.tri_edge[t, b])
                if eb not in cpos:
                    continue
                cb = m.tri_sign[t, b] * m.edge_len[eb] / (2 * A)
                fb = cb * (q - V[b])
                G[rpos[ea], cpos[eb]] += A * np.sum(w * np.einsum("ij,ij->i", nfa, fb))
    return G


@dataclass
class CellCBF:
    edges: np.ndarray        # Lambda_m
    CM: np.ndarray           # (N_m, L_m)
    CJ: np.ndarray           # (N_m, L_m)
    sigma: np.ndarray        # all singular values of G'_m (descending)
    L: int


def primary_cbfs(m: RWGMesh, cell: np.ndarray, ncell: int, eps_r: complex, gen: np.ndarray,
                 delta_svd: float, mu_r: float = 1.0, Lmax: int | None = None):
    """Steps 1-4 for every cell."""
    v = mom.rhs(m, gen)                          # (2 ne, s)
    ne = m.ne
    out = []
    for c in range(ncell):
        lam = np.nonzero(cell == c)[0]
        Nm = len(lam)
        Ks, Ta, Tb = mom.pmchwt_blocks(m, eps_r, mu_r, rows=lam, cols=lam)
        Zmm = np.block([[Ks, Ta], [Tb, Ks]])
        Vm = np.vstack([v[lam], v[ne + lam]])
        lu = sla.lu_factor(Zmm)
        Jm = sla.lu_solve(lu, Vm)
        out.append(cell_dual_cbfs(m, lam, Jm[:Nm], Jm[Nm:], delta_svd, Lmax))
    return out


def cell_dual_cbfs(m: RWGMesh, lam: np.ndarray, JM: np.ndarray, JJ: np.ndarray, delta_svd: float,
                   Lmax: int | None = None) -> CellCBF:
    """Steps 2-4 for one cell from its coefficient sets J^M, J^J (N_m x s)."""
    Gm = rwg_gram(m, lam, lam)
    Gp = JM.conj().T @ Gm @ JJ
    U, S, Vh = np.linalg.svd(Gp)
    L = int(np.sum(S / S[0] >= delta_svd))
    if Lmax is not None:
        L = min(L, Lmax)
    CM = JM @ U[:, :L]
    CJ = JJ @ Vh.conj().T[:, :L]
    return CellCBF(lam, CM, CJ, S, L)


def ipcbfs(m: RWGMesh, cell: np.ndarray, ncell: int, eps_r: complex, gen: np.ndarray, delta_r: float,
           delta_svd: float, mu_r: float = 1.0, Lmax: int | None = None, restart: int = 1000, maxit: int = 5000):
    """IPCBFs, GMRES version (Sec. III-A, after Eq. (ipcbf)): the whole MoM system,
    arranged as in Eq. (MoM_T) with its diagonal preconditioner, solved by GMRES
    for each generating wave and stopped at the relative residual delta_r; the
    coefficient sets J_m^M, J_m^J of cell m are those solutions restricted to the
    cell's RWG functions; steps 2-4 follow as for primary CBFs.  Returns (CBFs of
    every cell, GMRES iterations per wave)."""
    j, its = conventional_mom(m, eps_r, gen, delta_r, restart, maxit, mu_r)
    ne = m.ne
    out = []
    for c in range(ncell):
        lam = np.nonzero(cell == c)[0]
        out.append(cell_dual_cbfs(m, lam, j[lam], j[ne + lam], delta_svd, Lmax))
    return out, its


def block_C(cbfs, ne: int, which: str) -> np.ndarray:
    """Block-diagonal N_E x sum(L) matrix of C^M or C^J over all cells."""
    Ls = [c.L for c in cbfs]
    C = np.zeros((ne, sum(Ls)), np.complex128)
    off = 0
    for c in cbfs:
        C[c.edges, off:off + c.L] = c.CM if which == "M" else c.CJ
        off += c.L
    return C


def reduced_system(m: RWGMesh, cbfs, eps_r: complex, mu_r: float = 1.0, Z=None):
    """A = (C^JM)^H Z C^MJ with the dense Z (Eq. (CBFM_outer))."""
    ne = m.ne
    if Z is None:
        Z = mom.pmchwt_matrix(m, eps_r, mu_r)
    CM = block_C(cbfs, ne, "M")
    CJ = block_C(cbfs, ne, "J")
    Zr = np.zeros_like(CM)
    CJM = np.block([[CJ, Zr], [Zr, CM]])
    CMJ = np.block([[CM, Zr], [Zr, CJ]])
    return CJM.conj().T @ Z @ CMJ, CJM, CMJ


def reduced_block(m: RWGMesh, cbfs, eps_r: complex, mi: int, ni: int, mu_r: float = 1.0):
    """The 2x2 super-block of A for cells (m, n) from Z_mn only:
    [[CJ_m^H Ks CM_n, CJ_m^H Ta CJ_n], [CM_m^H Tb CM_n, CM_m^H Ks CJ_n]]."""
    cm, cn = cbfs[mi], cbfs[ni]
    Ks, Ta, Tb = mom.pmchwt_blocks(m, eps_r, mu_r, rows=cm.edges, cols=cn.edges)
    H = lambda X: X.conj().T  # noqa: E731
    return (H(cm.CJ) @ Ks @ cn.CM, H(cm.CJ) @ Ta @ cn.CJ, H(cm.CM) @ Tb @ cn.CM, H(cm.CM) @ Ks @ cn.CJ)


def cbf_gram(m: RWGMesh, cbfs, Gf=None) -> np.ndarray:
    """G^CBF = (C^JM)^H G_ffff C^MJ with G_ffff = diag(Gf, Gf) (Eq. (CBF_Gram_matrix))."""
    ne = m.ne
    if Gf is None:
        Gf = rwg_gram(m)
    CM = block_C(cbfs, ne, "M")
    CJ = block_C(cbfs, ne, "J")
    Gff = np.block([[Gf, np.zeros_like(Gf)], [np.zeros_like(Gf), Gf]])
    Zr = np.zeros_like(CM)
    CJM = np.block([[CJ, Zr], [Zr, CM]])
    CMJ = np.block([[CM, Zr], [Zr, CJ]])
    return CJM.conj().T @ Gff @ CMJ


def gmres(matvec, b: np.ndarray, tol: float, restart: int, maxit: int, precond=None):
    """Right-preconditioned restarted GMRES, x0 = 0, modified Gram-Schmidt.

    Solves (A P) y = b and returns (x = P y, iterations, residual history)
    where the residual is ||b - A P y|| / ||b|| from the Arnoldi least-squares
    problem.  `precond` applies P (identity when None)."""
    P = precond if precond is not None else (lambda z: z)
    n = b.shape[0]
    bn = np.linalg.norm(b)
    y = np.zeros(n, np.complex128)
    hist = []
    it = 0
    if bn == 0:
        return y, 0, [0.0]
    while it < maxit:
        r = b - matvec(P(y))
        beta = np.linalg.norm(r)
        hist.append(beta / bn)
        if beta / bn <= tol:
            break
        m = min(restart, maxit - it)
        Vb = np.zeros((n, m + 1), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        Vb[:, 0] = r / beta
        k_done = 0
        for k in range(m):
            w = matvec(P(Vb[:, k]))
            for i in range(k + 1):
                H[i, k] = np.vdot(Vb[:, i], w)
                w = w - H[i, k] * Vb[:, i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                Vb[:, k + 1] = w / H[k + 1, k]
            it += 1
            k_done = k + 1
            e1 = np.zeros(k + 2, np.complex128)
            e1[0] = beta
            z, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[:k + 2, :k + 1] @ z) / bn
            hist.append(res)
            if res <= tol or H[k + 1, k] == 0:
                break
        y = y + Vb[:, :k_done] @ z
        if hist[-1] <= tol:
            break
    return P(y), it, hist


@dataclass
class Solution:
    j: np.ndarray            # (2 ne, nrhs) RWG coefficients [alpha^M; alpha^J]
    jcbf: np.ndarray         # (N^CBF, nrhs)
    iters: list
    hist: list


def cmp_inexact(G: np.ndarray, inner_tol: float, restart: int = 200, maxit: int = 1000, its: list | None = None):
    """(G^CBF)^{-1} applied inexactly, as the paper proposes (Sec. III-C after Eq.
    (CBFM_inner), Sec. IV): GMRES on G^CBF z = v right-preconditioned by the
    diagonal D^CBF = 1 / diag(G^CBF), stopped at relative residual inner_tol.
    Inner iteration counts are appended to `its` when given."""
    d = np.diag(G).copy()

    def apply(v):
        z, it, _ = gmres(lambda u: G @ u, v, inner_tol, restart, maxit, lambda u: u / d)
        if its is not None:
            its.append(it)
        return z
    return apply


def solve_reduced(A: np.ndarray, Gcbf: np.ndarray, CMJ: np.ndarray, b: np.ndarray, tol: float,
                  restart: int = 200, maxit: int = 1000, use_cmp: bool = True,
                  inner_tol: float | None = None) -> Solution:
    """Step 7 for every right-hand side column of b; with inner_tol the CMP's
    (G^CBF)^{-1} is the inexact inner GMRES of cmp_inexact, else an LU solve."""
    if use_cmp and inner_tol is not None:
        P = cmp_inexact(Gcbf, inner_tol)
    elif use_cmp:
        lu = sla.lu_factor(Gcbf)
        P = lambda z: sla.lu_solve(lu, z)  # noqa: E731
    else:
        P = None
    X, its, hs = [], [], []
    for c in range(b.shape[1]):
        x, it, h = gmres(lambda z: A @ z, b[:, c], tol, restart, maxit, P)
        X.append(x)
        its.append(it)
        hs.append(h)
    jcbf = np.stack(X, axis=1)
    return Solution(CMJ @ jcbf, jcbf, its, hs)


def tdiag(A: np.ndarray) -> np.ndarray:
    """Eq. (MoM_T): a system in the unknown order of Eq. (Z) ([alpha^M;
    alpha^J], or the reduced system's [M-coefficient; J-coefficient] halves)
    rearranged for the unknowns [alpha^J; alpha^M] -- the same rows, the two
    column halves exchanged, so that the T blocks lie on the diagonal."""
    h = A.shape[1] // 2
    return np.concatenate([A[:, h:], A[:, :h]], axis=1)


def solve_tdiag(A: np.ndarray, b: np.ndarray, tol: float, restart: int = 200, maxit: int = 1000,
                jacobi: bool = True):
    """GMRES on Z_t D^{-1} j~ = b with j_t = D^{-1} j~ (Eq. (MoM_T)), Z_t = tdiag(A);
    D = diag(Z_t) when `jacobi` (the diagonal preconditioner of the paper's
    conventional MoM), else D = I (the T-diagonal CBFM, Eq. (cbfm_Tdiag)).
    Returns (x, iterations) with x = j_t brought back to A's unknown order."""
    Zt = tdiag(A)
    d = np.diag(Zt).copy() if jacobi else np.ones(Zt.shape[0], np.complex128)
    h = A.shape[1] // 2
    X, its = [], []
    for c in range(b.shape[1]):
        jt, it, _ = gmres(lambda z: Zt @ z, b[:, c], tol, restart, maxit, lambda z: z / d)
        X.append(np.concatenate([jt[h:], jt[:h]]))
        its.append(it)
    return np.stack(X, axis=1), its


def conventional_mom(m: RWGMesh, eps_r: complex, waves: np.ndarray, tol: float, restart: int = 1000,
                     maxit: int = 5000, mu_r: float = 1.0):
    """The paper's MoM (Sec. IV): PMCHWT matrix of Eq. (Z) in the T-diagonal
    arrangement with the diagonal preconditioner, solved by GMRES.  Returns
    (j in the order [alpha^M; alpha^J], iterations)."""
    Z = mom.pmchwt_matrix(m, eps_r, mu_r)
    return solve_tdiag(Z, mom.rhs(m, waves), tol, restart, maxit, jacobi=True)


def run(m: RWGMesh, cell, ncell, eps_r, gen, exc, delta_svd, tol, restart=200, maxit=1000,
        Lmax=None, use_cmp=True):
    """Whole pipeline on a small problem; returns a dict of intermediates."""
    cbfs = primary_cbfs(m, cell, ncell, eps_r, gen, delta_svd, Lmax=Lmax)
    Z = mom.pmchwt_matrix(m, eps_r)
    A, CJM, CMJ = reduced_system(m, cbfs, eps_r, Z=Z)
    v = mom.rhs(m, exc)
    b = CJM.conj().T @ v
    Gc = cbf_gram(m, cbfs)
    sol = solve_reduced(A, Gc, CMJ, b, tol, restart, maxit, use_cmp)
    return dict(cbfs=cbfs, Z=Z, A=A, b=b, G=Gc, CJM=CJM, CMJ=CMJ, sol=sol, v=v)
