"""PMCHWT method-of-moments pieces of the oracle (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper Sec. II-A/II-B:
  * media: exterior 1 (free space, k1 = 2 pi, eta1 = eta0), interior 2
    (k2 = k0 sqrt(eps_r mu_r) with Re > 0, Im <= 0; eta2 = eta0 sqrt(mu_r/eps_r));
  * Z = sum_i [[K_i, -eta_i T_i], [T_i/eta_i, K_i]]  (Eq. (Z)), unknowns
    j = [alpha^M; alpha^J]  (Eq. (coef_vector)),  v = [v^E; v^H]  (Eq. (v));
  * the three distinct RWG blocks: Ks = K1 + K2, Ta = -(eta1 T1 + eta2 T2),
    Tb = T1/eta1 + T2/eta2.
The operator entries come from zmat.c (see its header for the quadrature,
singularity extraction and sign reading).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import lib
from .mesh import RWGMesh

ETA0 = 376.730313668          # mu0 * c (CODATA 2018), ohm
K0 = 2.0 * math.pi            # lengths in free-space wavelengths
ALPHA_NEAR = 2.0              # near-pair factor (paper silent)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(_dp)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(_ip)


def media(eps_r: complex, mu_r: float = 1.0):
    """(k1, eta1, k2, eta2) for the exterior (free space) and interior media."""
    eps_r = complex(eps_r)
    n2 = np.sqrt(eps_r * mu_r)
    if n2.real < 0:
        n2 = -n2
    k2 = K0 * n2
    if k2.imag > 0:
        raise ValueError("active medium: Im(eps_r) must be <= 0 for exp(+j omega t)")
    eta2 = ETA0 * np.sqrt(mu_r / eps_r)
    return K0, ETA0, complex(k2), complex(eta2)


class _Arrs:
    """Keeps contiguous copies alive for the C calls."""

    def __init__(self, m: RWGMesh):
        self.verts = np.ascontiguousarray(m.verts, np.float64)
        self.tris = np.ascontiguousarray(m.tris, np.int32)
        self.tri_edge = np.ascontiguousarray(m.tri_edge, np.int32)
        self.tri_sign = np.ascontiguousarray(m.tri_sign, np.int32)
        self.edge_len = np.ascontiguousarray(m.edge_len, np.float64)
        self.edge_tri = np.ascontiguousarray(m.edge_tri, np.int32)
        self.edge_loc = np.ascontiguousarray(m.edge_loc, np.int32)
        self.nv = m.verts.shape[0]
        self.nt = m.tris.shape[0]
        self.ne = m.edges.shape[0]


def operator_block(m: RWGMesh, k: complex, rows=None, cols=None, alpha: float = ALPHA_NEAR):
    """K_i[rows][cols], T_i[rows][cols] for one medium with wavenumber k."""
    A = _Arrs(m)
    rows = np.arange(A.ne, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, np.int32)
    cols = np.arange(A.ne, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
    K = np.zeros((len(rows), len(cols)), np.complex128)
    T = np.zeros((len(rows), len(cols)), np.complex128)
    f = lib().orc_assemble
    f.restype = None
    f(ctypes.c_int(A.nv), _d(A.verts), ctypes.c_int(A.nt), _i(A.tris), _i(A.tri_edge), _i(A.tri_sign),
      _d(A.edge_len), _i(A.edge_tri), _i(A.edge_loc), ctypes.c_double(alpha),
      ctypes.c_double(complex(k).real), ctypes.c_double(complex(k).imag),
      ctypes.c_int(len(rows)), _i(rows), ctypes.c_int(len(cols)), _i(cols),
      K.ctypes.data_as(ctypes.c_void_p), T.ctypes.data_as(ctypes.c_void_p))
    return K, T


def local_block(m: RWGMesh, k: complex, t: int, s: int, alpha: float = ALPHA_NEAR):
    """3x3 local K and T of triangle pair (t, s) and the near flag."""
    A = _Arrs(m)
    Ko = np.zeros(18)
    To = np.zeros(18)
    near = ctypes.c_int(0)
    f = lib().orc_local_block
    f.restype = None
    f(ctypes.c_int(A.nv), _d(A.verts), ctypes.c_int(A.nt), _i(A.tris), _i(A.tri_edge), _i(A.tri_sign),
      _d(A.edge_len), ctypes.c_double(alpha), ctypes.c_double(complex(k).real),
      ctypes.c_double(complex(k).imag), ctypes.c_int(t), ctypes.c_int(s), _d(Ko), _d(To), ctypes.byref(near))
    return (Ko[0::2] + 1j * Ko[1::2]).reshape(3, 3), (To[0::2] + 1j * To[1::2]).reshape(3, 3), bool(near.value)


def pmchwt_blocks(m: RWGMesh, eps_r: complex, mu_r: float = 1.0, rows=None, cols=None,
                  alpha: float = ALPHA_NEAR):
    """Ks, Ta, Tb restricted to rows x cols (full matrices by default)."""
    k1, eta1, k2, eta2 = media(eps_r, mu_r)
    K1, T1 = operator_block(m, k1, rows, cols, alpha)
    K2, T2 = operator_block(m, k2, rows, cols, alpha)
    Ks = K1 + K2
    Ta = -(eta1 * T1 + eta2 * T2)
    Tb = T1 / eta1 + T2 / eta2
    return Ks, Ta, Tb


def pmchwt_matrix(m: RWGMesh, eps_r: complex, mu_r: float = 1.0, alpha: float = ALPHA_NEAR):
    """Full N x N PMCHWT matrix, Eq. (Z), unknown order [alpha^M; alpha^J]."""
    Ks, Ta, Tb = pmchwt_blocks(m, eps_r, mu_r, alpha=alpha)
    return np.block([[Ks, Ta], [Tb, Ks]])


def rhs(m: RWGMesh, waves: np.ndarray):
    """v = [v^E; v^H] for each plane wave (theta, phi, psi): (2 ne, nw)."""
    A = _Arrs(m)
    waves = np.ascontiguousarray(np.atleast_2d(waves), np.float64)
    nw = waves.shape[0]
    vE = np.zeros((A.ne, nw), np.complex128)
    vH = np.zeros((A.ne, nw), np.complex128)
    f = lib().orc_rhs
    f.restype = None
    f(ctypes.c_int(A.nv), _d(A.verts), ctypes.c_int(A.nt), _i(A.tris), _i(A.tri_edge), _i(A.tri_sign),
      _d(A.edge_len), ctypes.c_int(A.ne), ctypes.c_double(K0), ctypes.c_double(ETA0),
      ctypes.c_int(nw), _d(waves), vE.ctypes.data_as(ctypes.c_void_p), vH.ctypes.data_as(ctypes.c_void_p))
    return np.vstack([vE, vH])


def farfield(m: RWGMesh, j: np.ndarray, dirs: np.ndarray):
    """(F_theta, F_phi), each (nrhs, ndir), from j = [alpha^M; alpha^J] (2 ne, nrhs)."""
    A = _Arrs(m)
    j = np.atleast_2d(j.T).T
    aM = np.ascontiguousarray(j[:A.ne], np.complex128)
    aJ = np.ascontiguousarray(j[A.ne:], np.complex128)
    nrhs = j.shape[1]
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), np.float64)
    nd = dirs.shape[0]
    Fth = np.zeros((nrhs, nd), np.complex128)
    Fph = np.zeros((nrhs, nd), np.complex128)
    f = lib().orc_farfield
    f.restype = None
    f(ctypes.c_int(A.nv), _d(A.verts), ctypes.c_int(A.nt), _i(A.tris), _i(A.tri_edge), _i(A.tri_sign),
      _d(A.edge_len), ctypes.c_int(A.ne), ctypes.c_double(K0), ctypes.c_double(ETA0),
      ctypes.c_int(nrhs), aM.ctypes.data_as(ctypes.c_void_p), aJ.ctypes.data_as(ctypes.c_void_p),
      ctypes.c_int(nd), _d(dirs), Fth.ctypes.data_as(ctypes.c_void_p), Fph.ctypes.data_as(ctypes.c_void_p))
    return Fth, Fph


def rcs(Fth: np.ndarray, Fph: np.ndarray):
    """Partial RCS (sigma_theta, sigma_phi) = 4 pi |F_theta|^2, 4 pi |F_phi|^2
    for unit-amplitude incidence (Knott's definition, paper Sec. I)."""
    return 4.0 * math.pi * np.abs(Fth) ** 2, 4.0 * math.pi * np.abs(Fph) ** 2


def solve_mom(m: RWGMesh, eps_r: complex, waves: np.ndarray, mu_r: float = 1.0):
    """Conventional MoM: dense LU of Eq. (MoM).  Returns j (2 ne, nw)."""
    Z = pmchwt_matrix(m, eps_r, mu_r)
    v = rhs(m, waves)
    return np.linalg.solve(Z, v)


def rmse_db(sig_c: np.ndarray, sig_m: np.ndarray) -> float:
    """RMSE of a pattern sig_c against sig_m in dB, paper Eq. (RMSE)."""
    sig_c = np.asarray(sig_c, float)
    sig_m = np.asarray(sig_m, float)
    num = np.sqrt(np.mean((sig_c - sig_m) ** 2))
    return 10.0 * math.log10(num / (sig_m.max() - sig_m.min()))
