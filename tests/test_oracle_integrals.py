"""Pins for the oracle's quadrature rule and analytic potential integrals.

The 7-point rule is checked against exact monomial integrals; the closed-form
integrals of 1/R, (r'-r)/R and (r-r')/R^3 over a flat triangle are checked
against high-order Gauss-Legendre integration in Duffy-collapsed coordinates
(an independent numerical route), at observation points above, beside and in
the plane of the triangle.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle

_dp = ctypes.POINTER(ctypes.c_double)


def _quad7():
    bary = np.zeros((7, 3))
    w = np.zeros(7)
    oracle.lib().orc_quad7_bary(bary.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    return bary, w


def _potentials(tri, r):
    I1 = ctypes.c_double()
    Iv = np.zeros(3)
    I3 = np.zeros(3)
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in tri]
    rr = np.ascontiguousarray(r, dtype=np.float64)
    oracle.lib().orc_potentials(v[0].ctypes.data_as(_dp), v[1].ctypes.data_as(_dp), v[2].ctypes.data_as(_dp),
                                rr.ctypes.data_as(_dp), ctypes.byref(I1), Iv.ctypes.data_as(_dp),
                                I3.ctypes.data_as(_dp))
    return I1.value, Iv, I3


def test_quad7_exact_to_degree5():
    bary, w = _quad7()
    assert abs(w.sum() - 1.0) < 1e-15
    x, y = bary[:, 1], bary[:, 2]          # reference triangle (0,0),(1,0),(0,1), area 1/2
    for deg in range(0, 6):
        for i in range(deg + 1):
            j = deg - i
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            got = 0.5 * np.sum(w * x ** i * y ** j)
            assert abs(got - exact) < 1e-15, (i, j)
    # degree 6 is not integrated exactly
    errs = [abs(0.5 * np.sum(w * x ** i * y ** (6 - i)) - math.factorial(i) * math.factorial(6 - i) / math.factorial(8))
            for i in range(7)]
    assert max(errs) > 1e-6


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


def _ref_integrals(tri, r, n=64):
    """Numerical int over the triangle of 1/R, (r'-r)/R, (r-r')/R^3 via Duffy
    collapse from the projection of r (or vertex 0 when it lies outside)."""
    v0, v1, v2 = [np.asarray(x, float) for x in tri]
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    d = np.dot(nrm, r - v0)
    rho = r - d * nrm
    # barycentric of rho
    T = np.column_stack([v1 - v0, v2 - v0])
    lam, *_ = np.linalg.lstsq(T, rho - v0, rcond=None)
    inside = lam[0] >= -1e-14 and lam[1] >= -1e-14 and lam.sum() <= 1 + 1e-14
    apex = rho if inside else v0
    subs = [(v0, v1), (v1, v2), (v2, v0)] if inside else [(v1, v2)]
    # composite GL in u to resolve near-singular peaks
    us, uw = [], []
    for a, b in [(0, 1e-3), (1e-3, 1e-2), (1e-2, 0.1), (0.1, 1.0)]:
        x, w = _gl(n, a, b)
        us.append(x)
        uw.append(w)
    us = np.concatenate(us)
    uw = np.concatenate(uw)
    vs, vw = [], []
    edges_v = np.linspace(0.0, 1.0, 41)
    for a, b in zip(edges_v[:-1], edges_v[1:]):
        x, w = _gl(24, a, b)
        vs.append(x)
        vw.append(w)
    vs = np.concatenate(vs)
    vw = np.concatenate(vw)
    I1 = 0.0
    Iv = np.zeros(3)
    I3 = np.zeros(3)
    for A, B in subs:
        jac = np.dot(np.cross(A - apex, B - A), nrm)       # signed
        U, V = np.meshgrid(us, vs, indexing="ij")
        P = apex + U[..., None] * (A - apex) + (U * V)[..., None] * (B - A)
        Wt = (uw[:, None] * vw[None, :]) * U * jac
        D = P - r
        R = np.linalg.norm(D, axis=-1)
        I1 += np.sum(Wt / R)
        Iv += np.einsum("ij,ijk->k", Wt / R, D)
        I3 += np.einsum("ij,ijk->k", Wt / R ** 3, -D)
    return I1, Iv, I3


TRI = (np.array([0.1, -0.2, 0.05]), np.array([0.9, 0.1, -0.1]), np.array([0.2, 0.7, 0.3]))


@pytest.mark.parametrize("where", ["centroid", "near_edge", "near_vertex", "outside"])
@pytest.mark.parametrize("height", [0.5, 0.05, 0.01])
def test_potentials_off_plane(where, height):
    v0, v1, v2 = TRI
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    base = {"centroid": (v0 + v1 + v2) / 3,
            "near_edge": 0.5 * (v0 + v1) + 0.03 * ((v2 - 0.5 * (v0 + v1))),
            "near_vertex": v0 + 0.04 * (v1 - v0) + 0.03 * (v2 - v0),
            "outside": v1 + 0.3 * (v1 - v0)}[where]
    r = base + height * nrm
    I1, Iv, I3 = _potentials(TRI, r)
    R1, Rv, R3 = _ref_integrals(TRI, r)
    assert abs(I1 - R1) < 1e-9 * abs(R1)
    assert np.linalg.norm(Iv - Rv) < 1e-9 * np.linalg.norm(Rv)
    assert np.linalg.norm(I3 - R3) < 1e-7 * np.linalg.norm(R3)


@pytest.mark.parametrize("bary", [(1 / 3, 1 / 3), (0.05, 0.9), (0.47, 0.47), (0.8, 0.1)])
def test_potentials_in_plane_inside(bary):
    v0, v1, v2 = TRI
    r = v0 + bary[0] * (v1 - v0) + bary[1] * (v2 - v0)
    I1, Iv, _ = _potentials(TRI, r)
    R1, Rv, _ = _ref_integrals(TRI, r)
    assert abs(I1 - R1) < 1e-10 * abs(R1)
    assert np.linalg.norm(Iv - Rv) < 1e-10 * np.linalg.norm(Rv)


def test_potentials_in_plane_outside():
    v0, v1, v2 = TRI
    r = v2 + 0.6 * (v2 - 0.5 * (v0 + v1))
    I1, Iv, I3 = _potentials(TRI, r)
    R1, Rv, R3 = _ref_integrals(TRI, r)
    assert abs(I1 - R1) < 1e-10 * abs(R1)
    assert np.linalg.norm(Iv - Rv) < 1e-10 * np.linalg.norm(Rv)
    assert np.linalg.norm(I3 - R3) < 1e-9 * np.linalg.norm(R3)
    # in the plane, outside: no normal component
    nrm = np.cross(v1 - v0, v2 - v0)
    assert abs(np.dot(I3, nrm)) < 1e-12 * np.linalg.norm(I3) * np.linalg.norm(nrm)


def test_solid_angle_limit():
    """Just above the interior, n . int (r-r')/R^3 -> 2 pi (half-space solid angle)."""
    v0, v1, v2 = TRI
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    r = (v0 + v1 + v2) / 3 + 1e-9 * nrm
    _, _, I3 = _potentials(TRI, r)
    assert abs(np.dot(I3, nrm) - 2 * math.pi) < 1e-6
    r = (v0 + v1 + v2) / 3 - 1e-9 * nrm
    _, _, I3 = _potentials(TRI, r)
    assert abs(np.dot(I3, nrm) + 2 * math.pi) < 1e-6
