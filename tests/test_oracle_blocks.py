"""Pins for the oracle's triangle-pair blocks of K_i and T_i.

* far pairs: the 7x7-point result against a high-order product rule on both
  triangles (the quadrature error must be small, a wrong term is O(1));
* near pairs: singularity extraction against direct high-order integration of
  the unsplit kernel over the trial triangle at the same seven test points
  (same outer rule, same symmetrisation), which isolates the analytic parts;
* self pair: the K block vanishes on a flat triangle;
* exchange: L(s, t) = L(t, s)^T for K and T, far and near pairs, lossless
  and lossy wavenumbers.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mesh as OM, mom

K_EXT = 2 * math.pi
K_INT = 2 * math.pi * math.sqrt(4.0)


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


def _quad7(V):
    s15 = math.sqrt(15.0)
    b1, b2 = (6 - s15) / 21, (6 + s15) / 21
    bary = np.array([[1 / 3, 1 / 3, 1 / 3], [1 - 2 * b1, b1, b1], [b1, 1 - 2 * b1, b1], [b1, b1, 1 - 2 * b1],
                     [1 - 2 * b2, b2, b2], [b2, 1 - 2 * b2, b2], [b2, b2, 1 - 2 * b2]])
    w = np.array([9 / 40] + [(155 - s15) / 1200] * 3 + [(155 + s15) / 1200] * 3)
    A = 0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
    return bary @ V, w * A


def _duffy_rule(V, apex, nu=40, nv=40):
    """Points/weights of a Duffy collapse of triangle V from `apex` (any point
    in its plane); signed sub-triangles when apex is outside."""
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    us, uw = [], []
    for a, b in [(0, 1e-3), (1e-3, 1e-2), (1e-2, 0.1), (0.1, 1.0)]:
        x, w = _gl(nu, a, b)
        us.append(x)
        uw.append(w)
    us, uw = np.concatenate(us), np.concatenate(uw)
    vs, vw = [], []
    for a, b in zip(np.linspace(0, 1, 11)[:-1], np.linspace(0, 1, 11)[1:]):
        x, w = _gl(nv // 2, a, b)
        vs.append(x)
        vw.append(w)
    vs, vw = np.concatenate(vs), np.concatenate(vw)
    P, Wt = [], []
    for A, B in [(V[0], V[1]), (V[1], V[2]), (V[2], V[0])]:
        jac = np.dot(np.cross(A - apex, B - A), nrm)
        if abs(jac) < 1e-300:
            continue
        U, Vv = np.meshgrid(us, vs, indexing="ij")
        P.append((apex + U[..., None] * (A - apex) + (U * Vv)[..., None] * (B - A)).reshape(-1, 3))
        Wt.append(((uw[:, None] * vw[None, :]) * U * jac).reshape(-1))
    return np.concatenate(P), np.concatenate(Wt)


def _coef(m, t):
    c = np.array([m.tri_sign[t, a] * m.edge_len[m.tri_edge[t, a]] / (2 * m.area[t]) for a in range(3)])
    return c, m.verts[m.tris[t]]


def _kernels(k, R, part):
    """G and g = |grad G|/R pieces: 'full', the extracted 'singular' part
    1/(4 pi R), -1/(4 pi R^3) - k^2/(8 pi R), or the 'smooth' remainder."""
    zero = R == 0.0
    Rz = np.where(zero, 1.0, R)
    G = np.exp(-1j * k * Rz) / (4 * math.pi * Rz)
    g = -(1 + 1j * k * Rz) * np.exp(-1j * k * Rz) / (4 * math.pi * Rz ** 3)
    Gs = 1 / (4 * math.pi * Rz)
    gs = -1 / (4 * math.pi * Rz ** 3) - k ** 2 / (8 * math.pi * Rz)
    if part == "full":
        return G, g
    if part == "singular":
        return Gs + 0j, gs + 0j
    # coincident points: limits -jk/(4 pi) and jk^3/(12 pi) of the remainders
    return (np.where(zero, -1j * k / (4 * math.pi), G - Gs),
            np.where(zero, 1j * k ** 3 / (12 * math.pi), g - gs))


def _block_ref(m, k, t, s, inners):
    """Unsymmetrised block with the 7-point rule on t; `inners` is a list of
    (rule(r) -> (pts, w) on s, kernel part)."""
    ca, pa = _coef(m, t)
    cb, pb = _coef(m, s)
    qt, wt = _quad7(m.verts[m.tris[t]])
    Kl = np.zeros((3, 3), complex)
    Tl = np.zeros((3, 3), complex)
    for r, w in zip(qt, wt):
        for inner, part in inners:
            qs, ws = inner(r)
            d = r - qs
            R = np.linalg.norm(d, axis=1)
            G, g = _kernels(k, R, part)
            for a in range(3):
                ta = r - pa[a]
                for b in range(3):
                    fb = qs - pb[b]
                    cr = np.cross(d, fb)
                    Kl[a, b] += w * ca[a] * cb[b] * np.sum(ws * g * (cr @ ta))
                    Tl[a, b] += w * ca[a] * cb[b] * np.sum(ws * (-1j * k) * G * (fb @ ta - 4 / k ** 2))
    return Kl, Tl


@pytest.fixture(scope="module")
def sphere():
    g = W.icosphere(2, 0.3)
    return OM.build_rwg(g.verts, g.tris)


@pytest.mark.parametrize("k", [K_EXT, K_INT])
def test_far_block_vs_high_order(sphere, k):
    m = sphere
    c = (m.verts[m.tris].mean(axis=1))
    t = 0
    dist = np.linalg.norm(c - c[t], axis=1)
    for s in [int(np.argsort(dist)[40]), int(np.argmax(dist))]:
        Ko, To, near = mom.local_block(m, k, t, s)
        assert not near
        Vs = m.verts[m.tris[s]]
        qs, ws = _duffy_rule(Vs, Vs.mean(axis=0), nu=6, nv=12)
        Kr, Tr = _block_ref(m, k, t, s, [(lambda r: (qs, ws), 'full')])
        # outer rule is the same 7 points; compare against a converged outer too
        assert np.abs(To - Tr).max() < 2e-3 * np.abs(Tr).max()
        assert np.abs(Ko - Kr).max() < 2e-3 * np.abs(Kr).max()


@pytest.mark.parametrize("k", [K_EXT, K_INT])
@pytest.mark.parametrize("kind", ["self", "edge", "vertex"])
def test_near_block_singular_extraction(sphere, k, kind):
    m = sphere
    t = 5
    tv = set(m.tris[t].tolist())
    if kind == "self":
        s = t
    else:
        shared = [len(tv & set(m.tris[q].tolist())) for q in range(m.nt)]
        want = 2 if kind == "edge" else 1
        s = next(q for q in range(m.nt) if q != t and shared[q] == want)
    Ko, To, near = mom.local_block(m, k, t, s)
    assert near

    def inner_on(sidx):
        V = m.verts[m.tris[sidx]]
        nrm = np.cross(V[1] - V[0], V[2] - V[0])
        nrm /= np.linalg.norm(nrm)

        def f(r):
            rho = r - np.dot(nrm, r - V[0]) * nrm
            return _duffy_rule(V, rho, nu=40, nv=40)
        return f

    def seven_on(sidx):
        q, w = _quad7(m.verts[m.tris[sidx]])
        return lambda r: (q, w)

    # (1) same splitting, singular part by high-order quadrature: isolates the
    #     analytic integrals and how they are combined
    K1, T1 = _block_ref(m, k, t, s, [(inner_on(s), "singular"), (seven_on(s), "smooth")])
    K2, T2 = _block_ref(m, k, s, t, [(inner_on(t), "singular"), (seven_on(t), "smooth")])
    Kr = 0.5 * (K1 + K2.T)
    Tr = 0.5 * (T1 + T2.T)
    assert np.abs(To - Tr).max() < 1e-9 * np.abs(Tr).max()
    if kind == "self":
        assert np.abs(Ko).max() == 0.0
    else:
        assert np.abs(Ko - Kr).max() < 1e-8 * np.abs(Kr).max()
    # (2) against the exact inner integral of the unsplit kernel: the 7-point
    #     rule on the bounded remainder costs at most a small relative error
    K1, T1 = _block_ref(m, k, t, s, [(inner_on(s), "full")])
    K2, T2 = _block_ref(m, k, s, t, [(inner_on(t), "full")])
    Kx = 0.5 * (K1 + K2.T)
    Tx = 0.5 * (T1 + T2.T)
    assert np.abs(To - Tx).max() < 2e-3 * np.abs(Tx).max()
    if kind != "self":
        assert np.abs(Ko - Kx).max() < 2e-3 * np.abs(Kx).max()


@pytest.mark.parametrize("k", [K_EXT, K_INT, 2 * math.pi * complex(np.sqrt(3.0 - 0.1j))])
def test_blocks_transpose_under_exchange(sphere, k):
    """Exchanging test and trial triangle transposes a local block,
    L(s, t) = L(t, s)^T, for K and for T: G and |r - r'| are symmetric and the
    triple product f_a . ((r - r') x f_b') keeps its value when r <-> r' and
    a <-> b.  The discrete blocks keep it because both triangles use the same
    7-point rule (far pairs, each ordered pair evaluated on its own here) and
    because near blocks are symmetrised; the GPU path evaluates each unordered
    pair once on the strength of it."""
    m = sphere
    c = m.verts[m.tris].mean(axis=1)
    t = 3
    dist = np.linalg.norm(c - c[t], axis=1)
    order = np.argsort(dist)
    tv = set(m.tris[t].tolist())
    edge = next(q for q in range(m.nt) if q != t and len(tv & set(m.tris[q].tolist())) == 2)
    pairs = [(t, edge), (t, int(order[20])), (t, int(order[60])), (int(order[5]), int(np.argmax(dist)))]
    kinds = set()
    for (a, b) in pairs:
        K1, T1, n1 = mom.local_block(m, k, a, b)
        K2, T2, n2 = mom.local_block(m, k, b, a)
        assert n1 == n2
        kinds.add(n1)
        assert np.abs(K1 - K2.T).max() <= 1e-12 * np.abs(K1).max()
        assert np.abs(T1 - T2.T).max() <= 1e-12 * np.abs(T1).max()
    assert kinds == {True, False}   # near and far pairs both covered
