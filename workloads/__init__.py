"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only produces *inputs*: closed triangle meshes (vertex array +
outward-oriented triangle array), incident-wave direction sets and RCS
observation grids.  It contains none of the method's arithmetic (no RWG
functions, no cells, no Green's functions) so that the CPU oracle and the CUDA
path can both consume it without sharing any of the computation they are
compared on.

Units: lengths in free-space wavelengths (lambda0 = 1).  Angles in radians.
A direction triple (theta, phi, psi) names a plane wave *arriving from*
r_hat(theta, phi) with polarisation cos(psi) theta_hat + sin(psi) phi_hat.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "icosphere", "cube", "cylinder", "spheroid", "sphere_array",
    "fibonacci_dirs", "plane_wave_set", "bistatic_cut", "cube_c2", "sphere_c1",
    "scatterer_mix", "spheroid_c5",
]


@dataclass
class Mesh:
    """A closed, outward-oriented triangle surface."""
    verts: np.ndarray            # (nv, 3) float64
    tris: np.ndarray             # (nt, 3) int32, counter-clockwise seen from outside
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])


def _orient_outward(verts: np.ndarray, tris: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """Flip triangles whose normal points towards `centre` (star-shaped bodies only)."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    out = (a + b + c) / 3.0 - centre
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


def icosphere(level: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)) -> Mesh:
    """Icosahedron subdivided `level` times, vertices projected onto the sphere.

    level 2 gives 162 vertices / 320 triangles / 480 edges.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = list(f)
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(centre, dtype=np.float64)
    T = np.array(faces, dtype=np.int32)
    T = _orient_outward(V, T, np.asarray(centre, dtype=np.float64))
    return Mesh(V, T.astype(np.int32), f"icosphere{level}", {"radius": radius})


def _surface_grid(n: int):
    """Vertices of the n x n x n surface lattice of the unit cube [0,n]^3 (integer coords)."""
    idx = {}
    pts = []
    for i in range(n + 1):
        for j in range(n + 1):
            for k in range(n + 1):
                if i in (0, n) or j in (0, n) or k in (0, n):
                    idx[(i, j, k)] = len(pts)
                    pts.append((i, j, k))
    return idx, np.array(pts, dtype=np.float64)


def cube(n: int, side: float = 1.0, centre=(0.0, 0.0, 0.0)) -> Mesh:
    """Cube with n x n squares per face, every square split along the same
    face-local diagonal (from local (0,0) to (1,1)).  T = 12 n^2."""
    idx, P = _surface_grid(n)
    tris = []
    # each face: fixed axis `ax` at value `val`; local axes (u, w)
    for ax in range(3):
        u_ax, w_ax = [a for a in range(3) if a != ax]
        for val in (0, n):
            for i in range(n):
                for j in range(n):
                    def vid(di, dj):
                        c = [0, 0, 0]
                        c[ax] = val
                        c[u_ax] = i + di
                        c[w_ax] = j + dj
                        return idx[tuple(c)]
                    v00, v10, v01, v11 = vid(0, 0), vid(1, 0), vid(0, 1), vid(1, 1)
                    tris.append((v00, v10, v11))
                    tris.append((v00, v11, v01))
    V = (P / n - 0.5) * side + np.asarray(centre, dtype=np.float64)
    T = _orient_outward(V, np.array(tris, dtype=np.int32), np.asarray(centre, dtype=np.float64))
    return Mesh(V, T.astype(np.int32), f"cube{n}", {"side": side})


def cylinder(radius: float, height: float, n_phi: int, n_z: int, n_r: int,
             centre=(0.0, 0.0, 0.0)) -> Mesh:
    """Finite circular cylinder (axis z) with flat capped ends.

    Side: n_z rings of n_phi quads; caps: n_r concentric rings around a
    centre vertex.  Every quad is split along a fixed diagonal.
    """
    verts = []
    vid = {}

    def add(key, xyz):
        if key not in vid:
            vid[key] = len(verts)
            verts.append(xyz)
        return vid[key]

    def ring_pt(r_i, z_i, p):
        # r_i in 0..n_r (n_r = rim), z_i in 0..n_z (0 bottom, n_z top)
        z = -height / 2 + height * z_i / n_z
        if r_i == 0:
            return ("c", z_i), (0.0, 0.0, z)
        r = radius * r_i / n_r
        ph = 2 * math.pi * (p % n_phi) / n_phi
        key = ("rim", z_i, p % n_phi) if r_i == n_r else ("cap", z_i, r_i, p % n_phi)
        return key, (r * math.cos(ph), r * math.sin(ph), z)

    tris = []
    # side
    for zi in range(n_z):
        for p in range(n_phi):
            a = add(*ring_pt(n_r, zi, p))
            b = add(*ring_pt(n_r, zi, p + 1))
            c = add(*ring_pt(n_r, zi + 1, p + 1))
            d = add(*ring_pt(n_r, zi + 1, p))
            tris += [(a, b, c), (a, c, d)]
    # caps
    for zi in (0, n_z):
        for ri in range(n_r):
            for p in range(n_phi):
                if ri == 0:
                    c0 = add(*ring_pt(0, zi, 0))
                    a = add(*ring_pt(1, zi, p))
                    b = add(*ring_pt(1, zi, p + 1))
                    tris.append((c0, a, b))
                else:
                    a = add(*ring_pt(ri, zi, p))
                    b = add(*ring_pt(ri, zi, p + 1))
                    c = add(*ring_pt(ri + 1, zi, p + 1))
                    d = add(*ring_pt(ri + 1, zi, p))
                    tris += [(a, b, c), (a, c, d)]
    V = np.array(verts, dtype=np.float64) + np.asarray(centre, dtype=np.float64)
    T = _orient_outward(V, np.array(tris, dtype=np.int32), np.asarray(centre, dtype=np.float64))
    return Mesh(V, T.astype(np.int32), "cylinder", {"radius": radius, "height": height})


def spheroid(a_z: float, b_xy: float, n_rings: int, n_lon: int,
             centre=(0.0, 0.0, 0.0)) -> Mesh:
    """Prolate spheroid (semi-axis a_z along z, b_xy across) as a lat-long mesh.

    `n_rings` interior latitude rings spaced uniformly in meridian arc length,
    `n_lon` longitudes, two pole vertices.  T = 2 n_lon n_rings.
    """
    # meridian (x = b sin t, z = a cos t), t in [0, pi]; uniform arc length
    t = np.linspace(0.0, math.pi, 20001)
    dx = np.gradient(b_xy * np.sin(t), t)
    dz = np.gradient(a_z * np.cos(t), t)
    s = np.concatenate([[0.0], np.cumsum(0.5 * (np.hypot(dx[1:], dz[1:]) + np.hypot(dx[:-1], dz[:-1])) * np.diff(t))])
    targets = np.linspace(0.0, s[-1], n_rings + 2)[1:-1]
    tr = np.interp(targets, s, t)
    verts = [(0.0, 0.0, a_z)]
    for ti in tr:
        for p in range(n_lon):
            ph = 2 * math.pi * p / n_lon
            verts.append((b_xy * math.sin(ti) * math.cos(ph), b_xy * math.sin(ti) * math.sin(ph), a_z * math.cos(ti)))
    verts.append((0.0, 0.0, -a_z))
    south = len(verts) - 1

    def rv(r, p):
        return 1 + r * n_lon + (p % n_lon)

    tris = []
    for p in range(n_lon):
        tris.append((0, rv(0, p), rv(0, p + 1)))
    for r in range(n_rings - 1):
        for p in range(n_lon):
            a, b, c, d = rv(r, p), rv(r + 1, p), rv(r + 1, p + 1), rv(r, p + 1)
            tris += [(a, b, c), (a, c, d)]
    for p in range(n_lon):
        tris.append((south, rv(n_rings - 1, p + 1), rv(n_rings - 1, p)))
    V = np.array(verts, dtype=np.float64) + np.asarray(centre, dtype=np.float64)
    T = _orient_outward(V, np.array(tris, dtype=np.int32), np.asarray(centre, dtype=np.float64))
    return Mesh(V, T.astype(np.int32), "spheroid", {"a": a_z, "b": b_xy})


def sphere_array(nx: int, ny: int, nz: int, spacing: float, level: int = 2,
                 radius: float = 1.0 / 6.0) -> Mesh:
    """nx x ny x nz array of identical disjoint icospheres (one body each)."""
    vs, ts = [], []
    off = 0
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                c = ((ix - (nx - 1) / 2) * spacing, (iy - (ny - 1) / 2) * spacing, (iz - (nz - 1) / 2) * spacing)
                m = icosphere(level, radius, c)
                vs.append(m.verts)
                ts.append(m.tris + off)
                off += m.nv
    return Mesh(np.concatenate(vs), np.concatenate(ts).astype(np.int32), f"array{nx}x{ny}x{nz}",
                {"bodies": nx * ny * nz})


# ------------------------------------------------------------------ directions

def fibonacci_dirs(n: int) -> np.ndarray:
    """n directions (theta, phi) on a Fibonacci sphere lattice, shape (n, 2)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    th = np.arccos(np.clip(z, -1.0, 1.0))
    ph = np.mod(i * math.pi * (3.0 - math.sqrt(5.0)), 2.0 * math.pi)
    return np.stack([th, ph], axis=1)


def plane_wave_set(dirs: np.ndarray, pols=(0.0, math.pi / 2)) -> np.ndarray:
    """Every direction with every polarisation angle psi -> (s, 3) of (theta, phi, psi)."""
    out = [(t, p, q) for (t, p) in np.asarray(dirs) for q in pols]
    return np.array(out, dtype=np.float64)


def bistatic_cut(step_deg: float = 1.0, phis_deg=(0.0, 90.0)) -> np.ndarray:
    """Observation directions theta in [0, 180] deg for each listed phi -> (n, 2)."""
    th = np.deg2rad(np.arange(0.0, 180.0 + 1e-9, step_deg))
    return np.array([(t, math.radians(p)) for p in phis_deg for t in th], dtype=np.float64)


# ------------------------------------------------------------- named workloads

def sphere_c1():
    """Dielectric sphere, radius 0.3, eps_r 4, icosphere level 2 (N = 960),
    12 Fibonacci directions x 2 polarisations for CBF generation, one
    excitation arriving from theta = 0 with x polarisation."""
    mesh = icosphere(2, 0.3)
    gen = plane_wave_set(fibonacci_dirs(12))
    exc = np.array([[0.0, 0.0, 0.0]])
    return dict(mesh=mesh, eps=(4.0, 0.0), ncell=8, partition="octant", gen=gen, exc=exc,
                obs=bistatic_cut(1.0))


def cube_c2(n_rhs: int = 128):
    """Cube of side 1, eps_r 2.5, 16 x 16 squares per face (T = 3072, E = 4608,
    N = 9216), 32 cells, 64 Fibonacci directions x 2 polarisations (s = 128)
    for CBF generation.  Excitations: `n_rhs` monostatic plane waves on a
    Fibonacci set of n_rhs/2 directions x {theta, phi} polarisation."""
    mesh = cube(16, 1.0)
    gen = plane_wave_set(fibonacci_dirs(64))
    exc = plane_wave_set(fibonacci_dirs(max(1, n_rhs // 2)))[:n_rhs]
    obs = exc[:, :2].copy()
    return dict(mesh=mesh, eps=(2.5, 0.0), ncell=32, partition="rcb", gen=gen, exc=exc, obs=obs)


def spheroid_c5(n_dirs: int = 256):
    """Lossy prolate spheroid, semi-axes 2 (z) and 0.5 (x, y), eps_r 3 - 0.1j,
    100 rings x 150 longitudes (T = 30000, E = 45000, N = 90000), 256 RCB cells,
    `n_dirs` Fibonacci directions x 2 polarisations as generating waves and as
    monostatic excitations."""
    mesh = spheroid(2.0, 0.5, 100, 150)
    waves = plane_wave_set(fibonacci_dirs(n_dirs))
    return dict(mesh=mesh, eps=(3.0, -0.1), ncell=256, partition="rcb", gen=waves, exc=waves,
                obs=waves[:, :2].copy())


def scatterer_mix(count: int, seed: int = 0):
    """Seeded mix of spheres, cubes and finite cylinders of size 0.2-1.2,
    eps_r ~ U[1.5, 6], with meshes of 500-6000 unknowns."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = int(rng.integers(0, 3))
        size = float(rng.uniform(0.2, 1.2))
        eps = float(rng.uniform(1.5, 6.0))
        if kind == 0:
            lvl = int(rng.integers(2, 4))           # 960 or 3840 unknowns
            m = icosphere(lvl, size / 2)
        elif kind == 1:
            n = int(rng.integers(4, 13))            # N = 36 n^2
            m = cube(n, size)
        else:
            nphi = int(rng.integers(10, 25))
            m = cylinder(size / 2, size, nphi, int(rng.integers(3, 10)), 2)
        out.append(dict(mesh=m, eps=(eps, 0.0)))
    return out


def random_cbfs(Ns, Ls, seed: int = 0):
    """Seeded complex Gaussian blocks (N_m, L_m) standing in for C^M and C^J
    when the projection is tested on its own (the projection is linear in C)."""
    rng = np.random.default_rng(seed)
    CM = [(rng.standard_normal((n, l)) + 1j * rng.standard_normal((n, l))) / np.sqrt(2 * n) for n, l in zip(Ns, Ls)]
    CJ = [(rng.standard_normal((n, l)) + 1j * rng.standard_normal((n, l))) / np.sqrt(2 * n) for n, l in zip(Ns, Ls)]
    return CM, CJ
