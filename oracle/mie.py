"""Mie series for a homogeneous dielectric sphere (physics pin for the oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Written from the textbook treatment of Bohren & Huffman, "Absorption and
Scattering of Light by Small Particles" (1983), Ch. 4: coefficients a_n, b_n
from Riccati-Bessel functions psi_n, xi_n = psi_n - i chi_n and the
logarithmic derivative D_n(mx) (downward recurrence); angular functions
pi_n, tau_n by upward recurrence; amplitudes S1, S2.  The textbook uses
exp(-i omega t); intensities |S|^2 do not depend on that choice, and a passive
eps_r = e' - j e'' (exp(+j omega t)) enters as m = conj(sqrt(eps_r)).
"""
from __future__ import annotations

import math

import numpy as np


def mie_coefficients(x: float, m: complex, nmax: int | None = None):
    if nmax is None:
        nmax = int(round(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 4
    mx = m * x
    nmx = int(max(nmax, abs(mx))) + 30
    D = np.zeros(nmx + 1, np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_m1, psi_0 = math.cos(x), math.sin(x)
    chi_m1, chi_0 = -math.sin(x), math.cos(x)
    a = np.zeros(nmax, np.complex128)
    b = np.zeros(nmax, np.complex128)
    for n in range(1, nmax + 1):
        psi = (2 * n - 1) / x * psi_0 - psi_m1
        chi = (2 * n - 1) / x * chi_0 - chi_m1
        xi = psi - 1j * chi
        xi_1 = psi_0 - 1j * chi_0
        ta = D[n] / m + n / x
        tb = m * D[n] + n / x
        a[n - 1] = (ta * psi - psi_0) / (ta * xi - xi_1)
        b[n - 1] = (tb * psi - psi_0) / (tb * xi - xi_1)
        psi_m1, psi_0 = psi_0, psi
        chi_m1, chi_0 = chi_0, chi
    return a, b


def amplitudes(a: np.ndarray, b: np.ndarray, theta: np.ndarray):
    """S1(theta), S2(theta) with theta the scattering angle."""
    mu = np.cos(np.asarray(theta, float))
    S1 = np.zeros(mu.shape, np.complex128)
    S2 = np.zeros(mu.shape, np.complex128)
    p_nm2 = np.zeros_like(mu)          # pi_{n-2}
    p_nm1 = np.zeros_like(mu)          # pi_{n-1}
    for n in range(1, len(a) + 1):
        if n == 1:
            p_n = np.ones_like(mu)
        else:
            p_n = (2 * n - 1) / (n - 1) * mu * p_nm1 - n / (n - 1) * p_nm2
        t_n = n * mu * p_n - (n + 1) * p_nm1
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * p_n + b[n - 1] * t_n)
        S2 += f * (a[n - 1] * t_n + b[n - 1] * p_n)
        p_nm2, p_nm1 = p_nm1, p_n
    return S1, S2


def efficiencies(x: float, a: np.ndarray, b: np.ndarray):
    n = np.arange(1, len(a) + 1)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * (a + b).real)
    return qext, qsca


def sphere_rcs(radius: float, eps_r: complex, obs: np.ndarray, k0: float = 2.0 * math.pi):
    """Partial bistatic RCS (sigma_theta, sigma_phi) of a sphere at the origin
    for a unit plane wave arriving from theta = 0 (travelling along -z) with
    x polarisation, observed at directions obs (n, 2) = (theta, phi).

    Rotating the textbook frame (incidence along +z) by pi about x maps the
    observation (theta, phi) to scattering angle pi - theta, azimuth -phi.
    """
    m = np.conj(np.sqrt(complex(eps_r)))
    x = k0 * radius
    a, b = mie_coefficients(x, m)
    th = np.asarray(obs)[:, 0]
    ph = np.asarray(obs)[:, 1]
    S1, S2 = amplitudes(a, b, math.pi - th)
    c = 4.0 * math.pi / k0 ** 2
    return c * np.abs(S2) ** 2 * np.cos(ph) ** 2, c * np.abs(S1) ** 2 * np.sin(ph) ** 2
