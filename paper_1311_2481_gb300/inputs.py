"""Seeded synthetic initial states for the Taylor–Couette time step.

This module is shared by the CUDA path (tests, benchmark) and by the CPU oracle's
tests.  It draws random numbers and evaluates closed-form fields on radial nodes that
the caller supplies; it contains none of the time-step method's arithmetic (no finite
differences, transforms, products or solves).

Spectral layout (shared by every consumer): complex128 arrays of shape
``(3, N_r, M + 1, 2K + 1)`` holding (u_+, u_-, u_z) per radial node r_j, azimuthal mode
m = 0..M (the m < 0 half follows from the reality of u) and axial mode k = -K..K at index
k + K, where u_+ = u_r + i u_theta and u_- = u_r - i u_theta per Fourier mode (Sec. 3.1,
the change of variables before Eq. modalNSdecoup).

Recipes (all seeded through ``numpy.random.default_rng(seed)``):

* base flow: circular Couette flow U_theta = C1 r + C2 / r with the constants of Sec. 5.1,
  stored in the (m, k) = (0, 0) mode as u_+ = +i U, u_- = -i U;
* perturbation: u' = curl A with A_c(r, theta, z) = g(r) a_c exp(i(m m_p theta + k k_z z)),
  g = (r - r_i)^2 (r_o - r)^2, so that u' is divergence free and vanishes with its first
  radial derivative at both cylinders; the curl is written out analytically per mode;
* amplitude: the RMS of |u'| over the physical grid (mean over radial nodes, Parseval over
  theta and z) equals ``amp * Re_i``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "couette_constants",
    "couette_profile",
    "base_state",
    "curl_perturbation",
    "rms_amplitude",
    "initial_state",
    "random_spectral",
]


def couette_constants(eta: float, Re_i: float, Re_o: float):
    """C1, C2 of circular Couette flow U = C1 r + C2 / r (Sec. 5.1, laminar flow)."""
    C1 = (Re_o - eta * Re_i) / (1.0 + eta)
    C2 = eta * (Re_i - eta * Re_o) / ((1.0 - eta) * (1.0 - eta * eta))
    return C1, C2


def couette_profile(r, eta: float, Re_i: float, Re_o: float):
    C1, C2 = couette_constants(eta, Re_i, Re_o)
    r = np.asarray(r, dtype=np.float64)
    return C1 * r + C2 / r


def base_state(r, M: int, K: int, eta: float, Re_i: float, Re_o: float):
    """Circular Couette flow in the stored spectral layout."""
    r = np.asarray(r, dtype=np.float64)
    u = np.zeros((3, r.size, M + 1, 2 * K + 1), dtype=np.complex128)
    U = couette_profile(r, eta, Re_i, Re_o)
    u[0, :, 0, K] = 1j * U
    u[1, :, 0, K] = -1j * U
    return u


def _hermitian_m0(a, K):
    """Make the m = 0 line of coefficient array a[..., m, k] that of a real field."""
    a = a.copy()
    for k in range(1, K + 1):
        a[..., 0, K - k] = np.conj(a[..., 0, K + k])
    a[..., 0, K] = a[..., 0, K].real
    return a


def curl_perturbation(r, M, K, m_p, k_z, eta, coeff):
    """u' = curl(g(r) a) per Fourier mode, returned as (u_+, u_-, u_z) coefficients.

    ``coeff`` has shape (3, M + 1, 2K + 1): complex amplitudes a_r, a_theta, a_z.
    Cylindrical curl per mode (d_theta -> i m m_p, d_z -> i k k_z):
      (curl A)_r     = i m m_p A_z / r - i k k_z A_theta
      (curl A)_theta = i k k_z A_r - dA_z/dr
      (curl A)_z     = (1/r) d(r A_theta)/dr - i m m_p A_r / r
    """
    r = np.asarray(r, dtype=np.float64)
    r_i = eta / (1.0 - eta)
    r_o = 1.0 / (1.0 - eta)
    g = (r - r_i) ** 2 * (r_o - r) ** 2
    dg = 2.0 * (r - r_i) * (r_o - r) ** 2 - 2.0 * (r - r_i) ** 2 * (r_o - r)
    im = 1j * m_p * np.arange(M + 1)[None, :, None]
    ik = 1j * k_z * np.arange(-K, K + 1)[None, None, :]
    rr = r[:, None, None]
    gg = g[:, None, None]
    dgg = dg[:, None, None]
    a_r, a_t, a_z = (coeff[c][None, :, :] for c in range(3))
    ur = im * a_z * gg / rr - ik * a_t * gg
    ut = ik * a_r * gg - a_z * dgg
    uz = a_t * (gg / rr + dgg) - im * a_r * gg / rr
    out = np.empty((3, r.size, M + 1, 2 * K + 1), dtype=np.complex128)
    out[0] = ur + 1j * ut
    out[1] = ur - 1j * ut
    out[2] = uz
    return out


def rms_amplitude(u_pm_z, K):
    """RMS of |u| over the physical grid for (u_+, u_-, u_z) coefficients (Parseval)."""
    up, um, uz = u_pm_z
    dens = 0.5 * (np.abs(up) ** 2 + np.abs(um) ** 2) + np.abs(uz) ** 2  # |u_r|^2+|u_t|^2+|u_z|^2
    w = np.full(dens.shape[1], 2.0)
    w[0] = 1.0
    per_r = np.einsum("rmk,m->r", dens, w)
    return float(np.sqrt(per_r.mean()))


def _coeff_box(rng, M, K, mbox, kbox, taper=None):
    a = rng.standard_normal((3, M + 1, 2 * K + 1)) + 1j * rng.standard_normal((3, M + 1, 2 * K + 1))
    m = np.arange(M + 1)[:, None]
    k = np.arange(-K, K + 1)[None, :]
    mask = (m <= mbox) & (np.abs(k) <= kbox)
    mask[0, K] = False
    a = a * mask[None]
    if taper is not None:
        a = a * taper(m, k)[None]
    return _hermitian_m0(a, K)


def initial_state(r, M, K, m_p, L_z, eta, Re_i, Re_o, kind="box", amp=1e-3, seed=42,
                  mbox=4, kbox=4):
    """Couette flow plus a seeded divergence-free perturbation of RMS amp * Re_i.

    kind:
      'box'       random vector potential on |m| <= mbox, |k| <= kbox, (0,0) excluded;
      'taylor'    A_theta = g(r) cos(k_z z) scaled to amp, plus box noise (|m|<=4, |k|<=8)
                  scaled to amp / 10;
      'broadband' random coefficients on all stored modes with the Gaussian taper
                  exp(-(m/(M/4))^2 - (k/(K/4))^2).
    """
    k_z = 2.0 * np.pi / L_z
    rng = np.random.default_rng(seed)
    u = base_state(r, M, K, eta, Re_i, Re_o)
    target = amp * abs(Re_i)

    def scaled(coeff, level):
        up = curl_perturbation(r, M, K, m_p, k_z, eta, coeff)
        s = rms_amplitude(up, K)
        return up * (level / s) if s > 0 else up

    if kind == "box":
        u += scaled(_coeff_box(rng, M, K, mbox, kbox), target)
    elif kind == "taylor":
        c = np.zeros((3, M + 1, 2 * K + 1), dtype=np.complex128)
        if K >= 1:
            c[1, 0, K + 1] = 0.5
            c[1, 0, K - 1] = 0.5
        u += scaled(c, target)
        u += scaled(_coeff_box(rng, M, K, min(4, M), min(8, K)), target / 10.0)
    elif kind == "broadband":
        def taper(m, k):
            return np.exp(-(m / max(M / 4.0, 1e-300)) ** 2 - (k / max(K / 4.0, 1e-300)) ** 2)
        u += scaled(_coeff_box(rng, M, K, M, K, taper), target)
    else:
        raise ValueError(f"unknown perturbation kind {kind!r}")
    return u


def random_spectral(shape, seed, hermitian_K=None, scale=1.0):
    """Seeded complex normal coefficients (for operator-level parity tests).

    If ``hermitian_K`` is given the trailing two axes are (m, k) and the m = 0 line is made
    that of a real field."""
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale
    if hermitian_K is not None:
        a = _hermitian_m0(a, hermitian_K)
    return a
