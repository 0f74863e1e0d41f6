"""Far field of the marched currents and the Mie series for a dielectric sphere
(test infrastructure only).

Far field (paper Section VI-C computes scattered far fields from the Fourier-
transformed surface currents; the paper gives no formula, so the standard
radiation integrals are used, e^{+j w t} phasors):
  J^(w) = sum_i j_i int p_i(t) e^{-j w t} dt,  M^ likewise, kept loop/star apart
  (Eq. (dis_jm) and the remark below it);
  E_inf(r) = (j k / 4 pi) [eta r x (r x N) + r x L],
  N = int J^(y) e^{j k r.y} dy,  L = int M^(y) e^{j k r.y} dy,
normalised by the spectrum of the incident pulse at the origin.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def dft_weights(omega: float, dt: float, n_steps: int) -> np.ndarray:
    """int p_i(t) e^{-j w t} dt for i = 1..n_steps (p_i = 1 on ((i-1)dt, i dt))."""
    i = np.arange(1, n_steps + 1)
    if omega == 0.0:
        return np.full(n_steps, dt, dtype=complex)
    return np.exp(-1j * omega * i * dt) * (np.exp(1j * omega * dt) - 1.0) / (1j * omega)


def radiation(rwg, coeff: np.ndarray, k: float, dirs: np.ndarray) -> np.ndarray:
    """int sum_m coeff_m f_m(y) e^{j k r.y} dy for unit directions dirs (nd, 3);
    coeff (ne,) complex. Uses the RWG quadrature table."""
    x = rwg.x                        # (ne, q, 3)
    ph = np.exp(1j * k * np.einsum("eqd,ad->aeq", x, dirs))   # (nd, ne, q)
    return np.einsum("aeq,eqd,e->ad", ph, rwg.wf, coeff)


def far_field(rwg, Jw: np.ndarray, Mw: np.ndarray, k: float, eta: float, dirs: np.ndarray) -> np.ndarray:
    """E_inf(r) = (j k/4pi) [eta r x (r x N) + r x L] (standard radiation
    integrals, medium of wavenumber k and impedance eta)."""
    N = radiation(rwg, Jw, k, dirs)
    L = radiation(rwg, Mw, k, dirs)
    rxN = np.cross(dirs, N)
    return (1j * k / (4 * np.pi)) * (eta * np.cross(dirs, rxN) + np.cross(dirs, L))


def pulse_spectrum(exc, b: int, omega: float, c: float = 1.0) -> complex:
    """Fourier transform of the incident pulse of Eq. (hin) at the origin (per
    unit polarisation): (A/c) e^{-j w t0} exp(-(w w_p / (8c))^2)."""
    return (exc.A[b] / c) * np.exp(-1j * omega * exc.t0[b]) * np.exp(-(omega * exc.w[b] / (8.0 * c)) ** 2)


# ---------------------------------------------------------------------------
# Mie series (textbook Lorenz-Mie theory for a homogeneous sphere)
# ---------------------------------------------------------------------------


def mie_coefficients(x: float, m: float, nmax: int | None = None):
    """a_n, b_n for size parameter x = k a and relative index m (mu_r = 1):
    a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)] / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
    b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)] / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)]
    with Riccati-Bessel psi_n(r) = r j_n(r), xi_n(r) = r h_n^(1)(r)."""
    if nmax is None:
        nmax = int(np.ceil(x + 4 * x ** (1 / 3) + 2)) + 2
    n = np.arange(1, nmax + 1)

    def psi(r):
        return r * spherical_jn(n, r)

    def dpsi(r):
        return spherical_jn(n, r) + r * spherical_jn(n, r, derivative=True)

    def xi(r):
        return r * (spherical_jn(n, r) + 1j * spherical_yn(n, r))

    def dxi(r):
        h = spherical_jn(n, r) + 1j * spherical_yn(n, r)
        dh = spherical_jn(n, r, derivative=True) + 1j * spherical_yn(n, r, derivative=True)
        return h + r * dh

    mx = m * x
    a = (m * psi(mx) * dpsi(x) - psi(x) * dpsi(mx)) / (m * psi(mx) * dxi(x) - xi(x) * dpsi(mx))
    b = (psi(mx) * dpsi(x) - m * psi(x) * dpsi(mx)) / (psi(mx) * dxi(x) - m * xi(x) * dpsi(mx))
    return n, a, b


def mie_amplitudes(x: float, m: float, theta: np.ndarray):
    """S1(theta), S2(theta) = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n), (a_n tau_n + b_n pi_n),
    pi_n = P_n^1(cos t)/sin t, tau_n = d P_n^1(cos t)/dt (upward recurrences)."""
    n, a, b = mie_coefficients(x, m)
    mu = np.cos(theta)
    S1 = np.zeros_like(theta, dtype=complex)
    S2 = np.zeros_like(theta, dtype=complex)
    pim1 = np.zeros_like(theta)
    pin = np.ones_like(theta)
    for idx, nn in enumerate(n):
        tau = nn * mu * pin - (nn + 1) * pim1
        f = (2 * nn + 1) / (nn * (nn + 1))
        S1 += f * (a[idx] * pin + b[idx] * tau)
        S2 += f * (a[idx] * tau + b[idx] * pin)
        pnext = ((2 * nn + 1) * mu * pin - (nn + 1) * pim1) / nn
        pim1, pin = pin, pnext
    return S1, S2
