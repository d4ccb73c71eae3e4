"""Closed forms the paper fixes, written out in numpy (test infrastructure only).

Everything here is in nu-units at the interface (nu = omega / 2 pi, as MEEP and
the paper report frequencies) and angular inside.  Units: c = eps0 = mu0 = 1.

* ``chi_lorentz`` -- Eq. (chi_L); ``chi_drude`` -- its Drude limit (w0^2 := 0 in
  the denominator only).
* ``self_energy`` / ``chi_lorentz_bath`` -- Eq. (chi_LB) and (chi_LB_self_energy).
* ``chi_discrete`` -- the exact frequency response of the explicit ADE updates
  (Eq. Pz_1D_Lorentz, Pz_update-LB, Yzj_finite_difference): a z-transform of
  the recursions with z = exp(-i w dt), Omega = 2 sin(w dt/2)/dt and
  Omega_s = sin(w dt)/dt in place of w.  It tends to Eq. (chi_LB) as dt -> 0.
* ``bath_form`` -- Table I (uniform / lorentzian / gaussian baths).
* ``transmission_discrete`` -- transfer matrix of the 1D Yee lattice in the
  frequency domain (every cell carries eps_inf + chi_discrete): the exact
  frequency-domain response of the discrete scheme between two vacuum regions.
* ``transmission_continuum`` -- textbook thin-film transfer matrices with the
  continuum susceptibilities.
* ``yee_omega`` -- Yee numerical dispersion, sin^2(w dt/2)/dt^2 = sum_d sin^2(k_d dx/2)/dx^2.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------- susceptibilities
def chi_lorentz(nu, frequency, gamma, sigma):
    """Eq. (chi_L): w0^2 sigma / (w0^2 - w^2 - i gamma w)."""
    w = TWO_PI * np.asarray(nu, dtype=np.complex128)
    w0, g = TWO_PI * frequency, TWO_PI * gamma
    return w0 ** 2 * sigma / (w0 ** 2 - w ** 2 - 1j * g * w)


def chi_drude(nu, frequency, gamma, sigma):
    """Drude limit: w0^2 := 0 in the denominator, w0^2 sigma kept in the numerator."""
    w = TWO_PI * np.asarray(nu, dtype=np.complex128)
    w0, g = TWO_PI * frequency, TWO_PI * gamma
    return w0 ** 2 * sigma / (-w ** 2 - 1j * g * w)


def self_energy(nu, bath_frequencies, bath_gammas, bath_couplings):
    """Eq. (chi_LB_self_energy): sum_j k_j^2 w^2 / (w_j^2 - w^2 - i gamma_j w)."""
    w = TWO_PI * np.asarray(nu, dtype=np.complex128)[..., None]
    wj = TWO_PI * np.asarray(bath_frequencies, dtype=np.float64)
    gj = TWO_PI * np.asarray(bath_gammas, dtype=np.float64)
    kj = TWO_PI * np.asarray(bath_couplings, dtype=np.float64)
    return np.sum(kj ** 2 * w ** 2 / (wj ** 2 - w ** 2 - 1j * gj * w), axis=-1)


def chi_lorentz_bath(nu, frequency, gamma, sigma, bath_frequencies, bath_gammas, bath_couplings):
    """Eq. (chi_LB): w0^2 sigma / (w0^2 - w^2 - i gamma0 w - Sigma(w))."""
    w = TWO_PI * np.asarray(nu, dtype=np.complex128)
    w0, g = TWO_PI * frequency, TWO_PI * gamma
    S = self_energy(nu, bath_frequencies, bath_gammas, bath_couplings)
    return w0 ** 2 * sigma / (w0 ** 2 - w ** 2 - 1j * g * w - S)


def chi_material(nu, m):
    """Continuum susceptibility of a material dict."""
    if m["kind"] == "lorentz":
        return chi_lorentz(nu, m["frequency"], m["gamma"], m["sigma"])
    if m["kind"] == "drude":
        return chi_drude(nu, m["frequency"], m["gamma"], m["sigma"])
    if m["kind"] == "lorentz_bath":
        return chi_lorentz_bath(nu, m["frequency"], m["gamma"], m["sigma"],
                                m["bath_frequencies"], m["bath_gammas"], m["bath_couplings"])
    return np.zeros_like(np.asarray(nu, dtype=np.complex128))


def chi_discrete(nu, dt, m):
    """Exact response P/E of the explicit ADE recursion at angular w = 2 pi nu.

    Lorentz: w0^2 sigma / (w0^2 - Omega^2 - i gamma Omega_s); Drude: w0^2 -> 0 in the
    denominator; Lorentz-Bath: w0^2 sigma / (w0^2 - Omega^2 - i gamma0 Omega_s - Sigma_d),
    Sigma_d = sum_j k_j^2 Omega_s^2 / (w_j^2 - Omega^2 - i gamma_j Omega_s).
    """
    w = TWO_PI * np.asarray(nu, dtype=np.float64)
    Om2 = (2.0 * np.sin(w * dt / 2.0) / dt) ** 2
    Oms = np.sin(w * dt) / dt
    kind = m["kind"]
    if kind == "vacuum":
        return np.zeros_like(w, dtype=np.complex128)
    w0, g, sig = TWO_PI * m["frequency"], TWO_PI * m["gamma"], m["sigma"]
    rest = 0.0 if kind == "drude" else w0 ** 2
    den = rest - Om2 - 1j * g * Oms
    if kind == "lorentz_bath":
        wj = TWO_PI * np.asarray(m["bath_frequencies"], dtype=np.float64)
        gj = TWO_PI * np.asarray(m["bath_gammas"], dtype=np.float64)
        kj = TWO_PI * np.asarray(m["bath_couplings"], dtype=np.float64)
        Sd = np.sum(kj ** 2 * Oms[..., None] ** 2
                    / (wj ** 2 - Om2[..., None] - 1j * gj * Oms[..., None]), axis=-1)
        den = den - Sd
    return w0 ** 2 * sig / den


# --------------------------------------------------------------------- Table I
def bath_form(form, frequency, gamma, num_bath, bath_width, bath_gamma, bath_dephasing):
    """Table I: bath frequencies evenly spaced over frequency +/- width/2, equal dampings,
    and couplings k_b = sqrt(2 dw / pi * dephasing), dw = width / (N - 1), modulated by
    sqrt(G^2/(G^2 + (w_j - w0)^2)) ('lorentzian') or exp(-(w_j - w0)^2 / (4 G^2)) ('gaussian'),
    G = gamma + dephasing.  Returns (frequencies, gammas, couplings)."""
    N = int(num_bath)
    wj = np.linspace(frequency - bath_width / 2.0, frequency + bath_width / 2.0, N)
    gj = np.full(N, float(bath_gamma))
    dw = bath_width / (N - 1)
    kb = math.sqrt(2.0 * dw / math.pi * bath_dephasing)
    G = gamma + bath_dephasing
    if form == "uniform":
        kj = np.full(N, kb)
    elif form == "lorentzian":
        kj = kb * np.sqrt(G ** 2 / (G ** 2 + (wj - frequency) ** 2))
    elif form == "gaussian":
        kj = kb * np.exp(-(wj - frequency) ** 2 / (4.0 * G ** 2))
    else:
        raise ValueError(form)
    return wj, gj, kj


# --------------------------------------------------------------------- transfer matrices
def _eps_profile_1d(prob, chi_of):
    nz = int(prob["n"][2])
    eps = [None] * nz
    for m in prob.get("materials", []):
        lo, hi = int(m["z"][0]), int(m["z"][1])
        for k in range(lo, hi):
            eps[k] = m
    return eps


def transmission_discrete(nu, prob, k_left=None, k_right=None):
    """|t|^2 of the 1D Yee lattice between two vacuum regions.

    Frequency-domain Yee equations (fields ~ exp(-i w t) at their own time levels):
        H(k) = H(k-1) + i Omega dx eps_k E(k),   E(k+1) = E(k) + i Omega dx H(k),
    Omega = 2 sin(w dt/2)/dt and eps_k = eps_inf + chi_discrete in material cells.  A unit
    transmitted wave E = exp(i K k dx) (sin(K dx/2) = Omega dx/2) is carried back through the
    structure and split into incident and reflected waves on the left.
    """
    nu = np.atleast_1d(np.asarray(nu, dtype=np.float64))
    dx = 1.0 / float(prob["resolution"])
    dt = float(prob["courant"]) * dx
    nz = int(prob["n"][2])
    mats = _eps_profile_1d(prob, None)
    mat_k = [k for k in range(nz) if mats[k] is not None]
    kL = (min(mat_k) - 3) if k_left is None else k_left
    kR = (max(mat_k) + 2) if k_right is None else k_right
    out = np.empty(nu.shape)
    for q, f in enumerate(nu):
        w = TWO_PI * f
        Om = 2.0 * math.sin(w * dt / 2.0) / dt
        K = 2.0 * math.asin(Om * dx / 2.0) / dx
        chis = {}
        E_next = np.exp(1j * K * (kR + 1) * dx)
        H = np.exp(1j * K * (kR + 0.5) * dx) * 2.0 * math.sin(K * dx / 2.0) / (Om * dx)
        Ek = {}
        for k in range(kR, kL - 1, -1):
            Ecur = E_next - 1j * Om * dx * H          # E(k) from E(k+1), H(k)
            m = mats[k]
            if m is None:
                eps = 1.0
            else:
                key = id(m)
                if key not in chis:
                    chis[key] = m.get("eps_inf", 1.0) + complex(chi_discrete(f, dt, m))
                eps = chis[key]
            H = H - 1j * Om * dx * eps * Ecur        # H(k-1) from H(k), E(k)
            Ek[k] = Ecur
            E_next = Ecur
        # split E(kL), E(kL+1) into A exp(iKk dx) + B exp(-iKk dx)
        u0, u1 = np.exp(1j * K * kL * dx), np.exp(1j * K * (kL + 1) * dx)
        M = np.array([[u0, 1.0 / u0], [u1, 1.0 / u1]])
        A, _B = np.linalg.solve(M, np.array([Ek[kL], Ek[kL + 1]]))
        out[q] = abs(1.0 / A) ** 2
    return out


def _continuum_matrix(f, layers, dx):
    """Characteristic matrix of the layered structure at frequency f (normal incidence):
    the product over layers (and vacuum gaps) of [[cos d, -i sin d / n], [-i n sin d, cos d]],
    d = n w L, n = sqrt(eps_inf + chi)."""
    w = TWO_PI * f
    Mt = np.eye(2, dtype=np.complex128)
    prev_hi = None
    for m in layers:
        lo, hi = m["z"]
        if prev_hi is not None and lo > prev_hi:  # vacuum gap
            d = w * (lo - prev_hi) * dx
            Mt = Mt @ np.array([[math.cos(d), -1j * math.sin(d)],
                                [-1j * math.sin(d), math.cos(d)]])
        eps = m.get("eps_inf", 1.0) + complex(chi_material(f, m))
        n = np.sqrt(eps)
        if n.imag < 0:
            n = -n
        d = n * w * (hi - lo) * dx
        Mt = Mt @ np.array([[np.cos(d), -1j * np.sin(d) / n], [-1j * n * np.sin(d), np.cos(d)]])
        prev_hi = hi
    return Mt


def transmission_continuum(nu, prob):
    """|t|^2 of the layered structure with continuum susceptibilities (normal incidence,
    vacuum on both sides): t = 2 / (M00 + M01 + M10 + M11) of the characteristic matrix."""
    nu = np.atleast_1d(np.asarray(nu, dtype=np.float64))
    dx = 1.0 / float(prob["resolution"])
    layers = sorted(prob.get("materials", []), key=lambda m: m["z"][0])
    out = np.empty(nu.shape)
    for q, f in enumerate(nu):
        Mt = _continuum_matrix(f, layers, dx)
        t = 2.0 / (Mt[0, 0] + Mt[0, 1] + Mt[1, 0] + Mt[1, 1])
        out[q] = abs(t) ** 2
    return out


def reflectance_continuum(nu, prob):
    """|r|^2 of the same structure: r = (M00 + M01 - M10 - M11) / (M00 + M01 + M10 + M11).
    The absorbed fraction is 1 - |t|^2 - |r|^2."""
    nu = np.atleast_1d(np.asarray(nu, dtype=np.float64))
    dx = 1.0 / float(prob["resolution"])
    layers = sorted(prob.get("materials", []), key=lambda m: m["z"][0])
    out = np.empty(nu.shape)
    for q, f in enumerate(nu):
        Mt = _continuum_matrix(f, layers, dx)
        r = (Mt[0, 0] + Mt[0, 1] - Mt[1, 0] - Mt[1, 1]) / (Mt[0, 0] + Mt[0, 1] + Mt[1, 0] + Mt[1, 1])
        out[q] = abs(r) ** 2
    return out


# --------------------------------------------------------------------- dispersion
def yee_omega(kvec, dx, dt):
    """Angular frequency of a discrete Yee plane wave with wave vector kvec."""
    s = sum(math.sin(k * dx / 2.0) ** 2 for k in kvec) / dx ** 2
    return 2.0 / dt * math.asin(dt * math.sqrt(s))
