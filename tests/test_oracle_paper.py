"""P8: the paper's qualitative spectra (Sec. IV.A-B, Fig. 2) from the continuum transfer matrix
(CPU only), with the paper's parameters: 1-unit slab, nu0 = 1; Lorentz gamma = 0.04,
sigma = 5e-3; Lorentz-Bath gamma0 = 4e-4 with N = 100 bath modes over nu0 +/- 0.2 (Table I),
bath damping 4e-4, dephasing 0.0396; the cavity of Sec. IV.B (n = 10 mirrors) at sigma = 2e-2.

With bath modes 4e-4 wide and 0.004 apart the steady-state spectra of the Lorentz-Bath forms
are comb-like (each mode a sharp feature), so the checks are on what is robust: the Lorentz
line shape, and that the polaritons of the Lorentzian bath are the least damped (highest
transmission), the uniform bath next, the Lorentz medium of the same total width the most.

The reflectance used for the absorption is pinned first: for a lossless dielectric slab the
transfer matrix gives the Airy formula T = 1 / (1 + F sin^2 delta), F = ((n^2 - 1) / 2n)^2,
delta = n w L, and R = 1 - T."""
import json
import math
import pathlib

import numpy as np
import pytest

from oracle import closed_forms as cf
from test_oracle_tmm import paper_cavity

# the paper's printed parameters (tests/golden/paper_fig2_parameters.json, with citations)
GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_fig2_parameters.json").read_text())
NU0, GAMMA_L, SIGMA_SLAB = (GOLD["lorentz"][k] for k in ("frequency", "gamma", "sigma"))
LB = GOLD["lorentz_bath"]
CAV = GOLD["cavity"]
RES = 1.0 / GOLD["grid"]["dx"]


def slab(m):
    return dict(resolution=RES, materials=[dict(m, z=(0, int(round(CAV["gap"] * RES))))])


def lorentz(gamma=GAMMA_L, sigma=SIGMA_SLAB):
    return dict(kind="lorentz", eps_inf=1.0, frequency=NU0, gamma=gamma, sigma=sigma)


def bath(form, sigma=SIGMA_SLAB):
    width = 2.0 * LB["half_span_in_gamma"] * GAMMA_L
    f, g, k = cf.bath_form(form, NU0, LB["gamma0"], LB["num_bath"], width, LB["bath_gamma"], LB["dephasing"])
    return dict(kind="lorentz_bath", eps_inf=1.0, frequency=NU0, gamma=LB["gamma0"], sigma=sigma,
                bath_frequencies=f, bath_gammas=g, bath_couplings=k)


def absorption(nu, prob):
    return 1.0 - cf.transmission_continuum(nu, prob) - cf.reflectance_continuum(nu, prob)


def fwhm(nu, a):
    i = int(np.argmax(a))
    h = a[i] / 2.0
    lo, hi = i, i
    while lo > 0 and a[lo] > h:
        lo -= 1
    while hi < len(a) - 1 and a[hi] > h:
        hi += 1
    xl = nu[lo] + (h - a[lo]) * (nu[lo + 1] - nu[lo]) / (a[lo + 1] - a[lo])
    xr = nu[hi - 1] + (h - a[hi - 1]) * (nu[hi] - nu[hi - 1]) / (a[hi] - a[hi - 1])
    return nu[i], xr - xl


@pytest.mark.parametrize("eps", [2.25, 12.0])
def test_reflectance_airy_formula(eps):
    nu = np.linspace(0.3, 2.0, 171)
    p = dict(resolution=100.0, materials=[dict(kind="vacuum", z=(0, 37), eps_inf=eps)])
    n, L = math.sqrt(eps), 0.37
    F = ((n * n - 1.0) / (2.0 * n)) ** 2
    T = 1.0 / (1.0 + F * np.sin(n * 2.0 * math.pi * nu * L) ** 2)
    np.testing.assert_allclose(cf.transmission_continuum(nu, p), T, rtol=1e-12)
    np.testing.assert_allclose(cf.reflectance_continuum(nu, p), 1.0 - T, rtol=1e-11, atol=1e-14)


def test_p8_lorentz_slab_absorption_line():
    """Fig. 2a: the Lorentz slab absorbs at nu0 with a width set by gamma (the 1-unit slab
    absorbs ~half at the peak, which broadens the line; a thin slab shows gamma itself)."""
    nu = np.linspace(0.8, 1.2, 8001)
    peak, width = fwhm(nu, absorption(nu, slab(lorentz())))
    assert abs(peak - NU0) < 0.005
    assert GAMMA_L < width < 1.3 * GAMMA_L
    thin = dict(resolution=1000.0, materials=[dict(lorentz(), z=(0, 10))])   # 0.01 thick
    peak, width = fwhm(nu, absorption(nu, thin))
    assert abs(peak - NU0) < 0.002 and width == pytest.approx(GAMMA_L, rel=0.03)


def test_p8_bath_polaritons_least_damped():
    """Fig. 2b/2c: at sigma = 2e-2 the cavity splits into LP/UP near nu0 -/+ sqrt(sigma)/2 in
    every form; the Lorentzian bath (dephasing concentrated near nu0, weak at the polaritons)
    transmits the polaritons most, the uniform bath less, the Lorentz medium of the same total
    width (gamma = 0.04) least."""
    nu = np.linspace(0.85, 1.15, 15001)
    sig = CAV["sigma"][1]
    peaks = {}
    for name in ("lorentz", "uniform", "lorentzian"):
        p = (paper_cavity(sig, gamma=GAMMA_L) if name == "lorentz"
             else paper_cavity(sig, gamma=LB["gamma0"], kind="lorentz_bath"))
        if name != "lorentz":
            b = bath(name, sig)
            p["materials"][1].update({k: b[k] for k in ("bath_frequencies", "bath_gammas", "bath_couplings")})
        T = cf.transmission_continuum(nu, p)
        lp, up = T[nu < NU0], T[nu >= NU0]
        nlp, nup = nu[nu < NU0][np.argmax(lp)], nu[nu >= NU0][np.argmax(up)]
        assert nup - nlp == pytest.approx(math.sqrt(sig), rel=0.1), name
        peaks[name] = (lp.max(), up.max())
    for side in (0, 1):
        assert peaks["lorentzian"][side] > 1.5 * peaks["uniform"][side] > 1.5 * peaks["lorentz"][side]
