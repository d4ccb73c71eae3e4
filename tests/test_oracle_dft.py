"""P11: the running-DFT monitors against closed forms of the Yee lattice (no oracle formula
retyped).  A vacuum pulse passes two monitor planes in the 1D line.  For every frequency:

- the spectra of the two planes differ by the lattice propagator, F(z2) / F(z1) =
  exp(i kappa (z2 - z1) dx) with kappa the Yee wavenumber, sin(kappa dx / 2) / dx =
  sin(omega dt / 2) / dt (not the continuum omega, which is off by ~4e-2 here), so the DFT
  kernel is exp(+i omega t) with E sampled where the scheme puts it;
- at one plane, H (mean of the two H planes around the E plane, sampled at the step's end)
  over E (sampled at the half step) is the discrete impedance ratio cos(kappa dx / 2) for E_x /
  H_y and -cos(kappa dx / 2) for E_y / H_x, which fixes the half-step time offset between the E
  and H samples (an offset of dt / 2 would leave a phase of ~5e-2) and the averaging of the
  two H planes;
- the flux Re(E_x H_y* - E_y H_x*) of a +z travelling pulse is positive."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import workloads as wl

RES, PML = 50.0, 16
FREQS = np.linspace(0.5, 1.5, 21)
Z1, Z2 = PML + 150, PML + 350


def run(component: int):
    p = wl.slab_cavity(1, 1, (PML, 400, 0, 0, 0, 100), RES, num_bath=0, sigma=0.01,
                       phase_seed=None, nfreq=4, steps=10, src_z=PML + 50,
                       source_component=component)
    p = wl.vacuum_of(p)
    p["monitors"] = [dict(z=Z1, freqs=FREQS), dict(z=Z2, freqs=FREQS)]
    dx = 1.0 / RES
    dt = p["courant"] * dx
    tau = 1.0 / (2 * np.pi * p["sources"][0]["fwidth"])
    # until the pulse (12 widths long) has passed the far plane
    steps = int((p["sources"][0]["t0"] + 12 * tau + (Z2 - PML - 50) * dx + 1.0) / dt)
    o = O.OracleSim(p)
    o.step(steps)
    w = 2 * np.pi * FREQS
    kappa = 2.0 / dx * np.arcsin(dx / dt * np.sin(w * dt / 2))
    return o.dft(0), o.dft(1), kappa, w, dx


def rel(a, b):
    return float(np.max(np.abs(a / b - 1.0)))


@pytest.mark.parametrize("component", [0, 1])
def test_p11_monitor_spectra_follow_the_yee_propagator(component):
    F1, F2, kappa, w, dx = run(component)
    e = component          # spectra columns: E_x, E_y, H_x, H_y
    assert rel(F2[:, e] / F1[:, e], np.exp(1j * kappa * (Z2 - Z1) * dx)) < 1e-6
    assert rel(F2[:, e] / F1[:, e], np.exp(1j * w * (Z2 - Z1) * dx)) > 1e-2
    h, sign = (3, 1.0) if component == 0 else (2, -1.0)
    for F in (F1, F2):
        assert rel(F[:, h] / F[:, e], sign * np.cos(kappa * dx / 2)) < 1e-6
        assert np.all(O.flux(F) > 0)
        other = 1 - component
        assert np.max(np.abs(F[:, other])) == 0.0
