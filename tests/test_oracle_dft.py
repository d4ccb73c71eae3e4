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
- the flux Re(E_x H_y* - E_y H_x*) of a +z travelling pulse is positive;
- the absolute spectrum at a plane is the soft source's radiation on the lattice, dx J(omega) /
  (2 cos(kappa dx / 2)) exp(i kappa dz), with J(omega) the closed-form transform of the pulse,
  which fixes the source's amplitude, carrier, delay and sampling time and the dt of the DFT."""
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


def test_p11_source_sheet_radiates_the_pulse_spectrum():
    """The absolute spectrum of the soft source's pulse at a monitor plane.  A current sheet on
    one plane of the 1D Yee lattice, added as dt J(t_n) to D at t_n = n dt, radiates on either
    side the field amplitude dx J(omega) / (2 cos(kappa dx / 2)) per frequency (from the update
    at the source plane with outgoing lattice waves; dx J / 2 in the continuum limit), carried to
    the monitor by exp(i kappa dz).  J(omega) is the Fourier transform of the Gaussian-modulated
    sine in closed form, sqrt(2 pi) tau / (2i) e^{i omega t0} (e^{-tau^2 (omega + omega_c)^2 / 2}
    - e^{-tau^2 (omega - omega_c)^2 / 2}).  Agreement to 5e-5 (the pulse's truncation at t = 0,
    ~4e-6 of its peak, and the absorbers' 6e-6 reflections); sampling the source at (n + 1/2) dt
    would be off by 5e-2, the continuum formula by 4e-2."""
    S, M = PML + 50, PML + 250
    p = wl.slab_cavity(1, 1, (PML, 400, 0, 0, 0, 100), RES, num_bath=0, sigma=0.01,
                       phase_seed=None, nfreq=4, steps=10, src_z=S)
    p = wl.vacuum_of(p)
    p["monitors"] = [dict(z=M, freqs=FREQS)]
    src = p["sources"][0]
    dx = 1.0 / RES
    dt = p["courant"] * dx
    tau = 1.0 / (2 * np.pi * src["fwidth"])
    t0, wc, amp = src["t0"], 2 * np.pi * src["center"], src["amplitude"]
    steps = int((t0 + 12 * tau + (M - S) * dx + 1.0) / dt)
    o = O.OracleSim(p)
    o.step(steps)
    F = o.dft(0)[:, 0]
    w = 2 * np.pi * FREQS
    kappa = 2.0 / dx * np.arcsin(dx / dt * np.sin(w * dt / 2))
    J = amp * np.exp(1j * w * t0) * tau * np.sqrt(2 * np.pi) / 2j * (
        np.exp(-tau ** 2 * (w + wc) ** 2 / 2) - np.exp(-tau ** 2 * (w - wc) ** 2 / 2))
    want = dx / (2 * np.cos(kappa * dx / 2)) * np.exp(1j * kappa * (M - S) * dx) * J
    assert rel(F, want) < 5e-5
    assert rel(F, dx / 2 * np.exp(1j * w * (M - S) * dx) * J) > 1e-2
