"""The paper's own Fabry-Perot cavity through the GPU step kernels (Sec. IV.B, Fig. 1c, Figs.
2b/2c; the appendix's parameters, tests/golden/paper_fig2_parameters.json): two 0.02-thick
mirrors of refractive index 10 (eps_inf = 100, a vacuum-kind dielectric layer) 1 unit apart,
the gap filled by the molecular layer, dx = 0.01.

* Lorentz-Bath(L) layer, sigma = 2e-2 and 2e-3, gamma0 = 4e-4, the paper's N = 100 Lorentzian
  bath (Table I, dephasing 0.0396): GPU against the FP64 oracle over the pulse's transit of the
  cavity -- E, H, the layer's P and bath modes, the flux spectra and the energy traces of the
  gap (Fig. 2c's cavity energy, the polarization and bath shares).  With 100 modes the steps run
  the 3D step kernel's streamed-bath path on the 1D grid.
* The same cavity with a 16-mode bath runs the persistent 1D kernel (at most 32 modes).
* Transmission (Fig. 2b): with the Lorentz medium (gamma = 0.04, Fig. 2b top), which rings down
  within the run, the GPU's FDTD transmission (flux behind the cavity over the flux of the
  empty run) equals the discrete transfer matrix of the Yee lattice to the P4 level 3e-5; the
  paper's Lorentz-Bath cavity has bath resonances 4e-4 wide that ring for ~10^6 steps, so its
  transmission is compared with the oracle's over the same finite run instead (above).  Also the
  leaky Lorentz-Bath cavity of the P4 pin, on the persistent 1D kernel.
Tolerances: FP64 1e-12, FP32 1e-5 (fields, spectra, traces) / 1e-4 (P and bath modes)."""
import json
import pathlib

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb

pytestmark = pytest.mark.gpu

PAR = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_fig2_parameters.json").read_text())
CAV, LB = PAR["cavity"], PAR["lorentz_bath"]
TOL = {64: 1e-12, 32: 1e-5}
TOL_Y = {64: 1e-12, 32: 1e-4}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def cavity(layer, steps, nfreq=64):
    """CPML 16 | vacuum 200 | mirror 2 | gap 100 (layer) | mirror 2 | vacuum 200 | CPML 16 at
    dx = 0.01 (the paper's grid), a pulse 40 cells into the left vacuum, the flux monitor 40
    cells before the right CPML, the energy box = the gap."""
    res = 1.0 / PAR["grid"]["dx"]
    pml, vac = 16, 200
    gap, mir = int(round(CAV["gap"] * res)), int(round(CAV["mirror_thickness"] * res))
    z0 = pml + vac
    nz = 2 * pml + 2 * vac + gap + 2 * mir
    eps_m = CAV["mirror_index"] ** 2
    mats = [dict(kind="vacuum", z=(z0, z0 + mir), eps_inf=eps_m),
            dict(kind="vacuum", z=(z0 + mir + gap, z0 + 2 * mir + gap), eps_inf=eps_m)]
    if layer is not None:
        mats.insert(1, dict(layer, z=(z0 + mir, z0 + mir + gap)))
    t0 = 5.0 / (2.0 * np.pi * 0.5)
    return dict(name="paper_cavity", n=(1, 1, nz), resolution=res, courant=0.5, pml=pml, materials=mats,
                sources=[dict(component=0, z=pml + 40, center=1.0, fwidth=0.5, amplitude=1.0, t0=t0, phase=None)],
                monitors=[dict(z=nz - pml - 40, freqs=np.linspace(0.5, 1.5, nfreq))],
                energy_box=(z0 + mir, z0 + mir + gap), steps=steps)


def lb_layer(sigma, nb=LB["num_bath"]):
    width = 2 * LB["half_span_in_gamma"] * (LB["gamma0"] + LB["dephasing"])
    f, g, k = cf.bath_form("lorentzian", 1.0, LB["gamma0"], nb, width, LB["bath_gamma"], LB["dephasing"])
    return dict(kind="lorentz_bath", eps_inf=1.0, frequency=1.0, gamma=LB["gamma0"], sigma=sigma,
                bath_frequencies=f, bath_gammas=g, bath_couplings=k)


def check_against_oracle(prob, precision, steps):
    g = fb.Simulation(prob, precision=precision, energy_capacity=steps + 8)
    o = O.OracleSim(prob, trace_cap=steps + 8)
    g.step(steps)
    o.step(steps)
    for name in ("E", "H"):
        a = np.stack([g.get(name, comp=c) for c in range(3)])
        b = np.stack([o.get(name, comp=c) for c in range(3)])
        assert rel(a, b) < TOL[precision], name
    lo, hi = prob["materials"][1]["z"]
    for name in ("P", "Pm"):
        assert rel(g.get(name, comp=0)[lo:hi], o.get(name, comp=0)[lo:hi]) < TOL_Y[precision], name
    nb = len(prob["materials"][1]["bath_frequencies"])
    for j in (0, nb // 2, nb - 1):
        a = g.get("Y", comp=0, mode=j, level=0)[lo:hi]
        b = o.get("Y", comp=0, mode=j, level=0)[lo:hi]
        assert rel(a, b) < TOL_Y[precision], j
    assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    # U_EM to the field tolerance; U_P and U_bath, quadratic in P and the bath modes, to theirs
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < (TOL[precision] if col == 0 else TOL_Y[precision]), col
    assert to[:, 0].max() > 0 and to[:, 2].max() > 0   # the pulse entered the cavity, the bath took energy
    return g


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("sigma", CAV["sigma"])
def test_paper_cavity_lorentz_bath_100_modes_matches_oracle(precision, sigma):
    g = check_against_oracle(cavity(lb_layer(sigma), 3000), precision, 3000)
    assert not g.cavity_1d_kernel()   # 100 modes: the step kernel's streamed-bath path


@pytest.mark.parametrize("precision", [64, 32])
def test_paper_cavity_16_modes_on_the_1d_kernel(precision):
    g = check_against_oracle(cavity(lb_layer(CAV["sigma"][1], nb=16), 3000), precision, 3000)
    assert g.cavity_1d_kernel()


def transmission(prob, steps, precision=64):
    a = fb.Simulation(prob, precision=precision, energy=False)
    b = fb.Simulation(dict(prob, materials=[]), precision=precision, energy=False)
    a.step(steps)
    b.step(steps)
    flux = lambda s: np.real(s[:, 0] * np.conj(s[:, 3]) - s[:, 1] * np.conj(s[:, 2]))
    fa, fbv = flux(a.dft(0)), flux(b.dft(0))
    assert np.all(fbv > 0)
    return fa / fbv


def test_paper_cavity_lorentz_transmission_equals_discrete_tmm():
    lor = dict(kind="lorentz", eps_inf=1.0, frequency=1.0, gamma=PAR["lorentz"]["gamma"], sigma=CAV["sigma"][1])
    prob = cavity(lor, 0, nfreq=201)
    nu = prob["monitors"][0]["freqs"]
    # the cavity mode near 1.5 is 0.0054 wide: its amplitude falls by e every ~59 time units, so
    # the DFT needs ~1000 units (200000 steps) to hold less than 1e-7 of it
    T = transmission(prob, 200000)
    Td = cf.transmission_discrete(nu, prob)
    assert np.max(np.abs(T - Td)) < 3e-5
    assert T.max() > 0.5   # the uncoupled cavity mode near 0.5 transmits


def test_leaky_cavity_transmission_equals_discrete_tmm_on_gpu():
    from test_oracle_tmm import leaky_cavity
    p = leaky_cavity()
    nu = p["monitors"][0]["freqs"]
    T = transmission(p, 40000)
    assert np.max(np.abs(T - cf.transmission_discrete(nu, p))) < 3e-5
    assert T.max() > 0.9 and T.min() < 0.5
