"""P4: the oracle against transfer-matrix closed forms (CPU only).

* The FDTD transmission (DFT flux through a plane behind the structure, divided by the
  same flux without the structure) equals |t|^2 of the 1D Yee lattice solved in the
  frequency domain with chi_discrete in every material cell -- the exact frequency-domain
  response of the scheme -- up to CPML reflection.
* That discrete transfer matrix tends to the continuum one built from Eq. chi_L / chi_LB.
* In the paper's Fabry-Perot cavity (Sec. IV.B and the appendix: n = 10 mirrors 0.02 thick,
  d = 1, slab filling the cavity) the transfer-matrix polariton splitting equals the
  closed form w0 sqrt(sigma) that follows from Eq. chi_L for a resonant, filled cavity.
"""
import json
import math
import pathlib

import numpy as np
import pytest
from scipy.signal import find_peaks

from oracle import closed_forms as cf
from oracle import oracle as O
from paper_2505_23963_gb300 import workloads as wl

# the paper's cavity (tests/golden/paper_fig2_parameters.json, with citations)
CAV = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_fig2_parameters.json").read_text())["cavity"]


def leaky_cavity():
    """Lorentz-Bath layer between thin, weak Drude mirrors: rings down within ~40000 steps."""
    p = wl.slab_cavity(1, 1, (16, 200, 3, 300, 3, 200), 100.0, num_bath=16, sigma=0.05 ** 2,
                       bath_seed=0, drude_sigma=3.0, bath_gamma=0.03, gamma0=0.03,
                       phase_seed=None, src_z=40, nfreq=8, steps=0)
    p["monitors"][0]["freqs"] = np.linspace(0.5, 1.5, 101)
    return p


def paper_cavity(sigma, gamma=0.004, kind="lorentz"):
    """Sec. IV.B / appendix geometry at resolution 100: mirrors n = 10 (eps 100), 2 cells;
    1-unit gap filled by the slab; CPML 16; 200 vacuum cells on each side."""
    res = 100.0
    pml, vac = 16, 200
    gap, mir = int(round(CAV["gap"] * res)), int(round(CAV["mirror_thickness"] * res))
    eps_m = CAV["mirror_index"] ** 2
    z0 = pml + vac
    mats = [dict(kind="vacuum", z=(z0, z0 + mir), eps_inf=eps_m),
            dict(kind="vacuum", z=(z0 + mir + gap, z0 + 2 * mir + gap), eps_inf=eps_m)]
    if sigma > 0:
        mats.insert(1, dict(kind=kind, z=(z0 + mir, z0 + mir + gap), eps_inf=1.0, frequency=1.0,
                            gamma=gamma, sigma=sigma))
    return dict(n=(1, 1, 2 * pml + 2 * vac + gap + 2 * mir), resolution=res, courant=0.5, pml=pml,
                materials=mats, sources=[], monitors=[])


@pytest.mark.slow
def test_p4_fdtd_transmission_equals_discrete_tmm():
    p = leaky_cavity()
    vac = dict(p, materials=[])
    nu = p["monitors"][0]["freqs"]
    a, b = O.OracleSim(p), O.OracleSim(vac)
    a.step(40000)
    b.step(40000)
    T = O.flux(a.dft()) / O.flux(b.dft())
    Td = cf.transmission_discrete(nu, p)
    assert np.max(np.abs(T - Td)) < 3e-5
    assert T.max() > 0.9 and T.min() < 0.5      # a real spectrum, not a flat line
    # the vacuum flux is positive: the pulse travels towards +z through the monitor
    assert np.all(O.flux(b.dft()) > 0)


def test_p4_discrete_tmm_tends_to_continuum():
    nu = np.linspace(0.8, 1.2, 81)
    errs = []
    for res in (50.0, 100.0, 200.0):
        s = res / 100.0
        p = paper_cavity(0.01, gamma=0.02)
        p = dict(p, resolution=res, n=(1, 1, int(p["n"][2] * s)),
                 materials=[dict(m, z=(int(m["z"][0] * s), int(m["z"][1] * s))) for m in p["materials"]])
        errs.append(np.max(np.abs(cf.transmission_discrete(nu, p) - cf.transmission_continuum(nu, p))))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0   # O(dx^2)
    assert errs[1] < 0.02


@pytest.mark.parametrize("sigma", [2e-3, 2.5e-3, 1e-2, 2e-2])
def test_p4_rabi_splitting_closed_form(sigma):
    nu = np.linspace(0.8, 1.2, 40001)
    T = cf.transmission_discrete(nu, paper_cavity(sigma))
    idx, _ = find_peaks(T)
    pk = [nu[i] for i in idx if T[i] > 0.05]
    assert len(pk) == 2
    split = pk[1] - pk[0]
    assert split == pytest.approx(math.sqrt(sigma), rel=0.03)
    # lower and upper polaritons straddle the bare cavity mode near nu = 1
    empty = cf.transmission_discrete(nu, paper_cavity(0.0))
    nc = nu[np.argmax(empty)]
    assert pk[0] < nc < pk[1] and abs(nc - 1.0) < 0.02


def test_p4_paper_cavity_modes():
    """Sec. IV.B: uncoupled cavity modes near 0.5 and 1.5 and a polariton pair around 1."""
    nu = np.linspace(0.3, 1.7, 14001)
    T = cf.transmission_discrete(nu, paper_cavity(2e-2, gamma=0.04))
    idx, _ = find_peaks(T)
    strong = [nu[i] for i in idx if T[i] > 0.3]
    for mode in CAV["uncoupled_modes"]:
        assert any(abs(x - mode) < 0.06 for x in strong)
    # with the paper's Lorentz damping the polaritons transmit only weakly (Fig. 2b, top)
    pol = [nu[i] for i in idx if 0.85 < nu[i] < 1.15 and T[i] > 0.005]
    assert len(pol) == 2 and pol[1] - pol[0] == pytest.approx(math.sqrt(2e-2), rel=0.05)
