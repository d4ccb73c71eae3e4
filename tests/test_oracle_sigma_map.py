"""Pins of the oracle's per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz and
Eq. EOM_LorentzBath-1 let sigma vary with position; the mass density of Eq. H_full is
rho(r) = 1/(sigma(r) w0^2)) and of its sub-pixel box averaging (CPU only).

* box_fill against midpoint sub-sampling (exact for box bounds on multiples of 1/8).
* The exact discrete energy invariant of a closed, undamped box (P5) with a random sigma(r) map
  in a Drude, a Lorentz-Bath and a Lorentz layer: conserved only if both the drive term and the
  energy weight use the cell's own sigma.
* A 1D layer with a sigma(z) ramp: the FDTD transmission equals the discrete transfer matrix of
  the same planes as a stack of one-plane layers, each with its own sigma (P4 level), and differs
  from the layer without the map.
* A map equal to the material's sigma everywhere reproduces the run without a map bit for bit.
"""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import oracle as O
from paper_2505_23963_gb300 import workloads as wl


def test_box_fill_matches_subsampling():
    shape = (9, 5, 7)   # nz, ny, nx
    lo, hi = (1.375, 0.5, 2.125), (5.25, 4.875, 7.625)
    f = O.box_fill(shape, lo, hi)
    s = 8
    t = (np.arange(s) + 0.5) / s
    ref = np.zeros(shape)
    for k in range(shape[0]):
        for j in range(shape[1]):
            for i in range(shape[2]):
                x, y, z = np.meshgrid(i + t, j + t, k + t, indexing="ij")
                inside = ((x >= lo[0]) & (x < hi[0]) & (y >= lo[1]) & (y < hi[1]) &
                          (z >= lo[2]) & (z < hi[2]))
                ref[k, j, i] = inside.mean()
    assert np.max(np.abs(f - ref)) < 1e-15
    vol = np.prod([b - a for a, b in zip(lo, hi)])
    assert abs(f.sum() - vol) < 1e-12
    assert f.min() == 0.0 and f.max() == 1.0


def closed_box():
    bf = np.array([0.93, 1.02, 1.08])
    return dict(n=(5, 4, 20), resolution=10.0, courant=0.5, pml=0, sources=[], monitors=[],
                materials=[
                    dict(kind="drude", z=(2, 4), eps_inf=1.0, frequency=1.0, gamma=0.0, sigma=3.0),
                    dict(kind="lorentz_bath", z=(5, 12), eps_inf=2.0, frequency=1.0, gamma=0.0,
                         sigma=0.2, bath_frequencies=bf, bath_gammas=np.zeros(3),
                         bath_couplings=np.array([0.05, 0.08, 0.03])),
                    dict(kind="lorentz", z=(13, 16), eps_inf=1.0, frequency=0.8, gamma=0.0,
                         sigma=0.5),
                ], energy_box=(0, 20))


def seeded_run(prob, nsteps, smap=None):
    sim = O.OracleSim(prob, trace_cap=nsteps, record_invariant=True)
    if smap is not None:
        sim.set("S", smap)
    st = wl.random_state(prob, seed=11, scale=1.0)
    for key, arr in st.items():
        if key[0] == "Y":
            sim.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
        else:
            sim.set(key[0], arr, comp=key[1])
    eps = np.ones(prob["n"][::-1])
    eps[5:12] = 2.0
    for c in range(3):   # D = eps E + P^{n-1/2}
        sim.set("D", eps * st[("E", c)] + st[("Pm", c)], comp=c)
    sim.step(nsteps)
    return sim


def random_map(prob, seed):
    rng = np.random.default_rng(seed)
    smap = np.zeros(prob["n"][::-1])
    for m in prob["materials"]:
        lo, hi = m["z"]
        smap[lo:hi] = m["sigma"] * rng.uniform(0.25, 1.75, smap[lo:hi].shape)
    return smap


def test_sigma_map_read_back():
    prob = closed_box()
    sim = O.OracleSim(prob)
    s0 = sim.get("S")
    for m in prob["materials"]:   # the material's sigma before any map is written
        assert np.all(s0[m["z"][0]:m["z"][1]] == m["sigma"])
    assert not np.any(s0[:2]) and not np.any(s0[16:])
    smap = random_map(prob, 3)
    smap[0] = 7.0   # outside every layer: ignored
    sim.set("S", smap)
    got = sim.get("S")
    smap[0] = 0.0
    assert np.array_equal(got, smap)


def test_sigma_map_energy_invariant():
    prob = closed_box()
    nsteps = 6000
    smap = random_map(prob, 5)
    sim = seeded_run(prob, nsteps, smap)
    I = sim.trace()[:, 3]
    rel = np.abs(I - I[0]) / abs(I[0])
    assert rel.max() < 1e-11, rel.max()
    # the parts exchange energy: the invariant is not trivially constant
    for col in (0, 1):
        U = sim.trace()[:, col]
        assert (U.max() - U.min()) / U.max() > 0.1, col
    # the map changes the dynamics
    ref = seeded_run(prob, nsteps)
    assert np.max(np.abs(sim.get("E", comp=0) - ref.get("E", comp=0))) > 1e-3


def test_uniform_map_equals_scalar_sigma():
    prob = closed_box()
    smap = np.zeros(prob["n"][::-1])
    for m in prob["materials"]:
        smap[m["z"][0]:m["z"][1]] = m["sigma"]
    a, b = seeded_run(prob, 200, smap), seeded_run(prob, 200)
    for c in range(3):
        assert np.array_equal(a.get("E", comp=c), b.get("E", comp=c))
        assert np.array_equal(a.get("P", comp=c), b.get("P", comp=c))
    ta, tb = a.trace(), b.trace()
    assert np.array_equal(ta[:, :3], tb[:, :3])
    # the invariant's H.H term is an OpenMP reduction: its summation order may differ per run
    assert np.max(np.abs(ta[:, 3] - tb[:, 3]) / np.abs(tb[:, 3])) < 1e-14


def ramp_layer(res=20.0, lay=24):
    pml, vac = 16, 60
    z0 = pml + vac
    nz = 2 * pml + 2 * vac + lay
    layer = dict(kind="lorentz", z=(z0, z0 + lay), eps_inf=1.0, frequency=1.0, gamma=0.1,
                 sigma=0.05)
    src = dict(component=0, z=pml + 10, center=1.0, fwidth=0.5, amplitude=1.0,
               t0=wl.pulse_t0(0.5), phase=None)
    mon = dict(z=nz - pml - 10, freqs=np.linspace(0.6, 1.4, 41))
    prob = dict(n=(1, 1, nz), resolution=res, courant=0.5, pml=pml, materials=[layer],
                sources=[src], monitors=[mon])
    sig = np.linspace(0.02, 0.2, lay)
    return prob, sig


@pytest.mark.parametrize("res", [20.0])
def test_sigma_ramp_transmission_equals_stack_tmm(res):
    prob, sig = ramp_layer(res)
    lo, hi = prob["materials"][0]["z"]
    nu = prob["monitors"][0]["freqs"]
    a = O.OracleSim(prob)
    smap = np.zeros(prob["n"][::-1])
    smap[lo:hi, 0, 0] = sig
    a.set("S", smap)
    b = O.OracleSim(dict(prob, materials=[]))
    nsteps = 12000
    a.step(nsteps)
    b.step(nsteps)
    T = O.flux(a.dft()) / O.flux(b.dft())
    stack = dict(prob, materials=[dict(prob["materials"][0], z=(k, k + 1), sigma=float(s))
                                  for k, s in zip(range(lo, hi), sig)])
    Td = cf.transmission_discrete(nu, stack)
    err = np.max(np.abs(T - Td))
    assert err < 2e-5, err
    # the map is what the FDTD run saw: the unmapped layer's spectrum is far off
    Tu = cf.transmission_discrete(nu, prob)
    assert np.max(np.abs(Tu - Td)) > 20 * err
    assert T.min() < 0.8
