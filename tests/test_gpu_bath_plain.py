"""GPU parity of the plain-plane kernel's Lorentz-Bath form (FP32, 32 x 8 tiles; one cell per
thread with at most 8 bath modes per material, two threads per cell with 9 to 16, up to 128
streamed through a shared-memory ring) against the FP64 CPU oracle and against the general step
kernel.

The cavities are those of test_gpu_plain.py (CPML, vacuum with a phased source, an
eps_inf = 2.25 spacer, eps_inf = 1.5 Drude mirrors, an eps_inf = 2 Lorentz-Bath layer, the energy
box over spacer, mirrors and layer) on grids whose x extent is a multiple of 32 and y extent of 8.
Tolerances: FP32 1e-5 for E, H, spectra and energy traces, 1e-4 for polarizations and bath modes
(test_gpu_parity.py).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import TOL, assert_errs, compare, load_state, oracle_sensitivity, rel, stack

pytestmark = pytest.mark.gpu


class env:
    """Context: environment variables for the simulations created inside (read at creation)."""

    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def bath_cavity(nx=64, ny=16, steps=120, seed=3, nb=8, layer=10):
    """CPML 8 | vacuum 10 | spacer 4 | Drude 3 | Lorentz-Bath `layer` (nb modes) | Drude 3 |
    vacuum 12 | CPML 8, eps_inf as in plain_cavity."""
    p = wl.slab_cavity(nx, ny, (8, 14, 3, layer, 3, 12), 20.0, num_bath=nb, sigma=0.01, bath_seed=seed,
                       phase_seed=seed, src_z=12, nfreq=16, steps=steps, name="bath_cavity")
    mats = [dict(m, eps_inf=2.0 if m["kind"] == "lorentz_bath" else 1.5) for m in p["materials"]]
    z0 = mats[0]["z"][0]
    mats = [dict(kind="vacuum", z=(z0 - 4, z0), eps_inf=2.25)] + mats
    p["materials"] = mats
    p["energy_box"] = (z0 - 4, mats[-1]["z"][1])
    return p


@pytest.mark.parametrize("nb", [8, 4, 3, 16, 11, 100, 20])
def test_bath_form_from_rest_matches_oracle(nb):
    prob = bath_cavity(nb=nb)
    g = fb.Simulation(prob, precision=32, energy_capacity=200)
    assert g.bath_plain_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    assert_errs(compare(g, o, prob, 32), 32, sens=oracle_sensitivity(prob, 120))
    assert rel(g.dft(0), o.dft(0)) < TOL[32]
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[32], col
    # the bath energy column is nonzero: the modes moved
    assert np.max(np.abs(to[:, 2])) > 0


@pytest.mark.parametrize("shape,nb", [((64, 16), 8), ((32, 8), 8), ((96, 24), 8), ((64, 16), 16), ((32, 8), 13),
                                      ((64, 16), 100), ((32, 8), 33)])
def test_bath_form_random_state_matches_oracle(shape, nb):
    """Every field, polarization and bath-mode component nonzero; one tile per plane (32 x 8:
    every halo is the tile's own wrapped column / row) and several; one and two threads per cell."""
    prob = bath_cavity(nx=shape[0], ny=shape[1], steps=7, seed=5, nb=nb)
    st = wl.random_state(prob, seed=11)
    g = fb.Simulation(prob, precision=32, energy_capacity=16)
    assert g.bath_plain_kernel()
    o = O.OracleSim(prob, trace_cap=16)
    load_state(g, o, prob, st, 32)
    g.step(7)
    o.step(7)
    assert_errs(compare(g, o, prob, 32), 32)
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[32], col


@pytest.mark.parametrize("zchunk,nb", [("16", 8), ("5", 8), ("64", 8), ("16", 16), ("64", 16), ("16", 100),
                                       ("5", 37)])
def test_bath_form_equals_general_kernel(zchunk, nb):
    """The same run with the bath form and with the general kernel's bath instantiation: fields,
    polarizations and every bath mode to FP32 rounding; the layer cut into chunks of about 5, 16
    and 64 (one chunk) planes."""
    prob = bath_cavity(nx=64, ny=16, steps=60, layer=40, nb=nb)
    sims = []
    for flag in ("1", "0"):
        with env(FDTDBATH_BATHPLAIN=flag, FDTDBATH_BATH_ZCHUNK=zchunk):
            s = fb.Simulation(prob, precision=32, energy_capacity=64)
        assert s.bath_plain_kernel() == (flag == "1")
        s.step(60)
        sims.append(s)
    a, b = sims
    for name in ("E", "H", "P", "Pm"):
        assert rel(stack(a, name), stack(b, name)) < 1e-6, name
    lo, hi = prob["materials"][2]["z"]
    for j in range(nb):
        for lvl in (0, 1):
            assert rel(stack(a, "Y", mode=j, level=lvl)[:, lo:hi],
                       stack(b, "Y", mode=j, level=lvl)[:, lo:hi]) < 1e-6, (j, lvl)
    assert rel(a.dft(0), b.dft(0)) < 1e-6
    ta, tb = a.trace(), b.trace()
    for col in range(3):
        assert rel(ta[:, col], tb[:, col]) < 1e-6, col


def test_bath_form_zero_coupling_is_lorentz():
    """Bath couplings zero: the bath form's P equals the Lorentz update of the plain-plane kernel
    (the bath sum is an exact zero)."""
    base = bath_cavity(nx=128, ny=8, steps=50)
    mats = base["materials"]
    lb = mats[2]
    lb0 = dict(lb, bath_couplings=np.zeros_like(lb["bath_couplings"]))
    lor = dict(kind="lorentz", z=lb["z"], eps_inf=lb["eps_inf"], frequency=lb["frequency"],
               gamma=lb["gamma"], sigma=lb["sigma"])
    sa = fb.Simulation(dict(base, materials=[mats[0], mats[1], lb0, mats[3]]), precision=32)
    sb = fb.Simulation(dict(base, materials=[mats[0], mats[1], lor, mats[3]]), precision=32)
    assert sa.bath_plain_kernel() and sb.plain_kernel()
    sa.step(50)
    sb.step(50)
    for name in ("E", "H", "P", "Pm"):
        x, y = stack(sa, name), stack(sb, name)
        assert rel(x, y) < 1e-6, name
        assert np.max(np.abs(y)) > 0, name


def test_bath_form_not_used_outside_its_range():
    """FP64, bf16 bath storage with more than 16 modes, x not a multiple of 32, y not of 8, a
    source plane inside the layer: the general kernel."""
    cases = [(bath_cavity(steps=1), dict(precision=64)),
             (bath_cavity(steps=1, nb=17), dict(precision=32, bath_storage=1)),
             (bath_cavity(nx=48, steps=1), dict(precision=32)),
             (bath_cavity(ny=12, steps=1), dict(precision=32))]
    src_in = bath_cavity(steps=1)
    lo = src_in["materials"][2]["z"][0]
    src_in["sources"] = [dict(s, z=lo + 2) for s in src_in["sources"]]
    cases.append((src_in, dict(precision=32)))
    for prob, kw in cases:
        g = fb.Simulation(prob, **kw)
        assert not g.bath_plain_kernel(), kw
        g.close()
    for nb, kw in ((8, dict(precision=32)), (8, dict(precision=32, bath_storage=1)),
                   (17, dict(precision=32)), (100, dict(precision=32))):
        g = fb.Simulation(bath_cavity(steps=1, nb=nb), **kw)
        assert g.bath_plain_kernel(), (nb, kw)
        g.close()


@pytest.mark.parametrize("nb", [8, 16, 100])
def test_bath_form_snapshot_resume_bitwise(nb):
    """A snapshot taken between steps and restored into a fresh simulation continues bit for bit
    with the bath form (its pending H half-step stays pending across the snapshot)."""
    prob = bath_cavity(steps=40, nb=nb)
    a = fb.Simulation(prob, precision=32, energy_capacity=64)
    a.step(17)
    buf = a.snapshot()
    a.step(23)
    b = fb.Simulation(prob, precision=32, energy_capacity=64)
    b.restore(buf)
    b.step(23)
    for name in ("E", "H", "P", "Pm"):
        assert np.array_equal(stack(a, name), stack(b, name)), name
    assert np.array_equal(a.dft(0), b.dft(0))


@pytest.mark.parametrize("nb", [8, 16, 6])
def test_bath_form_bf16_storage_equals_general_kernel(nb):
    """bf16 bath storage (in-place (value, increment) pairs): the bath form against the general
    kernel's bf16 instantiation on the same run.  Both do the same FP32 arithmetic and round the
    same pairs, so the fields agree to FP32 rounding; a pair rounded to the other side of a bf16
    step by a last-bit difference moves a mode by 2^-8 relative, so the modes get 1e-3."""
    prob = bath_cavity(nx=64, ny=16, steps=60, layer=24, nb=nb)
    sims = []
    for flag in ("1", "0"):
        with env(FDTDBATH_BATHPLAIN=flag):
            s = fb.Simulation(prob, precision=32, bath_storage=1, energy_capacity=64)
        assert s.bath_plain_kernel() == (flag == "1")
        s.step(60)
        sims.append(s)
    a, b = sims
    for name in ("E", "H", "P", "Pm"):
        assert rel(stack(a, name), stack(b, name)) < 1e-5, name
    lo, hi = prob["materials"][2]["z"]
    for j in sorted({0, nb // 2, nb - 1}):
        for lvl in (0, 1):
            assert rel(stack(a, "Y", mode=j, level=lvl)[:, lo:hi],
                       stack(b, "Y", mode=j, level=lvl)[:, lo:hi]) < 1e-3, (j, lvl)
    ta, tb = a.trace(), b.trace()
    for col in range(3):
        assert rel(ta[:, col], tb[:, col]) < 1e-4, col


def two_layer_cavity(nx=64, ny=16, nbA=8, nbB=5, steps=120):
    """Two adjacent Lorentz-Bath layers with different baths (A: nbA modes, eps_inf 2; B: nbB
    modes, sigma 0.02, eps_inf 1.5), a second monitor inside layer A and an energy box that cuts
    through layer A: bath planes carrying monitor partials, box edges inside a chunk, and both
    materials' tensor maps."""
    p = bath_cavity(nx=nx, ny=ny, steps=steps, nb=nbA, layer=20)
    q = wl.slab_cavity(nx, ny, (8, 14, 3, 20, 3, 12), 20.0, num_bath=nbB, sigma=0.02, bath_seed=9,
                       phase_seed=3, src_z=12, nfreq=16, steps=steps, name="layer_b")
    mats = p["materials"]
    lo, hi = mats[2]["z"]
    mid = lo + 9
    lbB = [m for m in q["materials"] if m["kind"] == "lorentz_bath"][0]
    p["materials"] = [mats[0], mats[1], dict(mats[2], z=(lo, mid)), dict(lbB, z=(mid, hi), eps_inf=1.5),
                      mats[3]]
    p["monitors"] = p["monitors"] + [dict(z=lo + 4, freqs=np.linspace(0.5, 1.5, 16))]
    p["energy_box"] = (lo + 5, hi + 2)
    return p


@pytest.mark.parametrize("nbA,nbB", [(8, 5), (16, 12), (100, 20), (8, 16)])
def test_bath_form_two_layers_monitor_in_layer_matches_oracle(nbA, nbB):
    """Both Lorentz-Bath materials through the bath form (per-material maps and coefficient rows;
    the form set by the larger bath: registers, two threads per cell, or streamed), a monitor
    inside a layer, an energy box edge inside a layer."""
    prob = two_layer_cavity(nbA=nbA, nbB=nbB)
    g = fb.Simulation(prob, precision=32, energy_capacity=200)
    assert g.bath_plain_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    assert_errs(compare(g, o, prob, 32), 32, sens=oracle_sensitivity(prob, 120))
    for m in range(2):
        assert rel(g.dft(m), o.dft(m)) < TOL[32], m
        assert np.max(np.abs(o.dft(m))) > 0, m
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[32], col
