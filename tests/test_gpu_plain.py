"""GPU parity of the plain-plane kernel (the z-chunks without bath modes on grids tiled by its
128 x 8 FP32 / 64 x 8 FP64 tiles) against the FP64 CPU oracle and against the general step kernel.

The cavity puts every plane kind of that kernel on the grid: CPML at both ends, vacuum with a
phased soft source and a flux monitor, a dielectric (eps_inf = 2.25) spacer, Drude mirrors with
eps_inf = 1.5, and a Lorentz-Bath layer with eps_inf = 2 (run by the bath kernel); the energy box
spans the spacer, the mirrors and the layer, so the plain kernel's energy partials are exercised.
Tolerances as in test_gpu_parity.py: FP64 1e-12, FP32 1e-5 for E, H, spectra and energy traces,
1e-4 for the polarizations (the Drude polarization with the oracle's own one-ulp sensitivity).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import TOL, assert_errs, compare, load_state, oracle_sensitivity, rel, stack

pytestmark = pytest.mark.gpu


def plain_cavity(nx=256, ny=16, steps=120, seed=3):
    """CPML 8 | vacuum 10 | spacer 4 | Drude 3 | Lorentz-Bath 10 | Drude 3 | vacuum 12 | CPML 8."""
    p = wl.slab_cavity(nx, ny, (8, 14, 3, 10, 3, 12), 20.0, num_bath=4, sigma=0.01, bath_seed=seed,
                       phase_seed=seed, src_z=12, nfreq=16, steps=steps, name="plain_cavity")
    mats = []
    for m in p["materials"]:
        m = dict(m)
        m["eps_inf"] = 2.0 if m["kind"] == "lorentz_bath" else 1.5
        mats.append(m)
    z0 = mats[0]["z"][0]
    mats = [dict(kind="vacuum", z=(z0 - 4, z0), eps_inf=2.25)] + mats
    p["materials"] = mats
    p["energy_box"] = (z0 - 4, mats[-1]["z"][1])
    return p


def with_plain(flag):
    """Context: FDTDBATH_PLAIN for the simulations created inside (read at creation)."""
    class _Ctx:
        def __enter__(self):
            self.old = os.environ.get("FDTDBATH_PLAIN")
            os.environ["FDTDBATH_PLAIN"] = flag
        def __exit__(self, *exc):
            if self.old is None:
                os.environ.pop("FDTDBATH_PLAIN", None)
            else:
                os.environ["FDTDBATH_PLAIN"] = self.old
    return _Ctx()


@pytest.mark.parametrize("precision", [64, 32])
def test_plain_kernel_cavity_from_rest_matches_oracle(precision):
    prob = plain_cavity()
    g = fb.Simulation(prob, precision=precision, energy_capacity=200)
    assert g.plain_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    assert_errs(compare(g, o, prob, precision), precision, sens=oracle_sensitivity(prob, 120))
    assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[precision], col
    assert np.max(np.abs(o.get("E", comp=0))) > 1e-8


@pytest.mark.parametrize("precision", [64, 32])
def test_plain_kernel_random_state_matches_oracle(precision):
    """Every field component nonzero (all curl terms, both CPML memories, every P component)."""
    prob = plain_cavity(nx=128, ny=24, steps=7, seed=5)
    st = wl.random_state(prob, seed=11)
    g = fb.Simulation(prob, precision=precision, energy_capacity=16)
    assert g.plain_kernel()
    o = O.OracleSim(prob, trace_cap=16)
    load_state(g, o, prob, st, precision)
    g.step(7)
    o.step(7)
    assert_errs(compare(g, o, prob, precision), precision)
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[precision], col


@pytest.mark.parametrize("precision", [64, 32])
def test_plain_kernel_equals_general_kernel(precision):
    """The same run with the plain-plane kernel and with the general kernel's bath-free form: FP64
    fields bit for bit (same expressions, no contraction), FP32 to rounding; spectra and energy
    traces to rounding of their partial sums."""
    prob = plain_cavity(steps=90)
    sims = []
    for flag in ("1", "0"):
        with with_plain(flag):
            s = fb.Simulation(prob, precision=precision, energy_capacity=128)
        assert s.plain_kernel() == (flag == "1")
        s.step(90)
        sims.append(s)
    a, b = sims
    for name in ("E", "H", "P", "Pm"):
        x, y = stack(a, name), stack(b, name)
        if precision == 64:
            assert np.array_equal(x, y), name
        else:
            assert rel(x, y) < 1e-6, name
    assert rel(a.dft(0), b.dft(0)) < (1e-14 if precision == 64 else 1e-6)
    ta, tb = a.trace(), b.trace()
    for col in range(3):
        assert rel(ta[:, col], tb[:, col]) < (1e-14 if precision == 64 else 1e-6), col


def test_plain_kernel_not_used_on_untiled_grids():
    """Grids the tiles do not cover exactly keep the general kernel (and its ragged tiles)."""
    for n in ((200, 16), (256, 12), (40, 12)):
        prob = plain_cavity(nx=n[0], ny=n[1], steps=1)
        g = fb.Simulation(prob, precision=32)
        assert not g.plain_kernel(), n
        g.close()


def test_plain_kernel_step_calls_compose_bitwise():
    """Reads between step calls (each flushes the pending H half-step through the general
    kernel) leave the plain kernel's results unchanged."""
    prob = plain_cavity(steps=40)
    a = fb.Simulation(prob, precision=64, energy_capacity=64)
    b = fb.Simulation(prob, precision=64, energy_capacity=64)
    a.step(13)
    _ = a.get("H", comp=1)
    a.step(27)
    b.step(40)
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            assert np.array_equal(a.get(name, comp=c), b.get(name, comp=c)), (name, c)


@pytest.mark.parametrize("precision", [64, 32])
def test_eps_layers_on_ragged_tiles_match_oracle(precision):
    """The same cavity (eps_inf = 2.25 spacer, 1.5 Drude mirrors, 2.0 Lorentz-Bath layer) on a
    grid its tiles do not cover: every plane runs the general kernel with ragged x / y tiles."""
    prob = plain_cavity(nx=40, ny=12, steps=120)
    g = fb.Simulation(prob, precision=precision, energy_capacity=200)
    assert not g.plain_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    assert_errs(compare(g, o, prob, precision), precision, sens=oracle_sensitivity(prob, 120))
    assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[precision], col
