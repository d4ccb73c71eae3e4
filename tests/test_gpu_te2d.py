"""GPU parity of the TE form's register-streaming kernel (te2d.cuh: FP32, the z-chunks of
y-invariant grids driven through E_y, nx a multiple of 256; the Lorentz-Bath chunks with at most 8
modes) against the FP64 CPU oracle and against the general kernel's TE form.

The cavity: CPML | vacuum with a phased E_y source and a flux monitor | an eps_inf = 2.25 spacer |
eps_inf = 1.5 Drude mirrors | an eps_inf = 2 Lorentz-Bath layer | vacuum | CPML, the energy box
over spacer, mirrors and layer.  Tolerances as in test_gpu_parity.py (FP32 1e-5 for E, H, spectra
and energy traces, 1e-4 for polarizations and bath modes).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import TOL, TOL_Y, rel

pytestmark = pytest.mark.gpu

TE_KEYS = [("E", 1), ("H", 0), ("H", 2)]


def te_cavity(nx=512, steps=150, seed=3, nb=4):
    p = wl.slab_cavity(nx, 1, (8, 14, 3, 10, 3, 12), 20.0, num_bath=nb, sigma=0.01, bath_seed=seed,
                       phase_seed=seed, src_z=12, nfreq=16, steps=steps, name="te2d_cavity",
                       source_component=1)
    mats = [dict(m, eps_inf=2.0 if m["kind"] == "lorentz_bath" else 1.5) for m in p["materials"]]
    z0 = mats[0]["z"][0]
    p["materials"] = [dict(kind="vacuum", z=(z0 - 4, z0), eps_inf=2.25)] + mats
    p["energy_box"] = (z0 - 4, mats[-1]["z"][1])
    return p


class env:
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


def te_state(g, o, prob, seed):
    """Seeded random E_y, H_x, H_z, P_y (both levels) and y bath modes, float-rounded, into both
    (other components stay zero: the TE form is kept)."""
    rng = np.random.default_rng(seed)
    shp = prob["n"][::-1]
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    eps = np.ones(shp)
    for m in prob["materials"]:
        eps[m["z"][0]:m["z"][1]] = m.get("eps_inf", 1.0)
    vals = {}
    for name, c in TE_KEYS:
        vals[(name, c)] = f32(1e-2 * rng.standard_normal(shp))
    mask = np.zeros(shp, dtype=bool)
    for m in prob["materials"]:
        if m["kind"] != "vacuum":
            mask[m["z"][0]:m["z"][1]] = True
    for name in ("P", "Pm"):
        vals[(name, 1)] = f32(np.where(mask, 1e-3 * rng.standard_normal(shp), 0.0))
    for key, a in vals.items():
        g.set(key[0], a, comp=key[1])
        o.set(key[0], a, comp=key[1])
    for m in prob["materials"]:
        if m["kind"] != "lorentz_bath":
            continue
        lo, hi = m["z"]
        for j in range(len(m["bath_frequencies"])):
            for lvl in (0, 1):
                a = np.zeros(shp)
                a[lo:hi] = f32(1e-3 * rng.standard_normal((hi - lo,) + shp[1:]))
                g.set("Y", a, comp=1, mode=j, level=lvl)
                o.set("Y", a, comp=1, mode=j, level=lvl)
    o.set("D", eps * vals[("E", 1)] + vals[("Pm", 1)], comp=1)


def compare_te(g, o, prob):
    for name, c in TE_KEYS:
        assert rel(g.get(name, comp=c), o.get(name, comp=c)) < TOL[32], (name, c)
    for m in prob["materials"]:
        if m["kind"] == "vacuum":
            continue
        lo, hi = m["z"]
        for name in ("P", "Pm"):
            a, b = g.get(name, comp=1)[lo:hi], o.get(name, comp=1)[lo:hi]
            # the Drude mirrors' polarization is conditioning-limited (test_gpu_parity)
            tol = TOL_Y[32] if m["kind"] != "drude" else 1e-3
            assert rel(a, b) < tol, (name, m["kind"])


@pytest.mark.parametrize("nb", [4, 8, 16])
def test_te2d_from_rest_matches_oracle(nb):
    """N_b 4 and 8: the layer by the TE kernel too; 16: by the general kernel."""
    prob = te_cavity(nb=nb)
    g = fb.Simulation(prob, precision=32, energy_capacity=200)
    assert g.te_form() and g.te2d_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(150)
    o.step(150)
    compare_te(g, o, prob)
    lo, hi = prob["materials"][2]["z"]
    for j in sorted({0, nb - 1}):
        for lvl in (0, 1):
            assert rel(g.get("Y", comp=1, mode=j, level=lvl)[lo:hi],
                       o.get("Y", comp=1, mode=j, level=lvl)[lo:hi]) < TOL_Y[32], (j, lvl)
    assert rel(g.dft(0), o.dft(0)) < TOL[32]
    assert np.max(np.abs(o.dft(0))) > 0
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[32], col
    for c in (0, 2):   # the skipped components stay exactly zero
        assert not np.any(g.get("E", comp=c))


@pytest.mark.parametrize("nx", [256, 768])
def test_te2d_random_state_matches_oracle(nx):
    """Every TE component nonzero everywhere: both CPML memories, P_y in every layer, the periodic
    x wrap at the segments' ends (one and three CTAs per plane)."""
    prob = te_cavity(nx=nx, steps=7, seed=5)
    g = fb.Simulation(prob, precision=32, energy_capacity=16)
    o = O.OracleSim(prob, trace_cap=16)
    te_state(g, o, prob, 11)
    assert g.te_form() and g.te2d_kernel()
    g.step(7)
    o.step(7)
    compare_te(g, o, prob)
    tg, to = g.trace(), o.trace()
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[32], col


@pytest.mark.parametrize("nb", [4, 8])
def test_te2d_equals_general_te_form(nb):
    """The same run with the TE kernel and with the general kernel's TE form: every component,
    the layer's bath modes, the spectrum and the energy trace to FP32 rounding."""
    prob = te_cavity(steps=120, nb=nb)
    sims = []
    for flag in ("1", "0"):
        with env(FDTDBATH_TE2D=flag):
            s = fb.Simulation(prob, precision=32, energy_capacity=128)
        assert s.te_form() and s.te2d_kernel() == (flag == "1")
        s.step(120)
        sims.append(s)
    a, b = sims
    for name, c in TE_KEYS + [("P", 1), ("Pm", 1)]:
        assert rel(a.get(name, comp=c), b.get(name, comp=c)) < 1e-6, (name, c)
    lo, hi = prob["materials"][2]["z"]
    for j in range(nb):
        for lvl in (0, 1):
            assert rel(a.get("Y", comp=1, mode=j, level=lvl)[lo:hi],
                       b.get("Y", comp=1, mode=j, level=lvl)[lo:hi]) < 1e-6, (j, lvl)
    assert rel(a.dft(0), b.dft(0)) < 1e-6
    ta, tb = a.trace(), b.trace()
    for col in range(3):
        assert rel(ta[:, col], tb[:, col]) < 1e-6, col


def test_te2d_not_used_outside_its_range():
    """FP64, nx not a multiple of 256, an E_x write (the general form from then on)."""
    g = fb.Simulation(te_cavity(steps=1), precision=64)
    assert not g.te2d_kernel()
    g.close()
    g = fb.Simulation(te_cavity(nx=384, steps=1), precision=32)
    assert g.te_form() and not g.te2d_kernel()
    g.close()
    prob = te_cavity(steps=1)
    g = fb.Simulation(prob, precision=32)
    assert g.te2d_kernel()
    g.set("E", np.zeros(prob["n"][::-1]), comp=0)
    assert not g.te_form() and not g.te2d_kernel()
    g.close()
