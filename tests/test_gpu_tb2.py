"""GPU parity of the two-steps-per-pass kernel (temporal blocking, tb2.cuh) on grids without
polarizable material: the flux normalization run that every transmission spectrum needs (a slab
cavity with its layers removed: CPML at both ends, vacuum, a phased soft plane source, a flux
monitor, an energy box).

The kernel runs when FDTDBATH_TB=1 is set at creation.  Against two single steps of the other
step kernels (same chunk plan): FP64 bit for
bit over the snapshot's state -- E, H, both CPML memories -- and the running spectra and energy
trace to the rounding of their partial sums (the plain-plane kernel sums a tile's cells in another
order than the general kernel, whose order this kernel keeps), on several chunk plans (chunk starts whose ghost planes lie in the absorber, one-plane chunks),
with odd step counts and a read between calls (single steps mixed with pairs), and past the
partial-sum ring's capacity; FP32 to 1e-6.  Against the FP64 CPU oracle from rest: FP64 1e-12,
FP32 1e-5 for E, H, the spectra and the energy trace.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import TOL, rel, stack

pytestmark = pytest.mark.gpu


def vacuum_run(nx=64, ny=16, steps=60, seed=3):
    """CPML 8 | 56 vacuum planes | CPML 8 (the slab cavity's flux normalization run)."""
    p = wl.slab_cavity(nx, ny, (8, 14, 3, 10, 3, 12), 20.0, num_bath=4, sigma=0.01, bath_seed=seed,
                       phase_seed=seed, src_z=12, nfreq=16, steps=steps, name="tb_cavity")
    return wl.vacuum_of(p)


class env:
    """Environment variables for the simulations created inside (read at creation)."""
    def __init__(self, **kv):
        self.kv = {k: v for k, v in kv.items()}
    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        for k, v in self.kv.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def pair(prob, precision, zchunk=None, cap=200):
    """The same problem with and without the two-step kernel, on the same chunk plan (the energy
    partial sums are per chunk; by default the two-step kernel's grids take 32-plane chunks)."""
    chunk = dict(FDTDBATH_ZCHUNK=zchunk, FDTDBATH_PLAIN_ZCHUNK=zchunk or "32")
    with env(FDTDBATH_TB="1", **chunk):
        a = fb.Simulation(prob, precision=precision, energy_capacity=cap)
    with env(FDTDBATH_TB="0", **chunk):
        b = fb.Simulation(prob, precision=precision, energy_capacity=cap)
    assert a.tb2_kernel() and not b.tb2_kernel()
    return a, b


def load_random(sims, prob, precision, seed=11):
    st = wl.random_state(prob, seed=seed, with_bath=False)
    rnd = (lambda v: v.astype(np.float32).astype(np.float64)) if precision == 32 else (lambda v: v)
    for s in sims:
        for c in range(3):
            s.set("E", rnd(st[("E", c)]), comp=c)
            s.set("H", rnd(st[("H", c)]), comp=c)


def assert_same_state(a, b, prob):
    """E, H and the E- and H-side CPML memories (the snapshot's device-state pieces, each padded
    to 256 bytes behind a 256-byte header; no material arrays) bit for bit; the spectra and the
    energy trace to 1e-14."""
    nx, ny, nz = prob["n"]
    npml, plane = prob["pml"], nx * ny
    words = {"E": 3 * nx * ny * nz, "H": 3 * nx * ny * nz, "psiE": 2 * 2 * npml * plane,
             "psiH": 2 * (2 * npml + 1) * plane}
    assert a.steps_done == b.steps_done
    sa, sb = a.snapshot(), b.snapshot()
    assert sa.size == sb.size
    off = 256
    for name, w in words.items():
        x = sa[off:off + 8 * w].view(np.float64)
        y = sb[off:off + 8 * w].view(np.float64)
        assert np.array_equal(x, y), (name, float(np.max(np.abs(x - y))), float(np.max(np.abs(y))))
        off += (8 * w + 255) // 256 * 256
    da, db = a.dft(0), b.dft(0)
    assert np.all(np.isfinite(da)) and rel(da, db) < 1e-14, rel(da, db)
    ta, tb = a.trace(), b.trace()
    assert np.all(np.isfinite(ta)) and rel(ta, tb) < 1e-14, rel(ta, tb)


def run_calls(sim, calls):
    for n in calls:
        sim.step(n)
        sim.get("E", comp=0)   # a read flushes the pending H half-step: the next call starts single


@pytest.mark.parametrize("zchunk", [None, "3", "1"])
def test_tb2_fp64_bitwise_against_single_steps(zchunk):
    prob = vacuum_run(steps=0)
    a, b = pair(prob, 64, zchunk)
    load_random((a, b), prob, 64)
    calls = (1, 6, 3, 8)
    run_calls(a, calls)
    run_calls(b, calls)
    assert a.launches() < b.launches()
    assert_same_state(a, b, prob)


def test_tb2_fp64_bitwise_on_plain_kernel_grid_past_ring_capacity():
    """nx = 128: the single steps (the first of each call) run the plain-plane kernel; 300 steps
    wrap the 256-step partial-sum ring in pairs."""
    prob = vacuum_run(nx=128, ny=8, steps=0)
    a, b = pair(prob, 64, cap=400)
    assert a.plain_kernel()
    for s in (a, b):
        s.step(300)
        s.step(5)
    assert_same_state(a, b, prob)
    t = a.trace()
    assert t.shape[0] >= 305 and np.all(np.isfinite(t))


def test_tb2_fp32_against_single_steps():
    prob = vacuum_run(nx=128, ny=16, steps=0)
    a, b = pair(prob, 32)
    load_random((a, b), prob, 32)
    for s in (a, b):
        s.step(21)
    for name in ("E", "H"):
        assert rel(stack(a, name), stack(b, name)) < 1e-6, name
    assert rel(a.dft(0), b.dft(0)) < 1e-6
    assert rel(a.trace(), b.trace()) < 1e-6


@pytest.mark.parametrize("precision", [64, 32])
def test_tb2_from_rest_matches_oracle(precision):
    prob = vacuum_run(steps=120)
    with env(FDTDBATH_TB="1"):
        g = fb.Simulation(prob, precision=precision, energy_capacity=200)
    assert g.tb2_kernel()
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    for name in ("E", "H"):
        assert rel(stack(g, name), stack(o, name)) < TOL[precision], name
    assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    assert rel(tg[:, 0], to[:, 0]) < TOL[precision]
    assert np.max(np.abs(o.get("E", comp=0))) > 1e-8
