"""GPU parity of the per-cell oscillator strength sigma(r) (Eq. EOM_Lorentz and
Eq. EOM_LorentzBath-1 with sigma depending on the cell; rho(r) = 1/(sigma(r) w0^2) in the energy
of Eq. H_full) and of its sub-pixel box painting, through the C ABI, against the FP64 oracle given
the same map.  Tolerances as in test_gpu_parity.py.

* 3D ragged cavity (Drude mirrors and a Lorentz-Bath layer, every cell its own sigma) from rest
  and from a random state; the 1D cavity kernel with a sigma(z) map; a box painted with fractional
  bounds (the map read back against the oracle's box fill, then the run).
* A map equal to every layer's own sigma leaves the fields bit for bit as without a map (FP64,
  the plain-plane kernels reading the map); the plain-plane kernels' forms (bath-free with Drude
  mirrors, one-cell-per-thread, two-threads-per-cell and streamed Lorentz-Bath forms) against the
  general kernel with the same random map (FP32).
* Snapshot / restore carry the map; the refusals (adjoint, the allocation-free energy, negative
  and unstable values).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import TOL, assert_errs, compare, load_state, rel, stack

pytestmark = pytest.mark.gpu


def pair(prob, precision, smap, cap=200):
    g = fb.Simulation(prob, precision=precision, energy_capacity=cap)
    o = O.OracleSim(prob, trace_cap=cap)
    if precision == 32:
        smap = smap.astype(np.float32).astype(np.float64)
    g.set("S", smap)
    o.set("S", smap)
    assert g.sigma_map()
    return g, o


def sensitivity(prob, smap, steps):
    """The oracle against itself, both with the map, the source phase (or, without a phase
    table, the pulse delay t0) moved by one ulp: the bound of the conditioning-limited Drude
    polarization, as in test_gpu_parity.py."""
    p2 = dict(prob)
    p2["sources"] = [dict(s, phase=np.nextafter(s["phase"], 10.0)) if s.get("phase") is not None
                     else dict(s, t0=float(np.nextafter(s["t0"], 1e9))) for s in prob["sources"]]
    a, b = O.OracleSim(prob), O.OracleSim(p2)
    for sim in (a, b):
        sim.set("S", smap)
        sim.step(steps)
    return compare(b, a, prob, 64)


def check_run(g, o, prob, precision, steps, sens=None):
    assert_errs(compare(g, o, prob, precision), precision, sens=sens)
    if prob.get("monitors"):
        assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    assert tg.shape[0] == steps
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < TOL[precision], col


@pytest.mark.parametrize("precision", [64, 32])
def test_sigma_map_from_rest_matches_oracle(precision):
    prob = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=150, seed=1)
    smap = wl.random_sigma_map(prob, 3)
    g, o = pair(prob, precision, smap)
    g.step(150)
    o.step(150)
    check_run(g, o, prob, precision, 150, sens=sensitivity(prob, o.get("S"), 150))
    assert np.max(np.abs(o.get("P", comp=0))) > 0


@pytest.mark.parametrize("precision", [64, 32])
def test_sigma_map_random_state_matches_oracle(precision):
    prob = wl.slab_cavity(37, 11, (6, 6, 2, 12, 2, 6), 20.0, num_bath=5, sigma=0.01, bath_seed=4,
                          phase_seed=7, nfreq=12, steps=9)
    prob["courant"] = 0.5
    g, o = pair(prob, precision, wl.random_sigma_map(prob, 8, 0.2, 1.0), cap=16)
    load_state(g, o, prob, wl.random_state(prob, seed=21), precision)
    g.step(9)
    o.step(9)
    check_run(g, o, prob, precision, 9)


@pytest.mark.parametrize("precision", [64, 32])
def test_sigma_map_1d_kernel_matches_oracle(precision):
    # 260 steps: the pulse reflected by the first mirror is still inside the grid (once only the
    # small field between the mirrors is left, FP32 fields carry the cancellation residue of the
    # Drude metal, the conditioning noted in test_gpu_parity.py)
    prob = wl.slab_cavity(1, 1, (16, 40, 10, 60, 10, 40), 50.0, num_bath=8, sigma=0.02,
                          bath_seed=2, phase_seed=None, nfreq=24, steps=260)
    g, o = pair(prob, precision, wl.random_sigma_map(prob, 5), cap=300)
    assert g.cavity_1d_kernel()
    g.step(260)
    o.step(260)
    check_run(g, o, prob, precision, 260, sens=sensitivity(prob, o.get("S"), 260))


@pytest.mark.parametrize("precision", [64, 32])
def test_sigma_box_subpixel_matches_oracle(precision):
    prob = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=120, seed=2)
    lb = next(m for m in prob["materials"] if m["kind"] == "lorentz_bath")
    z0, z1 = lb["z"]
    lo, hi = (5.25, 2.5, z0 + 1.375), (31.625, 9.75, z1 - 2.5)
    g = fb.Simulation(prob, precision=precision, energy_capacity=200)
    o = O.OracleSim(prob, trace_cap=200)
    g.sigma_box(lo, hi, 4.0 * lb["sigma"])
    O.paint_sigma(o, lo, hi, 4.0 * lb["sigma"])
    sg, so = g.get("S"), o.get("S")
    assert np.max(np.abs(sg - so)) <= (0.0 if precision == 64 else 1e-7 * np.max(so))
    assert np.unique(np.round(so[z0:z1], 12)).size > 4   # fractional cells exist
    g.step(120)
    o.step(120)
    check_run(g, o, prob, precision, 120, sens=sensitivity(prob, so, 120))


def test_uniform_map_equals_no_map_fp64():
    prob = wl.small_3d(nx=128, ny=16, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=60, seed=3)
    a = fb.Simulation(prob, precision=64, energy_capacity=64)
    b = fb.Simulation(prob, precision=64, energy_capacity=64)
    assert a.plain_kernel()
    b.set("S", b.get("S"))   # every layer's own sigma, now as a map
    assert b.sigma_map() and b.plain_kernel()
    a.step(60)
    b.step(60)
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            assert np.array_equal(a.get(name, comp=c), b.get(name, comp=c)), (name, c)
    assert np.array_equal(a.dft(0), b.dft(0))
    # the energy weight rho_s / sigma(r) rounds differently from rho / dt^2
    assert rel(a.trace(), b.trace()) < 1e-14


class env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        import os
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *exc):
        import os
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("nb", [8, 13, 37])
def test_plain_kernel_forms_with_map_equal_general_kernel(nb):
    """FP32 128 x 16 grid: the bath-free form over the CPML, vacuum and Drude chunks, and the
    Lorentz-Bath form of nb modes (8: one cell per thread; 13: two threads per cell; 37:
    streamed), against the general kernel, both with the same random sigma(r) map."""
    prob = wl.slab_cavity(128, 16, (8, 6, 4, 20, 4, 6), 20.0, num_bath=nb, sigma=0.01, bath_seed=3,
                          phase_seed=3, nfreq=12, steps=80)
    prob["courant"] = 0.5
    smap = wl.random_sigma_map(prob, 9)
    sims = []
    for flag in ("1", "0"):
        with env(FDTDBATH_PLAIN=flag, FDTDBATH_BATHPLAIN=flag):
            s = fb.Simulation(prob, precision=32, energy_capacity=128)
        assert s.plain_kernel() == (flag == "1") and s.bath_plain_kernel() == (flag == "1")
        s.set("S", smap)
        s.step(80)
        sims.append(s)
    a, b = sims
    # the two kernels agree to FP32 rounding (normwise over the three components, ~1e-6; the FP32
    # parity bound 1e-5 here, the oracle comparison below being the parity test proper)
    for name in ("E", "H", "P", "Pm"):
        assert rel(stack(a, name), stack(b, name)) < TOL[32], name
    lo, hi = next(m for m in prob["materials"] if m["kind"] == "lorentz_bath")["z"]
    for j in sorted({0, nb // 2, nb - 1}):
        assert rel(stack(a, "Y", mode=j)[:, lo:hi], stack(b, "Y", mode=j)[:, lo:hi]) < TOL[32], j
    assert rel(a.dft(0), b.dft(0)) < TOL[32]
    ta, tb = a.trace(), b.trace()
    for col in range(3):
        assert rel(ta[:, col], tb[:, col]) < TOL[32], col
    # and the plain-plane kernels against the oracle given the same map
    o = O.OracleSim(prob, trace_cap=128)
    o.set("S", smap.astype(np.float32).astype(np.float64))
    o.step(80)
    check_run(a, o, prob, 32, 80, sens=sensitivity(prob, o.get("S"), 80))


@pytest.mark.parametrize("precision", [64, 32])
def test_sigma_map_snapshot_restore(precision):
    prob = wl.small_3d(nx=33, ny=9, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=80, seed=4)
    a = fb.Simulation(prob, precision=precision, energy_capacity=128)
    a.set("S", wl.random_sigma_map(prob, 6))
    a.step(30)
    snap = a.snapshot()
    a.step(25)
    b = fb.Simulation(prob, precision=precision, energy_capacity=128)
    assert not b.sigma_map()
    b.restore(snap)
    assert b.sigma_map()
    assert np.array_equal(a.get("S"), b.get("S"))
    b.step(25)
    for name in ("E", "H", "P"):
        for c in range(3):
            assert np.array_equal(a.get(name, comp=c), b.get(name, comp=c)), (name, c)
    # a snapshot without a map returns a simulation with one to the layers' own sigma
    c = fb.Simulation(prob, precision=precision, energy_capacity=128)
    plain = c.snapshot()
    b.restore(plain)
    assert not b.sigma_map()


def test_sigma_map_refusals():
    prob = wl.small_3d(nx=32, ny=8, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=10, seed=5)
    g = fb.Simulation(prob, precision=64, energy_capacity=16)
    smap = wl.random_sigma_map(prob, 1)
    bad = smap.copy()
    lb = next(m for m in prob["materials"] if m["kind"] == "lorentz_bath")
    bad[lb["z"][0], 0, 0] = -1.0
    with pytest.raises(fb.FdtdBathError) as e:
        g.set("S", bad)
    assert e.value.code == fb.ERR_ARG
    unstable = smap.copy()
    dr = next(m for m in prob["materials"] if m["kind"] == "drude")
    unstable[dr["z"][0], 3, 3] = 10.0 * dr["sigma"]
    with pytest.raises(fb.FdtdBathError) as e:
        g.set("S", unstable)
    assert e.value.code == fb.ERR_CFL
    assert not g.sigma_map()   # nothing changed
    g.set("S", smap)
    with pytest.raises(fb.FdtdBathError) as e:
        g.adjoint_forward(4, 2)
    assert e.value.code == fb.ERR_UNSUPPORTED
    with pytest.raises(fb.FdtdBathError) as e:
        fb.box_energy_noalloc(g.h, lb["z"][0], lb["z"][1])
    assert e.value.code == fb.ERR_UNSUPPORTED
    with pytest.raises(fb.FdtdBathError) as e:
        g.sigma_box((0, 0, 0), (33, 8, 4), 0.1)   # outside the grid in x
    assert e.value.code == fb.ERR_ARG
