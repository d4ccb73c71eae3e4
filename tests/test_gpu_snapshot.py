"""Checkpoint / resume of the whole state (fdtdbath_snapshot / fdtdbath_restore): a run
snapshotted after N steps and resumed -- in the same simulation after it moved on, or in a fresh
simulation of the same problem -- reproduces the uninterrupted run bit for bit: fields, the
polarization and bath modes, the CPML memories (the pulse is inside the absorbers), the running
spectra and the energy trace.  Covers the 3D step kernels (plain-plane and bath), the persistent
1D kernel and bf16 bath storage."""
import numpy as np
import pytest

from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def state(sim, prob):
    out = {}
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            out[(name, c)] = sim.get(name, comp=c)
    for m in prob["materials"]:
        if m["kind"] == "lorentz_bath":
            for j in (0, len(m["bath_frequencies"]) - 1):
                out[("Y", j)] = sim.get("Y", comp=0, mode=j, level=0)
    out["dft"] = sim.dft(0)
    out["trace"] = sim.trace()
    return out


def assert_same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


CASES = {
    "3d": lambda: wl.slab_cavity(128, 16, (8, 14, 3, 10, 3, 12), 20.0, num_bath=4, sigma=0.01,
                                 bath_seed=3, phase_seed=3, src_z=12, nfreq=16, steps=200),
    "3d_ragged": lambda: wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=200, seed=1),
    "1d": lambda: wl.slab_cavity(1, 1, (8, 60, 10, 120, 10, 60), 100.0, num_bath=6, sigma=0.01,
                                 bath_seed=3, phase_seed=None, src_z=30, nfreq=8, steps=700),
}


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_snapshot_resume_is_bitwise(precision, case):
    prob = CASES[case]()
    n1, n2 = (90, 70) if case != "1d" else (355, 301)
    ref = fb.Simulation(prob, precision=precision, energy_capacity=1000)
    ref.step(n1 + n2)
    want = state(ref, prob)

    a = fb.Simulation(prob, precision=precision, energy_capacity=1000)
    a.step(n1)
    snap = a.snapshot()
    a.step(n2 + 17)                      # the original moves on ...
    a.restore(snap)                      # ... and comes back
    assert a.steps_done == n1
    a.step(n2)
    assert_same(state(a, prob), want)

    b = fb.Simulation(prob, precision=precision, energy_capacity=1000)   # a fresh simulation
    b.restore(snap)
    b.step(n2)
    assert_same(state(b, prob), want)


def test_snapshot_resume_bf16_bath_storage():
    prob = CASES["3d_ragged"]()
    ref = fb.Simulation(prob, precision=32, bath_storage=1, energy_capacity=400)
    ref.step(150)
    a = fb.Simulation(prob, precision=32, bath_storage=1, energy_capacity=400)
    a.step(80)
    snap = a.snapshot()
    b = fb.Simulation(prob, precision=32, bath_storage=1, energy_capacity=400)
    b.restore(snap)
    b.step(70)
    assert_same(state(b, prob), state(ref, prob))


def test_restore_refuses_another_layout():
    p = CASES["3d_ragged"]()
    a = fb.Simulation(p, precision=64, energy_capacity=64)
    a.step(5)
    snap = a.snapshot()
    for other, kw in ((dict(p, n=(44, 12, p["n"][2])), {}), (p, {"precision": 32}), (p, {"energy_capacity": 65})):
        b = fb.Simulation(other, **{"precision": 64, "energy_capacity": 64, **kw})
        with pytest.raises(fb.FdtdBathError) as e:
            b.restore(snap)
        assert e.value.code == fb.ERR_ARG
    with pytest.raises(fb.FdtdBathError):
        a.restore(snap[:100])
