"""fdtdbath_box_energy_noalloc: the box energy of the current state, computed by the library
without allocating device memory (its scratch is a static device array), for callers that may
not allocate when they need the result -- a latency-bound loop (an allocation can synchronize
the device), a framework that owns the whole device memory pool, a fixed memory budget.  It
must agree with the energy trace that fdtdbath_energy records for the same box and state (the
last trace entry describes the state after the last step), call after call, and it must
allocate nothing: neither through the simulation's allocator (torch's caching allocator here)
nor on the library's side (the bytes the simulation holds stay the same).

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def allocations():
    """Allocation counters of torch's caching allocator (the simulations' device allocator)."""
    import torch
    st = torch.cuda.memory_stats()
    return st.get("allocation.all.allocated", 0), st.get("segment.all.allocated", 0)


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
@pytest.mark.parametrize("case", ["3d", "1d"])
def test_box_energy_noalloc_matches_energy_trace(precision, tol, case):
    """3D: the general step kernel; 1D (nx = ny = 1): the persistent cavity kernel, whose P level
    and pending H half-step bookkeeping differ -- after an odd and an even number of steps."""
    if case == "3d":
        prob = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=120, seed=1)
        chunks = (70, 35)
    else:
        prob = wl.slab_cavity(1, 1, (8, 60, 10, 120, 10, 60), 100.0, num_bath=6, sigma=0.01,
                              bath_seed=3, phase_seed=None, src_z=30, nfreq=8, steps=640)
        chunks = (401, 239)   # the pulse (peak at t0 = 318 steps) inside the layer
    lo, hi = prob["energy_box"]
    sim = fb.Simulation(prob, precision=precision, energy_capacity=700)
    for nsteps in chunks:
        sim.step(nsteps)
        want = sim.trace()[-1, :3]
        assert np.all(want > 0)
        held, allocs = fb.query(sim.h, 2), allocations()
        first = fb.box_energy_noalloc(sim.h, lo, hi)
        second = fb.box_energy_noalloc(sim.h, lo, hi)       # two calls in a row
        assert fb.query(sim.h, 2) == held and allocations() == allocs
        for got in (first, second):
            np.testing.assert_allclose(got, want, rtol=tol, atol=0)
        assert np.array_equal(first, second)


def test_box_energy_noalloc_device_output_and_limits():
    import torch
    prob = wl.small_3d(nx=33, ny=9, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=40, seed=2)
    lo, hi = prob["energy_box"]
    sim = fb.Simulation(prob, precision=64, energy_capacity=64)
    sim.step(40)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    fb.box_energy_noalloc(sim.h, lo, hi, out_ptr=out.data_ptr())
    np.testing.assert_allclose(out.cpu().numpy(), sim.trace()[-1, :3], rtol=1e-12, atol=0)
    for bad in ((hi, lo), (-1, hi), (lo, prob["n"][2] + 1)):
        with pytest.raises(fb.FdtdBathError) as e:
            fb.box_energy_noalloc(sim.h, *bad)
        assert e.value.code == fb.ERR_ARG
    # the static scratch holds one partial per plane: deeper boxes are refused
    deep = wl.slab_cavity(1, 1, (16, 2000, 0, 2100, 0, 2000), 100.0, num_bath=2, sigma=1e-3,
                          phase_seed=None, nfreq=4, steps=4)
    d = fb.Simulation(deep, precision=32, energy=False)
    d.step(2)
    with pytest.raises(fb.FdtdBathError) as e:
        fb.box_energy_noalloc(d.h, 0, 4097)
    assert e.value.code == fb.ERR_ARG and "4096" in str(e.value)
    assert fb.box_energy_noalloc(d.h, 0, 4096).shape == (3,)
