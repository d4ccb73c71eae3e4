"""P10: the oracle's absorber.  The paper runs MEEP's PML without specifying it; the oracle (and
the CUDA path) read it as a convolutional PML (Roden-Gedney, kappa = 1, cubic grading) on both z
ends.  What any absorbing layer must do, checked here on a vacuum pulse at normal incidence: the
reflection, read from the box energy while only the reflected pulses are inside the box (after
the direct pulses have entered the absorbers, before the reflections reach the far ends), falls
with every added cell and stays below 1e-3 in amplitude at 4 cells, 1e-4 at 8 and 1e-5 at 16 --
the level the transfer-matrix pin (P4) relies on.  With the convolution memories held at zero
the absorber becomes plain vacuum ending on the zero-field walls, and the pulse comes back
whole."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import workloads as wl

RES = 50.0
VAC = 300   # cells of vacuum on each side of the source: 6 time units of travel


def vacuum_line(pml: int) -> dict:
    p = wl.slab_cavity(1, 1, (pml, VAC, 0, 0, 0, VAC), RES, num_bath=0, sigma=0.01,
                       phase_seed=None, nfreq=4, steps=10, src_z=pml + VAC)
    p = wl.vacuum_of(p)
    p["energy_box"] = (pml, p["n"][2] - pml)
    return p


def reflection(pml: int, zero_memories: bool = False) -> float:
    """Amplitude reflection |R| = sqrt(max box energy in the reflection window / peak)."""
    p = vacuum_line(pml)
    dt = p["courant"] / RES
    t0 = p["sources"][0]["t0"]
    travel = VAC / RES
    steps = int((t0 + 3 * travel) / dt)
    o = O.OracleSim(p, trace_cap=steps)
    if zero_memories:
        zero = np.zeros(o.shape)
        for _ in range(steps):
            o.step(1)
            for name in ("psiE", "psiH"):
                for c in range(2):
                    o.set(name, zero, comp=c)
    else:
        o.step(steps)
    u = o.trace()[:, 0]
    t = (np.arange(u.size) + 1) * dt
    window = (t > t0 + travel + 2.0) & (t < t0 + 3 * travel - 2.0)
    assert window.sum() > 100
    return float(np.sqrt(u[window].max() / u.max()))


def test_p10_cpml_reflection_falls_with_thickness():
    R = {n: reflection(n) for n in (4, 8, 12, 16)}
    print("\nCPML amplitude reflection by thickness:", {n: f"{r:.2e}" for n, r in R.items()})
    assert R[4] < 1e-3 and R[8] < 1e-4 and R[16] < 1e-5
    assert R[4] > R[8] > R[12] > R[16] > 0


def test_p10_without_memories_the_pulse_reflects():
    """Sanity of the pin itself: the same layer without its convolution memories reflects."""
    assert reflection(8, zero_memories=True) > 0.5
