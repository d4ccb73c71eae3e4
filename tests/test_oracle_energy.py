"""P12: the energy traces against the exact discrete invariant.  The traces (U_EM, U_P, U_bath)
read the energy density of Eq. H_full off the stored state after a step -- E at the half step,
H at the step's end, P' and Y_j' as one-step differences -- so their sum differs from the
scheme's exact invariant (pinned as conserved by P5) by terms of first order in dt, and from
nothing else: on an undamped, source-free Lorentz-Bath box the largest gap over 20 time units
halves with every halving of dt, and at the smallest dt it is below 2% of the energy.  A term
dropped from a trace (the bath share is ~8% here, the polarization's ~30%) would leave an O(1)
gap that does not shrink."""
import numpy as np
import pytest

from oracle import oracle as O

NZ = 40


def gap(courant: float, couple: float) -> tuple[float, float]:
    """Largest |U_EM + U_P + U_bath - I| / I over the run, and the oscillator energy share."""
    res = 10.0
    prob = dict(n=(1, 1, NZ), resolution=res, courant=courant, pml=0, sources=[], monitors=[],
                materials=[dict(kind="lorentz_bath", z=(5, 30), eps_inf=2.0, frequency=1.0,
                                gamma=0.0, sigma=0.2, bath_frequencies=np.array([0.93, 1.02, 1.08]),
                                bath_gammas=np.zeros(3),
                                bath_couplings=couple * np.array([0.05, 0.08, 0.03]))],
                energy_box=(0, NZ))
    nsteps = int(round(20.0 / (courant / res)))
    sim = O.OracleSim(prob, trace_cap=nsteps, record_invariant=True)
    z = (np.arange(NZ) + 0.5) / NZ
    E = np.sin(np.pi * z).reshape(NZ, 1, 1)
    eps = np.ones((NZ, 1, 1))
    eps[5:30] = 2.0
    sim.set("E", E, comp=0)
    sim.set("D", eps * E, comp=0)
    sim.step(nsteps)
    tr = sim.trace()
    inv = tr[:, 3] / res          # the invariant is summed per cell; the traces carry dx
    total = tr[:, 0] + tr[:, 1] + tr[:, 2]
    share = float((tr[:, 1] + tr[:, 2]).max() / inv[0])
    return float(np.max(np.abs(total - inv)) / inv[0]), share


@pytest.mark.parametrize("couple", [0.0, 1.0])
def test_p12_traces_converge_to_the_invariant_at_first_order(couple):
    gaps = [gap(c, couple)[0] for c in (0.5, 0.25, 0.125)]
    print(f"\ncouplings x{couple}: trace-invariant gaps {gaps}")
    for a, b in zip(gaps, gaps[1:]):
        assert 1.8 < a / b < 2.2
    assert gaps[-1] < 0.02
    assert gap(0.125, couple)[1] > 0.25     # the oscillators hold a real share of the energy
