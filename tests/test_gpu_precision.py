"""Precision form: FP64, FP32 and FP32 with bf16-stored bath modes on the 64^3 crop of the
512 x 512 x 384 workload (resolution 8, N_b = 16, Rabi splitting 0.1), each against the FP64
oracle: the monitor-plane field trace (E_x on the plane, sampled every 40 steps), the final
fields, the monitor spectra, the two polariton peak positions of the transmitted spectrum, and
the energy trace.  Every error is printed; the bounds asserted are stated per precision below.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import analysis
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEPS, EVERY = 1600, 40


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(sim, prob):
    z = prob["monitors"][0]["z"]
    tr = []
    for _ in range(STEPS // EVERY):
        sim.step(EVERY)
        tr.append(np.asarray(sim.get("E", comp=0)[z], dtype=np.float64))
    spec = sim.dft(0)
    out = dict(trace=np.stack(tr), E=np.asarray(sim.get("E", comp=0), np.float64),
               H=np.asarray(sim.get("H", comp=1), np.float64), spec=spec, energy=sim.trace())
    power = np.abs(spec[:, 0]) ** 2
    out["peaks"] = analysis.spectral_peaks(prob["monitors"][0]["freqs"], power, 2)
    return out


@pytest.fixture(scope="module")
def reference():
    prob = wl.precision_crop(STEPS)
    return prob, run(O.OracleSim(prob, trace_cap=STEPS + 8), prob)


def errors(got, ref):
    return {"trace": rel(got["trace"], ref["trace"]), "E": rel(got["E"], ref["E"]),
            "H": rel(got["H"], ref["H"]), "spectrum": rel(got["spec"], ref["spec"]),
            "peaks": float(np.max(np.abs(got["peaks"] - ref["peaks"]) / ref["peaks"])),
            "energy": rel(got["energy"][:, :3], ref["energy"][:, :3])}


@pytest.mark.parametrize("precision,bath_storage", [(64, 0), (32, 0), (32, 1)])
def test_precision_errors_on_crop(reference, precision, bath_storage):
    prob, ref = reference
    sim = fb.Simulation(prob, precision=precision, bath_storage=bath_storage, energy_capacity=STEPS + 8)
    e = errors(run(sim, prob), ref)
    print(f"\nprecision {precision} bath_storage {bath_storage}: " +
          " ".join(f"{k} {v:.3e}" for k, v in e.items()) + f" peaks {ref['peaks']}")
    assert ref["peaks"].size == 2
    if precision == 64:
        bounds = {k: 1e-12 for k in e}
    elif bath_storage == 0:
        # the FP32 targets: field traces, fields, spectra and energies 1e-5, peak positions 1e-4
        bounds = dict(trace=1e-5, E=1e-5, H=1e-5, spectrum=1e-5, energy=1e-5, peaks=1e-4)
    else:
        # bf16 bath storage rounds every bath mode to 2^-9 relative each step; the fields see it
        # through the weak bath coupling (measured 3e-5 .. 1.3e-4 here).  Peak positions keep the
        # FP32 target.
        bounds = dict(trace=1e-3, E=1e-3, H=1e-3, spectrum=1e-3, energy=1e-3, peaks=1e-4)
    for k, v in e.items():
        assert v < bounds[k], (k, v, bounds[k])


def test_bf16_bath_storage_roundtrip_and_step():
    """bf16 bath storage: written levels read back within bf16 rounding (the value to 2^-8
    relative, the older level through value - increment), and a few steps from that stored state
    follow the oracle started from the same (read-back) state."""
    prob = wl.small_3d(nx=33, ny=9, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=20, seed=4)
    st = wl.random_state(prob, seed=9)
    g = fb.Simulation(prob, precision=32, bath_storage=1)
    o = O.OracleSim(prob)
    for key, arr in st.items():
        if key[0] == "Y":
            g.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
        else:
            g.set(key[0], arr, comp=key[1])
    lo, hi = prob["materials"][1]["z"]
    for key, arr in st.items():
        if key[0] != "Y":
            continue
        got = g.get("Y", comp=key[1], mode=key[2], level=key[3]).astype(np.float64)[lo:hi]
        want = arr[lo:hi]
        scale = np.max(np.abs(st[("Y", key[1], key[2], 0)][lo:hi]))
        assert np.max(np.abs(got - want)) <= 2.0 ** -7 * scale, key
    # the oracle starts from exactly what the GPU holds
    eps = np.ones(prob["n"][::-1])
    for m in prob["materials"]:
        eps[m["z"][0]:m["z"][1]] = m.get("eps_inf", 1.0)
    for key in st:
        if key[0] == "Y":
            o.set("Y", g.get("Y", comp=key[1], mode=key[2], level=key[3]).astype(np.float64),
                  comp=key[1], mode=key[2], level=key[3])
        else:
            o.set(key[0], g.get(key[0], comp=key[1]).astype(np.float64), comp=key[1])
    for c in range(3):
        o.set("D", eps * o.get("E", comp=c) + o.get("Pm", comp=c), comp=c)
    g.step(20)
    o.step(20)
    for name, tol in (("E", 1e-4), ("H", 1e-4)):
        for c in range(3):
            assert rel(g.get(name, comp=c), o.get(name, comp=c)) < tol, (name, c)
    y = rel(g.get("Y", comp=0, mode=3, level=0)[lo:hi], o.get("Y", comp=0, mode=3, level=0)[lo:hi])
    print(f"\nbf16 bath storage, 20 steps from a random state: Y rel err {y:.3e}")
    # worst case: one bf16 rounding (2^-9 relative) of the value and one of the increment per
    # step, accumulating linearly over the 20 steps
    assert y < 20 * 2.0 ** -8
    with pytest.raises(fb.FdtdBathError) as e:
        fb.box_energy_noalloc(g.h, lo, hi)
    assert e.value.code == fb.ERR_UNSUPPORTED
    with pytest.raises(fb.FdtdBathError) as e:
        fb.Simulation(prob, precision=64, bath_storage=1)
    assert e.value.code == fb.ERR_ARG
