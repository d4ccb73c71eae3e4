"""GPU parity of the batched 1D form (fdtdbath_batch_*) against the FP64 CPU oracle, cavity by
cavity: every cavity of a batch must evolve exactly as the same cavity run alone.

Tolerances as in test_gpu_parity (normwise relative errors): FP64 1e-12 for E_x, H_y, the
Lorentz / Lorentz-Bath polarization, bath modes and energy traces; FP32 1e-5 for E_x, H_y and
the energy traces, 1e-4 for polarization and bath modes; the Drude-mirror polarization against
30x the oracle's own one-ulp sensitivity in FP64, and 10x that sensitivity scaled by 2^29 (the
FP64 / FP32 unit-roundoff ratio) in FP32 -- one perturbation of the source timing samples the
conditioning; the FP32 path rounds at every one of its thousands of updates.  Polariton relaxation rates
and bath shares derived from FP32 traces: 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import analysis
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
TOL_PY = {64: 1e-12, 32: 1e-4}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_1d(p, steps, phase_ulp=False):
    q = p
    if phase_ulp:   # the source moved by one ulp of its carrier phase
        q = dict(p, sources=[dict(s, t0=np.nextafter(s["t0"], 10.0)) for s in p["sources"]])
    o = O.OracleSim(q, trace_cap=steps + 16)
    o.step(steps)
    return o


def field(sim, name, **kw):
    return sim.get(name, comp=0 if name in ("E", "P", "Pm", "Y") else 1, **kw)[:, 0, 0]


def cavity_errors(b, i, p, o):
    errs = {"E": rel(b.get(i, "E"), field(o, "E")), "H": rel(b.get(i, "H"), field(o, "H"))}
    for mi, m in enumerate(p["materials"]):
        lo, hi = m["z"]
        if m["kind"] == "vacuum":
            continue
        for name in ("P", "Pm"):
            errs[(name, m["kind"], mi)] = rel(b.get(i, name)[lo:hi], field(o, name)[lo:hi])
        if m["kind"] == "lorentz_bath":
            nb = len(m["bath_frequencies"])
            for j in sorted({0, nb // 2, nb - 1}):
                for lvl in (0, 1):
                    errs[("Y", mi, j, lvl)] = rel(b.get(i, "Y", mode=j, level=lvl)[lo:hi],
                                                 field(o, "Y", mode=j, level=lvl)[lo:hi])
    return errs


def check(errs, precision, sens):
    for k, e in errs.items():
        if k in ("E", "H"):
            tol = TOL[precision]
        elif k[0] == "Y" or k[1] in ("lorentz", "lorentz_bath"):
            tol = TOL_PY[precision]
        else:   # Drude mirror polarization: conditioning-limited (see test_gpu_parity)
            ulps = 1.0 if precision == 64 else 2.0 ** 29
            tol = max(TOL_PY[precision] if precision == 32 else TOL[precision],
                      (30.0 if precision == 64 else 10.0) * sens[k] * ulps)
        assert e < tol, (k, e, tol)


def sensitivity(p, o, steps):
    o2 = oracle_1d(p, steps, phase_ulp=True)
    out = {}
    for mi, m in enumerate(p["materials"]):
        if m["kind"] == "drude":
            lo, hi = m["z"]
            for name in ("P", "Pm"):
                out[(name, "drude", mi)] = rel(field(o2, name)[lo:hi], field(o, name)[lo:hi])
    return out


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("shape", [(4, 128), (1, 256), (0, 0)])
def test_batch_matches_oracle(precision, shape):
    probs = wl.batch_small(seed=0, steps=600)
    b = fb.Batch(probs, precision=precision, cluster_ctas=shape[0], block_threads=shape[1],
                 energy_capacity=700)
    b.step(250)
    b.step(350)   # two calls: the state is written back and reloaded between them
    assert b.query(7) == 600
    for i, p in enumerate(probs):
        o = oracle_1d(p, 600)
        errs = cavity_errors(b, i, p, o)
        check(errs, precision, sensitivity(p, o, 600))
        tg = b.trace(i)
        if p["energy_box"][1] > p["energy_box"][0]:
            to = o.trace()
            assert tg.shape[0] == 600 and to.shape[0] == 600
            for col in range(3):
                if np.any(to[:, col] != 0):
                    assert rel(tg[:, col], to[:, col]) < TOL[precision], (i, col)
            assert np.max(np.abs(tg[:, 0])) > 0
        else:
            assert np.all(tg == 0)
    b.close()


def test_batch_packing_and_graphs_do_not_change_fields():
    """The same FP64 batch under two launch shapes, with and without CUDA graphs: the per-cell
    arithmetic does not depend on the packing, so the fields agree bit for bit."""
    probs = wl.batch_small(seed=3, steps=500)
    runs = []
    for shape, graph in (((2, 128), True), ((8, 256), False), ((1, 512), True)):
        b = fb.Batch(probs, precision=64, cluster_ctas=shape[0], block_threads=shape[1],
                     use_graph=graph)
        b.step(500)
        runs.append([(b.get(i, "E"), b.get(i, "H"), b.get(i, "P")) for i in range(len(probs))])
        if graph:
            assert b.query(6) >= 1   # graph replays
        b.close()
    for r in runs[1:]:
        for a, c in zip(runs[0], r):
            for x, y in zip(a, c):
                assert np.array_equal(x, y)


def test_batch_many_cavities_share_ctas():
    """40 short cavities under 16-CTA clusters: several cavities per cluster and per CTA, cuts
    inside cavities; every cavity against the oracle (FP64)."""
    probs = []
    rng = np.random.default_rng(11)
    for k in range(40):
        L = int(rng.integers(80, 400))
        probs.append(wl.batch_cavity(L, rabi=float(rng.uniform(0.02, 0.2)),
                                     num_bath=int(rng.choice([4, 8, 16, 32])), pml=8, mirror=6,
                                     steps=300))
    b = fb.Batch(probs, precision=64, cluster_ctas=16, block_threads=128, energy_capacity=400)
    b.step(300)
    assert b.query(1) < len(probs)   # fewer clusters than cavities
    for i in range(0, 40, 3):
        o = oracle_1d(probs[i], 300)
        assert rel(b.get(i, "E"), field(o, "E")) < 1e-12, i
        assert rel(b.get(i, "H"), field(o, "H")) < 1e-12, i
        assert rel(b.trace(i)[:, 0], o.trace()[:, 0]) < 1e-12, i


def test_batch_relaxation_and_bath_share_fp32():
    """gamma_pol and the bath share from FP32 batch traces against the oracle's, 1e-4."""
    probs = [wl.batch_cavity(L, rabi=r, num_bath=nb, steps=16000)
             for L, r, nb in ((1000, 0.1, 8), (1200, 0.2, 16))]
    b = fb.Batch(probs, precision=32, energy_every=4)
    b.step(16000)
    for i, p in enumerate(probs):
        o = oracle_1d(p, 16000)
        to = o.trace()[::4]
        tg = b.trace(i)
        assert tg.shape == to.shape
        dtr = 4 * p["courant"] / p["resolution"]
        t0 = p["sources"][0]["t0"]
        gg, go = analysis.relaxation_rate(tg, dtr, 2 * t0), analysis.relaxation_rate(to, dtr, 2 * t0)
        assert np.isfinite(go) and go > 0
        assert abs(gg - go) <= 1e-4 * abs(go), (gg, go)
        sg, so = analysis.bath_share(tg, dtr, 2 * t0), analysis.bath_share(to, dtr, 2 * t0)
        assert so > 0 and abs(sg - so) <= 1e-4 * so, (sg, so)


def test_full_size_batch_sampled_cavities():
    """The 64-cavity sweep in the autotuned launch, sampled cavities (the longest, the shortest,
    the largest N_b, two more) against the oracle at the FP32 tolerances: fields at step 600,
    while the pulse is still inside the grid, to 1e-5; energy traces over 2000 steps to 2e-5
    (energy is quadratic in the fields, so its relative error is twice theirs).  Later field
    snapshots of the short cavities are not compared normwise: once the pulse has left through
    the absorber the remaining field is ~1e-3 of the pulse, a residue of cancellations in the
    metal mirrors that FP32 arithmetic resolves only to ~1e-3 of itself (an independent
    float32 emulation of the same updates shows the same)."""
    probs = wl.batch_sweep(steps=2000)
    b = fb.Batch(probs, precision=32)
    L = [p["n"][2] for p in probs]
    nb = [len(p["materials"][1].get("bath_frequencies", [])) for p in probs]
    sample = sorted({int(np.argmax(L)), int(np.argmin(L)), int(np.argmax(nb)), 5, 40})
    orc = {i: O.OracleSim(probs[i], trace_cap=2016) for i in sample}
    b.step(600)
    for i in sample:
        orc[i].step(600)
        assert rel(b.get(i, "E"), field(orc[i], "E")) < 1e-5, i
        assert rel(b.get(i, "H"), field(orc[i], "H")) < 1e-5, i
    b.step(1400)
    traces = {}
    for i in sample:
        orc[i].step(1400)
        traces[i] = (b.trace(i), orc[i].trace())
    scale = max(float(np.max(to[:, 0])) for _, to in traces.values())
    compared = 0
    for i, (tg, to) in traces.items():
        assert tg.shape == to.shape == (2000, 4)
        for col in range(3):
            # a cavity the pulse has not reached yet holds only the pulse's underflowing tail
            if np.max(to[:, col]) > 1e-10 * scale:
                assert rel(tg[:, col], to[:, col]) < 2e-5, (i, col)
                compared += 1
    assert compared >= 6
    b.close()


def test_batch_rejects_bad_cavities():
    p = wl.batch_cavity(1000, rabi=0.1, num_bath=4, steps=10)
    bad = dict(p, sources=[dict(p["sources"][0], component=1)])
    with pytest.raises(fb.FdtdBathError) as e:
        fb.Batch([p, bad])
    assert e.value.code == fb.ERR_ARG and "cavity 1" in str(e.value)
