"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (normwise relative error ||x_gpu - x_oracle|| / ||x_oracle|| of a vector field,
its three components stacked):
  FP64 path: 1e-12 for E, H, the Lorentz-Bath polarization and bath modes, spectra and
             energy traces.
  FP32 path: 1e-5 for E, H and spectra (the FP32 target), 1e-4 for the Lorentz-Bath
             polarization and bath modes, whose small amplitude raises their relative error.
The polarization of a Drude mirror is the one ill-conditioned quantity: inside the metal E is
evanescent (1e-3 .. 1e-4 of the vacuum field) while P ~ -(w_p/w)^2 E accumulates, so a
one-ulp change of the source phase moves it by ~1e-12 in the oracle itself.  Its FP64 bound
is 30x that measured one-ulp sensitivity; its FP32 bound is that sensitivity scaled from the
FP64 to the FP32 unit roundoff (x 2^29); never below the stated tolerance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
TOL_Y = {64: 1e-12, 32: 1e-4}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def eps_grid(prob):
    eps = np.ones(prob["n"][::-1])
    for m in prob["materials"]:
        eps[m["z"][0]:m["z"][1]] = m.get("eps_inf", 1.0)
    return eps


def load_state(g, o, prob, st, precision):
    """Write the same state into both; FP32 runs get float-rounded values on both sides."""
    rnd = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == 32 else (lambda a: a)
    st = {k: rnd(v) for k, v in st.items()}
    for key, arr in st.items():
        if key[0] == "Y":
            g.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
            o.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
        else:
            g.set(key[0], arr, comp=key[1])
            o.set(key[0], arr, comp=key[1])
    eps = eps_grid(prob)
    for c in range(3):
        o.set("D", eps * st[("E", c)] + st[("Pm", c)], comp=c)


def stack(sim, name, **kw):
    return np.stack([sim.get(name, comp=c, **kw) for c in range(3)])


def compare(g, o, prob, precision, check_bath=True):
    """Normwise relative errors: E, H over the grid; P, P^{n-1/2} and bath modes per material."""
    errs = {("E",): rel(stack(g, "E"), stack(o, "E")), ("H",): rel(stack(g, "H"), stack(o, "H"))}
    for mi, m in enumerate(prob["materials"]):
        if m["kind"] == "vacuum":
            continue
        lo, hi = m["z"]
        for name in ("P", "Pm"):
            errs[(name, m["kind"], mi)] = rel(stack(g, name)[:, lo:hi], stack(o, name)[:, lo:hi])
        if check_bath and m["kind"] == "lorentz_bath":
            nb = len(m["bath_frequencies"])
            for j in sorted({0, nb // 2, nb - 1}):
                for lvl in (0, 1):
                    errs[("Y", mi, j, lvl)] = rel(stack(g, "Y", mode=j, level=lvl)[:, lo:hi],
                                                 stack(o, "Y", mode=j, level=lvl)[:, lo:hi])
    return errs


def oracle_sensitivity(prob, steps):
    """The oracle against itself with the source phase (without a phase table: the pulse delay t0)
    moved by one ulp (same keys as compare)."""
    a = O.OracleSim(prob)
    p2 = dict(prob)
    p2["sources"] = [dict(s, phase=np.nextafter(s["phase"], 10.0)) if s.get("phase") is not None
                     else dict(s, t0=float(np.nextafter(s["t0"], 1e9))) for s in prob["sources"]]
    b = O.OracleSim(p2)
    a.step(steps)
    b.step(steps)
    return compare(b, a, prob, 64)


def assert_errs(errs, precision, sens=None):
    for k, e in errs.items():
        if k[0] in ("E", "H"):
            tol = TOL[precision]
        elif k[0] == "Y" or k[1] == "lorentz_bath" or k[1] == "lorentz":
            tol = TOL_Y[precision]
        else:   # Drude mirror polarization
            tol = TOL_Y[precision] if precision == 32 else TOL[precision]
            if sens is not None:
                # the oracle's one-ulp (2^-53) sensitivity, scaled to the path's unit roundoff
                ulps = 1.0 if precision == 64 else 2.0 ** 29
                tol = max(tol, 30.0 * sens[k] * (1.0 if precision == 64 else 1.0 / 30.0) * ulps)
        assert e < tol, (k, e, tol)


@pytest.mark.parametrize("precision", [64, 32])
def test_small_cavity_from_rest_matches_oracle(precision):
    prob = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=120, seed=1)
    g = fb.Simulation(prob, precision=precision, energy_capacity=200)
    o = O.OracleSim(prob, trace_cap=200)
    g.step(120)
    o.step(120)
    errs = compare(g, o, prob, precision)
    assert_errs(errs, precision, sens=oracle_sensitivity(prob, 120))
    # spectra and energy traces
    assert rel(g.dft(0), o.dft(0)) < TOL[precision]
    tg, to = g.trace(), o.trace()
    assert tg.shape[0] == 120
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < (1e-12 if precision == 64 else 1e-5), col
    assert np.max(np.abs(o.get("E", comp=0))) > 1e-8   # the pulse reached the grid


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("shape", [(37, 11, 46), (33, 9, 41), (1, 1, 60), (64, 1, 40)])
def test_random_state_ragged_tiles(precision, shape):
    nx, ny, nz = shape
    layout = (6, nz - 6 - 6 - 2 - 2 - 12 - 6, 2, 12, 2, 6)
    prob = wl.slab_cavity(nx, ny, layout, 20.0, num_bath=5, sigma=0.01, bath_seed=4,
                          phase_seed=7, nfreq=12, steps=9)
    prob["courant"] = 0.5 if (nx > 1 and ny > 1) else 0.6
    st = wl.random_state(prob, seed=21)
    g = fb.Simulation(prob, precision=precision, energy_capacity=16)
    o = O.OracleSim(prob, trace_cap=16)
    load_state(g, o, prob, st, precision)
    g.step(9)
    o.step(9)
    assert_errs(compare(g, o, prob, precision), precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_step_calls_compose_bitwise(precision):
    prob = wl.small_3d(nx=35, ny=10, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=40, seed=2)
    a = fb.Simulation(prob, precision=precision, energy_capacity=64)
    b = fb.Simulation(prob, precision=precision, energy_capacity=64)
    a.step(17)
    a.step(0)
    _ = a.get("E", comp=0)        # a read flushes the pending H half-step
    a.step(23)
    b.step(40)
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            assert np.array_equal(a.get(name, comp=c), b.get(name, comp=c)), (name, c)
    assert np.array_equal(a.dft(0), b.dft(0))
    assert a.steps_done == b.steps_done == 40


@pytest.mark.parametrize("precision", [64, 32])
def test_zero_coupling_is_lorentz_bitwise_on_gpu(precision):
    base = wl.small_3d(nx=34, ny=9, layout=(6, 5, 3, 10, 3, 5), nb=6, steps=50, seed=3)
    lb = base["materials"][1]
    lb0 = dict(lb, bath_couplings=np.zeros_like(lb["bath_couplings"]))
    lor = dict(kind="lorentz", z=lb["z"], eps_inf=1.0, frequency=lb["frequency"],
               gamma=lb["gamma"], sigma=lb["sigma"])
    sa = fb.Simulation(dict(base, materials=[base["materials"][0], lb0, base["materials"][2]]),
                       precision=precision)
    sb = fb.Simulation(dict(base, materials=[base["materials"][0], lor, base["materials"][2]]),
                       precision=precision)
    sa.step(50)
    sb.step(50)
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            x, y = sa.get(name, comp=c), sb.get(name, comp=c)
            assert np.array_equal(x, y), (name, c)


def test_cavity_1d_fp64_matches_oracle():
    prob = wl.cavity_1d(steps=3000)
    g = fb.Simulation(prob, precision=64, energy_capacity=3100)
    o = O.OracleSim(prob, trace_cap=3100)
    g.step(3000)
    o.step(3000)
    assert_errs(compare(g, o, prob, 64), 64, sens=oracle_sensitivity(prob, 3000))
    assert rel(g.dft(0), o.dft(0)) < 1e-12
    assert rel(g.trace()[:, 0], o.trace()[:, 0]) < 1e-12


def test_uniform_3d_equals_1d_on_gpu():
    p1 = wl.slab_cavity(1, 1, (8, 10, 3, 12, 3, 10), 20.0, num_bath=4, sigma=0.01, bath_seed=2,
                        phase_seed=None, nfreq=8, steps=200)
    p3 = dict(p1, n=(40, 9, p1["n"][2]))
    a = fb.Simulation(p1, precision=64)
    b = fb.Simulation(p3, precision=64)
    a.step(200)
    b.step(200)
    x = a.get("E", comp=0)[:, 0, 0]
    y = b.get("E", comp=0)
    assert np.max(np.abs(y - x[:, None, None])) <= 1e-13 * np.max(np.abs(x))
    assert np.max(np.abs(x)) > 1e-8


@pytest.mark.slow
@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_3d_random_state(precision):
    """The 256^3 / N_b = 8 workload in the bench's launch configuration: two steps from a
    seeded random state, every cell of every field compared with the oracle."""
    prob = wl.slab_3d(steps=2)
    st = wl.random_state(prob, seed=5)
    g = fb.Simulation(prob, precision=precision, energy_capacity=8)
    o = O.OracleSim(prob, trace_cap=8)
    load_state(g, o, prob, st, precision)
    g.step(2)
    o.step(2)
    assert_errs(compare(g, o, prob, precision), precision)
    assert rel(g.trace()[:, 0], o.trace()[:, 0]) < (1e-12 if precision == 64 else 1e-5)


def test_bad_step_argument_and_empty_step():
    prob = wl.small_3d(nx=32, ny=8, steps=1)
    g = fb.Simulation(prob, precision=32)
    with pytest.raises(fb.FdtdBathError):
        fb.step(g.h, -1)
    g.step(0)
    assert g.steps_done == 0
    assert np.all(g.get("E", comp=0) == 0)


@pytest.mark.parametrize("precision", [64, 32])
def test_1d_cavity_moving_to_3d_kernel_keeps_traces(precision):
    """A 1D cavity runs on the persistent 1D kernel until a y component is written, then on the
    3D kernel, whose energy partials have their own layout: the trace must stay the oracle's."""
    prob = wl.slab_cavity(1, 1, (8, 200, 10, 200, 10, 164), 100.0, num_bath=4, sigma=0.01,
                          bath_seed=3, phase_seed=None, src_z=60, mon_z=560, nfreq=16, steps=600)
    g = fb.Simulation(prob, precision=precision, energy_capacity=700)
    o = O.OracleSim(prob, trace_cap=700)
    g.step(300)
    o.step(300)
    ey = 1e-3 * np.random.default_rng(5).standard_normal(prob["n"][::-1])
    if precision == 32:
        ey = ey.astype(np.float32).astype(np.float64)
    g.set("E", ey, comp=1)
    o.set("E", ey, comp=1)
    eps = eps_grid(prob)
    o.set("D", eps * o.get("E", comp=1) + o.get("Pm", comp=1), comp=1)
    g.step(300)
    o.step(300)
    tol = TOL[precision]
    tg, to = g.trace(), o.trace()
    assert tg.shape == to.shape == (600, 4)
    for col in range(3):
        assert rel(tg[:, col], to[:, col]) < tol, col
    assert rel(g.dft(0), o.dft(0)) < tol
    assert rel(stack(g, "E"), stack(o, "E")) < tol
