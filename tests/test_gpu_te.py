"""The TE form of y-invariant grids (ny = 1, every source on E_y; Sec. II.C's 2D case): the step
kernel carries only E_y, H_x, H_z, P_y and the y bath modes.

Checks: (1) against the general three-component form of the same run (forced by a write to
E_x before the first step): every field, spectrum and energy trace bit-identical in FP64, and
in FP32 within the FP32 tolerances of the parity tests, 1e-5 for fields, spectra and traces,
1e-4 for the layer's polarization and bath modes (normwise relative; the two kernels are
compiled separately, so FMA contraction places roundings differently); the components the TE form skips stay exactly 0;
(2) the TE form against the FP64 oracle at the parity tolerance 1e-12 (fields, the layer's
polarization, spectrum, energy trace); (3) the switch back to
the general form on a write to a skipped component."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 400


def rel(a, b):
    a, b = np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def snapshot(s, prob):
    out = {}
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            out[(name, c)] = s.get(name, comp=c)
    nb = len(prob["materials"][1]["bath_frequencies"])
    for j in range(nb):
        for lvl in (0, 1):
            for c in range(3):
                out[("Y", c, j, lvl)] = s.get("Y", comp=c, mode=j, level=lvl)
    out["dft"] = s.dft(0)
    out["trace"] = s.trace()
    return out


def run(prob, precision, general):
    s = fb.Simulation(prob, precision=precision, energy_capacity=STEPS + 8)
    assert s.te_form()
    if general:
        s.set("E", np.zeros(prob["n"][::-1]), comp=0)   # E_x written: general form from now on
        assert not s.te_form()
    s.step(STEPS)
    snap = snapshot(s, prob)
    s.close()
    return snap


@pytest.mark.parametrize("precision", [64, 32])
def test_te_form_matches_general_form(precision):
    prob = wl.adjoint_crop(steps=STEPS, nb=8)
    te, gen = run(prob, precision, False), run(prob, precision, True)
    live = 0
    for key in te:
        a, b = te[key], gen[key]
        dead = isinstance(key, tuple) and (
            (key[0] in ("E", "P", "Pm", "Y") and key[1] != 1) or (key[0] == "H" and key[1] == 1))
        if dead:
            assert not np.any(a) and not np.any(b), key
            continue
        if precision == 64:
            assert np.array_equal(a, b), key
        elif isinstance(key, tuple) and key[0] in ("P", "Pm", "Y"):
            # FP32 polarization and bath modes: the Lorentz-Bath layer at 1e-4 (the Drude
            # mirrors' polarization is conditioning-limited, see test_gpu_parity)
            lo, hi = prob["materials"][1]["z"]
            assert rel(a[lo:hi], b[lo:hi]) < 1e-4, (key, rel(a[lo:hi], b[lo:hi]))
        else:
            assert rel(a, b) < 1e-5, (key, rel(a, b))
        live += int(np.any(b))
    assert live >= 10


def test_te_form_matches_oracle():
    prob = wl.adjoint_crop(steps=STEPS, nb=8)
    s = fb.Simulation(prob, precision=64, energy_capacity=STEPS + 8)
    assert s.te_form()
    s.step(STEPS)
    o = O.OracleSim(prob, trace_cap=STEPS + 8)
    o.step(STEPS)
    for name in ("E", "H"):
        g = np.stack([s.get(name, comp=c) for c in range(3)])
        r = np.stack([o.get(name, comp=c) for c in range(3)])
        assert rel(g, r) < 1e-12, name
    # the Lorentz-Bath layer's polarization (the Drude mirrors' is conditioning-limited at the
    # 1e-12 level in the oracle itself; the general parity tests bound it separately)
    lo, hi = prob["materials"][1]["z"]
    for name in ("P", "Pm"):
        assert rel(s.get(name, comp=1)[lo:hi], o.get(name, comp=1)[lo:hi]) < 1e-12, name
    assert rel(s.dft(0), o.dft(0)) < 1e-12
    tg, to = s.trace(), o.trace()
    n = min(len(tg), len(to))
    for col in range(3):
        if np.any(to[:n, col]):
            assert rel(tg[:n, col], to[:n, col]) < 1e-12, col
    s.close()


def test_write_to_skipped_component_leaves_te_form():
    prob = wl.adjoint_crop(steps=40, nb=4)
    s = fb.Simulation(prob, precision=32)
    assert s.te_form()
    s.set("H", np.zeros(prob["n"][::-1]), comp=0)   # H_x is carried by the TE form
    s.set("P", np.zeros(prob["n"][::-1]), comp=1)
    assert s.te_form()
    s.step(20)
    s.set("H", np.zeros(prob["n"][::-1]), comp=1)   # H_y is not
    assert not s.te_form()
    s.step(20)
    assert s.steps_done == 40
    s.close()


def adjoint_gradient(prob, precision, general, dLdF, steps=STEPS, every=96):
    s = fb.Simulation(prob, precision=precision)
    if general:
        s.set("E", np.zeros(prob["n"][::-1]), comp=0)
    s.adjoint_forward(steps, every)
    g = s.adjoint_backward(dLdF, material=1)
    te = s.adjoint_te_form()
    s.close()
    return g, te


@pytest.mark.parametrize("precision", [64, 32])
def test_te_reverse_sweep_matches_general_form(precision):
    """The reverse sweep of a TE run with dL/dF zero on the E_x and H_y spectra runs the TE
    form of the adjoint kernels: its gradient equals the general form's (bit for bit in FP64,
    within 1e-5 in FP32).
    A nonzero E_x entry sends the same TE run through the general reverse sweep."""
    prob = wl.adjoint_crop(steps=STEPS, nb=8)
    nf = len(prob["monitors"][0]["freqs"])
    d = np.random.default_rng(5).standard_normal((nf, 4, 2))
    d[:, 0, :] = 0.0   # E_x spectrum
    d[:, 3, :] = 0.0   # H_y spectrum
    g_te, te = adjoint_gradient(prob, precision, False, d)
    g_gen, te_gen = adjoint_gradient(prob, precision, True, d)
    assert te and not te_gen
    assert np.all(np.isfinite(g_te)) and np.any(g_te)
    if precision == 64:
        assert np.array_equal(g_te, g_gen)
    else:
        assert rel(g_te, g_gen) < 1e-5, rel(g_te, g_gen)
    d[:, 0, 0] = 1.0
    g1, te1 = adjoint_gradient(prob, precision, False, d)
    g2, _ = adjoint_gradient(prob, precision, True, d)
    assert not te1
    if precision == 64:
        assert np.array_equal(g1, g2)
    else:
        assert rel(g1, g2) < 1e-5
