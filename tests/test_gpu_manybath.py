"""N_b = 100 bath modes per Lorentz-Bath cell (the baths of the paper's Fig. 2: Table I's
Lorentzian form, N = 100 over nu0 +/- 0.2, bath damping 4e-4, dephasing 0.0396).  Above 32
modes the step kernel streams the bath modes from memory instead of holding them in registers.

Parity against the FP64 oracle at the tolerances of test_gpu_parity (normwise relative):
FP64 1e-12 for E, H, the layer's P and bath modes, spectra and energy traces; FP32 1e-5 for
E, H and spectra, 1e-4 for the layer's P and bath modes.  Cases: a ragged 3D cavity (tiles cut
in x and y) and the paper's free-space slab of Fig. 2a in 1D (600 cells at dx = 0.01, 50-cell
CPML, a 1-unit slab), which runs on the step kernel (the register-resident 1D kernel holds at
most 32 modes); the slab again beside a Drude-mirror cavity in one batched launch.  The bath
arrays come from the oracle's Table I expansion (pinned by P7)."""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}
TOL_Y = {64: 1e-12, 32: 1e-4}
NB = 100


def rel(a, b):
    a, b = np.asarray(a, dtype=np.complex128), np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def with_paper_bath(prob, mat, sigma):
    f, g, k = cf.bath_form("lorentzian", 1.0, 4e-4, NB, 0.4, 4e-4, 0.0396)
    mats = list(prob["materials"])
    mats[mat] = dict(mats[mat], kind="lorentz_bath", gamma=4e-4, sigma=sigma, bath_frequencies=f,
                     bath_gammas=g, bath_couplings=k)
    return dict(prob, materials=mats)


def ragged_3d(steps):
    p = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=steps, seed=4)
    return with_paper_bath(p, 1, 2e-2), 1


def paper_slab_1d(steps):
    # cell 6 at dx = 0.01: CPML 50 | vacuum 200 | slab 100 | vacuum 200 | CPML 50
    p = wl.slab_cavity(1, 1, (50, 200, 0, 100, 0, 200), 100.0, num_bath=8, sigma=5e-3,
                       phase_seed=None, nfreq=64, steps=steps, name="paper_slab_fig2a")
    return with_paper_bath(p, 0, 5e-3), 0


def compare(prob, mat, precision, steps):
    s = fb.Simulation(prob, precision=precision, energy_capacity=steps + 8)
    s.step(steps)
    o = O.OracleSim(prob, trace_cap=steps + 8)
    o.step(steps)
    lo, hi = prob["materials"][mat]["z"]
    for name in ("E", "H"):
        g = np.stack([s.get(name, comp=c) for c in range(3)])
        r = np.stack([o.get(name, comp=c) for c in range(3)])
        assert rel(g, r) < TOL[precision], (name, rel(g, r))
    for name in ("P", "Pm"):
        g = np.stack([s.get(name, comp=c)[lo:hi] for c in range(3)])
        r = np.stack([o.get(name, comp=c)[lo:hi] for c in range(3)])
        assert rel(g, r) < TOL_Y[precision], (name, rel(g, r))
    for j in (0, 37, NB - 1):
        for lvl in (0, 1):
            g = np.stack([s.get("Y", comp=c, mode=j, level=lvl)[lo:hi] for c in range(3)])
            r = np.stack([o.get("Y", comp=c, mode=j, level=lvl)[lo:hi] for c in range(3)])
            assert rel(g, r) < TOL_Y[precision], (j, lvl, rel(g, r))
    assert rel(s.dft(0), o.dft(0)) < TOL[precision]
    tg, to = s.trace(), o.trace()
    n = min(len(tg), len(to))
    for col in range(3):
        if np.any(to[:n, col]):
            assert rel(tg[:n, col], to[:n, col]) < 2 * TOL[precision], col
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_many_bath_modes_3d(precision):
    prob, mat = ragged_3d(120)
    compare(prob, mat, precision, 120)


@pytest.mark.parametrize("precision", [64, 32])
def test_paper_slab_fig2a_1d(precision):
    prob, mat = paper_slab_1d(1500)
    compare(prob, mat, precision, 1500)


def test_mode_limits_of_the_forms():
    """The adjoint holds at most 32 bath modes per material, the batch (like the step kernel)
    at most 128."""
    prob, _ = paper_slab_1d(10)
    s = fb.Simulation(prob, precision=32)
    with pytest.raises(fb.FdtdBathError) as e:
        s.adjoint_forward(10, 4)
    assert e.value.code == fb.ERR_UNSUPPORTED
    s.close()
    f, g, k = cf.bath_form("lorentzian", 1.0, 4e-4, 129, 0.4, 4e-4, 0.0396)
    m0 = dict(prob["materials"][0], bath_frequencies=f, bath_gammas=g, bath_couplings=k)
    with pytest.raises(fb.FdtdBathError) as e:
        fb.Batch([dict(prob, materials=[m0])])
    assert e.value.code == fb.ERR_ARG


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_with_paper_baths(precision):
    """The batched form with N_b = 100: the paper's Fig. 2a slab and a Drude-mirror cavity whose
    360-cell bath layer (800 B of bath state per cell in FP32) spans the CTAs of a cluster, each
    cavity against the FP64 oracle: E_x, H_y, the layer's P and bath modes 0 / 37 / 99 and the
    energy traces."""
    steps = 600
    slab, _ = paper_slab_1d(steps)
    cav = with_paper_bath(wl.batch_cavity(900, rabi=0.1, num_bath=8, steps=steps), 1, 1e-2)
    probs = [slab, cav]
    b = fb.Batch(probs, precision=precision, cluster_ctas=4, block_threads=256,
                 energy_capacity=steps + 16)
    b.step(steps)
    for i, (p, mat) in enumerate(((slab, 0), (cav, 1))):
        o = O.OracleSim(p, trace_cap=steps + 16)
        o.step(steps)
        lo, hi = p["materials"][mat]["z"]
        assert rel(b.get(i, "E"), o.get("E", comp=0)[:, 0, 0]) < TOL[precision], (i, "E")
        assert rel(b.get(i, "H"), o.get("H", comp=1)[:, 0, 0]) < TOL[precision], (i, "H")
        for name in ("P", "Pm"):
            e = rel(b.get(i, name)[lo:hi], o.get(name, comp=0)[lo:hi, 0, 0])
            assert e < TOL_Y[precision], (i, name, e)
        for j in (0, 37, NB - 1):
            for lvl in (0, 1):
                e = rel(b.get(i, "Y", mode=j, level=lvl)[lo:hi],
                        o.get("Y", comp=0, mode=j, level=lvl)[lo:hi, 0, 0])
                assert e < TOL_Y[precision], (i, j, lvl, e)
        tg, to = b.trace(i), o.trace()
        n = min(len(tg), len(to))
        assert n == steps
        for col in range(3):
            if np.any(to[:n, col]):
                assert rel(tg[:n, col], to[:n, col]) < 2 * TOL[precision], (i, col)
    b.close()


def test_many_bath_modes_2d_te_form():
    """A y-invariant, E_y-driven 2D crop with N_b = 100: the TE form of the streamed kernel
    (128-wide single-row tiles) against the FP64 oracle."""
    p = wl.adjoint_crop(steps=300, nb=8)
    prob = with_paper_bath(p, 1, 2e-2)
    s = fb.Simulation(prob, precision=64, energy_capacity=308)
    assert s.te_form()
    s.close()
    compare(prob, 1, 64, 300)


def test_many_bath_modes_bf16_storage():
    """bf16 bath storage with N_b = 100 (value / increment pairs, streamed): fields, spectrum
    and the layer's polarization within the bf16 bounds of the precision form (1e-3)."""
    prob, mat = ragged_3d(120)
    s = fb.Simulation(prob, precision=32, bath_storage=1, energy_capacity=128)
    s.step(120)
    o = O.OracleSim(prob, trace_cap=128)
    o.step(120)
    lo, hi = prob["materials"][mat]["z"]
    for name in ("E", "H"):
        g = np.stack([s.get(name, comp=c) for c in range(3)])
        r = np.stack([o.get(name, comp=c) for c in range(3)])
        assert rel(g, r) < 1e-3, (name, rel(g, r))
    g = np.stack([s.get("P", comp=c)[lo:hi] for c in range(3)])
    r = np.stack([o.get("P", comp=c)[lo:hi] for c in range(3)])
    assert rel(g, r) < 1e-3, rel(g, r)
    assert rel(s.dft(0), o.dft(0)) < 1e-3
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_zero_coupling_is_lorentz_bitwise_streamed(precision):
    """Pin P2 on the streamed path: N_b = 100 bath modes with every coupling zero give the plain
    Lorentz medium bit for bit (E, H, P)."""
    prob, mat = ragged_3d(60)
    lb = prob["materials"][mat]
    lb0 = dict(lb, bath_couplings=np.zeros_like(lb["bath_couplings"]))
    lor = dict(kind="lorentz", z=lb["z"], eps_inf=1.0, frequency=lb["frequency"], gamma=lb["gamma"],
               sigma=lb["sigma"])
    mats = list(prob["materials"])
    sa = fb.Simulation(dict(prob, materials=mats[:mat] + [lb0] + mats[mat + 1:]), precision=precision)
    sb = fb.Simulation(dict(prob, materials=mats[:mat] + [lor] + mats[mat + 1:]), precision=precision)
    sa.step(60)
    sb.step(60)
    for name in ("E", "H", "P", "Pm"):
        for c in range(3):
            assert np.array_equal(sa.get(name, comp=c), sb.get(name, comp=c)), (name, c)
    sa.close()
    sb.close()
