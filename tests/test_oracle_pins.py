"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

P1  Yee numerical dispersion: discrete plane / standing eigenmodes, hand-derived from
    Maxwell's curl equations (Eq. 1a,b) on the Yee lattice, must evolve as exp(-i w t)
    with sin^2(w dt/2)/dt^2 = sum_d sin^2(k_d dx/2)/dx^2 -- every curl term and sign.
P2  Lorentz-Bath with all k_j = 0 reproduces the Lorentz update bit for bit.
P3  A single cell driven at one frequency settles to P/E = chi_discrete, the exact
    z-transform of Eq. Pz_1D_Lorentz / Pz_update-LB / Yzj_finite_difference; it tends to
    Eq. chi_L / chi_LB as dt -> 0.
P5  With all damping zero, no source and no absorber, the discrete energy derived from
    Eq. H_full is conserved to rounding.
P6  A transversely uniform 3D run equals the 1D run cell for cell (Sec. IV.C: 2D = 1D).
P7  Table I: the uniform bath's (1/w) Im Sigma(w0) equals bath_dephasing in the continuum
    limit (Eq. int_countor_simplified, bath_dephasing_value_uniform) and the Lorentzian
    bath follows the Im I(w) approximation that follows Eq. self-energy-lorentz-bath-code.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from paper_2505_23963_gb300 import workloads as wl


def vacuum(nx, ny, nz, res=10.0, courant=0.5, pml=0):
    return dict(n=(nx, ny, nz), resolution=res, courant=courant, pml=pml, materials=[],
                sources=[], monitors=[])


def grid_idx(nx, ny, nz):
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return I.astype(float), J.astype(float), K.astype(float)


def mode(kind, nx, ny, nz, dx, dt, m=(1, 1)):
    """Return (omega, fields(tE, tH) -> {(name, comp): array}) of a discrete eigenmode."""
    I, J, K = grid_idx(nx, ny, nz)
    S = dt / dx
    # standing wave along z in the closed box: E ~ cos(K (k+1/2) dx), H ~ sin(K (k+1) dx)
    Kz = math.pi * (m[1] + 0.5) / ((nz + 0.5) * dx)
    C = np.cos(Kz * (K + 0.5) * dx)
    Sk = np.sin(Kz * (K + 1.0) * dx)
    if kind == "xz_te":         # Ey, Hx, Hz
        kx = 2 * math.pi * m[0] / (nx * dx)
        w = cf.yee_omega([kx, Kz], dx, dt)
        hx = -1j * S * math.sin(Kz * dx / 2) / math.sin(w * dt / 2)
        hz = S * math.sin(kx * dx / 2) / math.sin(w * dt / 2)

        def f(tE, tH):
            return {("E", 1): np.real(C * np.exp(1j * (kx * I * dx - w * tE))),
                    ("H", 0): np.real(hx * Sk * np.exp(1j * (kx * I * dx - w * tH))),
                    ("H", 2): np.real(hz * C * np.exp(1j * (kx * (I + 0.5) * dx - w * tH)))}
        return w, f
    if kind == "yz_te":         # Ex, Hy, Hz
        ky = 2 * math.pi * m[0] / (ny * dx)
        w = cf.yee_omega([ky, Kz], dx, dt)
        hy = 1j * S * math.sin(Kz * dx / 2) / math.sin(w * dt / 2)
        hz = -S * math.sin(ky * dx / 2) / math.sin(w * dt / 2)

        def f(tE, tH):
            return {("E", 0): np.real(C * np.exp(1j * (ky * J * dx - w * tE))),
                    ("H", 1): np.real(hy * Sk * np.exp(1j * (ky * J * dx - w * tH))),
                    ("H", 2): np.real(hz * C * np.exp(1j * (ky * (J + 0.5) * dx - w * tH)))}
        return w, f
    if kind == "xz_tm":         # Ex, Ez, Hy  (h = 1)
        kx = 2 * math.pi * m[0] / (nx * dx)
        w = cf.yee_omega([kx, Kz], dx, dt)
        st, sx, sz = math.sin(w * dt / 2), math.sin(kx * dx / 2), math.sin(Kz * dx / 2)
        ex, ez = -1j * S * sz / st, -S * sx / st

        def f(tE, tH):
            return {("E", 0): np.real(ex * C * np.exp(1j * (kx * (I + 0.5) * dx - w * tE))),
                    ("E", 2): np.real(ez * Sk * np.exp(1j * (kx * I * dx - w * tE))),
                    ("H", 1): np.real(Sk * np.exp(1j * (kx * (I + 0.5) * dx - w * tH)))}
        return w, f
    if kind == "yz_tm":         # Ey, Ez, Hx  (h = 1)
        ky = 2 * math.pi * m[0] / (ny * dx)
        w = cf.yee_omega([ky, Kz], dx, dt)
        st, sy, sz = math.sin(w * dt / 2), math.sin(ky * dx / 2), math.sin(Kz * dx / 2)
        ey, ez = 1j * S * sz / st, S * sy / st

        def f(tE, tH):
            return {("E", 1): np.real(ey * C * np.exp(1j * (ky * (J + 0.5) * dx - w * tE))),
                    ("E", 2): np.real(ez * Sk * np.exp(1j * (ky * J * dx - w * tE))),
                    ("H", 0): np.real(Sk * np.exp(1j * (ky * (J + 0.5) * dx - w * tH)))}
        return w, f
    raise KeyError(kind)


@pytest.mark.parametrize("kind,shape,m", [
    ("xz_tm", (24, 1, 17), (2, 1)),
    ("yz_tm", (1, 20, 19), (3, 2)),
    ("xz_te", (18, 1, 23), (2, 3)),
    ("yz_te", (1, 16, 21), (1, 4)),
    ("yz_te", (1, 1, 40), (0, 5)),       # pure z standing wave (1D)
])
def test_p1_yee_dispersion(orc, kind, shape, m):
    nx, ny, nz = shape
    prob = vacuum(nx, ny, nz, res=10.0, courant=0.6 if sum(d > 1 for d in shape) == 2 else 0.9)
    sim = orc.OracleSim(prob)
    dx, dt = 1.0 / prob["resolution"], sim.dt
    w, f = mode(kind, nx, ny, nz, dx, dt, m)
    for (name, c), arr in f(-0.5 * dt, 0.0).items():
        sim.set(name, arr, comp=c)
        if name == "E":
            sim.set("D", arr, comp=c)
    nsteps = 157
    sim.step(nsteps)
    want = f((nsteps - 0.5) * dt, nsteps * dt)
    for (name, c), arr in want.items():
        got = sim.get(name, comp=c)
        scale = max(np.max(np.abs(arr)), 1e-30)
        assert np.max(np.abs(got - arr)) / scale < 1e-11, (kind, name, c)
    # components absent from the mode stay zero
    for name in ("E", "H"):
        for c in range(3):
            if (name, c) not in want:
                assert np.max(np.abs(sim.get(name, comp=c))) < 1e-14


def test_p1_wrong_sign_is_caught(orc):
    """Sanity of the pin itself: the mode with the opposite H sign does not evolve correctly."""
    nx, nz = 24, 17
    prob = vacuum(nx, 1, nz, res=10.0, courant=0.6)
    sim = orc.OracleSim(prob)
    dx, dt = 0.1, sim.dt
    w, f = mode("xz_tm", nx, 1, nz, dx, dt, (2, 1))
    for (name, c), arr in f(-0.5 * dt, 0.0).items():
        sim.set(name, -arr if name == "H" else arr, comp=c)
        if name == "E":
            sim.set("D", arr, comp=c)
    sim.step(40)
    want = f(39.5 * dt, 40 * dt)
    assert np.max(np.abs(sim.get("E", comp=2) - want[("E", 2)])) > 0.05


# ------------------------------------------------------------------ P3
def drive_cell(orc, m, nu, dt, nsteps=60000):
    """Drive one cell with E^n = cos(w t_n) and fit the steady state to Re(chi e^{-i w t})."""
    w = 2 * math.pi * nu
    P = Pm = 0.0
    nb = len(m.get("bath_frequencies", [])) if m["kind"] == "lorentz_bath" else 0
    Y = np.zeros(max(nb, 1))
    Ym = np.zeros(max(nb, 1))
    w0, g, sig = 2 * math.pi * m["frequency"], 2 * math.pi * m["gamma"], m["sigma"]
    tail = []
    for n in range(nsteps):
        E = math.cos(w * n * dt)
        if m["kind"] == "lorentz":
            Pn = orc.lorentz_update(E, P, Pm, w0, g, sig, dt)
        elif m["kind"] == "drude":
            Pn = orc.drude_update(E, P, Pm, w0, g, sig, dt)
        else:
            Pn = orc.lorentz_bath_update(E, P, Pm, w0, g, sig,
                                         2 * math.pi * np.asarray(m["bath_frequencies"]),
                                         2 * math.pi * np.asarray(m["bath_gammas"]),
                                         2 * math.pi * np.asarray(m["bath_couplings"]), Y, Ym, dt)
        Pm, P = P, Pn
        if n >= nsteps - 4000:
            tail.append((n, Pn))
    # P^{n+1} responds to E^n: P at index n+1 = Re(chi exp(-i w (n+1) dt) * z^{-1}) with the
    # lag folded into chi_discrete's definition: P^{m+1} from E^m.  Fit P^{n+1} = a cos(w n dt) + b sin.
    n = np.array([t[0] for t in tail], dtype=float)
    p = np.array([t[1] for t in tail])
    # a constant column absorbs the free DC offset a Drude polarization can carry
    A = np.stack([np.cos(w * (n + 1) * dt), np.sin(w * (n + 1) * dt), np.ones_like(n)], axis=1)
    a, b, _ = np.linalg.lstsq(A, p, rcond=None)[0]
    return a + 1j * b   # Re(chi e^{-i w t}) = Re(chi) cos + Im(chi) sin


def test_p3_discrete_susceptibility(orc):
    dt = 0.5 / 40.0
    bf, bg, bk = cf.bath_form("lorentzian", 1.0, 0.01, 12, 0.2, 0.02, 0.03)
    mats = [
        dict(kind="lorentz", frequency=1.0, gamma=0.05, sigma=0.3),
        dict(kind="drude", frequency=1.0, gamma=0.4, sigma=2.0),
        dict(kind="lorentz_bath", frequency=1.0, gamma=0.05, sigma=0.3,
             bath_frequencies=bf, bath_gammas=bg, bath_couplings=bk),
    ]
    for m in mats:
        for nu in (0.7, 0.97, 1.3):
            got = drive_cell(orc, m, nu, dt)
            # the recursion's P^{m+1} answers E^m: chi_discrete is defined with that lag
            want = complex(cf.chi_discrete(nu, dt, m))
            assert abs(got - want) / abs(want) < 1e-9, (m["kind"], nu, got, want)


def test_p3_discrete_tends_to_continuum():
    bf, bg, bk = cf.bath_form("gaussian", 1.0, 0.01, 16, 0.3, 0.01, 0.02)
    m = dict(kind="lorentz_bath", frequency=1.0, gamma=0.02, sigma=0.1, bath_frequencies=bf,
             bath_gammas=bg, bath_couplings=bk)
    nu = np.array([0.8, 0.95, 1.0, 1.1])
    want = cf.chi_material(nu, m)
    errs = []
    for dt in (1e-2, 5e-3, 2.5e-3):
        errs.append(np.max(np.abs(cf.chi_discrete(nu, dt, m) - want) / np.abs(want)))
    # second-order convergence in dt
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[2] < 2e-3


# ------------------------------------------------------------------ P2
def test_p2_zero_coupling_is_lorentz_bitwise(orc):
    base = wl.small_3d(nx=6, ny=5, layout=(4, 4, 2, 6, 2, 4), nb=5, steps=80, seed=3)
    lb = base["materials"][1]
    assert lb["kind"] == "lorentz_bath"
    lb0 = dict(lb, bath_couplings=np.zeros_like(lb["bath_couplings"]))
    lor = dict(kind="lorentz", z=lb["z"], eps_inf=1.0, frequency=lb["frequency"],
               gamma=lb["gamma"], sigma=lb["sigma"])
    pa = dict(base, materials=[base["materials"][0], lb0, base["materials"][2]])
    pb = dict(base, materials=[base["materials"][0], lor, base["materials"][2]])
    sa, sb = orc.OracleSim(pa), orc.OracleSim(pb)
    sa.step(80)
    sb.step(80)
    for name in ("E", "H", "P", "Pm", "D"):
        for c in range(3):
            a, b = sa.get(name, comp=c), sb.get(name, comp=c)
            assert np.array_equal(a.view(np.int64), b.view(np.int64)), (name, c)
    assert np.max(np.abs(sa.get("E", comp=0))) > 0  # the run did something


# ------------------------------------------------------------------ P5
def test_p5_energy_invariant(orc):
    bf = np.array([0.93, 1.02, 1.08])
    prob = dict(n=(5, 4, 20), resolution=10.0, courant=0.5, pml=0, sources=[], monitors=[],
                materials=[
                    dict(kind="drude", z=(2, 4), eps_inf=1.0, frequency=1.0, gamma=0.0, sigma=3.0),
                    dict(kind="lorentz_bath", z=(5, 12), eps_inf=2.0, frequency=1.0, gamma=0.0,
                         sigma=0.2, bath_frequencies=bf, bath_gammas=np.zeros(3),
                         bath_couplings=np.array([0.05, 0.08, 0.03])),
                    dict(kind="lorentz", z=(13, 16), eps_inf=1.0, frequency=0.8, gamma=0.0,
                         sigma=0.5),
                ], energy_box=(0, 20))
    nsteps = 20000
    sim = orc.OracleSim(prob, trace_cap=nsteps, record_invariant=True)
    st = wl.random_state(prob, seed=11, scale=1.0)
    for (key, arr) in st.items():
        if key[0] == "Y":
            sim.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
        else:
            sim.set(key[0], arr, comp=key[1])
    eps = np.ones(prob["n"][::-1])
    eps[5:12] = 2.0
    for c in range(3):   # D = eps E + P^{n-1/2}
        sim.set("D", eps * st[("E", c)] + st[("Pm", c)], comp=c)
    sim.step(nsteps)
    I = sim.trace()[:, 3]
    rel = np.abs(I - I[0]) / abs(I[0])
    assert rel.max() < 1e-11, rel.max()
    # the individual parts exchange energy: the invariant is not trivially constant
    U = sim.trace()[:, 0]
    assert (U.max() - U.min()) / abs(I[0]) > 1e-3


def test_p5_damping_dissipates(orc):
    """Same box with gamma0 > 0: the invariant must decrease monotonically (no source)."""
    prob = dict(n=(3, 3, 12), resolution=10.0, courant=0.5, pml=0, sources=[], monitors=[],
                materials=[dict(kind="lorentz", z=(3, 9), eps_inf=1.0, frequency=1.0,
                                gamma=0.2, sigma=0.5)], energy_box=(0, 12))
    sim = orc.OracleSim(prob, trace_cap=3000, record_invariant=True)
    st = wl.random_state(prob, seed=5, scale=1.0, with_bath=False)
    for key, arr in st.items():
        sim.set(key[0], arr, comp=key[1])
    for c in range(3):
        sim.set("D", st[("E", c)] + st[("Pm", c)], comp=c)
    sim.step(3000)
    I = sim.trace()[:, 3]
    assert I[-1] < 0.5 * I[0]


# ------------------------------------------------------------------ P6
def test_p6_uniform_3d_equals_1d(orc):
    p1 = wl.slab_cavity(1, 1, (8, 10, 3, 12, 3, 10), 20.0, num_bath=4, sigma=0.01, bath_seed=2,
                        phase_seed=None, nfreq=8, steps=300)
    p3 = dict(p1, n=(3, 2, p1["n"][2]), courant=0.5)
    p1 = dict(p1, courant=0.5)
    a, b = orc.OracleSim(p1), orc.OracleSim(p3)
    a.step(300)
    b.step(300)
    for name in ("E", "H", "P"):
        x = a.get(name, comp=0)[:, 0, 0] if name != "H" else a.get(name, comp=1)[:, 0, 0]
        c = 0 if name != "H" else 1
        y3 = b.get(name, comp=c)
        for jj in range(2):
            for ii in range(3):
                assert np.max(np.abs(y3[:, jj, ii] - x)) <= 1e-13 * np.max(np.abs(x)), name
    assert np.max(np.abs(a.get("E", comp=0))) > 1e-6
    sa, sb = a.dft(0), b.dft(0)
    assert np.max(np.abs(sa - sb)) <= 1e-12 * np.max(np.abs(sa))


# ------------------------------------------------------------------ P7
def test_p7_table1_uniform_bath_dephasing():
    """(1/w) Im Sigma(w0) -> bath_dephasing for a dense uniform bath (gamma_b << dw << width)."""
    dephasing = 0.02
    bf, bg, bk = cf.bath_form("uniform", 1.0, 0.001, 801, 0.8, 0.004, dephasing)
    dw = 0.8 / 800
    assert np.allclose(bk, math.sqrt(2 * dw / math.pi * dephasing))
    assert np.allclose(np.diff(bf), dw) and bf[0] == pytest.approx(0.6) and bf[-1] == pytest.approx(1.4)
    S = cf.self_energy(np.array([1.0]), bf, bg, bk)[0]
    # Sigma is in angular units; (1/w) Im Sigma / 2pi is the dephasing in nu-units
    got = S.imag / (2 * math.pi * 1.0) / (2 * math.pi)
    assert got == pytest.approx(dephasing, rel=0.02)


def test_p7_table1_lorentzian_and_gaussian():
    # dense bath (gamma_b = 5 dw) so the sum over modes is the paper's integral
    dephasing, gamma, gb = 0.03, 0.01, 0.002
    G = gamma + dephasing
    bf, bg, bk = cf.bath_form("lorentzian", 1.0, gamma, 4001, 1.6, gb, dephasing)
    kb = bk[2000]
    assert bf[2000] == pytest.approx(1.0)
    assert np.allclose(bk ** 2 / kb ** 2, G ** 2 / (G ** 2 + (bf - 1.0) ** 2))
    S = cf.self_energy(np.array([1.0]), bf, bg, bk)[0]
    got = S.imag / (2 * math.pi) / (2 * math.pi)
    # Im I(w0) ~ (pi w0/2) G/(G + gamma_b/2)  =>  (1/w) Im Sigma = dephasing G/(G + gamma_b/2)
    assert got == pytest.approx(dephasing * G / (G + gb / 2), rel=1e-3)
    bfg, _, bkg = cf.bath_form("gaussian", 1.0, gamma, 41, 0.4, gb, dephasing)
    assert np.allclose(bkg / bkg[20], np.exp(-(bfg - 1.0) ** 2 / (4 * G ** 2)))
