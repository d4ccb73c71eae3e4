"""Seeded synthetic inputs for the FDTD-Bath path.

This module only builds problem descriptions -- grid sizes, planar material
layers with their Lorentz / Drude / Lorentz-Bath parameters, Gaussian-pulse
sources, DFT monitors and random initial states -- as plain dicts and numpy
arrays.  It performs none of the method's arithmetic (no field, polarization,
bath, absorber or DFT update) and imports nothing else from this package, so
both the CUDA library's binding and the CPU oracle can consume its output.

Conventions: c = eps0 = mu0 = 1; lengths in units of a with dx = 1/resolution
and dt = courant * dx; every frequency-like parameter (frequency, gamma, sigma
is dimensionless, bath frequencies/dampings/couplings, pulse centre and width,
DFT frequencies) is in nu-units (nu = omega / 2 pi), the unit MEEP and the paper
use.  Grids are [nz][ny][nx] with x fastest, periodic in x and y, with the
absorber and all layers stacked along z.

Problem dict keys:
    n=(nx, ny, nz), resolution, courant, pml (cells at each z end),
    materials=[{kind, z=(lo, hi), eps_inf, frequency, gamma, sigma,
                bath_frequencies, bath_gammas, bath_couplings}],
    sources=[{component, z, center, fwidth, amplitude, t0, phase (ny, nx) or None}],
    monitors=[{z, freqs}], energy_box=(lo, hi), steps, name.
"""
from __future__ import annotations

import math

import numpy as np


def ohmic_bath(num_bath: int, freqs: np.ndarray, frequency: float, dephasing: float,
               width: float, bath_gamma: float):
    """Bath arrays for the 'Ohmic-like' weighted coupling used by the cavity workloads.

    Frequencies are given; dampings are all ``bath_gamma``; couplings are
    k_j = k_b sqrt(w_j) with the weight w_j = (f_j/f0) exp(1 - f_j/f0) and the
    uniform-bath scale k_b = sqrt(2 df / pi * dephasing), df = width / (N - 1).
    """
    freqs = np.asarray(freqs, dtype=np.float64)
    df = width / (num_bath - 1)
    kb = math.sqrt(2.0 * df / math.pi * dephasing)
    wgt = (freqs / frequency) * np.exp(1.0 - freqs / frequency)
    return freqs, np.full(num_bath, float(bath_gamma)), kb * np.sqrt(wgt)


def pulse_t0(fwidth: float) -> float:
    """Pulse delay: five Gaussian widths, tau = 1/(2 pi fwidth)."""
    return 5.0 / (2.0 * math.pi * fwidth)


def slab_cavity(nx: int, ny: int, layout, resolution: float, *, num_bath: int, sigma: float,
                bath_seed: int | None = None, phase_seed: int | None = 0,
                src_z: int | None = None, mon_z: int | None = None, nfreq: int = 256,
                steps: int = 100, name: str = "slab", drude_sigma: float = 25.0,
                drude_gamma: float = 0.01, gamma0: float = 0.01, bath_gamma: float = 0.005,
                dephasing: float = 0.01, courant: float = 0.5, source_component: int = 0,
                phase_scale: float = math.pi / 8.0) -> dict:
    """Planar Fabry-Perot cavity: CPML | vacuum | Drude | Lorentz-Bath | Drude | vacuum | CPML.

    ``layout`` = (pml, vac_left, mirror, layer, mirror, vac_right) in cells along z.
    Bath frequencies are linspace(0.9, 1.1) or, with ``bath_seed``, uniform in
    [0.9, 1.1] from numpy.random.default_rng(bath_seed).  The source is an Ex
    plane in the left vacuum with a per-(x,y) phase (pi/8) U[-1, 1] drawn from
    default_rng(phase_seed) (None: zero phase).
    """
    pml, vl, mir, lay, mir2, vr = (int(v) for v in layout)
    nz = pml + vl + mir + lay + mir2 + vr + pml
    z_m1 = pml + vl
    z_lb = z_m1 + mir
    z_m2 = z_lb + lay
    z_end = z_m2 + mir2
    if num_bath > 0:
        if bath_seed is None:
            bf = np.linspace(0.9, 1.1, num_bath)
        else:
            bf = np.random.default_rng(bath_seed).uniform(0.9, 1.1, num_bath)
        bf, bg, bk = ohmic_bath(num_bath, bf, 1.0, dephasing, 0.2, bath_gamma)
        layer = dict(kind="lorentz_bath", z=(z_lb, z_m2), eps_inf=1.0, frequency=1.0,
                     gamma=gamma0, sigma=sigma, bath_frequencies=bf, bath_gammas=bg,
                     bath_couplings=bk)
    else:
        layer = dict(kind="lorentz", z=(z_lb, z_m2), eps_inf=1.0, frequency=1.0, gamma=gamma0,
                     sigma=sigma)
    mats = []
    if mir > 0:
        mats.append(dict(kind="drude", z=(z_m1, z_lb), eps_inf=1.0, frequency=1.0,
                         gamma=drude_gamma, sigma=drude_sigma))
    if lay > 0:
        mats.append(layer)
    if mir2 > 0:
        mats.append(dict(kind="drude", z=(z_m2, z_end), eps_inf=1.0, frequency=1.0,
                         gamma=drude_gamma, sigma=drude_sigma))
    if src_z is None:
        src_z = pml + max(1, vl // 3)
    if mon_z is None:
        mon_z = nz - pml - max(1, vr // 3)
    phase = None
    if phase_seed is not None and nx * ny > 1:
        rng = np.random.default_rng(phase_seed)
        phase = phase_scale * rng.uniform(-1.0, 1.0, size=(ny, nx))
    fwidth = 0.5
    return dict(
        name=name, n=(nx, ny, nz), resolution=float(resolution), courant=float(courant), pml=pml,
        materials=mats,
        sources=[dict(component=source_component, z=src_z, center=1.0, fwidth=fwidth,
                      amplitude=1.0, t0=pulse_t0(fwidth), phase=phase)],
        monitors=[dict(z=mon_z, freqs=np.linspace(0.5, 1.5, nfreq))],
        energy_box=(z_lb, z_m2), steps=int(steps))


# ----------------------------------------------------------------- named workloads
def cavity_1d(steps: int = 20000) -> dict:
    """1D Fabry-Perot, plain method: Nz = 2000 at resolution 100, Courant 0.5, two 20-cell
    Drude mirrors around an 800-cell Lorentz-Bath layer (f0 = 1, gamma0 = 0.01, sigma =
    0.05^2 for a Rabi splitting of 0.05 f0), N_b = 16 bath modes with frequencies from
    default_rng(0) uniform in [0.9, 1.1], bath damping 0.005, Ohmic-like couplings;
    16-cell CPML, pulse centred at 1.0 with width 0.5, 500 DFT frequencies."""
    p = slab_cavity(1, 1, (16, 564, 20, 800, 20, 564), 100.0, num_bath=16, sigma=0.05 ** 2,
                    bath_seed=0, phase_seed=None, src_z=40, mon_z=1960, nfreq=500, steps=steps,
                    name="cavity1d_nz2000_nb16")
    return p


def slab_3d(steps: int = 4000) -> dict:
    """3D slab cavity: 256^3 at resolution 32, periodic x/y, 16-cell CPML in z, 8-cell Drude
    mirrors around a 64-cell (1/4 of z) Lorentz-Bath layer with N_b = 8 (frequencies
    linspace(0.9, 1.1)), sigma = 0.05^2; Ex plane source at z = 24 with a seeded random
    transverse phase; 256 DFT frequencies at z = 232."""
    return slab_cavity(256, 256, (16, 72, 8, 64, 8, 72), 32.0, num_bath=8, sigma=0.05 ** 2,
                       phase_seed=0, src_z=24, mon_z=232, nfreq=256, steps=steps,
                       name="slab3d_256cubed_nb8")


def precision_3d(steps: int = 3000) -> dict:
    """Precision form: 512 x 512 x 384 at resolution 48, N_b = 16, sigma = 0.1^2 (Rabi 0.1)."""
    return slab_cavity(512, 512, (16, 120, 8, 96, 8, 120), 48.0, num_bath=16, sigma=0.1 ** 2,
                       phase_seed=0, src_z=40, mon_z=344, nfreq=256, steps=steps,
                       name="precision3d_512x512x384_nb16")


def precision_crop(steps: int = 1600) -> dict:
    """64^3 crop of the precision form at resolution 8 (layer 16, mirrors 2, CPML 16), N_b = 16,
    sigma = 0.1^2.  The mirrors' plasma strength is sigma_D = 4 (nu_p = 2): the cavity workloads'
    sigma_D = 25 gives w_p dt = 1.96 at this resolution, outside the stability limit
    w_max^2 dt^2 + 4 S^2 dims / eps_inf <= 4.  1600 steps (T = 100) resolve the 0.1 Rabi
    splitting in the monitor spectrum."""
    return slab_cavity(64, 64, (16, 6, 2, 16, 2, 6), 8.0, num_bath=16, sigma=0.1 ** 2,
                       phase_seed=0, src_z=18, mon_z=46, nfreq=256, steps=steps,
                       name="crop64_nb16", drude_sigma=4.0)


def small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=8, steps=60, seed=0) -> dict:
    """Small 3D case with ragged x/y tiles for element-wise parity against the oracle
    (resolution 20 keeps the Drude mirrors inside the coupled stability limit)."""
    return slab_cavity(nx, ny, layout, 20.0, num_bath=nb, sigma=0.05 ** 2, bath_seed=seed,
                       phase_seed=seed, nfreq=16, steps=steps, name=f"small3d_{nx}x{ny}_nb{nb}")


def batch_cavity(L: int, *, rabi: float, num_bath: int, resolution: float = 100.0,
                 pml: int = 16, mirror: int = 20, layer_frac: float = 0.4, steps: int = 50000,
                 name: str = "") -> dict:
    """One cavity of the batching form: L cells = CPML | vacuum | Drude | Lorentz-Bath (40% of L)
    | Drude | vacuum | CPML, the vacuum remainder split evenly; sigma = (Omega_R / f0)^2 for the
    requested Rabi splitting (ideal-cavity relation Omega_R = w0 sqrt(sigma)); bath frequencies
    linspace(0.9, 1.1) with Ohmic-like couplings; the source 24 cells into the left vacuum, the
    energy box = the layer between the mirrors."""
    layer = int(round(layer_frac * L))
    vac = L - 2 * pml - 2 * mirror - layer
    if vac < 4:
        raise ValueError("cavity too short for its layout")
    vl = vac // 2
    vr = vac - vl
    return slab_cavity(1, 1, (pml, vl, mirror, layer, mirror, vr), resolution, num_bath=num_bath,
                       sigma=float(rabi) ** 2, phase_seed=None, src_z=pml + min(24, vl // 2),
                       mon_z=L - pml - min(24, vr // 2), nfreq=8, steps=steps,
                       name=name or f"batch_L{L}_nb{num_bath}_rabi{rabi:.4f}")


def batch_sweep(n: int = 64, steps: int = 50000, len_seed: int = 0, nb_seed: int = 1,
                lmin: int = 1000, lmax: int = 8000, rabi_lo: float = 0.01,
                rabi_hi: float = 0.2) -> list:
    """Batching form: n independent 1D cavities, lengths default_rng(len_seed).integers(lmin,
    lmax + 1), Rabi splittings linspace(rabi_lo, rabi_hi, n) (sigma = Omega_R^2), N_b drawn by
    default_rng(nb_seed).choice([4, 8, 16, 32]); resolution 100, Courant 0.5."""
    lengths = np.random.default_rng(len_seed).integers(lmin, lmax + 1, size=n)
    nbs = np.random.default_rng(nb_seed).choice([4, 8, 16, 32], size=n)
    rabis = np.linspace(rabi_lo, rabi_hi, n)
    return [batch_cavity(int(L), rabi=float(r), num_bath=int(nb), steps=steps)
            for L, r, nb in zip(lengths, rabis, nbs)]


def batch_small(seed: int = 0, steps: int = 600) -> list:
    """A small ragged batch for element-wise parity: lengths 64..700, N_b in {0 (plain Lorentz),
    4, 8, 16, 32}, one cavity with a dielectric (eps_inf = 2.25) spacer, one without an energy
    box."""
    rng = np.random.default_rng(seed)
    out = []
    for i, nb in enumerate((0, 4, 8, 16, 32, 8)):
        L = int(rng.integers(64, 701))
        pml = 8
        mir = 6
        layer = max(8, int(0.35 * L))
        vac = L - 2 * pml - 2 * mir - layer
        vl = vac // 2
        p = slab_cavity(1, 1, (pml, vl, mir, layer, mir, vac - vl), 100.0, num_bath=nb,
                        sigma=float(rng.uniform(1e-4, 0.04)), bath_seed=seed + i,
                        phase_seed=None, src_z=pml + max(1, vl // 2), mon_z=L - pml - 2,
                        nfreq=4, steps=steps, name=f"batch_small_{i}")
        if i == 2:
            z0 = pml + 1
            p["materials"] = [dict(kind="vacuum", z=(z0, z0 + max(2, vl // 3)), eps_inf=2.25)] + p["materials"]
        if i == 5:
            p["energy_box"] = (0, 0)
        out.append(p)
    return out


def adjoint_2d(steps: int = 8000) -> dict:
    """Differentiation form: 2D TE cavity, 2048 x 2048 cells (x periodic, CPML along z),
    resolution 64, out-of-plane E (E_y here, with the in-plane H_x, H_z), z: CPML 16 | vacuum 744
    | Drude 16 | Lorentz-Bath 512 (N_b = 8, sigma = 0.05^2) | Drude 16 | vacuum 728 | CPML 16;
    E_y plane source with the seeded transverse phase; 128 DFT frequencies.  The mirrors take
    sigma_D = 4 (nu_p = 2): with the cavity workloads' sigma_D = 25 a 0.25-unit mirror is ~8 skin
    depths thick and the cavity transmits below 2e-9, which leaves a transmission loss without
    signal; at sigma_D = 4 the transmission peaks near 0.15."""
    return slab_cavity(2048, 1, (16, 744, 16, 512, 16, 728), 64.0, num_bath=8, sigma=0.05 ** 2,
                       phase_seed=0, src_z=16 + 372, mon_z=2048 - 16 - 364, nfreq=128, steps=steps,
                       source_component=1, name="adjoint2d_2048x2048_nb8", drude_sigma=4.0)


def adjoint_crop(steps: int = 2000, nb: int = 8) -> dict:
    """128 x 128 crop of the differentiation form at resolution 16 (32-cell layer, 4-cell
    mirrors with sigma_D = 4), for oracle and finite-difference gradients."""
    return slab_cavity(128, 1, (16, 24, 4, 32, 4, 32), 16.0, num_bath=nb, sigma=0.05 ** 2,
                       phase_seed=0, src_z=28, mon_z=96, nfreq=128, steps=steps,
                       source_component=1, name=f"adjoint_crop128_nb{nb}", drude_sigma=4.0)


def vacuum_of(prob: dict) -> dict:
    """The same problem with every layer removed (the flux normalization run)."""
    q = dict(prob)
    q["materials"] = []
    q["name"] = prob.get("name", "") + "_vacuum"
    return q


def adjoint_target_params(params: np.ndarray, seed: int = 0) -> np.ndarray:
    """Perturbed parameters of the seeded target spectrum: sigma x 1.1, gamma x 0.9,
    coupling_j x (1 + 0.1 N(0, 1)) from default_rng(seed)."""
    p = np.array(params, dtype=np.float64)
    rng = np.random.default_rng(seed)
    p[0] *= 1.1
    p[1] *= 0.9
    p[2:] *= 1.0 + 0.1 * rng.standard_normal(p.size - 2)
    return p


# ----------------------------------------------------------------- random states
def random_sigma_map(prob: dict, seed: int, lo: float = 0.3, hi: float = 1.0) -> np.ndarray:
    """Seeded per-cell oscillator strengths sigma(r): every cell of a Lorentz, Drude or
    Lorentz-Bath layer gets its layer's sigma times a factor drawn uniformly from [lo, hi) by
    default_rng(seed) (factors below 1 keep each layer inside its stability limit); zero elsewhere.
    float64, shape (nz, ny, nx)."""
    nx, ny, nz = prob["n"]
    rng = np.random.default_rng(seed)
    out = np.zeros((nz, ny, nx))
    for m in prob["materials"]:
        if m["kind"] == "vacuum":
            continue
        a, b = m["z"]
        out[a:b] = float(m["sigma"]) * rng.uniform(lo, hi, (b - a, ny, nx))
    return out


def random_state(prob: dict, seed: int, scale: float = 1e-2, with_bath: bool = True) -> dict:
    """Seeded random E, H, P (two levels) and Y (two levels) for every cell of a polarizable
    layer (a vacuum-kind layer, a plain dielectric, has no polarization).

    Returns {("E", c): arr, ("H", c): arr, ("P", c): arr, ("Pm", c): arr,
    ("Y", c, j, level): arr}; material-only quantities are zero outside their
    layers.  Arrays are float64 with shape (nz, ny, nx)."""
    nx, ny, nz = prob["n"]
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    st = {}
    for c in range(3):
        st[("E", c)] = scale * rng.standard_normal(shp)
        st[("H", c)] = scale * rng.standard_normal(shp)
    mask = np.zeros(shp, dtype=bool)
    for m in prob["materials"]:
        if m["kind"] != "vacuum":
            mask[m["z"][0]:m["z"][1]] = True
    for c in range(3):
        st[("P", c)] = np.where(mask, 0.1 * scale * rng.standard_normal(shp), 0.0)
        st[("Pm", c)] = np.where(mask, 0.1 * scale * rng.standard_normal(shp), 0.0)
    if with_bath:
        for m in prob["materials"]:
            if m["kind"] != "lorentz_bath":
                continue
            lo, hi = m["z"]
            for c in range(3):
                for j in range(len(m["bath_frequencies"])):
                    for lvl in (0, 1):
                        a = st.get(("Y", c, j, lvl))
                        if a is None:
                            a = np.zeros(shp)
                            st[("Y", c, j, lvl)] = a
                        a[lo:hi] = 0.1 * scale * rng.standard_normal((hi - lo, ny, nx))
    return st
