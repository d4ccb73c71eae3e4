"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

The time stepping lives in ``fdtd_oracle.c``; this module only marshals a
problem description (the plain dict the seeded workload generators produce)
into it and reads state back as numpy arrays.  Only tests, the smoke check and
the benchmark's CPU-baseline leg and reference arm import it.

Field ids follow the C file: 0..2 E, 3..5 H, 6..8 D, 9..11 P^{n+1/2},
12..14 P^{n-1/2}; bath mode j of component c at level l (0: Y^{n+1/2},
1: Y^{n-1/2}) is ``64 + (2c + l) * 128 + j``; 32..33 / 34..35 are the CPML
memories of the E / H updates; 16 is the per-cell oscillator strength sigma(r).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

KINDS = {"vacuum": 0, "lorentz": 1, "drude": 2, "lorentz_bath": 3}
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
        dp = C.POINTER(C.c_double)
        L.orc_new.restype = vp
        L.orc_new.argtypes = [i64, i64, i64, d, d, i32]
        L.orc_add_material.restype = i32
        L.orc_add_material.argtypes = [vp, i32, i64, i64, d, d, d, d, i32, dp, dp, dp]
        L.orc_add_source.restype = i32
        L.orc_add_source.argtypes = [vp, i32, i64, d, d, d, d, dp]
        L.orc_add_monitor.restype = i32
        L.orc_add_monitor.argtypes = [vp, i64, i32, dp]
        L.orc_set_energy_box.restype = None
        L.orc_set_energy_box.argtypes = [vp, i64, i64, i64, i32]
        L.orc_step.restype = None
        L.orc_step.argtypes = [vp, i64]
        L.orc_get_field.restype = i32
        L.orc_get_field.argtypes = [vp, i32, dp]
        L.orc_set_field.restype = i32
        L.orc_set_field.argtypes = [vp, i32, dp]
        L.orc_get_dft.restype = i32
        L.orc_get_dft.argtypes = [vp, i32, dp]
        L.orc_get_trace.restype = i64
        L.orc_get_trace.argtypes = [vp, dp, i64]
        L.orc_steps_done.restype = i64
        L.orc_steps_done.argtypes = [vp]
        L.orc_dt.restype = d
        L.orc_dt.argtypes = [vp]
        L.orc_free.restype = None
        L.orc_free.argtypes = [vp]
        for name in ("orc_lorentz_update", "orc_drude_update"):
            f = getattr(L, name)
            f.restype = d
            f.argtypes = [d, d, d, d, d, d, d]
        L.orc_lorentz_bath_update.restype = d
        L.orc_lorentz_bath_update.argtypes = [d, d, d, d, d, d, i32, dp, dp, dp, dp, dp, d]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def field_id(name: str, comp: int = 0, mode: int = 0, level: int = 0) -> int:
    base = {"E": 0, "H": 3, "D": 6, "P": 9, "Pm": 12}
    if name in base:
        return base[name] + comp
    if name == "Y":
        return 64 + (2 * comp + level) * 128 + mode
    if name == "psiE":
        return 32 + comp
    if name == "psiH":
        return 34 + comp
    if name == "S":   # sigma(r), the per-cell oscillator strength
        return 16
    raise KeyError(name)


class OracleSim:
    """FP64 oracle simulation built from a problem dict (see the workload generators)."""

    def __init__(self, prob: dict, trace_cap: int = 0, record_invariant: bool = False):
        L = lib()
        nx, ny, nz = (int(v) for v in prob["n"])
        self.shape = (nz, ny, nx)
        self.prob = prob
        self._h = L.orc_new(nx, ny, nz, float(prob["resolution"]), float(prob["courant"]),
                            int(prob.get("pml", 0)))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self._keep = []
        for m in prob.get("materials", []):
            nb = int(len(m.get("bath_frequencies", []))) if m["kind"] == "lorentz_bath" else 0
            bf = _f64(m.get("bath_frequencies", np.zeros(1)) if nb else np.zeros(1))
            bg = _f64(m.get("bath_gammas", np.zeros(1)) if nb else np.zeros(1))
            bk = _f64(m.get("bath_couplings", np.zeros(1)) if nb else np.zeros(1))
            rc = L.orc_add_material(self._h, KINDS[m["kind"]], int(m["z"][0]), int(m["z"][1]),
                                    float(m.get("eps_inf", 1.0)), float(m.get("frequency", 0.0)),
                                    float(m.get("gamma", 0.0)), float(m.get("sigma", 0.0)), nb,
                                    _dp(bf), _dp(bg), _dp(bk))
            if rc:
                raise ValueError(f"oracle rejected material {m['kind']} z={m['z']} (rc={rc})")
        for s in prob.get("sources", []):
            ph = s.get("phase")
            php = None
            if ph is not None:
                ph = _f64(ph).reshape(-1)
                if ph.size != nx * ny:
                    raise ValueError("phase must hold nx*ny values")
                self._keep.append(ph)
                php = _dp(ph)
            rc = L.orc_add_source(self._h, int(s["component"]), int(s["z"]), float(s["center"]),
                                  float(s["fwidth"]), float(s.get("amplitude", 1.0)),
                                  float(s["t0"]), php)
            if rc:
                raise ValueError("oracle rejected source")
        self.nfreq = []
        for mon in prob.get("monitors", []):
            fr = _f64(mon["freqs"])
            rc = L.orc_add_monitor(self._h, int(mon["z"]), int(fr.size), _dp(fr))
            if rc:
                raise ValueError("oracle rejected monitor")
            self.nfreq.append(int(fr.size))
        self.trace_cap = int(trace_cap)
        if trace_cap:
            lo, hi = prob.get("energy_box", (0, nz))
            L.orc_set_energy_box(self._h, int(lo), int(hi), int(trace_cap), int(record_invariant))

    # -- stepping and state ---------------------------------------------------------
    def step(self, n: int) -> None:
        lib().orc_step(self._h, int(n))

    @property
    def steps_done(self) -> int:
        return int(lib().orc_steps_done(self._h))

    @property
    def dt(self) -> float:
        return float(lib().orc_dt(self._h))

    def get(self, name: str, comp: int = 0, mode: int = 0, level: int = 0) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        rc = lib().orc_get_field(self._h, field_id(name, comp, mode, level), _dp(out))
        if rc:
            raise KeyError(name)
        return out

    def set(self, name: str, arr, comp: int = 0, mode: int = 0, level: int = 0) -> None:
        a = _f64(arr).reshape(self.shape)
        rc = lib().orc_set_field(self._h, field_id(name, comp, mode, level), _dp(a))
        if rc:
            raise KeyError(name)

    def dft(self, mon: int = 0) -> np.ndarray:
        """Complex plane-mean spectra, shape (nfreq, 4) for (Ex, Ey, Hx, Hy)."""
        out = np.empty((self.nfreq[mon], 8), dtype=np.float64)
        if lib().orc_get_dft(self._h, int(mon), _dp(out)):
            raise IndexError(mon)
        return out[:, 0::2] + 1j * out[:, 1::2]

    def trace(self) -> np.ndarray:
        """Energy traces per step, shape (steps, 4): U_EM, U_P, U_bath, discrete invariant."""
        out = np.empty((max(self.trace_cap, 1), 4), dtype=np.float64)
        n = lib().orc_get_trace(self._h, _dp(out), self.trace_cap)
        return out[:n].copy()

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flux(spec: np.ndarray) -> np.ndarray:
    """Normal flux through the monitor plane, Re(Ex Hy* - Ey Hx*) (z-directed Poynting vector)."""
    return np.real(spec[:, 0] * np.conj(spec[:, 3]) - spec[:, 1] * np.conj(spec[:, 2]))


# -- single-cell ADE updates (for the discrete-susceptibility pin) ------------------
def lorentz_update(E, P, Pm, w0, g, sigma, dt):
    return lib().orc_lorentz_update(E, P, Pm, w0, g, sigma, dt)


def drude_update(E, P, Pm, w0, g, sigma, dt):
    return lib().orc_drude_update(E, P, Pm, w0, g, sigma, dt)


def lorentz_bath_update(E, P, Pm, w0, g0, sigma, wj, gj, kj, Y, Ym, dt):
    """One Eq. (Pz_update-LB) + Eq. (Yzj_finite_difference) step; Y, Ym updated in place."""
    wj, gj, kj = _f64(wj), _f64(gj), _f64(kj)
    return lib().orc_lorentz_bath_update(E, P, Pm, w0, g0, sigma, int(wj.size), _dp(wj), _dp(gj),
                                         _dp(kj), _dp(Y), _dp(Ym), dt)


def two_pi() -> float:
    return 2.0 * math.pi


# -- per-cell sigma(r) with sub-pixel averaging --------------------------------------
def box_fill(shape, lo, hi) -> np.ndarray:
    """Fraction of each cell covered by the box [lo, hi) (cell units, x, y, z order).

    Cell (i, j, k) is the unit cube [i, i+1) x [j, j+1) x [k, k+1); its covered fraction is the
    product over the axes of the overlap length max(0, min(hi, i+1) - max(lo, i)).  Returned as a
    [nz][ny][nx] array (``shape`` = (nz, ny, nx)).
    """
    out = np.ones(shape)
    for ax, n in zip((2, 1, 0), shape[::-1]):   # x, y, z
        a, b = float(lo[2 - ax]), float(hi[2 - ax])
        i = np.arange(n, dtype=np.float64)
        f = np.clip(np.minimum(b, i + 1.0) - np.maximum(a, i), 0.0, 1.0)
        sh = [1, 1, 1]
        sh[ax] = n
        out = out * f.reshape(sh)
    return out


def paint_sigma(sim: "OracleSim", lo, hi, sigma: float) -> None:
    """sigma(r) <- f sigma + (1 - f) sigma_old in every cell of the dispersive layers that the box
    covers by the fraction f (the cell average of the coupling strength: the susceptibility of
    Eq. chi_L is linear in sigma)."""
    old = sim.get("S")
    f = box_fill(sim.shape, lo, hi)
    sim.set("S", f * float(sigma) + (1.0 - f) * old)
