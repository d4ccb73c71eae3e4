"""Python binding of the C ABI in ``include/fdtdbath.h`` (argument marshalling only).

The functions below carry the C names without the ``fdtdbath_`` prefix and do
nothing but convert arguments: every step of the method runs in the CUDA
library.  Loading fails loudly when the library is missing or no CUDA device is
present -- there is no CPU fallback.

PyTorch supplies device memory and streams: by default a simulation allocates
through ``torch.cuda.caching_allocator_alloc`` and queues work on the current
torch stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_CFL, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(-1, -8, -1)
KINDS = {"vacuum": 0, "lorentz": 1, "drude": 2, "lorentz_bath": 3}
BATH_SHAPES = {"uniform": 0, "lorentzian": 1, "gaussian": 2}

EXPORTED = ["fdtdbath_create", "fdtdbath_step", "fdtdbath_sync", "fdtdbath_read_fields",
            "fdtdbath_write_fields", "fdtdbath_dft", "fdtdbath_energy", "fdtdbath_steps_done",
            "fdtdbath_last_error", "fdtdbath_destroy", "fdtdbath_bath_form", "fdtdbath_query",
            "fdtdbath_box_energy_noalloc", "fdtdbath_batch_create", "fdtdbath_batch_autotune",
            "fdtdbath_batch_step", "fdtdbath_batch_sync", "fdtdbath_batch_read_field",
            "fdtdbath_batch_energy", "fdtdbath_batch_query", "fdtdbath_batch_last_error",
            "fdtdbath_batch_destroy", "fdtdbath_batch_plan", "fdtdbath_adjoint_forward",
            "fdtdbath_adjoint_backward", "fdtdbath_sigma_box"]


def field_E(c): return 0 + c
def field_H(c): return 3 + c
def field_P(c): return 6 + c
def field_PM(c): return 9 + c
def field_Y(c, j, level): return 1024 + (c * 2 + level) * 256 + j
FIELD_SIGMA = 12   # the per-cell oscillator strength sigma(r)


class Grid(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("pml_cells", C.c_int32)]


class Material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("z_lo", C.c_int64), ("z_hi", C.c_int64),
                ("eps_inf", C.c_double), ("frequency", C.c_double), ("gamma", C.c_double),
                ("sigma", C.c_double), ("num_bath", C.c_int32),
                ("bath_frequencies", C.POINTER(C.c_double)),
                ("bath_gammas", C.POINTER(C.c_double)),
                ("bath_couplings", C.POINTER(C.c_double))]


class Source(C.Structure):
    _fields_ = [("component", C.c_int32), ("z", C.c_int64), ("center", C.c_double),
                ("fwidth", C.c_double), ("amplitude", C.c_double), ("t0", C.c_double),
                ("phase", C.POINTER(C.c_double))]


class Monitor(C.Structure):
    _fields_ = [("z", C.c_int64), ("nfreq", C.c_int32), ("freqs", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("bath_storage", C.c_int32),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("energy_lo", C.c_int64), ("energy_hi", C.c_int64),
                ("energy_capacity", C.c_int64), ("device", C.c_int32)]


class Cavity(C.Structure):
    _fields_ = [("nz", C.c_int64), ("pml_cells", C.c_int32), ("materials", C.POINTER(Material)),
                ("nmat", C.c_int32), ("source", C.POINTER(Source)), ("energy_lo", C.c_int64),
                ("energy_hi", C.c_int64)]


class BatchOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("energy_every", C.c_int32),
                ("energy_capacity", C.c_int64), ("cluster_ctas", C.c_int32),
                ("block_threads", C.c_int32), ("use_graph", C.c_int32), ("device", C.c_int32)]


_lib = None


def lib(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raise if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = C.CDLL(path)
        vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
        L.fdtdbath_create.restype = i32
        L.fdtdbath_create.argtypes = [C.POINTER(Grid), C.c_double, C.c_double,
                                      C.POINTER(Material), i32, C.POINTER(Source), i32,
                                      C.POINTER(Monitor), i32, C.POINTER(Options), C.POINTER(vp)]
        L.fdtdbath_step.restype = i32
        L.fdtdbath_step.argtypes = [vp, i64]
        L.fdtdbath_sync.restype = i32
        L.fdtdbath_sync.argtypes = [vp]
        L.fdtdbath_read_fields.restype = i32
        L.fdtdbath_read_fields.argtypes = [vp, i32, vp, C.c_size_t, i32]
        L.fdtdbath_write_fields.restype = i32
        L.fdtdbath_write_fields.argtypes = [vp, i32, vp, C.c_size_t, i32]
        L.fdtdbath_dft.restype = i32
        L.fdtdbath_dft.argtypes = [vp, i32, dp]
        L.fdtdbath_energy.restype = i32
        L.fdtdbath_energy.argtypes = [vp, dp, i64, C.POINTER(i64)]
        L.fdtdbath_steps_done.restype = i64
        L.fdtdbath_steps_done.argtypes = [vp]
        L.fdtdbath_last_error.restype = C.c_char_p
        L.fdtdbath_last_error.argtypes = [vp]
        L.fdtdbath_destroy.restype = None
        L.fdtdbath_destroy.argtypes = [vp]
        L.fdtdbath_snapshot_size.restype = i32
        L.fdtdbath_snapshot_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.fdtdbath_snapshot.restype = i32
        L.fdtdbath_snapshot.argtypes = [vp, vp, C.c_size_t, i32]
        L.fdtdbath_restore.restype = i32
        L.fdtdbath_restore.argtypes = [vp, vp, C.c_size_t, i32]
        L.fdtdbath_measure_fma_rate.restype = i32
        L.fdtdbath_measure_fma_rate.argtypes = [i32, i32, i32, dp]
        L.fdtdbath_bath_form.restype = i32
        L.fdtdbath_bath_form.argtypes = [i32, C.c_double, C.c_double, i32, C.c_double,
                                         C.c_double, C.c_double, dp, dp, dp]
        L.fdtdbath_query.restype = i64
        L.fdtdbath_query.argtypes = [vp, i32]
        L.fdtdbath_box_energy_noalloc.restype = i32
        L.fdtdbath_box_energy_noalloc.argtypes = [vp, i64, i64, vp, i32]
        L.fdtdbath_adjoint_forward.restype = i32
        L.fdtdbath_adjoint_forward.argtypes = [vp, i64, i32]
        L.fdtdbath_adjoint_backward.restype = i32
        L.fdtdbath_adjoint_backward.argtypes = [vp, i32, dp, i32, dp]
        L.fdtdbath_sigma_box.restype = i32
        L.fdtdbath_sigma_box.argtypes = [vp, dp, dp, C.c_double]
        i32p, i64p = C.POINTER(i32), C.POINTER(i64)
        L.fdtdbath_batch_create.restype = i32
        L.fdtdbath_batch_create.argtypes = [C.POINTER(Cavity), i32, C.c_double, C.c_double,
                                            C.POINTER(BatchOptions), C.POINTER(vp)]
        L.fdtdbath_batch_autotune.restype = i32
        L.fdtdbath_batch_autotune.argtypes = [vp, i32, i32p, i32p, C.POINTER(C.c_float)]
        L.fdtdbath_batch_step.restype = i32
        L.fdtdbath_batch_step.argtypes = [vp, i64]
        L.fdtdbath_batch_sync.restype = i32
        L.fdtdbath_batch_sync.argtypes = [vp]
        L.fdtdbath_batch_read_field.restype = i32
        L.fdtdbath_batch_read_field.argtypes = [vp, i32, i32, vp, C.c_size_t]
        L.fdtdbath_batch_energy.restype = i32
        L.fdtdbath_batch_energy.argtypes = [vp, i32, dp, i64, i64p]
        L.fdtdbath_batch_query.restype = i64
        L.fdtdbath_batch_query.argtypes = [vp, i32]
        L.fdtdbath_batch_last_error.restype = C.c_char_p
        L.fdtdbath_batch_last_error.argtypes = [vp]
        L.fdtdbath_batch_destroy.restype = None
        L.fdtdbath_batch_destroy.argtypes = [vp]
        L.fdtdbath_batch_plan.restype = i32
        L.fdtdbath_batch_plan.argtypes = [C.POINTER(Cavity), i32, C.c_double, C.c_double, i32,
                                          i32, i32, i32, i32, i64p, i32p, i32p, i32p]
        _lib = L
    return _lib


class FdtdBathError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fdtdbath error {code}: {msg}")
        self.code = code


def _check(rc: int, handle=None):
    if rc != OK:
        msg = lib().fdtdbath_last_error(handle)
        raise FdtdBathError(rc, msg.decode() if msg else "")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ------------------------------------------------------------------ C-named wrappers
def measure_fma_rate(precision: int, device: int = 0, reps: int = 5) -> float:
    """fdtdbath_measure_fma_rate: the device's measured FMA throughput in flops per second."""
    out = C.c_double(0.0)
    _check(lib().fdtdbath_measure_fma_rate(int(precision), int(device), int(reps), C.byref(out)))
    return float(out.value)


def bath_form(shape: str, frequency: float, gamma: float, num_bath: int, width: float,
              bath_gamma: float, dephasing: float):
    """Table I expansion (fdtdbath_bath_form): returns (frequencies, gammas, couplings)."""
    f, g, k = (np.empty(num_bath) for _ in range(3))
    _check(lib().fdtdbath_bath_form(BATH_SHAPES[shape], frequency, gamma, num_bath, width,
                                    bath_gamma, dephasing, _dptr(f), _dptr(g), _dptr(k)))
    return f, g, k


class _TorchAllocator:
    """Device allocator callbacks backed by torch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch
        self._torch = torch
        self.device, self.stream = device, stream

        def _alloc(size, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), self.device,
                                                              self.stream or None))
            except Exception:
                return None

        def _free(ptr, _ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def _materials(mats, keep):
    marr = (Material * max(1, len(mats)))()
    for i, m in enumerate(mats):
        nb = len(m.get("bath_frequencies", [])) if m["kind"] == "lorentz_bath" else 0
        arrs = [_f64(m.get(k, np.zeros(1)) if nb else np.zeros(1))
                for k in ("bath_frequencies", "bath_gammas", "bath_couplings")]
        keep += arrs
        marr[i] = Material(KINDS[m["kind"]], int(m["z"][0]), int(m["z"][1]),
                           float(m.get("eps_inf", 1.0)), float(m.get("frequency", 0.0)),
                           float(m.get("gamma", 0.0)), float(m.get("sigma", 0.0)), nb,
                           _dptr(arrs[0]), _dptr(arrs[1]), _dptr(arrs[2]))
    keep.append(marr)
    return marr


def _source(s, keep) -> "Source":
    ph = s.get("phase")
    php = None
    if ph is not None:
        ph = _f64(ph).reshape(-1)
        keep.append(ph)
        php = _dptr(ph)
    return Source(int(s["component"]), int(s["z"]), float(s["center"]), float(s["fwidth"]),
                  float(s.get("amplitude", 1.0)), float(s["t0"]), php)


def create(prob: dict, precision: int = 64, stream=None, use_torch_allocator: bool = True,
           energy: bool = True, energy_capacity: int = 0, device: int = 0, bath_storage: int = 0):
    """fdtdbath_create from a problem dict; returns (handle, keepalive)."""
    L = lib()
    nx, ny, nz = (int(v) for v in prob["n"])
    grid = Grid((C.c_int64 * 3)(nx, ny, nz), int(prob.get("pml", 0)))
    keep = []
    mats = prob.get("materials", [])
    marr = _materials(mats, keep)
    srcs = prob.get("sources", [])
    sarr = (Source * max(1, len(srcs)))()
    for i, src in enumerate(srcs):
        sarr[i] = _source(src, keep)
    mons = prob.get("monitors", [])
    monarr = (Monitor * max(1, len(mons)))()
    for i, mo in enumerate(mons):
        fr = _f64(mo["freqs"])
        keep.append(fr)
        monarr[i] = Monitor(int(mo["z"]), int(fr.size), _dptr(fr))
    opt = Options()
    opt.precision = int(precision)
    opt.bath_storage = int(bath_storage)
    opt.device = int(device)
    sptr = 0
    if stream is not None:
        sptr = int(getattr(stream, "cuda_stream", stream))
    opt.cuda_stream = sptr or None
    if use_torch_allocator:
        alloc = _TorchAllocator(device, sptr)
        keep.append(alloc)
        opt.alloc, opt.free = alloc.alloc, alloc.free
    lo, hi = prob.get("energy_box", (0, 0)) if energy else (0, 0)
    opt.energy_lo, opt.energy_hi = int(lo), int(hi)
    opt.energy_capacity = int(energy_capacity or max(1, int(prob.get("steps", 1024))) + 16)
    h = C.c_void_p()
    rc = L.fdtdbath_create(C.byref(grid), float(prob["resolution"]), float(prob["courant"]),
                           marr, len(mats), sarr, len(srcs), monarr, len(mons), C.byref(opt),
                           C.byref(h))
    _check(rc, None)
    return h, keep


def step(h, n: int):
    _check(lib().fdtdbath_step(h, int(n)), h)


def sync(h):
    _check(lib().fdtdbath_sync(h), h)


def read_fields(h, field: int, shape, dtype) -> np.ndarray:
    out = np.empty(shape, dtype=dtype)
    _check(lib().fdtdbath_read_fields(h, int(field), out.ctypes.data, out.nbytes, 0), h)
    return out


def write_fields(h, field: int, arr: np.ndarray):
    a = np.ascontiguousarray(arr)
    _check(lib().fdtdbath_write_fields(h, int(field), a.ctypes.data, a.nbytes, 0), h)


def dft(h, monitor: int, nfreq: int) -> np.ndarray:
    out = np.empty((nfreq, 8), dtype=np.float64)
    _check(lib().fdtdbath_dft(h, int(monitor), _dptr(out)), h)
    return out[:, 0::2] + 1j * out[:, 1::2]


def energy(h, maxlen: int) -> np.ndarray:
    out = np.empty((max(1, maxlen), 4), dtype=np.float64)
    n = C.c_int64(0)
    _check(lib().fdtdbath_energy(h, _dptr(out), int(maxlen), C.byref(n)), h)
    return out[:n.value].copy()


def steps_done(h) -> int:
    return int(lib().fdtdbath_steps_done(h))


def query(h, key: int) -> int:
    return int(lib().fdtdbath_query(h, int(key)))


def destroy(h):
    lib().fdtdbath_destroy(h)


def box_energy_noalloc(h, z_lo: int, z_hi: int, out_ptr: int | None = None) -> np.ndarray | None:
    """fdtdbath_box_energy_noalloc: (U_EM, U_P, U_bath) of planes [z_lo, z_hi) of the current
    state, computed by the library without allocating memory.  With out_ptr (a device address
    of 3 doubles) the result stays on the device and None is returned."""
    if out_ptr is not None:
        _check(lib().fdtdbath_box_energy_noalloc(h, int(z_lo), int(z_hi), int(out_ptr), 1), h)
        return None
    out = np.zeros(3, dtype=np.float64)
    _check(lib().fdtdbath_box_energy_noalloc(h, int(z_lo), int(z_hi), out.ctypes.data, 0), h)
    return out


# ------------------------------------------------------------------ convenience class
class Simulation:
    """A simulation built from a problem dict (see ``workloads``), owning its handle."""

    def __init__(self, prob: dict, precision: int = 64, stream=None, energy: bool = True,
                 use_torch_allocator: bool = True, energy_capacity: int = 0,
                 bath_storage: int = 0):
        self.prob = prob
        self.precision = precision
        nx, ny, nz = (int(v) for v in prob["n"])
        self.shape = (nz, ny, nx)
        self.dtype = np.float64 if precision == 64 else np.float32
        self.nfreq = [len(m["freqs"]) for m in prob.get("monitors", [])]
        self.h, self._keep = create(prob, precision, stream=stream, energy=energy,
                                    use_torch_allocator=use_torch_allocator,
                                    energy_capacity=energy_capacity, bath_storage=bath_storage)

    def step(self, n: int):
        step(self.h, n)

    def sync(self):
        sync(self.h)

    @property
    def steps_done(self) -> int:
        return steps_done(self.h)

    @staticmethod
    def _field(name: str, comp: int, mode: int, level: int) -> int:
        if name == "S":   # sigma(r)
            return FIELD_SIGMA
        fid = {"E": field_E, "H": field_H, "P": field_P, "Pm": field_PM}.get(name)
        if fid:
            return fid(comp)
        if name != "Y":
            raise KeyError(name)
        return field_Y(comp, mode, level)

    def get(self, name: str, comp: int = 0, mode: int = 0, level: int = 0) -> np.ndarray:
        """Read a field: E, H, P, Pm, Y (bath mode `mode` at `level`) or S (sigma(r))."""
        return read_fields(self.h, self._field(name, comp, mode, level), self.shape, self.dtype)

    def set(self, name: str, arr, comp: int = 0, mode: int = 0, level: int = 0):
        """Overwrite a field (names as for get)."""
        write_fields(self.h, self._field(name, comp, mode, level),
                     np.asarray(arr, dtype=self.dtype).reshape(self.shape))

    def sigma_box(self, lo, hi, sigma: float):
        """fdtdbath_sigma_box: paint a box [lo, hi) (x, y, z in cell units) of oscillator strength
        sigma into the sigma(r) map, each cell weighted by the fraction the box covers."""
        lo_a = np.ascontiguousarray(lo, dtype=np.float64)
        hi_a = np.ascontiguousarray(hi, dtype=np.float64)
        _check(lib().fdtdbath_sigma_box(self.h, _dptr(lo_a), _dptr(hi_a), float(sigma)), self.h)

    def sigma_map(self) -> bool:
        """Whether a per-cell sigma(r) map is set (query key 11)."""
        return query(self.h, 11) == 1

    def dft(self, mon: int = 0) -> np.ndarray:
        return dft(self.h, mon, self.nfreq[mon])

    def trace(self, maxlen: int | None = None) -> np.ndarray:
        return energy(self.h, maxlen or self.steps_done + 1)

    def launches(self) -> int:
        return query(self.h, 1)

    def te_form(self) -> bool:
        """Whether the step kernel runs the y-invariant TE form (query key 5)."""
        return query(self.h, 5) == 1

    def adjoint_te_form(self) -> bool:
        """Whether the last reverse sweep ran the TE form (query key 6)."""
        return query(self.h, 6) == 1

    def snapshot(self) -> np.ndarray:
        """fdtdbath_snapshot into host memory: the whole state as an opaque byte array."""
        n = C.c_size_t(0)
        _check(lib().fdtdbath_snapshot_size(self.h, C.byref(n)), self.h)
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().fdtdbath_snapshot(self.h, buf.ctypes.data, buf.nbytes, 0), self.h)
        return buf

    def restore(self, buf: np.ndarray):
        """fdtdbath_restore from a host snapshot taken by snapshot()."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().fdtdbath_restore(self.h, buf.ctypes.data, buf.nbytes, 0), self.h)

    def cavity_1d_kernel(self) -> bool:
        """Whether the steps run on the persistent 1D cavity kernel (query key 8)."""
        return query(self.h, 8) == 1

    def plain_kernel(self) -> bool:
        """Whether the z-chunks without bath modes run the plain-plane kernel (query key 7)."""
        return query(self.h, 7) == 1

    def te2d_kernel(self) -> bool:
        """Whether the TE form's bath-free chunks run the register-streaming kernel (query key 10)."""
        return query(self.h, 10) == 1

    def tb2_kernel(self) -> bool:
        """Whether pairs of steps run in one launch of the two-steps-per-pass kernel (query key 12:
        grids without polarizable material tiled exactly by 32 x 8 tiles)."""
        return query(self.h, 12) == 1

    def bath_plain_kernel(self) -> bool:
        """Whether the z-chunks with bath modes run the plain-plane kernel's Lorentz-Bath form
        (query key 9)."""
        return query(self.h, 9) == 1

    def adjoint_forward(self, nsteps: int, checkpoint_every: int = 256):
        """fdtdbath_adjoint_forward: advance nsteps steps keeping checkpoints for the adjoint."""
        _check(lib().fdtdbath_adjoint_forward(self.h, int(nsteps), int(checkpoint_every)), self.h)

    def adjoint_backward(self, dL_dF, material: int, monitor: int = 0) -> np.ndarray:
        """fdtdbath_adjoint_backward: dL_dF (nfreq, 4, 2) = dL/d(Re, Im) of the monitor spectra
        (Ex, Ey, Hx, Hy); returns dL/d(sigma, gamma, coupling_1..N_b) of layer `material`."""
        g = _f64(dL_dF).reshape(-1)
        nb = len(self.prob["materials"][material].get("bath_frequencies", [])) \
            if self.prob["materials"][material]["kind"] == "lorentz_bath" else 0
        out = np.zeros(2 + nb)
        _check(lib().fdtdbath_adjoint_backward(self.h, int(monitor), _dptr(g), int(material), _dptr(out)), self.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched 1D cavities
def _bcheck(rc: int, handle=None):
    if rc < 0:
        msg = lib().fdtdbath_batch_last_error(handle)
        raise FdtdBathError(rc, msg.decode() if msg else "")


def _cavities(probs, energy: bool, keep):
    """Cavity array from 1D problem dicts (n = (1, 1, nz)) sharing resolution and Courant."""
    res, cour = float(probs[0]["resolution"]), float(probs[0]["courant"])
    cav = (Cavity * len(probs))()
    for i, p in enumerate(probs):
        if tuple(int(v) for v in p["n"][:2]) != (1, 1):
            raise ValueError("batched cavities are 1D: n = (1, 1, nz)")
        if float(p["resolution"]) != res or float(p["courant"]) != cour:
            raise ValueError("the cavities of a batch share resolution and Courant number")
        marr = _materials(p.get("materials", []), keep)
        srcs = p.get("sources", [])
        if len(srcs) > 1:
            raise ValueError("a batched cavity takes at most one source")
        sp = None
        if srcs:
            src = (Source * 1)(_source(srcs[0], keep))
            keep.append(src)
            sp = C.cast(src, C.POINTER(Source))
        lo, hi = p.get("energy_box", (0, 0)) if energy else (0, 0)
        cav[i] = Cavity(int(p["n"][2]), int(p.get("pml", 0)), C.cast(marr, C.POINTER(Material)),
                        len(p.get("materials", [])), sp, int(lo), int(hi))
    keep.append(cav)
    return cav, res, cour


def batch_plan(probs, precision: int, cluster_ctas: int, nclusters: int, smem_per_cta: int,
               block_threads: int = 1):
    """fdtdbath_batch_plan (host only): per-CTA work / cells / shared-memory bytes and the
    cluster of every cavity, balanced for CTAs of block_threads threads."""
    keep = []
    cav, res, cour = _cavities(probs, True, keep)
    nmax = cluster_ctas * nclusters
    work = np.zeros(nmax, np.int64)
    cells = np.zeros(nmax, np.int32)
    smem = np.zeros(nmax, np.int32)
    clus = np.zeros(len(probs), np.int32)
    rc = lib(build_if_missing=True).fdtdbath_batch_plan(
        cav, len(probs), res, cour, int(precision), int(cluster_ctas), int(block_threads),
        int(nclusters), int(smem_per_cta), work.ctypes.data_as(C.POINTER(C.c_int64)),
        cells.ctypes.data_as(C.POINTER(C.c_int32)), smem.ctypes.data_as(C.POINTER(C.c_int32)),
        clus.ctypes.data_as(C.POINTER(C.c_int32)))
    _bcheck(rc, None)
    return {"work": work[:rc], "cells": cells[:rc], "smem": smem[:rc], "cluster": clus}


class Batch:
    """Batched 1D cavities (fdtdbath_batch_*): one persistent launch per chunk of steps."""

    def __init__(self, probs, precision: int = 32, stream=None, energy: bool = True,
                 energy_every: int = 1, energy_capacity: int = 0, cluster_ctas: int = 0,
                 block_threads: int = 0, use_graph: bool = True, use_torch_allocator: bool = True,
                 device: int = 0):
        L = lib()
        self.probs = list(probs)
        self.precision = precision
        self.dtype = np.float64 if precision == 64 else np.float32
        self.every = max(1, int(energy_every))
        self._keep = []
        cav, res, cour = _cavities(self.probs, energy, self._keep)
        opt = BatchOptions()
        opt.precision = int(precision)
        opt.device = int(device)
        sptr = 0
        if stream is not None:
            sptr = int(getattr(stream, "cuda_stream", stream))
        opt.cuda_stream = sptr or None
        if use_torch_allocator:
            alloc = _TorchAllocator(device, sptr)
            self._keep.append(alloc)
            opt.alloc, opt.free = alloc.alloc, alloc.free
        opt.energy_every = self.every
        steps = max(int(p.get("steps", 1024)) for p in self.probs)
        opt.energy_capacity = int(energy_capacity or steps // self.every + 16)
        opt.cluster_ctas = int(cluster_ctas)
        opt.block_threads = int(block_threads)
        opt.use_graph = int(bool(use_graph))
        h = C.c_void_p()
        _bcheck(L.fdtdbath_batch_create(cav, len(self.probs), res, cour, C.byref(opt), C.byref(h)))
        self.h = h

    def autotune(self, probe_steps: int = 64):
        c, t, ms = C.c_int32(0), C.c_int32(0), C.c_float(0)
        _bcheck(lib().fdtdbath_batch_autotune(self.h, int(probe_steps), C.byref(c), C.byref(t),
                                              C.byref(ms)), self.h)
        return c.value, t.value, ms.value

    def step(self, n: int):
        _bcheck(lib().fdtdbath_batch_step(self.h, int(n)), self.h)

    def sync(self):
        _bcheck(lib().fdtdbath_batch_sync(self.h), self.h)

    def get(self, cavity: int, name: str, mode: int = 0, level: int = 0) -> np.ndarray:
        f = {"E": field_E(0), "H": field_H(1), "P": field_P(0), "Pm": field_PM(0)}.get(name)
        if f is None:
            f = field_Y(0, mode, level)
        out = np.empty(int(self.probs[cavity]["n"][2]), dtype=self.dtype)
        _bcheck(lib().fdtdbath_batch_read_field(self.h, int(cavity), int(f), out.ctypes.data,
                                                out.nbytes), self.h)
        return out

    def trace(self, cavity: int, maxlen: int | None = None) -> np.ndarray:
        maxlen = maxlen or self.query(7) // self.every + 2
        out = np.empty((max(1, maxlen), 4), dtype=np.float64)
        n = C.c_int64(0)
        _bcheck(lib().fdtdbath_batch_energy(self.h, int(cavity), _dptr(out), int(maxlen),
                                            C.byref(n)), self.h)
        return out[:n.value].copy()

    def query(self, key: int) -> int:
        return int(lib().fdtdbath_batch_query(self.h, int(key)))

    def shape(self) -> dict:
        return {"clusters": self.query(1), "ctas": self.query(2), "cluster_ctas": self.query(3),
                "threads": self.query(4), "smem": self.query(8)}

    def close(self):
        if getattr(self, "h", None):
            lib().fdtdbath_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
