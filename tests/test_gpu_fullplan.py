"""The 512 x 512 x 384 precision workload (N_b = 16) through its full-size launch plan -- the
plain-plane kernel's bath-free form over the vacuum / CPML / mirror chunks and its two-threads-
per-cell Lorentz-Bath form over the 96-plane layer -- compared with the FP64 oracle cell by cell
on sampled windows, FP32 and bf16 bath storage.

Two steps from a seeded random state move information at most a few cells in x and y (each
half-step reads the nearest neighbours; reading H back adds the pending H half-step), so the
state of a window's centre after two steps depends only on the window's initial state and its
source columns.  The GPU grid holds random values inside two 28 x 28-column windows (all z; one
window wraps around the periodic x / y edges) and zeros elsewhere; the oracle runs each window as
its own 28 x 28 x 384 periodic grid from the same values (for bf16 storage, from the bath modes
as the GPU stored them) and the central 16 x 16 columns are compared: every field component over
all z, P and P^{n-1/2} and three bath modes (both levels) over the layer.  Tolerances are the
parity tests' (FP32 1e-5 for fields, 1e-4 for P and modes; bf16 storage 1e-3, and 2^-8 for the
modes themselves, which it returns rounded to bf16).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl
from test_gpu_parity import rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W, MARGIN = 28, 6
WINDOWS = [(100, 37), (496, 500)]   # (x0, y0); the second wraps around both edges


def window_index(n, o):
    return (o + np.arange(W)) % n


def window_values(prob, win, seed):
    """Random state of one window: {key: (nz, W, W) array}, FP64, zero where a quantity does
    not exist (P outside polarizable layers, modes outside the Lorentz-Bath layer)."""
    sub = dict(prob, n=(W, W, prob["n"][2]))
    return wl.random_state(sub, seed=seed)


def crop_problem(prob, win):
    """The window as a periodic W x W x nz grid: same layers, CPML, source (its phase table
    cropped), monitor and energy box."""
    nx, ny, _ = prob["n"]
    xi, yi = window_index(nx, win[0]), window_index(ny, win[1])
    srcs = []
    for s in prob["sources"]:
        ph = s.get("phase")
        srcs.append(dict(s, phase=None if ph is None else ph[np.ix_(yi, xi)]))
    return dict(prob, n=(W, W, prob["n"][2]), sources=srcs, name=prob["name"] + "_window")


@pytest.mark.parametrize("bath_storage", [0, 1])
def test_precision_workload_full_plan_matches_oracle_on_windows(bath_storage):
    prob = wl.precision_3d(steps=2)
    nx, ny, nz = prob["n"]
    g = fb.Simulation(prob, precision=32, bath_storage=bath_storage, energy_capacity=8)
    assert g.plain_kernel() and g.bath_plain_kernel()
    lb = [m for m in prob["materials"] if m["kind"] == "lorentz_bath"][0]
    nb = len(lb["bath_frequencies"])
    lo, hi = lb["z"]
    states = [window_values(prob, w, seed=20 + i) for i, w in enumerate(WINDOWS)]
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    states = [{k: f32(v) for k, v in st.items()} for st in states]
    # the GPU state: zeros outside the windows, one full array at a time
    for key in states[0]:
        full = np.zeros((nz, ny, nx), dtype=np.float32)
        for st, win in zip(states, WINDOWS):
            full[np.ix_(np.arange(nz), window_index(ny, win[1]), window_index(nx, win[0]))] = st[key]
        if key[0] == "Y":
            g.set("Y", full, comp=key[1], mode=key[2], level=key[3])
        else:
            g.set(key[0], full, comp=key[1])
        del full
    if bath_storage:
        # the modes as stored (bf16 pairs): the oracle starts from what the GPU holds
        for key in states[0]:
            if key[0] != "Y":
                continue
            back = g.get("Y", comp=key[1], mode=key[2], level=key[3])
            for st, win in zip(states, WINDOWS):
                st[key] = back[np.ix_(np.arange(nz), window_index(ny, win[1]),
                                      window_index(nx, win[0]))].astype(np.float64)
            del back
    g.step(2)
    c = slice(MARGIN, W - MARGIN)
    sel_modes = sorted({0, nb // 2, nb - 1})
    got = {}
    for name in ("E", "H", "P", "Pm"):
        for comp in range(3):
            a = g.get(name, comp=comp)
            got[(name, comp)] = [a[np.ix_(np.arange(nz), window_index(ny, w[1]), window_index(nx, w[0]))]
                                 for w in WINDOWS]
            del a
    for j in sel_modes:
        for lvl in (0, 1):
            for comp in range(3):
                a = g.get("Y", comp=comp, mode=j, level=lvl)
                got[("Y", comp, j, lvl)] = [a[np.ix_(np.arange(nz), window_index(ny, w[1]),
                                                     window_index(nx, w[0]))] for w in WINDOWS]
                del a
    g.close()
    tol_f = 1e-5 if bath_storage == 0 else 1e-3
    tol_m = 1e-4 if bath_storage == 0 else 1e-3
    # bf16 storage returns each mode rounded to bf16 (2^-9 relative): their bound is 2^-8
    tol_y = tol_m if bath_storage == 0 else 2.0 ** -8
    eps = np.ones((nz, W, W))
    for m in prob["materials"]:
        eps[m["z"][0]:m["z"][1]] = m.get("eps_inf", 1.0)
    for wi, (win, st) in enumerate(zip(WINDOWS, states)):
        sub = crop_problem(prob, win)
        o = O.OracleSim(sub)
        for key, arr in st.items():
            if key[0] == "Y":
                o.set("Y", arr, comp=key[1], mode=key[2], level=key[3])
            else:
                o.set(key[0], arr, comp=key[1])
        for comp in range(3):
            o.set("D", eps * st[("E", comp)] + st[("Pm", comp)], comp=comp)
        o.step(2)
        for name in ("E", "H"):
            for comp in range(3):
                want = o.get(name, comp=comp)[:, c, c]
                assert np.max(np.abs(want)) > 0, (name, comp)
                assert rel(got[(name, comp)][wi][:, c, c], want) < tol_f, (wi, name, comp)
        for name in ("P", "Pm"):
            for comp in range(3):
                want = o.get(name, comp=comp)[lo:hi, c, c]
                assert rel(got[(name, comp)][wi][lo:hi, c, c], want) < tol_m, (wi, name, comp)
        for j in sel_modes:
            for lvl in (0, 1):
                for comp in range(3):
                    want = o.get("Y", comp=comp, mode=j, level=lvl)[lo:hi, c, c]
                    assert rel(got[("Y", comp, j, lvl)][wi][lo:hi, c, c], want) < tol_y, (wi, j, lvl, comp)
