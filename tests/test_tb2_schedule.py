"""Host check of the two-steps-per-pass schedule (tb2.cuh, temporal blocking) without a GPU.

A plain-Python model of one CTA's march follows the kernel's schedule step for step: the 32 x 8
tile, the shared-memory frames (origin (x0-4, y0-2), 40 columns; E^{n-1/2} frames 12 rows, every
other array 11), the staging rings (E^{n-1/2} 3 planes, H^{n-1} 2, one plane ahead, a slot being
refilled unreadable until the next plane), the rings of H^n and its CPML memories (3) and of
E^{n+1/2} (2), the halo boxes and their halo-cell enumeration, the ghost planes at the chunk
ends, the two phases per plane ({H^n(k), H^{n+1}(k-2)}, then {E^{n+1/2}(k), E^{n+3/2}(k-2)}) and
the own-cell values carried between planes.  Every frame entry that has not been staged or
computed is NaN, so a read of one shows up in the outputs.  The model's result for all CTAs of
a chunk plan is compared with two single fused steps of the same update (Eq. 1a / Eq. 1b in the
3D curl form, CPML memories on the z terms, a phased soft plane source) evaluated directly on the
whole grid, and must agree exactly; the monitor / energy bookkeeping must visit every plane of the
grid exactly once per step.  Chunk plans include one-plane chunks, chunk starts whose ghost planes
lie inside the absorber and a top ghost plane inside it.
"""
import numpy as np
import pytest

TX, TY = 32, 8                    # tile (kTbTX, kTbTY)
FX, FY = TX + 8, TY + 4           # frame columns, rows of the E^{n-1/2} frames
FH = FY - 1                       # rows of every other frame
RE, RH, RH1, RE1 = 3, 2, 3, 2     # rings: E^{n-1/2}, H^{n-1}, H^n (+ memories), E^{n+1/2}
H1B = (2, TX + 5, 0, TY + 3)      # boxes as (first column, end column, first row, end row)
E1B = (3, TX + 5, 1, TY + 3)
H2B = (3, TX + 4, 1, TY + 2)
OWN = [(ty + 2, tx + 4) for ty in range(TY) for tx in range(TX)]
OWN_SET = set(OWN)


def halo_cell(t, c0, c1, r0, r1):
    """Halo cell t of a box: its rows above the tile, then below, then the side columns."""
    w = c1 - c0
    ntop = (2 - r0) * w
    if t < ntop:
        return (r0 + t // w, c0 + t % w)
    t -= ntop
    nbot = (r1 - (2 + TY)) * w
    if t < nbot:
        return (2 + TY + t // w, c0 + t % w)
    t -= nbot
    nl, nr = 4 - c0, c1 - (4 + TX)
    r = t % (nl + nr)
    return (2 + t // (nl + nr), c0 + r if r < nl else 4 + TX + (r - nl))


def box_cells(box):
    """Own cells then halo cells of a box; each cell of the box exactly once."""
    c0, c1, r0, r1 = box
    halo = [halo_cell(t, *box) for t in range((c1 - c0) * (r1 - r0) - TX * TY)]
    cells = OWN + halo
    assert len(set(cells)) == len(cells)
    assert set(cells) == {(r, c) for r in range(r0, r1) for c in range(c0, c1)}
    return cells


def psi_e_plane(k, nz, npml):
    if k < npml:
        return k
    if k >= nz - npml:
        return npml + (k - (nz - npml))
    return -1


def psi_h_plane(k, nz, npml):
    if npml <= 0:
        return -1
    if k < npml:
        return k
    if k >= nz - npml - 1:
        return npml + (k - (nz - npml - 1))
    return -1


class Grid:
    """A random state: E, H, both CPML memories and their coefficients, a phased source on E_y."""

    def __init__(self, nx, ny, nz, npml, seed=1):
        r = np.random.default_rng(seed)
        self.nx, self.ny, self.nz, self.npml = nx, ny, nz, npml
        self.S, self.dt = 0.5, 0.5 / 16
        self.E = r.standard_normal((3, nz, ny, nx))
        self.H = r.standard_normal((3, nz, ny, nx))
        self.psiE = r.standard_normal((2, 2 * npml, ny, nx))
        self.psiH = r.standard_normal((2, 2 * npml + 1, ny, nx))
        self.pmlE = r.uniform(0.5, 1.0, (nz, 2))
        self.pmlH = r.uniform(0.5, 1.0, (nz, 2))
        self.srcz, self.srcc = min(7, nz - 2), 1
        self.cos, self.sin = r.standard_normal((ny, nx)), r.standard_normal((ny, nx))
        self.amp = [(0.3, 0.7), (-0.2, 0.4)]   # (a, b) of the two steps


def fused_step(g, E, H, psiE, psiH, amp):
    """One step on the whole grid: H^n from E^{n-1/2}, then E^{n+1/2} (no E above the grid, no H
    below it, periodic x and y)."""
    nz, S, dt = g.nz, g.S, g.dt
    Ez1 = np.concatenate([E[:, 1:], np.zeros_like(E[:, :1])], axis=1)
    Ej1, Ei1 = np.roll(E, -1, axis=2), np.roll(E, -1, axis=3)
    dyEz, dzEy, dzEx = Ej1[2] - E[2], Ez1[1] - E[1], Ez1[0] - E[0]
    dxEz, dxEy, dyEx = Ei1[2] - E[2], Ei1[1] - E[1], Ej1[0] - E[0]
    Hn, psiHn = H.copy(), psiH.copy()
    for k in range(nz):
        ip = psi_h_plane(k, nz, g.npml)
        if ip >= 0:
            b, c = g.pmlH[k]
            psiHn[0, ip] = b * psiH[0, ip] + c * dzEy[k]
            psiHn[1, ip] = b * psiH[1, ip] + c * dzEx[k]
            Hn[0, k] = H[0, k] - S * (dyEz[k] - (dzEy[k] + psiHn[0, ip]))
            Hn[1, k] = H[1, k] - S * ((dzEx[k] + psiHn[1, ip]) - dxEz[k])
        else:
            Hn[0, k] = H[0, k] - S * (dyEz[k] - dzEy[k])
            Hn[1, k] = H[1, k] - S * (dzEx[k] - dxEz[k])
        Hn[2, k] = H[2, k] - S * (dxEy[k] - dyEx[k])
    Hm = np.concatenate([np.zeros_like(Hn[:, :1]), Hn[:, :-1]], axis=1)
    Hjm, Him = np.roll(Hn, 1, axis=2), np.roll(Hn, 1, axis=3)
    dyHz, dzHy, dzHx = Hn[2] - Hjm[2], Hn[1] - Hm[1], Hn[0] - Hm[0]
    dxHz, dxHy, dyHx = Hn[2] - Him[2], Hn[1] - Him[1], Hn[0] - Hjm[0]
    En, psiEn = E.copy(), psiE.copy()
    for k in range(nz):
        ip = psi_e_plane(k, nz, g.npml)
        if ip >= 0:
            b, c = g.pmlE[k]
            px = b * psiE[0, ip] + c * dzHy[k]
            py = b * psiE[1, ip] + c * dzHx[k]
            psiEn[0, ip], psiEn[1, ip] = px, py
            curl = [dyHz[k] - (dzHy[k] + px), (dzHx[k] + py) - dxHz[k]]
        else:
            curl = [dyHz[k] - dzHy[k], dzHx[k] - dxHz[k]]
        curl.append(dxHy[k] - dyHx[k])
        for c in range(3):
            e = E[c, k] + S * curl[c]
            if k == g.srcz and c == g.srcc:
                e = e + dt * (amp[0] * g.cos + amp[1] * g.sin)
            En[c, k] = e
    return En, Hn, psiEn, psiHn


def h_cell(e, en, h, r, c, S, psi=None, bc=None):
    """H at frame cell (r, c) from E frames e (plane k) and en (plane k+1) and H frame h."""
    dyEz = e[2, r + 1, c] - e[2, r, c]
    dzEy = en[1, r, c] - e[1, r, c]
    dzEx = en[0, r, c] - e[0, r, c]
    dxEz = e[2, r, c + 1] - e[2, r, c]
    dxEy = e[1, r, c + 1] - e[1, r, c]
    dyEx = e[0, r + 1, c] - e[0, r, c]
    hx, hy, hz = h[:, r, c]
    ps = (np.nan, np.nan)
    if psi is not None:
        b, cf = bc
        ps = (b * psi[0] + cf * dzEy, b * psi[1] + cf * dzEx)
        hx = hx - S * (dyEz - (dzEy + ps[0]))
        hy = hy - S * ((dzEx + ps[1]) - dxEz)
    else:
        hx = hx - S * (dyEz - dzEy)
        hy = hy - S * (dzEx - dxEz)
    hz = hz - S * (dxEy - dyEx)
    return (hx, hy, hz), ps


def e_curl(h, r, c, hxm, hym, psi=None, bc=None):
    """curl H at frame cell (r, c) (the z-neighbour values given), with the E-side memories."""
    Hx, Hy, Hz = h[:, r, c]
    dyHz, dzHy, dzHx = Hz - h[2, r - 1, c], Hy - hym, Hx - hxm
    dxHz, dxHy, dyHx = Hz - h[2, r, c - 1], Hy - h[1, r, c - 1], Hx - h[0, r - 1, c]
    ps = (np.nan, np.nan)
    if psi is not None:
        b, cf = bc
        ps = (b * psi[0] + cf * dzHy, b * psi[1] + cf * dzHx)
        curl = [dyHz - (dzHy + ps[0]), (dzHx + ps[1]) - dxHz]
    else:
        curl = [dyHz - dzHy, dzHx - dxHz]
    return curl + [dxHy - dyHx], ps


def march(g, starts):
    """Every CTA of the chunk plan `starts`, in the kernel's order of work; returns the outputs and
    the planes whose monitor / energy partials each step recorded."""
    nx, ny, nz, npml, S, dt = g.nx, g.ny, g.nz, g.npml, g.S, g.dt
    out = {k: np.full(getattr(g, k).shape, np.nan) for k in ("E", "H", "psiE", "psiH")}
    visits = {("H", 1): [], ("E", 1): [], ("H", 2): [], ("E", 2): []}
    h1cells, e1cells, h2cells = box_cells(H1B), box_cells(E1B), box_cells(H2B)
    for ci in range(len(starts) - 1):
        zb, ze = starts[ci], starts[ci + 1]
        for by in range(ny // TY):
            for bx in range(nx // TX):
                x0, y0 = bx * TX, by * TY
                ys = [(y0 - 2 + r) % ny for r in range(FY)]
                xs = [(x0 - 4 + c) % nx for c in range(FX)]
                sE0 = np.full((RE, 3, FY, FX), np.nan)
                sH0 = np.full((RH, 3, FH, FX), np.nan)
                sH1 = np.full((RH1, 3, FH, FX), np.nan)
                sPH = np.full((RH1, 2, FH, FX), np.nan)
                sE1 = np.full((RE1, 3, FH, FX), np.nan)
                sH2 = np.full((3, FH, FX), np.nan)
                kA, a1 = max(zb - 2, 0), max(zb - 1, 0)
                kE_last, kH_last = ze + 1, min(ze, nz - 1)
                landing = []

                def stage_e(k):
                    sE0[k % RE] = np.nan
                    v = g.E[:, k][:, ys][:, :, xs] if k < nz else np.zeros((3, FY, FX))
                    landing.append((sE0, k % RE, v))

                def stage_h(k):
                    sH0[k % RH] = np.nan
                    landing.append((sH0, k % RH, g.H[:, k][:, ys[:FH]][:, :, xs]))

                stage_e(kA)
                stage_e(kA + 1)
                stage_h(kA)
                hm = {rc: (0.0, 0.0) for rc in OWN}          # H^{n+1} below, own cells
                q0, q1 = {}, {}                                # E^{n+1/2} and memories, own cells
                for k in range(kA, ze + 2):
                    for arr, slot, v in landing:               # wait + barrier
                        arr[slot] = v
                    landing.clear()
                    if k + 2 <= kE_last:
                        stage_e(k + 2)
                    if k + 1 <= kH_last:
                        stage_h(k + 1)
                    m = k - 2
                    h1, h1m, ph1, e1 = sH1[k % RH1], sH1[(k + 2) % RH1], sPH[k % RH1], sE1[k & 1]
                    # phase 1: H^n(k) on the H1 box, H^{n+1}(m) on the H2 box
                    if k <= ze and k < nz:
                        e0, e0n, hin = sE0[k % RE], sE0[(k + 1) % RE], sH0[k % RH]
                        ip = psi_h_plane(k, nz, npml)
                        for (r, c) in h1cells:
                            psi = g.psiH[:, ip, ys[r], xs[c]] if ip >= 0 else None
                            h1[:, r, c], ps = h_cell(e0, e0n, hin, r, c, S, psi, g.pmlH[k])
                            if ip >= 0:
                                ph1[:, r, c] = ps
                        if zb <= k < ze:
                            visits[("H", 1)].append(k)
                    h2own = {}
                    if a1 <= m < ze:
                        ea, eb = sE1[m & 1], sE1[(m + 1) & 1]
                        ha, pa = sH1[(k + 1) % RH1], sPH[(k + 1) % RH1]
                        ip = psi_h_plane(m, nz, npml)
                        for (r, c) in h2cells:
                            psi = pa[:, r, c] if ip >= 0 else None
                            sH2[:, r, c], ps = h_cell(ea, eb, ha, r, c, S, psi, g.pmlH[m])
                            if (r, c) in OWN_SET:
                                h2own[(r, c)] = sH2[:2, r, c].copy()
                                if zb <= m < ze:
                                    out["H"][:, m, ys[r], xs[c]] = sH2[:, r, c]
                                    if ip >= 0:
                                        out["psiH"][:, ip, ys[r], xs[c]] = ps
                        if zb <= m < ze:
                            visits[("H", 2)].append(m)
                    # phase 2: E^{n+3/2}(m) on the tile, E^{n+1/2}(k) on the E1 box
                    if zb <= m < ze:
                        ip = psi_e_plane(m, nz, npml)
                        for (r, c) in OWN:
                            hx, hy = hm[(r, c)]
                            psi = q0[(r, c)][1] if ip >= 0 else None
                            curl, ps = e_curl(sH2, r, c, hx, hy, psi, g.pmlE[m])
                            for cc in range(3):
                                e = q0[(r, c)][0][cc] + S * curl[cc]
                                if m == g.srcz and cc == g.srcc:
                                    a, b = g.amp[1]
                                    e = e + dt * (a * g.cos[ys[r], xs[c]] + b * g.sin[ys[r], xs[c]])
                                out["E"][cc, m, ys[r], xs[c]] = e
                            if ip >= 0:
                                out["psiE"][:, ip, ys[r], xs[c]] = ps
                        visits[("E", 2)].append(m)
                    e1own = {rc: ((np.nan,) * 3, (np.nan,) * 2) for rc in OWN}
                    if a1 <= k <= ze and k < nz:
                        e0 = sE0[k % RE]
                        ip = psi_e_plane(k, nz, npml)
                        for (r, c) in e1cells:
                            hxm, hym = (0.0, 0.0) if k == 0 else (h1m[0, r, c], h1m[1, r, c])
                            psi = g.psiE[:, ip, ys[r], xs[c]] if ip >= 0 else None
                            curl, ps = e_curl(h1, r, c, hxm, hym, psi, g.pmlE[k])
                            for cc in range(3):
                                e = e0[cc, r, c] + S * curl[cc]
                                if k == g.srcz and cc == g.srcc:
                                    a, b = g.amp[0]
                                    e = e + dt * (a * g.cos[ys[r], xs[c]] + b * g.sin[ys[r], xs[c]])
                                e1[cc, r, c] = e
                            if (r, c) in OWN_SET:
                                e1own[(r, c)] = (e1[:, r, c].copy(), ps)
                        if zb <= k < ze:
                            visits[("E", 1)].append(k)
                    elif k == nz:
                        e1[:] = 0.0
                    if k >= a1:
                        q0, q1 = q1, e1own
                    if a1 <= m < ze:
                        hm = h2own
    return out, visits


@pytest.mark.parametrize("nx,ny,nz,npml,starts", [
    (64, 16, 30, 4, [0, 5, 9, 17, 26, 30]),           # ghost planes next to the absorbers
    (32, 8, 14, 2, [0, 3, 8, 11, 14]),                # chunk starts inside the absorber's reach
    (64, 16, 20, 1, [0, 1, 2, 3, 10, 19, 20]),        # one-plane chunks, top ghost plane in the CPML
])
def test_two_step_schedule_equals_two_single_steps(nx, ny, nz, npml, starts):
    g = Grid(nx, ny, nz, npml)
    E1, H1, pE1, pH1 = fused_step(g, g.E, g.H, g.psiE, g.psiH, g.amp[0])
    E2, H2, pE2, pH2 = fused_step(g, E1, H1, pE1, pH1, g.amp[1])
    out, visits = march(g, starts)
    for name, want in (("E", E2), ("H", H2), ("psiE", pE2), ("psiH", pH2)):
        assert not np.isnan(out[name]).any(), name
        np.testing.assert_array_equal(out[name], want, err_msg=name)
    tiles = (nx // TX) * (ny // TY)
    for key, planes in visits.items():   # each step's partials: every plane once per tile
        assert sorted(planes) == sorted(list(range(nz)) * tiles), key


def test_halo_enumeration_covers_each_box_once():
    for box in (H1B, E1B, H2B):
        cells = box_cells(box)
        assert len(cells) - TX * TY <= TX * TY
