"""Host analysis of energy traces: polariton relaxation rate and bath-energy share.

Plain numpy on recorded traces (any producer: the CUDA library or the CPU oracle), not part of
the simulated path.  Definitions (the paper shows energy traces but fixes no estimator):

* gamma_pol: U_cav(t) is the electromagnetic energy inside the cavity's energy box.  From the
  largest value of U_cav after the source has ended (t > 2 t0) -- the pulse needs time to reach
  and fill a long cavity -- take the local maxima of U_cav, fit ln U_cav at those maxima by least
  squares against t, and report minus the slope (an energy decay rate, 1/time).  With fewer than
  three maxima the fit uses every record from that point on.
* bath_share: the largest fraction of the box energy held by the bath modes after the source,
  max_t U_bath / (U_EM + U_P + U_bath).
"""
from __future__ import annotations

import numpy as np


def relaxation_rate(trace: np.ndarray, dt_record: float, t_start: float) -> float:
    """Polariton energy decay rate from trace[:, 0] (records dt_record apart, record r at
    t = r * dt_record), using records after t_start."""
    u = np.asarray(trace, dtype=np.float64)[:, 0]
    t = np.arange(u.size) * dt_record
    after = np.nonzero(t > t_start)[0]
    if after.size == 0:
        return float("nan")
    top = after[np.argmax(u[after])]
    keep = (np.arange(u.size) >= top) & (u > 0)
    idx = np.nonzero(keep)[0]
    if idx.size < 3:
        return float("nan")
    inner = idx[(idx > 0) & (idx < u.size - 1)]
    peaks = inner[(u[inner] >= u[inner - 1]) & (u[inner] > u[inner + 1])]
    sel = peaks if peaks.size >= 3 else idx
    slope = np.polyfit(t[sel], np.log(u[sel]), 1)[0]
    return float(-slope)


def bath_share(trace: np.ndarray, dt_record: float, t_start: float) -> float:
    """Largest share of the box energy held by the bath modes after t_start."""
    tr = np.asarray(trace, dtype=np.float64)
    t = np.arange(tr.shape[0]) * dt_record
    tot = tr[:, 0] + tr[:, 1] + tr[:, 2]
    ok = (t > t_start) & (tot > 0)
    if not np.any(ok):
        return float("nan")
    return float(np.max(tr[ok, 2] / tot[ok]))


def spectral_peaks(freqs: np.ndarray, power: np.ndarray, count: int = 2) -> np.ndarray:
    """Positions of the `count` largest local maxima of a sampled spectrum, each refined by a
    3-point parabola through the maximum and its neighbours; sorted by frequency."""
    f = np.asarray(freqs, dtype=np.float64)
    p = np.asarray(power, dtype=np.float64)
    i = np.arange(1, p.size - 1)
    loc = i[(p[i] >= p[i - 1]) & (p[i] > p[i + 1])]
    loc = loc[np.argsort(p[loc])[::-1][:count]]
    out = []
    for k in loc:
        y0, y1, y2 = p[k - 1], p[k], p[k + 1]
        den = y0 - 2.0 * y1 + y2
        d = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        out.append(f[k] + d * (f[k + 1] - f[k]))
    return np.sort(np.array(out))
