"""The trace and spectrum estimators of paper_2505_23963_gb300/analysis.py on signals whose
answers are known in closed form (no simulation): an exponentially decaying energy with and
without a Rabi-like beat, a fixed bath share, and peaks of known position."""
import numpy as np
import pytest

from paper_2505_23963_gb300 import analysis


def trace_of(u_em, u_p=None, u_b=None):
    z = np.zeros_like(u_em)
    return np.stack([u_em, z if u_p is None else u_p, z if u_b is None else u_b, z], axis=1)


def test_relaxation_rate_of_a_pure_exponential():
    """Without local maxima the fit takes every record after the peak: exact for e^{-g t}."""
    dt, g = 0.05, 0.137
    t = np.arange(4000) * dt
    u = np.where(t < 3.0, t / 3.0, np.exp(-g * (t - 3.0)))
    assert analysis.relaxation_rate(trace_of(u), dt, 1.0) == pytest.approx(g, rel=1e-10)


@pytest.mark.parametrize("g,omega", [(0.02, 2.0), (0.11, 5.3)])
def test_relaxation_rate_through_a_beat(g, omega):
    """U = e^{-g t} (1 + 0.6 cos(omega t)): the maxima of U sit one fixed shift after the beat's,
    so ln U at the maxima falls with slope -g exactly; sampling at 2000 points per beat period
    leaves ~1e-4 of jitter."""
    period = 2 * np.pi / omega
    dt = period / 2000
    t = np.arange(int(12 * period / dt)) * dt
    u = np.exp(-g * t) * (1.0 + 0.6 * np.cos(omega * t))
    assert analysis.relaxation_rate(trace_of(u), dt, 0.0) == pytest.approx(g, rel=2e-3)


def test_bath_share_is_the_largest_fraction_after_the_start():
    dt = 0.1
    t = np.arange(500) * dt
    em = 1.0 + 0.5 * np.cos(t)
    p = np.full_like(t, 0.25)
    b = 0.25 * (1.0 - np.cos(t)) + np.where(t < 5.0, 100.0, 0.0)   # ignored before t_start
    share = b / (em + p + b)
    want = share[t > 5.0].max()
    assert analysis.bath_share(trace_of(em, p, b), dt, 5.0) == pytest.approx(want, rel=1e-12)
    assert 0.39 < want <= 0.4          # 0.5 / 1.25 where cos t = -1


def test_spectral_peaks_of_quadratic_tops_are_exact():
    """The 3-point parabola refinement recovers the vertex of a peak that is a parabola near its
    top, wherever the vertex falls between samples; the two largest maxima, sorted by
    frequency."""
    f = np.linspace(0.8, 1.2, 401)
    a, b = 0.93137, 1.06421
    p = np.maximum(0.0, 1.0 - ((f - a) / 0.01) ** 2) + 0.7 * np.maximum(0.0, 1.0 - ((f - b) / 0.01) ** 2)
    p = p + 0.1 * np.maximum(0.0, 1.0 - ((f - 1.15) / 0.01) ** 2)         # a third, smaller peak
    got = analysis.spectral_peaks(f, p, 2)
    assert got == pytest.approx([a, b], abs=1e-12)
