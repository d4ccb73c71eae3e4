"""Why the FP32 path advances each oscillator by increments (no GPU): a numpy emulation of one
driven Lorentz cell (Eq. Pz_1D_Lorentz at the 1D cavity's resolution, w0 dt = 0.031) in float32,
once in the literal two-level form and once in the increment form V = P^n - P^{n-1}, against the
same recursion in float64.  The literal form stores (2 - w0^2 dt^2) / A, whose float32 rounding
shifts the oscillator frequency by ~eps / (w0 dt)^2; the increment form never forms that
number.  Both forms are the same recursion in exact arithmetic (checked in float64)."""
import numpy as np


def lorentz_cell(dtype, form, E, w2, g, s):
    f = dtype
    w2, g, s, one, two = f(w2), f(g), f(s), f(1), f(2)
    A = one + g
    P = Pm = f(0)
    out = np.empty(E.size, np.float64)
    if form == "literal":
        c1, c2, cs = (two - w2) / A, (one - g) / A, s / A
        for i, e in enumerate(E.astype(dtype)):
            P, Pm = c1 * P - c2 * Pm + cs * e, P
            out[i] = P
    else:
        cw, cg, cs = w2 / A, (one - g) / A, s / A
        V = f(0)
        for i, e in enumerate(E.astype(dtype)):
            V = cs * e - cw * P + cg * V
            P = P + V
            out[i] = P
    return out


def setup(n=40000):
    dt = 0.005                                   # resolution 100, Courant 0.5
    w0, gamma, sigma = 2 * np.pi, 2 * np.pi * 0.01, 0.05 ** 2
    t = np.arange(n) * dt
    E = np.exp(-((t - 1.6) / 0.32) ** 2 / 2) * np.sin(2 * np.pi * (t - 1.6))
    return E, (w0 * dt) ** 2, gamma * dt / 2, sigma * (w0 * dt) ** 2


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forms_agree_in_float64():
    E, w2, g, s = setup(8000)
    a = lorentz_cell(np.float64, "literal", E, w2, g, s)
    b = lorentz_cell(np.float64, "increment", E, w2, g, s)
    assert rel(b, a) < 1e-11


def test_increment_form_is_the_accurate_float32_form():
    E, w2, g, s = setup()
    ref = lorentz_cell(np.float64, "literal", E, w2, g, s)
    lit = rel(lorentz_cell(np.float32, "literal", E, w2, g, s), ref)
    inc = rel(lorentz_cell(np.float32, "increment", E, w2, g, s), ref)
    print(f"\nfloat32 error: literal {lit:.2e}, increment {inc:.2e}")
    assert inc < 1e-4 and lit > 20 * inc
