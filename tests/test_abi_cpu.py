"""The C-ABI library without a GPU: it builds, loads, exports every declared entry point,
and its host-side logic (Table I expansion, argument validation) behaves (CPU only)."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from oracle import closed_forms as cf
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdtdbath_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = fb.lib()
    decl = declared_functions()
    assert len(decl) >= 12
    for name in decl:
        assert hasattr(L, name), name
    assert set(fb.EXPORTED) <= set(decl)


@pytest.mark.parametrize("shape", ["uniform", "lorentzian", "gaussian"])
def test_bath_form_matches_table1(shape):
    f, g, k = fb.bath_form(shape, 1.0, 0.0004, 100, 0.4, 0.0004, 0.0396)
    f2, g2, k2 = cf.bath_form(shape, 1.0, 0.0004, 100, 0.4, 0.0004, 0.0396)
    np.testing.assert_allclose(f, f2, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(g, g2)
    np.testing.assert_allclose(k, k2, rtol=1e-13, atol=1e-16)


def test_bath_form_rejects_bad_arguments():
    with pytest.raises(fb.FdtdBathError) as e:
        fb.bath_form("uniform", 1.0, 0.01, 1, 0.2, 0.001, 0.01)
    assert e.value.code == fb.ERR_ARG


def _create_err(prob, **kw):
    with pytest.raises(fb.FdtdBathError) as e:
        fb.create(prob, use_torch_allocator=False, **kw)
    return e.value.code


def test_create_validates_before_touching_the_gpu():
    p = wl.small_3d()
    assert _create_err(dict(p, courant=0.7)) == fb.ERR_CFL            # > 1/sqrt(3)
    assert _create_err(p, precision=16) == fb.ERR_ARG
    bad = dict(p, materials=[dict(p["materials"][0], z=(5, 500))])
    assert _create_err(bad) == fb.ERR_ARG
    over = dict(p, materials=[p["materials"][0], dict(p["materials"][1], z=(p["materials"][0]["z"][0], 30))])
    assert _create_err(over) == fb.ERR_ARG
    assert _create_err(dict(p, pml=40)) == fb.ERR_ARG
    assert _create_err(p, precision=64, bath_storage=1) == fb.ERR_ARG   # bf16 bath modes need FP32
    assert _create_err(p, precision=32, bath_storage=2) == fb.ERR_ARG
    fast = dict(p, materials=[dict(p["materials"][1], frequency=40.0)])   # w0 dt >= 2
    assert _create_err(fast) == fb.ERR_CFL
    assert _create_err(dict(p, monitors=[dict(z=0, freqs=np.ones(3))])) == fb.ERR_ARG
    # Drude mirrors with w_p dt too large for the coupled field-oscillator update
    assert _create_err(dict(p, resolution=10.0)) == fb.ERR_CFL
    # at most 128 bath modes per material (the step kernel streams them above 32)
    lb = p["materials"][1]
    many = dict(p, materials=[dict(lb, bath_frequencies=np.linspace(0.9, 1.1, 129),
                                   bath_gammas=np.full(129, 0.005), bath_couplings=np.full(129, 0.001))])
    assert _create_err(many) == fb.ERR_ARG
