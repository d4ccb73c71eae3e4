"""Error reporting of a diverged state through the C ABI: once NaN reaches the state, the spectra
and the energy trace read out are flagged FDTDBATH_ERR_NONFINITE (the outputs are still filled);
before that both read out cleanly.  The NaN is written from the host into E_x: the kernels only
carry it through their arithmetic, no index or branch depends on a field value."""
import numpy as np
import pytest

from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [64, 32])
def test_nan_in_the_state_is_reported(precision):
    prob = wl.small_3d(nx=8, ny=4, nb=4, steps=8, seed=1)
    s = fb.Simulation(prob, precision=precision, energy_capacity=16)
    s.step(3)
    assert np.all(np.isfinite(s.dft(0)))
    assert len(s.trace()) == 3
    e = s.get("E", comp=0)
    e[...] = np.nan
    s.set("E", e, comp=0)
    s.step(2)
    for read in (lambda: s.dft(0), lambda: s.trace()):
        with pytest.raises(fb.FdtdBathError) as err:
            read()
        assert err.value.code == fb.ERR_NONFINITE
        assert "NaN or Inf" in str(err.value)
    s.close()
