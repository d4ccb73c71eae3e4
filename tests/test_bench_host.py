"""Host arithmetic of bench.py (no GPU): the algorithmic bytes behind the roofline fraction,
the batch form's flop count and derived FP32 peak, and the finite-spectrum probe."""
import pytest

import bench
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl


def test_algorithmic_bytes_of_the_measured_workloads():
    """256^3, N_b = 8: 34624 B per (x, y) column = 135.25 B per cell-update (FP32), twice that in
    FP64; 512 x 512 x 384, N_b = 16: 205.2 B (157.2 B with bf16 value/increment bath pairs)."""
    p = wl.slab_3d(steps=10)
    assert bench.algorithmic_bytes(p, 4) == 34624 * 256 * 256
    assert bench.algorithmic_bytes(p, 8) == 2 * 34624 * 256 * 256
    q = wl.precision_3d(steps=10)
    cells = 512 * 512 * 384
    assert bench.algorithmic_bytes(q, 4) / cells == pytest.approx(205.2, abs=0.05)
    assert bench.algorithmic_bytes(q, 4, 8.0) / cells == pytest.approx(157.2, abs=0.05)


def test_batch_flop_count():
    """One 1000-cell batch cavity with N_b = 4: 6 per cell, 8 x 2 x 16 CPML, 8 x 40 Drude,
    (10 x 4 + 8) x 400 Lorentz-Bath."""
    p = wl.batch_cavity(1000, rabi=0.1, num_bath=4, steps=10)
    assert bench.batch_flops_per_step([p]) == 6 * 1000 + 8 * 2 * 16 + 8 * 40 + 48 * 400
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.548, rel=1e-4)


def test_spectrum_is_finite_reads_the_error_code():
    class Sim:
        def __init__(self, code=None):
            self.code = code

        def dft(self, mon):
            if self.code is not None:
                raise fb.FdtdBathError(self.code, "")
            return None

    assert bench.spectrum_is_finite(fb, Sim())
    assert not bench.spectrum_is_finite(fb, Sim(fb.ERR_NONFINITE))
    with pytest.raises(fb.FdtdBathError):
        bench.spectrum_is_finite(fb, Sim(fb.ERR_CUDA))


def test_fp64_flop_count():
    """FP64 literal path: vacuum 30 per cell, +16 in the CPML, Drude +24, a Lorentz-Bath plane
    51 N_b + 112, +7 inside the energy box.  256^3, N_b = 8: (144 x 30 + 32 x 46 + 16 x 54 +
    64 x (520 + 7)) per column."""
    p = wl.slab_3d(steps=10)
    col = 144 * 30 + 32 * 46 + 16 * 54 + 64 * (51 * 8 + 112 + 7)
    assert bench.algorithmic_flops_fp64(p) == col * 256 * 256
    q = dict(p, materials=[], energy_box=(0, 0))
    assert bench.algorithmic_flops_fp64(q) == (224 * 30 + 32 * 46) * 256 * 256
