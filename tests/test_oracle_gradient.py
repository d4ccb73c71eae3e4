"""The oracle gradient of the differentiation form is a central finite difference of the FP64
oracle's loss.  Pin of that procedure (no GPU): on a small 2D cavity the central differences
converge at second order -- the change from step h to h/2 shrinks about 4x per halving -- so
h = 1e-4 relative carries an error near 1e-8 relative."""
import numpy as np

from oracle import oracle as O
from paper_2505_23963_gb300 import adjoint as adj
from paper_2505_23963_gb300 import workloads as wl


def test_central_differences_converge_at_second_order():
    prob = wl.slab_cavity(4, 1, (8, 12, 3, 16, 3, 12), 16.0, num_bath=2, sigma=0.05 ** 2,
                          phase_seed=1, src_z=14, mon_z=52, nfreq=24, steps=400,
                          source_component=1, drude_sigma=4.0)
    mat = 1

    def spec(p):
        o = O.OracleSim(p)
        o.step(p["steps"])
        return o.dft(0)

    fv = O.flux(spec(wl.vacuum_of(prob)))
    p0 = adj.layer_params(prob, mat)
    target = O.flux(spec(adj.with_params(prob, mat, wl.adjoint_target_params(p0)))) / fv

    def loss(p):
        return float(np.sum((O.flux(spec(adj.with_params(prob, mat, p))) / fv - target) ** 2))

    def fd(h, i):
        d = h * abs(p0[i])
        a, b = p0.copy(), p0.copy()
        a[i] += d
        b[i] -= d
        return (loss(a) - loss(b)) / (2 * d)

    for i in (0, 2):   # sigma and the first coupling
        g = [fd(h, i) for h in (4e-2, 2e-2, 1e-2)]
        d1, d2 = abs(g[0] - g[1]), abs(g[1] - g[2])
        assert d1 > 0 and 3.0 < d1 / d2 < 5.0, (i, g, d1 / d2)
