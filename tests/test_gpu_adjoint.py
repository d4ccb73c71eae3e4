"""Differentiation form on the GPU: the library's discrete adjoint (through torch.autograd)
against central finite differences of the loss (h = 1e-4 relative) -- of the GPU FP64 forward and
of the FP64 oracle -- on the 128 x 128 crop (resolution 16, N_b Lorentz-Bath layer, E_y source
with the seeded transverse phase, CPML, Drude mirrors).  The loss is sum_k (T_k - T*_k)^2 with
T = flux / flux of the empty run and T* the transmission at perturbed parameters.
Tolerances (normwise over the gradient vector): FP64 adjoint vs FD 1e-6 (the FD truncation error
is ~h^2 = 1e-8 relative); FP32 adjoint vs FP64 adjoint 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2505_23963_gb300 import adjoint as adj
from paper_2505_23963_gb300 import fdtdbath as fb
from paper_2505_23963_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAT = 1   # the Lorentz-Bath layer (0 and 2 are the mirrors)


def gpu_T(prob, params, precision=64):
    s = fb.Simulation(adj.with_params(prob, MAT, params), precision=precision, energy=False)
    s.step(prob["steps"])
    out = s.dft(0)
    s.close()
    return out


def setup(prob, precision=64):
    fv = O.flux(_vac_spec(prob, precision))
    p0 = adj.layer_params(prob, MAT)
    target = O.flux(gpu_T(prob, wl.adjoint_target_params(p0), precision)) / fv
    return p0, fv, target


def _vac_spec(prob, precision):
    s = fb.Simulation(wl.vacuum_of(prob), precision=precision, energy=False)
    s.step(prob["steps"])
    out = s.dft(0)
    s.close()
    return out


def loss_value(prob, params, fv, target, precision=64):
    T = O.flux(gpu_T(prob, params, precision)) / fv
    return float(np.sum((T - target) ** 2))


def adjoint_grad(prob, params, fv, target, every, precision=64):
    x = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    L = adj.transmission_loss(x, prob, MAT, fv, target, prob["steps"], every, precision)
    L.backward()
    return float(L.detach()), x.grad.numpy().copy()


def central_fd(f, p0, h=1e-4):
    g = np.zeros_like(p0)
    for i in range(p0.size):
        d = h * abs(p0[i])
        a, b = p0.copy(), p0.copy()
        a[i] += d
        b[i] -= d
        g[i] = (f(a) - f(b)) / (2 * d)
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_adjoint_fp64_matches_gpu_finite_differences():
    prob = wl.adjoint_crop(steps=800, nb=4)
    p0, fv, target = setup(prob)
    L, g = adjoint_grad(prob, p0, fv, target, every=96)   # 96 does not divide 800
    assert abs(L - loss_value(prob, p0, fv, target)) <= 1e-12 * L
    fd = central_fd(lambda p: loss_value(prob, p, fv, target), p0)
    print(f"\nadjoint {g}\nFD      {fd}\nrel {rel(g, fd):.3e}")
    assert rel(g, fd) < 1e-6


def test_adjoint_fp32_close_to_fp64():
    prob = wl.adjoint_crop(steps=800, nb=4)
    p0, fv, target = setup(prob)
    _, g64 = adjoint_grad(prob, p0, fv, target, every=128, precision=64)
    _, g32 = adjoint_grad(prob, p0, fv, target, every=128, precision=32)
    print(f"\nFP32 vs FP64 adjoint gradient: rel {rel(g32, g64):.3e}")
    assert rel(g32, g64) < 1e-3


def test_adjoint_matches_oracle_gradient():
    """The FP64 oracle's own gradient: central differences of its loss on the crop."""
    prob = wl.adjoint_crop(steps=2000, nb=8)
    p0 = adj.layer_params(prob, MAT)

    def o_spec(p):
        o = O.OracleSim(p)
        o.step(prob["steps"])
        return o.dft(0)

    fv = O.flux(o_spec(wl.vacuum_of(prob)))
    target = O.flux(o_spec(adj.with_params(prob, MAT, wl.adjoint_target_params(p0)))) / fv
    f = lambda p: float(np.sum((O.flux(o_spec(adj.with_params(prob, MAT, p))) / fv - target) ** 2))
    g_or = central_fd(f, p0)
    _, g = adjoint_grad(prob, p0, fv, target, every=256)
    print(f"\nadjoint {g}\noracle  {g_or}\nrel {rel(g, g_or):.3e}")
    assert rel(g, g_or) < 1e-6


def test_adjoint_3d_fp64_matches_gpu_finite_differences():
    """A ragged 3D cavity (40 x 12 cells, tiles cut in x and y, E_x source with a transverse
    phase): the general three-component adjoint kernels, and their cell-index arithmetic on a
    grid with ny > 1, against central differences of the GPU FP64 forward."""
    prob = wl.small_3d(nx=40, ny=12, layout=(6, 5, 3, 10, 3, 5), nb=4, steps=300, seed=2)
    p0, fv, target = setup(prob)
    L, g = adjoint_grad(prob, p0, fv, target, every=64)
    assert abs(L - loss_value(prob, p0, fv, target)) <= 1e-12 * L
    fd = central_fd(lambda p: loss_value(prob, p, fv, target), p0)
    print(f"\n3D adjoint {g}\nFD         {fd}\nrel {rel(g, fd):.3e}")
    assert rel(g, fd) < 1e-6
