"""Differentiation form: gradients of a spectral loss through torch.autograd.

``Spectrum`` is a torch.autograd.Function whose forward runs the simulation through the C ABI
with checkpoints (fdtdbath_adjoint_forward) and returns the monitor spectra, and whose backward
runs the library's discrete adjoint (fdtdbath_adjoint_backward).  The differentiable inputs are
the oscillator parameters of one layer in nu-units: (sigma, gamma, coupling_1..coupling_N_b).
Everything after the spectra (flux, transmission, loss) is ordinary torch arithmetic, so any
loss of the spectra can be differentiated.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import fdtdbath as fb


def layer_params(prob: dict, material: int) -> np.ndarray:
    """(sigma, gamma, coupling_1..N_b) of layer `material` (nu-units)."""
    m = prob["materials"][material]
    k = np.asarray(m.get("bath_couplings", []), dtype=np.float64) if m["kind"] == "lorentz_bath" else np.zeros(0)
    return np.concatenate([[float(m["sigma"]), float(m["gamma"])], k])


def with_params(prob: dict, material: int, params) -> dict:
    """A copy of prob whose layer `material` takes the given (sigma, gamma, couplings)."""
    p = np.asarray(params, dtype=np.float64)
    q = copy.deepcopy(prob)
    m = q["materials"][material]
    m["sigma"] = float(p[0])
    m["gamma"] = float(p[1])
    if m["kind"] == "lorentz_bath":
        m["bath_couplings"] = p[2:].copy()
    return q


def flux(spec: torch.Tensor) -> torch.Tensor:
    """Normal flux Re(Ex Hy* - Ey Hx*) from spectra (nfreq, 4, 2) = (Ex, Ey, Hx, Hy) x (re, im)."""
    ex, ey, hx, hy = (torch.complex(spec[:, c, 0], spec[:, c, 1]) for c in range(4))
    return torch.real(ex * torch.conj(hy) - ey * torch.conj(hx))


class Spectrum(torch.autograd.Function):
    """params (float64, 2 + N_b) -> monitor spectra (nfreq, 4, 2), backward by the adjoint."""

    @staticmethod
    def forward(ctx, params, prob, material, nsteps, checkpoint_every, precision):
        sim = fb.Simulation(with_params(prob, material, params.detach().cpu().numpy()),
                            precision=precision, energy=False)
        sim.adjoint_forward(nsteps, checkpoint_every)
        spec = sim.dft(0)
        ctx.sim, ctx.material = sim, material
        out = np.stack([spec.real, spec.imag], axis=-1)
        return torch.from_numpy(np.ascontiguousarray(out)).to(params.device)

    @staticmethod
    def backward(ctx, grad_spec):
        g = ctx.sim.adjoint_backward(grad_spec.detach().cpu().numpy(), ctx.material)
        ctx.sim.close()
        return torch.from_numpy(g).to(grad_spec.device), None, None, None, None, None


def transmission_loss(params: torch.Tensor, prob: dict, material: int, flux_vac: np.ndarray,
                      target: np.ndarray, nsteps: int, checkpoint_every: int = 256,
                      precision: int = 32) -> torch.Tensor:
    """L = sum_k (T_k - T*_k)^2 with T = flux / flux of the empty (vacuum) run."""
    spec = Spectrum.apply(params, prob, material, nsteps, checkpoint_every, precision)
    T = flux(spec) / torch.as_tensor(flux_vac, dtype=spec.dtype)
    return torch.sum((T - torch.as_tensor(target, dtype=spec.dtype)) ** 2)
