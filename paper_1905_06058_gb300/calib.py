"""Calibration of the dispersion coefficients and the focal depth by gradient
descent through the model and through unrolled FISTA iterations.

The paper notes that the dispersion coefficients a (Eq. 7) may be found by an
autofocus method and places the focus at a known depth (§2, §4.1).  These
torch.autograd.Function wrappers make the model differentiable in
theta = (a1, a2, a3, a4, z0) so both can be fitted to data instead.  Every
derivative is computed by the library (isam_param_grad, the adjoint operator,
isam_fista_unrolled_vjp); this module only marshals tensors.

theta is a float64 CPU tensor of shape [5] in the plan's units (a_i in
rad m^i about k0, z0 in m).  Every op first makes the plan's model equal to
theta (isam_set_model); lambda and L of the unrolled solve are constants.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from .isam import N_PARAMS, Plan


def _apply_theta(plan: Plan, theta: torch.Tensor) -> None:
    t = theta.detach().to("cpu", torch.float64)
    if getattr(plan, "_theta", None) is None or not torch.equal(plan._theta, t):
        plan.set_model(t[:4].tolist(), float(t[4]))
        plan._theta = t.clone()


class IsamA(torch.autograd.Function):
    """s = A_theta eta.  Backward: A^H g for eta, <dA/dtheta eta, g> for theta."""

    @staticmethod
    def forward(ctx, eta, theta, plan: Plan):
        _apply_theta(plan, theta)
        ctx.plan = plan
        ctx.save_for_backward(eta, theta)
        return plan.forward(eta.contiguous())

    @staticmethod
    def backward(ctx, g):
        eta, theta = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        g = g.contiguous()
        d_eta = plan.adjoint(g) if ctx.needs_input_grad[0] else None
        d_theta = None
        if ctx.needs_input_grad[1]:
            d_theta = torch.from_numpy(plan.param_grad(eta.contiguous(), g))
        return d_eta, d_theta, None


class IsamAH(torch.autograd.Function):
    """x = A_theta^H y.  Backward: A x_bar for y, <dA/dtheta x_bar, y> for theta."""

    @staticmethod
    def forward(ctx, y, theta, plan: Plan):
        _apply_theta(plan, theta)
        ctx.plan = plan
        ctx.save_for_backward(y, theta)
        return plan.adjoint(y.contiguous())

    @staticmethod
    def backward(ctx, xb):
        y, theta = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        xb = xb.contiguous()
        d_y = plan.forward(xb) if ctx.needs_input_grad[0] else None
        d_theta = None
        if ctx.needs_input_grad[1]:
            d_theta = torch.from_numpy(plan.param_grad(xb, y.contiguous()))
        return d_y, d_theta, None


class UnrolledFista(torch.autograd.Function):
    """z^K of K FISTA iterations (Alg. 1, fixed lambda and step 1/L) from z^0 = 0.

    The forward keeps checkpoints every `every` iterations; the backward
    recomputes each segment from its checkpoint and runs the reverse
    recursion (isam_fista_unrolled_vjp)."""

    @staticmethod
    def forward(ctx, s_d, theta, plan: Plan, lam: float, L: float, K: int, every: int, w=None):
        _apply_theta(plan, theta)
        s_d = s_d.contiguous()
        z, ck = plan.fista_unrolled(s_d, lam, L, K, every, w=w, checkpoints=True)
        ctx.plan, ctx.lam, ctx.L, ctx.K, ctx.every, ctx.w = plan, lam, L, K, every, w
        ctx.save_for_backward(s_d, theta, ck)
        return z

    @staticmethod
    def backward(ctx, z_bar):
        s_d, theta, ck = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        grad, s_bar = plan.fista_unrolled_vjp(s_d, ctx.lam, ctx.L, ctx.K, ctx.every, ck,
                                              z_bar.contiguous(),
                                              want_s_bar=ctx.needs_input_grad[0], w=ctx.w)
        d_theta = torch.from_numpy(grad) if ctx.needs_input_grad[1] else None
        return s_bar, d_theta, None, None, None, None, None, None


def model(eta, theta, plan: Plan):
    return IsamA.apply(eta, theta, plan)


def model_adjoint(y, theta, plan: Plan):
    return IsamAH.apply(y, theta, plan)


def unrolled_fista(s_d, theta, plan: Plan, lam: float, L: float, K: int = 20, every: int = 5,
                   w=None):
    return UnrolledFista.apply(s_d, theta, plan, lam, L, K, every, w)


def data_fidelity(s_d, theta, plan: Plan, lam: float, L: float, K: int, every: int, w=None):
    """1/2 ||A_theta z^K(theta) - s_d||^2 with z^K the unrolled reconstruction."""
    z = unrolled_fista(s_d, theta, plan, lam, L, K, every, w)
    r = model(z, theta, plan) - s_d
    return 0.5 * torch.sum(r.double() * r.double())


# ----------------------------------------------------------------------------
# Fitting (a2, a3, z0) over several B-scans of one geometry with Adam
# ----------------------------------------------------------------------------

@dataclass
class CalibResult:
    theta: np.ndarray        # fitted (a1..a4, z0)
    losses: list             # normalised data fidelity per step
    seconds: float           # wall time of the steps


def theta_scales(geom) -> np.ndarray:
    """Units in which Adam moves theta: a_i in radians of phase at the band
    edge (a_i (B/2)^i), z0 in fractions of the full depth range pi/dk."""
    half = 0.5 * (geom.k_max - geom.k_min)
    dk = (geom.k_max - geom.k_min) / (geom.nk - 1)
    return np.array([1 / half, 1 / half ** 2, 1 / half ** 3, 1 / half ** 4, math.pi / dk])


def calibrate(plan: Plan, spectra: list, theta0, lam: list, L: float, K: int = 20,
              every: int = 5, steps: int = 50, lr: float = 1e-2, fit=(1, 2, 4)) -> CalibResult:
    """Adam on the normalised data fidelity summed over `spectra` (device tensors
    of one geometry), moving the components `fit` of theta (default a2, a3, z0)."""
    import time
    scale = torch.from_numpy(theta_scales(plan.geom))
    base = torch.as_tensor(np.asarray(theta0, dtype=np.float64))
    mask = torch.zeros(N_PARAMS, dtype=torch.float64)
    mask[list(fit)] = 1.0
    p = torch.zeros(N_PARAMS, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr)
    norm = sum(float(torch.sum(s.double() ** 2)) for s in spectra)
    losses = []
    t0 = time.perf_counter()
    for _ in range(steps):
        opt.zero_grad()
        theta = base + mask * p * scale
        loss = sum(data_fidelity(s, theta, plan, lm, L, K, every) for s, lm in zip(spectra, lam))
        loss = loss / norm
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    theta = (base + mask * p.detach() * scale).numpy()
    return CalibResult(theta, losses, seconds)
