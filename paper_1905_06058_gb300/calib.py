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


class DataFidelity(torch.autograd.Function):
    """1/2 ||A_theta z - s_d||^2, evaluated by the library (isam_data_fidelity),
    which also returns the residual r = A_theta z - s_d.  Backward: A^H r for z
    and <dA/dtheta z, r> for theta, both from the library, times the incoming
    scalar."""

    @staticmethod
    def forward(ctx, z, theta, plan: Plan, s_d):
        _apply_theta(plan, theta)
        z = z.contiguous()
        value, r = plan.data_fidelity(z, s_d.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(z, theta, r)
        # a device scalar: autograd then runs this node's backward on the same
        # device thread as the other nodes of the plan (a plan's calls must not
        # overlap: they share its workspace)
        return torch.tensor(value, dtype=torch.float64, device=z.device)

    @staticmethod
    def backward(ctx, g):
        z, theta, r = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        gs = float(g)
        d_z = d_theta = None
        if ctx.needs_input_grad[0]:
            d_z = plan.adjoint(r)
            if gs != 1.0:
                d_z = d_z * gs
        if ctx.needs_input_grad[1]:
            d_theta = torch.from_numpy(plan.param_grad(z, r) * gs)
        return d_z, d_theta, None, None


def model(eta, theta, plan: Plan):
    return IsamA.apply(eta, theta, plan)


def model_adjoint(y, theta, plan: Plan):
    return IsamAH.apply(y, theta, plan)


def unrolled_fista(s_d, theta, plan: Plan, lam: float, L: float, K: int = 20, every: int = 5,
                   w=None):
    return UnrolledFista.apply(s_d, theta, plan, lam, L, K, every, w)


def data_fidelity(s_d, theta, plan: Plan, lam: float, L: float, K: int, every: int, w=None):
    """1/2 ||A_theta z^K(theta) - s_d||^2 with z^K the unrolled reconstruction
    (a float64 device scalar; its value and gradient come from the library)."""
    z = unrolled_fista(s_d, theta, plan, lam, L, K, every, w)
    return DataFidelity.apply(z, theta, plan, s_d)


# ----------------------------------------------------------------------------
# Fitting (a2, a3, z0) over several B-scans of one geometry with Adam
# ----------------------------------------------------------------------------

@dataclass
class CalibResult:
    theta: np.ndarray        # theta after the last step
    losses: list             # normalised data fidelity per step, at the theta the step started from
    seconds: float           # wall time of the steps
    best_theta: np.ndarray   # the theta with the lowest loss seen
    best_loss: float


def theta_scales(geom) -> np.ndarray:
    """Units in which Adam moves theta: a_i in radians of phase at the band
    edge (a_i (B/2)^i), z0 in fractions of the full depth range pi/dk."""
    half = 0.5 * (geom.k_max - geom.k_min)
    dk = (geom.k_max - geom.k_min) / (geom.nk - 1)
    return np.array([1 / half, 1 / half ** 2, 1 / half ** 3, 1 / half ** 4, math.pi / dk])


def calibrate(plan: Plan, spectra: list, theta0, lam: list, L: float, K: int = 20,
              every: int = 5, steps: int = 50, lr: float = 5e-2, fit=(1, 2, 4),
              lr_final: float = 0.02, z0_step: float = 1 / 32) -> CalibResult:
    """Adam on the normalised data fidelity summed over `spectra` (device tensors
    of one geometry), moving the components `fit` of theta (default a2, a3, z0).

    The step size follows a half cosine from lr down to lr * lr_final over the
    steps (lr_final = 1 keeps it constant): the fidelity through the unrolled
    solve is not convex in the phase coefficients, and a constant step keeps
    Adam bouncing across the valley it has found.  Adam moves every component
    by about the step size in its own unit; z0 moves in units of z0_step of
    the depth range, a_i in radians at the band edge (theta_scales), so that
    one step shifts the focus by a fraction of a depth pixel, not by tens."""
    import time
    scale = torch.from_numpy(theta_scales(plan.geom))
    scale[4] *= z0_step
    base = torch.as_tensor(np.asarray(theta0, dtype=np.float64))
    mask = torch.zeros(N_PARAMS, dtype=torch.float64)
    mask[list(fit)] = 1.0
    p = torch.zeros(N_PARAMS, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr)
    anneal = lambda i: lr_final + (1.0 - lr_final) * 0.5 * (1.0 + math.cos(math.pi * i / max(steps, 1)))
    sched = torch.optim.lr_scheduler.LambdaLR(opt, anneal)
    norm = sum(float(torch.sum(s.double() ** 2)) for s in spectra)
    losses = []
    best_theta, best_loss = base.numpy().copy(), math.inf
    t0 = time.perf_counter()
    for _ in range(steps):
        opt.zero_grad()
        theta = base + mask * p * scale
        loss = sum(data_fidelity(s, theta, plan, lm, L, K, every) for s, lm in zip(spectra, lam))
        loss = loss / norm
        loss.backward()
        value = float(loss.detach())
        if value < best_loss:
            best_theta, best_loss = theta.detach().numpy().copy(), value
        opt.step()
        sched.step()
        losses.append(value)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    theta = (base + mask * p.detach() * scale).numpy()
    return CalibResult(theta, losses, seconds, best_theta, best_loss)
