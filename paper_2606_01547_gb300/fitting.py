"""Lens-model fitting on top of the batched likelihood (the paper's lens-modelling section:
particle swarm optimisation as in lenstronomy, and L-BFGS with automatic-differentiation
gradients).  Both are host-side orchestration only: every likelihood and gradient evaluation
is one call into the CUDA library (lens_sim_grad), batched over all particles or starts.

Parameters are the 15 free parameters of lens_sim_grad in its order: EPL_E1E2 (theta_E,
gamma, e1, e2, cx, cy), SHEAR (g1, g2), SERSIC_ELLIPSE (amp, R, n, e1, e2, cx, cy).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import lenssim
from . import workloads as W

# Box of the priors the workloads draw from (used to bound the swarm).
PRIOR_LO = np.array([0.8, 1.8, -0.15, -0.15, -0.05, -0.05, -0.08, -0.08, 5.0, 0.05, 0.5, -0.15, -0.15, -0.1, -0.1],
                    np.float32)
PRIOR_HI = np.array([1.4, 2.2, 0.15, 0.15, 0.05, 0.05, 0.08, 0.08, 15.0, 0.5, 4.0, 0.15, 0.15, 0.1, 0.1],
                    np.float32)


@dataclasses.dataclass
class FitResult:
    params: np.ndarray        # [n, 15] best parameters
    logL: np.ndarray          # [n] log-likelihood at them
    history: list             # best logL per iteration
    evaluations: int          # likelihood evaluations (parameter points) issued


def lbfgs_fit(sim: lenssim.Simulator, system: W.LensSystem, data: torch.Tensor, sigma_bkg: float, t_exp: float,
              starts: np.ndarray, iters: int = 50, lr: float = 1.0, subhalo_table: int = -1,
              restarts: int = 10, scale: Optional[np.ndarray] = None) -> FitResult:
    """Maximise logL from each row of `starts` ([n, 15]) with L-BFGS (strong-Wolfe line search).

    The n problems are independent; their negative log-likelihoods are summed so that one
    batched lens_sim_grad call serves all of them at every function evaluation.  L-BFGS runs on
    parameters divided by `scale` (default: the prior widths), which evens out the very different
    sensitivities of the 15 parameters, and is restarted with a fresh history from the best point
    seen (up to `restarts` times, `iters` iterations each) until a restart no longer improves the
    summed likelihood.  Points outside the profiles' domain (non-finite likelihood) count as a
    very large loss, so the line search backs off from them; the best finite point is returned."""
    sc = torch.tensor(np.asarray(PRIOR_HI - PRIOR_LO if scale is None else scale, np.float32), device=data.device)
    Z = (torch.tensor(np.asarray(starts, np.float32), device=data.device) / sc).requires_grad_(True)
    history = []
    evals = [0]
    best = {"total": -float("inf"), "P": (Z * sc).detach().clone()}

    def closure_for(opt):
        def closure():
            opt.zero_grad()
            L = lenssim.LensLogLike.apply(Z * sc, sim, system, data, sigma_bkg, t_exp, subhalo_table)
            evals[0] += Z.shape[0]
            if not bool(torch.isfinite(L).all()):
                # outside the profiles' domain (|e| >= 1, n <= 0, ...): a large loss with zero
                # gradient, so that the line search backs off
                loss = (Z * 0.0).sum() + 1e30
                loss.backward()
                return loss
            total = float(L.detach().sum())
            if total > best["total"]:
                best["total"] = total
                best["P"] = (Z * sc).detach().clone()
            loss = -L.sum()
            loss.backward()
            history.append(float(L.detach().max()))
            return loss
        return closure

    prev = -float("inf")
    for _ in range(max(1, restarts)):
        opt = torch.optim.LBFGS([Z], lr=lr, max_iter=iters, history_size=20, line_search_fn="strong_wolfe",
                                tolerance_grad=1e-12, tolerance_change=1e-14)
        opt.step(closure_for(opt))
        with torch.no_grad():
            Z.copy_(best["P"] / sc)   # restart from the best point seen
        if best["total"] <= prev + 1e-7 * abs(prev):
            break
        prev = best["total"]
    P = best["P"]
    with torch.no_grad():
        L = sim.grad(system, data, sigma_bkg, t_exp, P, want_grad=False, subhalo_table=subhalo_table)
    return FitResult(P.cpu().numpy(), L.cpu().numpy(), history, evals[0] + P.shape[0])


def pso_fit(sim: lenssim.Simulator, system: W.LensSystem, data: torch.Tensor, sigma_bkg: float, t_exp: float,
            n_particles: int = 64, iters: int = 50, lo: Optional[np.ndarray] = None, hi: Optional[np.ndarray] = None,
            seed: int = 0, inertia: float = 0.7, c_cognitive: float = 1.5, c_social: float = 1.5,
            subhalo_table: int = -1) -> FitResult:
    """Particle swarm optimisation (Kennedy & Eberhart 1995) of logL inside the box [lo, hi].

    Each iteration evaluates the whole swarm in one batched likelihood call; particles move by
    v <- w v + c1 r1 (pbest - x) + c2 r2 (gbest - x), x <- clip(x + v, lo, hi)."""
    lo = PRIOR_LO if lo is None else np.asarray(lo, np.float32)
    hi = PRIOR_HI if hi is None else np.asarray(hi, np.float32)
    dev = data.device
    g = torch.Generator(device="cpu").manual_seed(seed)
    lo_t = torch.tensor(lo, device=dev)
    hi_t = torch.tensor(hi, device=dev)
    span = hi_t - lo_t
    x = lo_t + span * torch.rand((n_particles, 15), generator=g).to(dev)
    v = 0.1 * span * (torch.rand((n_particles, 15), generator=g).to(dev) - 0.5)

    def evaluate(pts):
        L = sim.grad(system, data, sigma_bkg, t_exp, pts, want_grad=False, subhalo_table=subhalo_table)
        return torch.nan_to_num(L, nan=-3.0e38, neginf=-3.0e38)

    f = evaluate(x)
    pbest, pbest_f = x.clone(), f.clone()
    k = int(torch.argmax(pbest_f))
    gbest, gbest_f = pbest[k].clone(), float(pbest_f[k])
    history = [gbest_f]
    evals = n_particles
    for _ in range(iters):
        r1 = torch.rand((n_particles, 15), generator=g).to(dev)
        r2 = torch.rand((n_particles, 15), generator=g).to(dev)
        v = inertia * v + c_cognitive * r1 * (pbest - x) + c_social * r2 * (gbest[None] - x)
        x = torch.minimum(torch.maximum(x + v, lo_t), hi_t)
        f = evaluate(x)
        evals += n_particles
        better = f > pbest_f
        pbest[better] = x[better]
        pbest_f[better] = f[better]
        k = int(torch.argmax(pbest_f))
        if float(pbest_f[k]) > gbest_f:
            gbest, gbest_f = pbest[k].clone(), float(pbest_f[k])
        history.append(gbest_f)
    return FitResult(gbest.cpu().numpy()[None], np.array([gbest_f]), history, evals)
