"""Predictor multi-corrector Newton step of the generalized-alpha scheme
(oracle; test infrastructure only). §3.3, each linear system solved directly.

Readings where the paper is silent or garbled:
* eq. gen_alpha_def_y_n_plus_1 has a stray comma; read as
  y_{n+1} = y_n + dt ydot_n + gamma dt (ydot_{n+1} - ydot_n).
* The corrector update uses the previous iterate on the right:
  ydot_{(l)} = ydot_{(l-1)} + Delta ydot, y_{(l)} = y_{(l-1)} + gamma dt Delta ydot.
* ||R_(0)|| of the relative test is the residual of the first evaluation
  (the predictor state).
* Residual components on Dirichlet dofs are excluded from the norm; the
  prescribed values are imposed in the predictor (u = g(t_{n+1}),
  v = dg/dt(t_{n+1}), rates from the generalized-alpha update), and the
  increments there are zero.
"""
from __future__ import annotations

import numpy as np

from . import system as sysm


def dirichlet_targets(prob, t):
    """Prescribed g(t) and dg/dt(t) on Dirichlet components: the values in the
    mesh scale with the same ramp s(t) = min(t / t_ramp, 1) as the load."""
    T = prob.load["t_ramp"]
    s = min(t / T, 1.0)
    sd = 1.0 / T if t < T else 0.0
    return prob.dir_vals * s, prob.dir_vals * sd


def predictor(prob, yn, ydn, t_np1, dt, gam):
    """y_{n+1,(0)} = y_n, ydot_{n+1,(0)} = (gamma-1)/gamma ydot_n (§3.3), then
    Dirichlet components set to their prescribed values at t_{n+1}."""
    y1 = {k: v.copy() for k, v in yn.items()}
    yd1 = {k: (gam - 1.0) / gam * v for k, v in ydn.items()}
    m = prob.dir_mask
    if np.any(m):
        g, gd = dirichlet_targets(prob, t_np1)
        y1["u"] = np.where(m, g, y1["u"])
        y1["v"] = np.where(m, gd, y1["v"])
        # rates consistent with y_{n+1} = y_n + dt ydot_n + gamma dt (ydot_{n+1} - ydot_n)
        for yk, ydk in (("u", "udot"), ("v", "vdot")):
            rate = ydn[ydk] + (y1[yk] - yn[yk] - dt * ydn[ydk]) / (gam * dt)
            yd1[ydk] = np.where(m, rate, yd1[ydk])
    return y1, yd1


def corrector_update(y1, yd1, dyd, gam, dt):
    """ydot_{n+1,(l)} = ydot_{n+1,(l-1)} + Delta ydot,
    y_{n+1,(l)} = y_{n+1,(l-1)} + gamma dt Delta ydot (§3.3, step 7)."""
    y = dict(y1)
    yd = dict(yd1)
    for yk, ydk in (("u", "udot"), ("p", "pdot"), ("v", "vdot")):
        if ydk in dyd:
            yd[ydk] = yd1[ydk] + dyd[ydk]
            y[yk] = y1[yk] + gam * dt * dyd[ydk]
    return y, yd


def newton_step(prob, yn, ydn, t_n, dt, rho_inf=0.5, tol_r=1e-6, tol_a=1e-6, l_max=20,
                exact_rhs=True, record=None):
    """One generalized-alpha time step by Newton with a direct linear solve.

    Returns (y_{n+1}, ydot_{n+1}, info) with info = {iterations, converged,
    norms}. ``record`` (a list) receives per-iteration (K, rhs, dx) tuples when
    given.
    """
    am, af, gam = sysm.gen_alpha(rho_inf)
    ga = (am, af, gam, dt)
    t_alpha = t_n + af * dt
    y1, yd1 = predictor(prob, yn, ydn, t_n + dt, dt, gam)
    dofs = sysm.dirichlet_dofs(prob)
    mask = prob.dir_mask
    norms = []
    norm0 = None
    for l in range(1, l_max + 1):
        st = sysm.stage_values(yn, ydn, y1, yd1, am, af)
        rhs, Rm, Rp, Rk = sysm.newton_rhs(prob, st, t_alpha, ga, exact=exact_rhs)
        free = ~mask
        nrm = np.sqrt(np.sum(Rk[free] ** 2) + np.sum(Rp ** 2) + np.sum(Rm[free] ** 2))
        norms.append(nrm)
        if norm0 is None:
            norm0 = nrm
        if nrm / norm0 <= tol_r or nrm <= tol_a:
            return y1, yd1, {"iterations": l - 1, "converged": True, "norms": norms}
        K = sysm.assemble_matrix(prob, st, ga)
        Kd, r = sysm.apply_dirichlet(K, rhs, dofs)
        dx = sysm.direct_solve(Kd, r)
        if record is not None:
            record.append((Kd, r, dx))
        N = prob.N
        dvd = dx[:3 * N].reshape(N, 3)
        dpd = dx[3 * N:]
        # eq. NR_smaller_eqn_2
        dud = (af * gam * dt / am) * dvd - Rk / am
        dud = np.where(mask, 0.0, dud)
        y1, yd1 = corrector_update(y1, yd1, {"udot": dud, "pdot": dpd, "vdot": dvd}, gam, dt)
    return y1, yd1, {"iterations": l_max, "converged": False, "norms": norms}
