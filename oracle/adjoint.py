"""Discrete adjoint of the generalized-alpha Newton time stepping (oracle;
test infrastructure only).

Plain definition, for small meshes. One time step is the map
s_n = (y_n, ydot_n) -> s_{n+1}: z = ydot_{n+1} solves F(z; s_n, theta) = 0 with
F = [R_k bar ; R_p ; R_m] at the stage values (§3.2, eq. gen_alpha_def_*), and
y_{n+1} = y_n + dt ydot_n + gamma dt (z - ydot_n). For J = w . y_N the reverse
sweep is
    K^T lam = ydotbar_{n+1} + gamma dt ybar_{n+1},          K = dF/dz,
    ybar_n    = ybar_{n+1} - (dF/dy_n)^T lam,
    ydotbar_n = dt (1 - gamma) ybar_{n+1} - (dF/dydot_n)^T lam,
    dJ/dtheta -= (dF/dtheta)^T lam,
with every Jacobian formed densely by complex-step differentiation of the
step residual (y_{n+1} and the stage values recomputed inside), on the free
dofs. Homogeneous Dirichlet components are identically zero, so they are left
out of the unknowns, and their adjoint components are set to zero.
"""
from __future__ import annotations

import numpy as np

from . import element as el
from . import newton as Nw
from . import system as S

_KEYS_Y = ("u", "p", "v")
_KEYS_YD = ("udot", "pdot", "vdot")


def pack(d, keys):
    return np.concatenate([np.asarray(d[k]).ravel() for k in keys])


def unpack(x, N, keys):
    return {keys[0]: x[:3 * N].reshape(N, 3), keys[1]: x[3 * N:4 * N], keys[2]: x[4 * N:].reshape(N, 3)}


def with_params(prob, mu_e, kappa_e):
    """A shallow copy of the problem with per-element mu, kappa (complex-safe)."""
    q = S.Problem.__new__(S.Problem)
    q.__dict__.update(prob.__dict__)
    me = dict(prob.me)
    me["mu"] = mu_e
    me["kappa"] = kappa_e
    q.me = me
    q.tau = el.tau_m(prob.geo, me)
    return q


def step_residual(prob, yn, ydn, z, t_n, dt, rho_inf=0.5):
    """F = [R_k bar ; R_p ; R_m] (7N) at ydot_{n+1} = z; inputs are packed 7N vectors."""
    N = prob.N
    am, af, gam = S.gen_alpha(rho_inf)
    y1 = yn + dt * ydn + gam * dt * (z - ydn)
    st = S.stage_values(unpack(yn, N, _KEYS_Y), unpack(ydn, N, _KEYS_YD), unpack(y1, N, _KEYS_Y),
                        unpack(z, N, _KEYS_YD), am, af)
    Rm, Rp = S.assemble_residual(prob, st, t_n + af * dt)
    Rk = S.kinematic_residual(st)
    return np.concatenate([Rk.ravel(), Rp, Rm.ravel()])


def free_mask(prob):
    m = prob.dir_mask.ravel()
    return np.concatenate([~m, np.ones(prob.N, bool), ~m])


def _cs_jacobian(fun, x0, cols, h=1e-30):
    out = []
    for c in cols:
        x = x0.astype(np.complex128)
        x[c] += 1j * h
        out.append(fun(x).imag / h)
    return np.stack(out, axis=1)


def forward(prob, nsteps, dt, tol=1e-13):
    """Oracle time stepping from rest; returns the list of packed (y_n, ydot_n)."""
    N = prob.N
    states = [(np.zeros(7 * N), np.zeros(7 * N))]
    yn = unpack(states[0][0], N, _KEYS_Y)
    ydn = unpack(states[0][1], N, _KEYS_YD)
    for n in range(nsteps):
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, n * dt, dt, tol_r=tol, tol_a=1e-300)
        assert info["converged"], info
        states.append((pack(y1, _KEYS_Y), pack(yd1, _KEYS_YD)))
        yn, ydn = y1, yd1
    return states


def gradient(prob, states, w, dt, rho_inf=0.5):
    """dJ/d(mu_e, kappa_e) for J = w . y_N by the reverse sweep above."""
    N = prob.N
    am, af, gam = S.gen_alpha(rho_inf)
    fm = free_mask(prob)
    free = np.flatnonzero(fm)
    ybar = w.copy()
    ydbar = np.zeros(7 * N)
    grad = np.zeros((prob.E, 2))
    nsteps = len(states) - 1
    for n in range(nsteps - 1, -1, -1):
        yn, ydn = states[n]
        _, z = states[n + 1]
        t_n = n * dt
        K = _cs_jacobian(lambda zz: step_residual(prob, yn, ydn, zz, t_n, dt, rho_inf), z, free)[free]
        g = ydbar + gam * dt * ybar
        lam = np.zeros(7 * N)
        lam[free] = np.linalg.solve(K.T, g[free])
        Gy = _cs_jacobian(lambda yy: step_residual(prob, yy, ydn, z, t_n, dt, rho_inf), yn, range(7 * N))
        Gyd = _cs_jacobian(lambda dd: step_residual(prob, yn, dd, z, t_n, dt, rho_inf), ydn, range(7 * N))
        ybar_new = ybar - Gy.T @ lam
        ydbar_new = dt * (1.0 - gam) * ybar - Gyd.T @ lam
        ybar, ydbar = ybar_new * fm, ydbar_new * fm
        # parameters: element e's residual depends only on (mu_e, kappa_e), so
        # one complex evaluation with all elements perturbed gives every dR_e/dtheta_e
        y1 = yn + dt * ydn + gam * dt * (z - ydn)
        st = S.stage_values(unpack(yn, N, _KEYS_Y), unpack(ydn, N, _KEYS_YD), unpack(y1, N, _KEYS_Y),
                            unpack(z, N, _KEYS_YD), am, af)
        es = el.gather(prob.tets, st)
        lm = lam[4 * N:].reshape(N, 3)[prob.tets]
        lp = lam[3 * N:4 * N][prob.tets]
        for k in range(2):
            mu = prob.me["mu"].astype(np.complex128)
            ka = prob.me["kappa"].astype(np.complex128)
            if k == 0:
                mu = mu + 1e-30j * prob.me["mu"]
                scale = prob.me["mu"]
            else:
                ka = ka + 1e-30j * prob.me["kappa"]
                scale = prob.me["kappa"]
            q = with_params(prob, mu, ka)
            Rm_e, Rp_e = el.element_residual(q.geo, q.me, q.tau, es)
            dRm = Rm_e.imag / (1e-30 * scale)[:, None, None]
            dRp = Rp_e.imag / (1e-30 * scale)[:, None]
            grad[:, k] -= np.einsum("eai,eai->e", lm, dRm) + np.einsum("ea,ea->e", lp, dRp)
    return grad


def top_uz_weights(mesh):
    """w with J = w . y = mean of u_z over the top-face nodes (§5.1 block, top face)."""
    X = mesh["X"]
    N = X.shape[0]
    top = np.flatnonzero(np.abs(X[:, 2] - X[:, 2].max()) < 1e-12)
    w = np.zeros(7 * N)
    w[3 * top + 2] = 1.0 / len(top)
    return w
