"""Gradient of a linear functional of the final state with respect to the
per-element moduli, through generalized-alpha time stepping (discrete adjoint).

``HyelObjective.apply(mu_e, kappa_e, problem)`` returns J = w . y_N after
``problem.nsteps`` Newton time steps from rest; its backward pass returns
dJ/dmu_e and dJ/dkappa_e. The forward pass keeps the state every
``checkpoint_every`` steps; the backward pass recomputes one segment at a time
from its checkpoint and runs ``hyel_adjoint_step`` (transposed nested solve,
partial Jacobians, parameter sensitivities -- all inside libhyel) from the last
step back to the first. This module only moves pointers and orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hyel as H


class AdjointProblem:
    """A mesh on one GPU context, a load schedule and the controls of the
    forward and adjoint solves."""

    def __init__(self, mesh, mat, load, dt, nsteps, weights, checkpoint_every=5, solver=None,
                 adjoint_solver=None, tol_r=1e-6, tol_a=1e-300, device=0, rho_inf=0.5):
        self.mesh, self.mat, self.load = mesh, mat, load
        self.dt, self.nsteps, self.k = dt, nsteps, checkpoint_every
        self.rho_inf, self.tol_r, self.tol_a = rho_inf, tol_r, tol_a
        self.solver = solver or H.solver_params(outer_rtol=1e-10)
        self.adjoint_solver = adjoint_solver or self.solver
        self.device = device
        self.stream = torch.cuda.current_stream(device).cuda_stream
        self.ctx = H.hyel_create(device, self.stream)
        self.inp = H.MeshInputs(mesh, mat, None, load)
        H.hyel_mesh_upload(self.ctx, self.inp.X, self.inp.tets, self.inp.bc, self.inp.mat)
        self.N = mesh["X"].shape[0]
        self.E = mesh["tets"].shape[0]
        self.w = torch.as_tensor(np.asarray(weights, dtype=np.float64), device=f"cuda:{device}")
        self.newton_its = 0
        self.adjoint_its = 0

    def close(self):
        if self.ctx is not None:
            H.hyel_destroy(self.ctx)
            self.ctx = None

    # -- helpers -----------------------------------------------------------
    def set_params(self, mu_e, kappa_e):
        fields = {"mu_e": mu_e.detach().cpu().double().numpy(), "kappa_e": kappa_e.detach().cpu().double().numpy()}
        m, keep = H.material_struct(self.mat, fields, self.mesh)
        H.hyel_update_material(self.ctx, m)

    def _struct(self, y, yd):
        N = self.N
        b, d = y.data_ptr(), yd.data_ptr()
        return H.HyelState(b, b + 8 * 3 * N, b + 8 * 4 * N, d, d + 8 * 3 * N, d + 8 * 4 * N)

    def _tp(self, n):
        return H.time_params(dt=self.dt, t_n=n * self.dt, rho_inf=self.rho_inf, tol_r=self.tol_r,
                             tol_a=self.tol_a)

    def step(self, n, y, yd):
        """Advance (y, yd) in place from t_n to t_{n+1}."""
        st, _ = H.hyel_newton_step(self.ctx, self._tp(n), self.solver, self._struct(y, yd))
        self.newton_its += st.iterations

    def zeros(self):
        return torch.zeros(7 * self.N, dtype=torch.float64, device=self.w.device)


class HyelObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, mu_e, kappa_e, problem):
        problem.set_params(mu_e, kappa_e)
        y, yd = problem.zeros(), problem.zeros()
        ckpt = {0: (y.clone(), yd.clone())}
        for n in range(problem.nsteps):
            problem.step(n, y, yd)
            if (n + 1) % problem.k == 0 and n + 1 < problem.nsteps:
                ckpt[n + 1] = (y.clone(), yd.clone())
        fctx.problem = problem
        fctx.ckpt = ckpt
        # the moduli this forward ran with: another forward on the same problem
        # may replace the context's material before this backward runs
        fctx.params = (mu_e.detach().clone(), kappa_e.detach().clone())
        fctx.shapes = (mu_e.shape, kappa_e.shape, mu_e.dtype, mu_e.device)
        return torch.dot(problem.w, y).reshape(())

    @staticmethod
    def backward(fctx, gJ):
        P = fctx.problem
        P.set_params(*fctx.params)
        ybar = (gJ.to(P.w.device) * P.w).contiguous()
        ydbar = P.zeros()
        grad = torch.zeros((P.E, 4), dtype=torch.float64, device=P.w.device)
        starts = sorted(fctx.ckpt)
        for s in reversed(starts):
            e = min(s + P.k, P.nsteps)
            y, yd = (t.clone() for t in fctx.ckpt[s])
            states = [(y.clone(), yd.clone())]
            for n in range(s, e):  # recompute the segment
                P.step(n, y, yd)
                states.append((y.clone(), yd.clone()))
            for n in range(e - 1, s - 1, -1):
                sn = P._struct(*states[n - s])
                s1 = P._struct(*states[n - s + 1])
                st = H.hyel_adjoint_step(P.ctx, P._tp(n), P.adjoint_solver, sn, s1, ybar.data_ptr(),
                                         ydbar.data_ptr(), grad.data_ptr())
                P.adjoint_its += st.outer_its
        mu_shape, ka_shape, dtype, device = fctx.shapes
        gm = grad[:, 0].to(device=device, dtype=dtype).reshape(mu_shape)
        gk = grad[:, 1].to(device=device, dtype=dtype).reshape(ka_shape)
        return gm, gk, None
