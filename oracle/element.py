"""P1 tetrahedral element residuals of the VMS formulation (oracle; test
infrastructure only).

Follows the residual formulas of Appendix A, written in the reference
configuration:

  R_p,A   = int J N_A (beta pdot + v_i,i)
            + sum_e int tau_M N_A,i (rho J vdot_i - P~_iJ,J + J p_,i - rho J b_i)
  R_m,A^i = int N_A J rho vdot_i + N_A,I P~_iI - N_A,i J p - N_A J rho b_i
            - int_{Gamma_H} N_A H_i      (the traction term lives in ``system``)

with N_A,i = N_A,I F^-1_Ii and p_,i = p_,I F^-1_Ii. For P1 elements F and P~
are constant per element, so P~_iJ,J = 0. Every integral uses the symmetric
4-point rule (barycentric (a,b,b,b) and permutations, a = (5+3 sqrt5)/20,
b = (5-sqrt5)/20, weights V/4); the paper does not state its quadrature.
tau_M = c_m h^e/(c rho0) with h^e the longest reference edge (§3.1).

All arithmetic is complex-safe for complex-step differentiation.
"""
from __future__ import annotations

import numpy as np

from . import constitutive as cm

QA = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
QB = (5.0 - np.sqrt(5.0)) / 20.0
# NQ[q, A] = N_A at quadrature point q
NQ = np.array([[QA, QB, QB, QB], [QB, QA, QB, QB], [QB, QB, QA, QB], [QB, QB, QB, QA]])
_DN_DXI = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def reference_geometry(X, tets):
    """Shape-function gradients G[e, A, I] = dN_A/dX_I, volume V[e] and the
    longest edge h[e] of each tetrahedron in the reference configuration."""
    Xe = X[tets]
    Jxi = np.stack([Xe[:, 1] - Xe[:, 0], Xe[:, 2] - Xe[:, 0], Xe[:, 3] - Xe[:, 0]], axis=-1)
    V = cm.det3(Jxi) / 6.0
    Jinv = cm.inv3(Jxi)  # [e, a, I] = dxi_a / dX_I
    G = np.einsum("Aa,eaI->eAI", _DN_DXI, Jinv)
    h = np.max(np.stack([np.linalg.norm(Xe[:, a] - Xe[:, b], axis=1) for a, b in _EDGES], 1), 1)
    return {"G": G, "V": V, "h": h}


def element_material(mat, n_tets, fields=None, fibres=None):
    """Per-element material arrays: mu, kappa, tau_M inputs, fibre data."""
    fields = fields or {}
    mu = np.asarray(fields.get("mu_e", np.full(n_tets, mat["mu"])), dtype=np.float64)
    kappa = np.asarray(fields.get("kappa_e", np.full(n_tets, mat["kappa"])), dtype=np.float64)
    out = {"mu": mu, "kappa": kappa, "rho0": mat["rho0"], "vol": mat["vol"],
           "body": np.asarray(mat["body"], dtype=np.float64), "c_m": mat["c_m"], "fib": None}
    if mat["fibres"]:
        k1 = np.asarray(fields.get("k1_e", np.full(n_tets, mat["k1"])), dtype=np.float64)
        k2 = np.asarray(fields.get("k2_e", np.full(n_tets, mat["k2"])), dtype=np.float64)
        H1, H2 = cm.structure_tensors(fibres[0], fibres[1], mat["kd"])
        out["fib"] = (k1, k2, H1, H2)
    return out


def tau_m(geo, me):
    """tau_M^e = c_m h^e / (c rho0) (§3.1), c from the element's moduli."""
    c = cm.wave_speed(me["mu"], me["kappa"], me["rho0"], me["vol"])
    return me["c_m"] * geo["h"] / (c * me["rho0"])


def gather(tets, st):
    """Element-local copies of a nodal state dict (u, v, vdot [N,3]; p, pdot [N])."""
    return {k: st[k][tets] for k in ("u", "v", "p", "vdot", "pdot")}


def element_residual(geo, me, tau, es):
    """Element residual vectors R_m [E,4,3] and R_p [E,4] (Appendix A) at the
    stage values es = {u, p, v at n+alpha_f; vdot, pdot at n+alpha_m}."""
    G, V = geo["G"], geo["V"]
    u, v, p, vd, pd = es["u"], es["v"], es["p"], es["vdot"], es["pdot"]
    b = me["body"]
    F = np.eye(3) + np.einsum("eAi,eAI->eiI", u, G)
    P, J, Fi = cm.piola_dev(F, me["mu"], me["fib"])
    n = np.einsum("eAI,eIi->eAi", G, Fi)            # N_A,i
    gradv = np.einsum("eAi,eAj->eij", v, n)         # v_i,j
    divv = gradv[:, 0, 0] + gradv[:, 1, 1] + gradv[:, 2, 2]
    gradp = np.einsum("eA,eAi->ei", p, n)           # p_,i
    pq = np.einsum("qA,eA->eq", NQ, p)
    pdq = np.einsum("qA,eA->eq", NQ, pd)
    vdq = np.einsum("qA,eAi->eqi", NQ, vd)
    rho, beta, _, _ = cm.rho_beta(pq, me["kappa"][:, None], me["rho0"], me["vol"])
    wJ = (V / 4.0) * J                              # quadrature weight times J
    # momentum: inertia and body force, stress divergence (weak), pressure
    inert = np.einsum("qA,eq,eqi->eAi", NQ, rho * wJ[:, None], vdq - b)
    stress = V[:, None, None] * np.einsum("eAI,eiI->eAi", G, P)
    pres = n * (wJ * pq.sum(axis=1))[:, None, None]
    Rm = inert + stress - pres
    # mass: compressibility and divergence, plus the tau_M stabilisation
    mass = np.einsum("qA,eq->eA", NQ, wJ[:, None] * (beta * pdq + divv[:, None]))
    strong = rho[:, :, None] * J[:, None, None] * (vdq - b) + (J[:, None] * gradp)[:, None, :]
    stab = (tau * V / 4.0)[:, None] * np.einsum("eAi,eqi->eA", n, strong)
    Rp = mass + stab
    return Rm, Rp
