"""Global residual, consistent tangent and linear-algebra definitions (oracle;
test infrastructure only).

Unknown ordering of the reduced linear system (§4): x = [x_v ; x_p] with
x_v[3a + i] = Delta vdot of node a, component i, and x_p[a] = Delta pdot.

The consistent tangent is the exact Jacobian of the residual with respect to
the Newton unknowns (§3.3: K entries are partial derivatives of R). With the
kinematic block factorization (eq. K_block_decomposition) the reduced system
(eq. NR_smaller_eqn_1, blocks def_matrix_A / def_matrix_D) is the Jacobian of
[R_m ; R_p] along directions in which Delta udot = (alpha_f gamma dt / alpha_m)
Delta vdot. Through the generalized-alpha relations (eq. gen_alpha_def_*),
a unit Delta vdot_{n+1} moves vdot_{n+alpha_m} by alpha_m, v_{n+alpha_f} by
alpha_f gamma dt, and (through the tied Delta udot) u_{n+alpha_f} by
(alpha_f gamma dt)^2 / alpha_m; a unit Delta pdot moves pdot_{n+alpha_m} by
alpha_m and p_{n+alpha_f} by alpha_f gamma dt. Each column is taken by
complex-step differentiation, which is exact to rounding.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import element as el

CS_H = 1e-30  # complex-step size


def gen_alpha(rho_inf):
    """alpha_m, alpha_f, gamma of the first-order generalized-alpha method (§3.2)."""
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = 1.0 / (1.0 + rho_inf)
    return am, af, af


class Problem:
    """A mesh, a material and a load, with precomputed reference geometry."""

    def __init__(self, mesh, mat, fields=None, load=None):
        self.mesh = mesh
        self.mat = mat
        self.X = mesh["X"]
        self.tets = mesh["tets"].astype(np.int64)
        self.N = self.X.shape[0]
        self.E = self.tets.shape[0]
        self.geo = el.reference_geometry(self.X, self.tets)
        fib = None
        if mat["fibres"]:
            fib = (mesh["fibre_a1"], mesh["fibre_a2"])
        self.me = el.element_material(mat, self.E, fields, fib)
        self.tau = el.tau_m(self.geo, self.me)
        self.load = load or {"p_max": 0.0, "t_ramp": 1.0}
        mask = np.zeros((self.N, 3), dtype=bool)
        d = mesh["dirichlet"]
        mask[d[:, 0], d[:, 1]] = True
        self.dir_mask = mask
        self.dir_vals = np.zeros((self.N, 3))
        self.dir_vals[d[:, 0], d[:, 1]] = mesh["dirichlet_values"]

    # ------------------------------------------------------------ subsets
    def subset(self, elems):
        """Geometry/material restricted to an element subset (for sampling)."""
        g = {k: v[elems] for k, v in self.geo.items()}
        me = dict(self.me)
        me["mu"] = self.me["mu"][elems]
        me["kappa"] = self.me["kappa"][elems]
        if self.me["fib"] is not None:
            k1, k2, H1, H2 = self.me["fib"]
            me["fib"] = (k1[elems], k2[elems], H1[elems], H2[elems])
        return g, me, self.tau[elems]

    # ------------------------------------------------------------ loads
    def load_factor(self, t):
        return min(t / self.load["t_ramp"], 1.0)

    def traction_nodal(self, t):
        """int_{Gamma_H} N_A H_i dGamma for the dead nominal traction
        H = P(t) * traction_dir on the reference faces: each triangle passes a
        third of its area to each vertex."""
        f = np.zeros((self.N, 3))
        tris = self.mesh["traction_tris"].astype(np.int64)
        if tris.shape[0] == 0 or self.load["p_max"] == 0.0:
            return f
        Xt = self.X[tris]
        area = 0.5 * np.linalg.norm(np.cross(Xt[:, 1] - Xt[:, 0], Xt[:, 2] - Xt[:, 0]), axis=1)
        H = self.load["p_max"] * self.load_factor(t) * np.asarray(self.mesh["traction_dir"])
        for a in range(3):
            np.add.at(f, tris[:, a], (area / 3.0)[:, None] * H[None, :])
        return f


def stage_values(yn, ydn, y1, yd1, am, af):
    """ydot_{n+alpha_m} = ydot_n + alpha_m (ydot_{n+1} - ydot_n),
    y_{n+alpha_f} = y_n + alpha_f (y_{n+1} - y_n)  (§3.2)."""
    st = {}
    for k in ("u", "p", "v"):
        st[k] = yn[k] + af * (y1[k] - yn[k])
    for k in ("udot", "pdot", "vdot"):
        st[k] = ydn[k] + am * (yd1[k] - ydn[k])
    return st


def kinematic_residual(st):
    """R_k bar = udot_{n+alpha_m} - v_{n+alpha_f} (eq. gen_alpha_fully_discrete_kinematic_new)."""
    return st["udot"] - st["v"]


def assemble_residual(prob, st, t_alpha):
    """Global R_m [N,3] (with the traction term) and R_p [N] at a stage state."""
    Rm_e, Rp_e = el.element_residual(prob.geo, prob.me, prob.tau, el.gather(prob.tets, st))
    Rm = np.zeros((prob.N, 3), dtype=Rm_e.dtype)
    Rp = np.zeros(prob.N, dtype=Rp_e.dtype)
    for a in range(4):
        np.add.at(Rm, prob.tets[:, a], Rm_e[:, a])
        np.add.at(Rp, prob.tets[:, a], Rp_e[:, a])
    Rm -= prob.traction_nodal(t_alpha)
    return Rm, Rp


def _complex_state(es):
    return {k: v.astype(np.complex128) for k, v in es.items()}


def element_tangent(geo, me, tau, es, ga):
    """Element blocks A [E,4,3,4,3], B [E,4,3,4], C [E,4,4,3], D [E,4,4] of the
    reduced system, as the exact derivative of the element residual along the
    kinematically reduced unknown directions (see module docstring)."""
    am, af, gam, dt = ga
    c_vd, c_v, c_u = am, af * gam * dt, (af * gam * dt) ** 2 / am
    c_pd, c_p = am, af * gam * dt
    E = geo["V"].shape[0]
    A = np.zeros((E, 4, 3, 4, 3))
    B = np.zeros((E, 4, 3, 4))
    C = np.zeros((E, 4, 4, 3))
    D = np.zeros((E, 4, 4))
    base = _complex_state(es)
    for b in range(4):
        for j in range(3):
            st = {k: v.copy() for k, v in base.items()}
            st["u"][:, b, j] += 1j * CS_H * c_u
            st["v"][:, b, j] += 1j * CS_H * c_v
            st["vdot"][:, b, j] += 1j * CS_H * c_vd
            Rm, Rp = el.element_residual(geo, me, tau, st)
            A[:, :, :, b, j] = Rm.imag / CS_H
            C[:, :, b, j] = Rp.imag / CS_H
        st = {k: v.copy() for k, v in base.items()}
        st["p"][:, b] += 1j * CS_H * c_p
        st["pdot"][:, b] += 1j * CS_H * c_pd
        Rm, Rp = el.element_residual(geo, me, tau, st)
        B[:, :, :, b] = Rm.imag / CS_H
        D[:, :, b] = Rp.imag / CS_H
    return A, B, C, D


def element_udot_product(geo, me, tau, es, ga, Rk_e):
    """(1/alpha_m) K_{m,udot} R_k bar and (1/alpha_m) K_{p,udot} R_k bar per
    element (the right-hand-side terms of eq. NR_smaller_eqn_1): the
    derivative along Delta udot_{n+1} = R_k bar / alpha_m, which moves
    u_{n+alpha_f} by alpha_f gamma dt R_k bar / alpha_m."""
    am, af, gam, dt = ga
    st = _complex_state(es)
    st["u"] = st["u"] + 1j * CS_H * (af * gam * dt / am) * Rk_e
    Rm, Rp = el.element_residual(geo, me, tau, st)
    return Rm.imag / CS_H, Rp.imag / CS_H


def dof_v(nodes, comp):
    return 3 * nodes + comp


def assemble_matrix(prob, st, ga):
    """The reduced tangent [[A, B], [C, D]] (4N x 4N, CSR), no Dirichlet."""
    N = prob.N
    A, B, C, D = element_tangent(prob.geo, prob.me, prob.tau, el.gather(prob.tets, st), ga)
    t = prob.tets
    vd = 3 * t[:, :, None] + np.arange(3)        # [E, a, i] velocity dof of (a, i)
    pd = 3 * N + t                               # [E, a]    pressure dof of a
    rA = np.broadcast_to(vd[:, :, :, None, None], A.shape)
    cA = np.broadcast_to(vd[:, None, None, :, :], A.shape)
    rB = np.broadcast_to(vd[:, :, :, None], B.shape)
    cB = np.broadcast_to(pd[:, None, None, :], B.shape)
    rC = np.broadcast_to(pd[:, :, None, None], C.shape)
    cC = np.broadcast_to(vd[:, None, :, :], C.shape)
    rD = np.broadcast_to(pd[:, :, None], D.shape)
    cD = np.broadcast_to(pd[:, None, :], D.shape)
    rows = np.concatenate([rA.ravel(), rB.ravel(), rC.ravel(), rD.ravel()])
    cols = np.concatenate([cA.ravel(), cB.ravel(), cC.ravel(), cD.ravel()])
    vals = np.concatenate([A.ravel(), B.ravel(), C.ravel(), D.ravel()])
    K = sp.coo_matrix((vals, (rows, cols)), shape=(4 * N, 4 * N)).tocsr()
    K.sum_duplicates()
    return K


def assemble_rows(prob, st, ga, nodes):
    """The reduced tangent restricted to the elements that touch ``nodes``:
    the block rows of those nodes are complete, all other rows are partial.
    For sampled parity checks on meshes too large to assemble whole."""
    elems = np.unique(np.nonzero(np.isin(prob.tets, nodes))[0])
    geo, me, tau = prob.subset(elems)
    sub = Problem.__new__(Problem)
    sub.__dict__.update(prob.__dict__)
    sub.tets, sub.geo, sub.me, sub.tau, sub.E = prob.tets[elems], geo, me, tau, len(elems)
    return assemble_matrix(sub, st, ga)


def newton_rhs(prob, st, t_alpha, ga, exact=True):
    """Right-hand side of the reduced system.

    exact=True: -[R_m - (1/a_m) K_{m,udot} Rk ; R_p - (1/a_m) K_{p,udot} Rk]
    (eq. NR_smaller_eqn_1); exact=False: -[R_m ; R_p] as printed in step 5 of
    the multi-corrector stage. Rk is zeroed on Dirichlet displacement
    components (those components never change). Returns (rhs [4N], Rm, Rp, Rk).
    """
    Rm, Rp = assemble_residual(prob, st, t_alpha)
    Rk = kinematic_residual(st) * (~prob.dir_mask)
    gm, gp = np.zeros_like(Rm), np.zeros_like(Rp)
    if exact and np.any(Rk != 0.0):
        es = el.gather(prob.tets, st)
        cm_e, cp_e = element_udot_product(prob.geo, prob.me, prob.tau, es, ga, Rk[prob.tets])
        for a in range(4):
            np.add.at(gm, prob.tets[:, a], cm_e[:, a])
            np.add.at(gp, prob.tets[:, a], cp_e[:, a])
    rhs_v = -(Rm - gm)
    rhs_p = -(Rp - gp)
    rhs = np.concatenate([rhs_v.ravel(), rhs_p])
    return rhs, Rm, Rp, Rk


def dirichlet_dofs(prob):
    return np.flatnonzero(prob.dir_mask.ravel())


def apply_dirichlet(K, rhs, dofs):
    """Constrained velocity-rate dofs: zero row and column, unit diagonal,
    zero right-hand side (homogeneous increments on Gamma_g)."""
    n = K.shape[0]
    keep = np.ones(n)
    keep[dofs] = 0.0
    Dk = sp.diags(keep)
    Kd = (Dk @ K @ Dk).tocsr()
    Kd = Kd + sp.diags(1.0 - keep)
    r = rhs.copy()
    r[dofs] = 0.0
    return Kd.tocsr(), r


def diag_scaling(K, eps=1e-15):
    """W_ii = |A_ii|^{-1/2} if |A_ii| >= eps_diag, else 1 (§4.1)."""
    d = np.abs(K.diagonal())
    w = np.ones_like(d)
    big = d >= eps
    w[big] = 1.0 / np.sqrt(d[big])
    return w


def split_blocks(K, N):
    """Views A (3N x 3N), B (3N x N), C (N x 3N), D (N x N) of the 2x2 block matrix."""
    K = K.tocsr()
    return K[:3 * N, :3 * N], K[:3 * N, 3 * N:], K[3 * N:, :3 * N], K[3 * N:, 3 * N:]


def explicit_schur(K, N):
    """Dense S = D - C A^-1 B (§4.2); for small meshes only."""
    A, B, C, D = split_blocks(K, N)
    AinvB = np.linalg.solve(A.toarray(), B.toarray())
    return D.toarray() - C.toarray() @ AinvB


def schur_hat_diag(K, N):
    """diag of S^ = D - C diag(A)^-1 B (§4.2), with the scalar diagonal of A."""
    A, B, C, D = split_blocks(K, N)
    Bs = sp.diags(1.0 / A.diagonal()) @ B          # diag(A)^-1 B   (3N x N)
    CB = np.asarray(C.multiply(Bs.T.tocsr()).sum(axis=1)).ravel()
    return D.diagonal() - CB


def block_jacobi_inverse(K, N):
    """Inverses of the 3x3 node-diagonal blocks of A."""
    A = split_blocks(K, N)[0].tocsr()
    blocks = np.zeros((N, 3, 3))
    for i in range(3):
        for j in range(3):
            blocks[:, i, j] = np.asarray(A[np.arange(N) * 3 + i, np.arange(N) * 3 + j]).ravel()
    return np.linalg.inv(blocks)


def direct_solve(K, rhs):
    """Direct solve of the assembled system, x = W (W K W)^-1 W rhs with the
    symmetric diagonal scaling W of §4.1 (it leaves x unchanged in exact
    arithmetic): dense LAPACK LU for small systems, SuperLU otherwise (library
    primitives). Without the scaling the velocity and pressure rows differ by
    about ten orders of magnitude and the LU loses digits in the pressure (a
    1e-16 relative change of the entries moved the unscaled solution of a
    16^3-hex cube by 2e-9; the scaled one by 5e-16)."""
    n = K.shape[0]
    w = diag_scaling(K)
    Ks = (sp.diags(w) @ K @ sp.diags(w))
    b = w * rhs
    if n <= 4000:
        return w * np.linalg.solve(Ks.toarray(), b)
    lu = spla.splu(Ks.tocsc(), permc_spec="COLAMD")
    return w * lu.solve(b)


BLOCK_KINDS = ("LDU", "DU", "D", "SIMPLE")


def block_precond_matrix(K, N, kind):
    """The block preconditioner P as a dense matrix, in the expanded forms of
    §4.3–4.4 (small systems only): LDU = the full factorization, i.e. K itself;
    DU = [[A, B], [O, S]]; D = [[A, O], [O, S]]; SIMPLE (H1 = H2 = diag(A)^-1) =
    [[A, A diag(A)^-1 B], [C, D]]; S = D - C A^-1 B."""
    A, B, C, D = (m.toarray() for m in split_blocks(K, N))
    if kind == "LDU":
        return K.toarray()
    if kind == "SIMPLE":
        return np.block([[A, A @ (B / np.diag(A)[:, None])], [C, D]])
    S = explicit_schur(K, N)
    if kind == "DU":
        return np.block([[A, B], [np.zeros((N, 3 * N)), S]])
    if kind == "D":
        return np.block([[A, np.zeros((3 * N, N))], [np.zeros((N, 3 * N)), S]])
    raise ValueError(kind)


def block_precond_apply(K, N, kind, r):
    """z = P^-1 r by the block steps, every sub-system solved exactly (dense
    LAPACK; small systems only). LDU is Algorithm 1: A xhat = r_v,
    r_p' = r_p - C xhat, S x_p = r_p', A x_v = r_v - B x_p. DU: S x_p = r_p,
    A x_v = r_v - B x_p. D: A x_v = r_v, S x_p = r_p. SIMPLE: A xhat = r_v,
    S^ x_p = r_p - C xhat, x_v = xhat - diag(A)^-1 B x_p."""
    A, B, C, D = (m.toarray() for m in split_blocks(K, N))
    rv, rp = r[:3 * N], r[3 * N:]
    if kind == "SIMPLE":
        xhat = np.linalg.solve(A, rv)
        Sh = D - C @ (B / np.diag(A)[:, None])
        xp = np.linalg.solve(Sh, rp - C @ xhat)
        return np.concatenate([xhat - (B @ xp) / np.diag(A), xp])
    S = explicit_schur(K, N)
    if kind == "LDU":
        xhat = np.linalg.solve(A, rv)
        xp = np.linalg.solve(S, rp - C @ xhat)
    elif kind == "DU":
        xp = np.linalg.solve(S, rp)
    elif kind == "D":
        return np.concatenate([np.linalg.solve(A, rv), np.linalg.solve(S, rp)])
    else:
        raise ValueError(kind)
    return np.concatenate([np.linalg.solve(A, rv - B @ xp), xp])


def symmetrized_schur(K, N):
    """Dense S_sym = D - C A_sym^-1 B with A_sym = (A + A^T) / 2: the Schur
    product when the inner A-solve of Algorithm 2 runs on the symmetrized
    velocity block (the paper's conclusion: symmetrize and use CG as the inner
    solver). Small systems only."""
    A, B, C, D = split_blocks(K, N)
    Asym = 0.5 * (A + A.T).toarray()
    return D.toarray() - C.toarray() @ np.linalg.solve(Asym, B.toarray())


def block_jacobi_pcg(Asym, Minv_blocks, b, rtol, maxit=10000):
    """Preconditioned CG for Asym x = b from x = 0 with the 3x3 block-Jacobi
    preconditioner (Minv_blocks [N, 3, 3]), in the textbook form (Saad,
    Iterative Methods for Sparse Linear Systems, Algorithm 9.1); stops when
    ||r|| <= rtol ||b||. Returns (x, iterations)."""
    N = Minv_blocks.shape[0]
    prec = lambda v: np.einsum("nij,nj->ni", Minv_blocks, v.reshape(N, 3)).ravel()
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0
    for k in range(1, maxit + 1):
        q = Asym @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(r) <= rtol * nb:
            return x, k
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit
