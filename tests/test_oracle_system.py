"""Pins of the oracle's time integration, consistent tangent and linear algebra.

* generalized-alpha (§3.2) on ydot = lambda y: the amplification matrix's
  spectral radius tends to rho_inf as lambda dt -> -inf, the scheme is second
  order, and the predictor is consistent with eq. gen_alpha_def_y_n_plus_1;
* the complex-step tangent equals a central finite-difference Jacobian taken
  through the whole pipeline (perturb ydot_{n+1}, rebuild y_{n+1} and the
  stage values, reassemble the residual);
* at the stress-free reference state the tangent equals its closed form:
  consistent P1 mass, linearised deviatoric elasticity, discrete gradient and
  divergence, tau_M Laplacian;
* the kinematic block factorization (eq. K_block_decomposition): the full
  7-dof-per-node Newton system solved directly equals the two-stage solve;
* Newton converges quadratically (third residual scales with load^4);
* the LDU identity, the S^ diagonal and the diagonal scaling definitions.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1809_06350_gb300 import inputs
from oracle import element as el
from oracle import newton as Nw
from oracle import system as S


# ------------------------------------------------------------ generalized-alpha

def _scalar_step(lam, y, yd, dt, rho_inf):
    am, af, gam = S.gen_alpha(rho_inf)
    z = np.zeros(1)
    yn = {"u": np.array([y]), "p": z, "v": z}
    ydn = {"udot": np.array([yd]), "pdot": z, "vdot": z}
    y1 = {k: v.copy() for k, v in yn.items()}
    yd1 = {k: (gam - 1) / gam * v for k, v in ydn.items()}
    for _ in range(2):  # linear: one correction is exact, the second is ~0
        st = S.stage_values(yn, ydn, y1, yd1, am, af)
        R = st["udot"] - lam * st["u"]
        d = -R / (am - lam * af * gam * dt)
        y1, yd1 = Nw.corrector_update(y1, yd1, {"udot": d}, gam, dt)
    # predictor consistency: y_{n+1} = y_n + dt ydot_n + gamma dt (ydot_{n+1} - ydot_n)
    terms = abs(y) + abs(dt * yd) + abs(gam * dt * yd1["udot"][0]) + abs(gam * dt * yd)
    assert abs(y1["u"][0] - (y + dt * yd + gam * dt * (yd1["udot"][0] - yd))) <= 1e-14 * terms
    return y1["u"][0], yd1["udot"][0]


@pytest.mark.parametrize("rho_inf", [0.0, 0.5, 1.0])
def test_gen_alpha_high_frequency_spectral_radius(rho_inf):
    # for rho_inf = 0 the limit is a defective double zero: the eigenvalues
    # approach it like |lambda dt|^-1/2, hence the large |lambda dt|
    lam, dt = -1e14, 1.0
    cols = [_scalar_step(lam, 1.0, 0.0, dt, rho_inf), _scalar_step(lam, 0.0, 1.0, dt, rho_inf)]
    Amp = np.array(cols).T
    assert np.max(np.abs(np.linalg.eigvals(Amp))) == pytest.approx(rho_inf, abs=1e-6)


def test_gen_alpha_second_order():
    lam = -1.3
    errs = []
    for nsteps in (40, 80, 160):
        dt = 1.0 / nsteps
        y, yd = 1.0, lam
        for _ in range(nsteps):
            y, yd = _scalar_step(lam, y, yd, dt, 0.5)
        errs.append(abs(y - np.exp(lam)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


# ------------------------------------------------------------ tangent

def _problem(kind):
    if kind == "hgo":
        m = inputs.tube_mesh(2, 8, 2)
        mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.1)
        fields = inputs.element_fields(m["tets"].shape[0], mat, seed=4, with_fibres=True)
    elif kind == "incompressible":
        m = inputs.cube_mesh(2, jitter=0.05, seed=5)
        mat = inputs.material_nh(1e5, np.inf, 1e3, body=(0.3, -0.2, -9.81))
        fields = inputs.element_fields(m["tets"].shape[0], mat, seed=6)
    else:
        m = inputs.cube_mesh(2, jitter=0.05, seed=7)
        mat = inputs.material_nh(1e5, 1e6, 1e3, body=(0.3, -0.2, -9.81))
        fields = inputs.element_fields(m["tets"].shape[0], mat, seed=8)
    return S.Problem(m, mat, fields=fields, load={"p_max": 1e4, "t_ramp": 1.0})


def _random_newton_iterate(prob, seed, dt, gam):
    h = np.cbrt(prob.geo["V"].mean())
    yn = inputs.random_state(prob.N, seed=seed, u_scale=0.03 * h, v_scale=0.05, p_scale=3e3)
    ydn = inputs.random_state(prob.N, seed=seed + 1, u_scale=0.0, v_scale=0.05, p_scale=3e3,
                              rate_scale=5.0)
    ydn = {"udot": ydn["udot"], "pdot": ydn["pdot"], "vdot": ydn["vdot"]}
    yn = {k: yn[k] for k in ("u", "p", "v")}
    yd1 = {k: v * 0.7 + 0.1 for k, v in ydn.items()}
    y1 = {k: yn[k] + dt * ydn[k + "dot"] + gam * dt * (yd1[k + "dot"] - ydn[k + "dot"])
          for k in ("u", "p", "v")}
    return yn, ydn, y1, yd1


@pytest.mark.parametrize("kind", ["gibbs", "incompressible", "hgo"])
def test_tangent_equals_finite_difference_jacobian(kind):
    prob = _problem(kind)
    dt, rho_inf = 1e-3, 0.5
    am, af, gam = S.gen_alpha(rho_inf)
    yn, ydn, y1, yd1 = _random_newton_iterate(prob, 21, dt, gam)
    st = S.stage_values(yn, ydn, y1, yd1, am, af)
    K = S.assemble_matrix(prob, st, (am, af, gam, dt)).toarray()
    N = prob.N

    def residual(yd1p):
        y1p = {k: yn[k] + dt * ydn[k + "dot"] + gam * dt * (yd1p[k + "dot"] - ydn[k + "dot"])
               for k in ("u", "p", "v")}
        s = S.stage_values(yn, ydn, y1p, yd1p, am, af)
        Rm, Rp = S.assemble_residual(prob, s, 0.0)
        return np.concatenate([Rm.ravel(), Rp])

    Kfd = np.zeros_like(K)
    tie = af * gam * dt / am  # Delta udot = tie * Delta vdot (kinematic factorization)
    for col in range(4 * N):
        dp = {k: v.copy() for k, v in yd1.items()}
        dm = {k: v.copy() for k, v in yd1.items()}
        if col < 3 * N:
            a, i = divmod(col, 3)
            eps = 1e-3
            for d, s in ((dp, 1), (dm, -1)):
                d["vdot"][a, i] += s * eps
                d["udot"][a, i] += s * eps * tie
        else:
            a = col - 3 * N
            eps = 1.0
            dp["pdot"][a] += eps
            dm["pdot"][a] -= eps
        Kfd[:, col] = (residual(dp) - residual(dm)) / (2 * eps)
    for rows, cols in ((slice(0, 3 * N), slice(0, 3 * N)), (slice(0, 3 * N), slice(3 * N, None)),
                       (slice(3 * N, None), slice(0, 3 * N)), (slice(3 * N, None), slice(3 * N, None))):
        blk, fd = K[rows, cols], Kfd[rows, cols]
        assert np.max(np.abs(blk - fd)) <= 2e-6 * np.max(np.abs(blk)), (kind, rows, cols)


def test_tangent_closed_form_at_reference_state():
    """Zero state, no load, no body force: A = a_m rho0 M + c^2/a_m K_lin,
    B = -c (V/4) g_Ai, C = a_m tau rho0 (V/4) g_Aj + c (V/4) g_Bj,
    D = a_m M / kappa + c tau V g_A . g_B,  c = alpha_f gamma dt, with
    M_AB = V (1 + delta_AB)/20 and K_lin = V mu [d_ij g_A.g_B + g_Aj g_Bi - 2/3 g_Ai g_Bj]."""
    m = inputs.cube_mesh(2, jitter=0.05, seed=3)
    mu, kappa, rho0 = 1e5, 1e6, 1e3
    prob = S.Problem(m, inputs.material_nh(mu, kappa, rho0))
    dt = 1e-3
    am, af, gam = S.gen_alpha(0.5)
    st = inputs.zero_state(prob.N)
    K = S.assemble_matrix(prob, st, (am, af, gam, dt)).toarray()
    X, t = m["X"], m["tets"].astype(np.int64)
    Mx = np.concatenate([np.ones((t.shape[0], 4, 1)), X[t]], axis=2)
    g = np.swapaxes(np.linalg.inv(Mx)[:, 1:, :], 1, 2)          # [e, A, I]
    V = np.abs(np.linalg.det(Mx)) / 6.0
    tau = prob.tau
    c = af * gam * dt
    N = prob.N
    Kc = np.zeros_like(K)
    Mloc = (np.ones((4, 4)) + np.eye(4)) / 20.0
    I3 = np.eye(3)
    for e in range(t.shape[0]):
        gg = g[e] @ g[e].T
        for A in range(4):
            for B in range(4):
                a_, b_ = t[e, A], t[e, B]
                Klin = V[e] * mu * (I3 * gg[A, B] + np.outer(g[e, B], g[e, A])
                                    - 2.0 / 3.0 * np.outer(g[e, A], g[e, B]))
                Ablk = am * rho0 * V[e] * Mloc[A, B] * I3 + c * c / am * Klin
                Kc[3 * a_:3 * a_ + 3, 3 * b_:3 * b_ + 3] += Ablk
                Kc[3 * a_:3 * a_ + 3, 3 * N + b_] += -c * V[e] / 4.0 * g[e, A]
                Kc[3 * N + a_, 3 * b_:3 * b_ + 3] += (am * tau[e] * rho0 * V[e] / 4.0 * g[e, A]
                                                      + c * V[e] / 4.0 * g[e, B])
                Kc[3 * N + a_, 3 * N + b_] += (am * V[e] * Mloc[A, B] / kappa
                                              + c * tau[e] * V[e] * gg[A, B])
    for rows, cols in ((slice(0, 3 * N), slice(0, 3 * N)), (slice(0, 3 * N), slice(3 * N, None)),
                       (slice(3 * N, None), slice(0, 3 * N)), (slice(3 * N, None), slice(3 * N, None))):
        assert np.max(np.abs(K[rows, cols] - Kc[rows, cols])) <= 1e-12 * np.max(np.abs(Kc[rows, cols]))


def test_A_block_symmetric_without_inertia_load():
    """A is symmetric when rho J (vdot - b) = 0 (hyperelastic major symmetry)."""
    prob = _problem("hgo")
    dt = 1e-3
    am, af, gam = S.gen_alpha(0.5)
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=2, u_scale=0.05 * h, v_scale=0.05, p_scale=2e3)
    st["vdot"][:] = 0.0
    K = S.assemble_matrix(prob, st, (am, af, gam, dt)).toarray()
    A = K[:3 * prob.N, :3 * prob.N]
    assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A))


def _full_system(prob, yn, ydn, y1, yd1, dt, rho_inf, t_alpha):
    """The 7-dof-per-node Newton system [Delta udot, Delta pdot, Delta vdot]
    with rows [R_k bar ; R_p ; R_m], by complex step of the element residual."""
    am, af, gam = S.gen_alpha(rho_inf)
    N = prob.N
    st = S.stage_values(yn, ydn, y1, yd1, am, af)
    Rm, Rp = S.assemble_residual(prob, st, t_alpha)
    Rk = S.kinematic_residual(st)
    n = 7 * N
    K = np.zeros((n, n))
    h = 1e-30
    es = el.gather(prob.tets, st)
    cs = {k: v.astype(np.complex128) for k, v in es.items()}
    # column blocks: udot (0..3N), pdot (3N..4N), vdot (4N..7N)
    for a in range(N):
        elems, loc = np.nonzero(prob.tets == a)
        sub_geo, sub_me, sub_tau = prob.subset(elems)
        for kind in ("udot", "pdot", "vdot"):
            comps = range(1) if kind == "pdot" else range(3)
            for i in comps:
                s = {k: v[elems].copy() for k, v in cs.items()}
                if kind == "udot":
                    s["u"][np.arange(len(elems)), loc, i] += 1j * h * af * gam * dt
                    col = 3 * a + i
                elif kind == "pdot":
                    s["p"][np.arange(len(elems)), loc] += 1j * h * af * gam * dt
                    s["pdot"][np.arange(len(elems)), loc] += 1j * h * am
                    col = 3 * N + a
                else:
                    s["v"][np.arange(len(elems)), loc, i] += 1j * h * af * gam * dt
                    s["vdot"][np.arange(len(elems)), loc, i] += 1j * h * am
                    col = 4 * N + 3 * a + i
                Rme, Rpe = el.element_residual(sub_geo, sub_me, sub_tau, s)
                dRm = np.zeros((N, 3))
                dRp = np.zeros(N)
                for b in range(4):
                    np.add.at(dRm, prob.tets[elems, b], Rme[:, b].imag / h)
                    np.add.at(dRp, prob.tets[elems, b], Rpe[:, b].imag / h)
                K[3 * N:4 * N, col] = dRp
                K[4 * N:, col] = dRm.ravel()
    # kinematic rows: d(udot_am - v_af) = a_m d udot - a_f gamma dt d vdot
    K[np.arange(3 * N), np.arange(3 * N)] = am
    K[np.arange(3 * N), 4 * N + np.arange(3 * N)] = -af * gam * dt
    r = -np.concatenate([Rk.ravel(), Rp, Rm.ravel()])
    return K, r


def test_kinematic_factorization_two_stage_equals_full_solve():
    prob = _problem("gibbs")
    dt, rho_inf = 1e-3, 0.5
    am, af, gam = S.gen_alpha(rho_inf)
    yn, ydn, y1, yd1 = _random_newton_iterate(prob, 31, dt, gam)
    for k in ("udot", "vdot"):
        yd1[k] = np.where(prob.dir_mask, 0.0, yd1[k])
    t_alpha = 0.3
    N = prob.N
    Kf, rf = _full_system(prob, yn, ydn, y1, yd1, dt, rho_inf, t_alpha)
    dm = np.flatnonzero(prob.dir_mask.ravel())
    fixed = np.concatenate([dm, 4 * N + dm])  # constrained udot and vdot components
    keep = np.ones(7 * N)
    keep[fixed] = 0
    Kf = Kf * keep[:, None] * keep[None, :] + np.diag(1 - keep)
    rf = rf * keep
    xf = np.linalg.solve(Kf, rf)
    st = S.stage_values(yn, ydn, y1, yd1, am, af)
    ga = (am, af, gam, dt)
    for exact in (True, False):
        rhs, Rm, Rp, Rk = S.newton_rhs(prob, st, t_alpha, ga, exact=exact)
        K = S.assemble_matrix(prob, st, ga)
        Kd, r = S.apply_dirichlet(K, rhs, S.dirichlet_dofs(prob))
        x = S.direct_solve(Kd, r)
        dvd = x[:3 * N].reshape(N, 3)
        dud = np.where(prob.dir_mask, 0.0, (af * gam * dt / am) * dvd - Rk / am)
        xr = np.concatenate([dud.ravel(), x[3 * N:], dvd.ravel()])
        err = np.linalg.norm(xr - xf) / np.linalg.norm(xf)
        if exact:
            assert err < 1e-10
        else:  # the printed step-5 right-hand side drops the R_k terms
            assert err > 1e-6


def test_newton_quadratic_convergence():
    m = inputs.cube_mesh(3, jitter=0.05, seed=0)
    res = []
    for pmax in (2e4, 2e5):
        prob = S.Problem(m, inputs.material_nh(1e5, 1e6, 1e3), load={"p_max": pmax, "t_ramp": 1e-3})
        z = inputs.zero_state(prob.N)
        _, _, info = Nw.newton_step(prob, z, z, 0.0, 1e-3, tol_r=1e-13, tol_a=0.0)
        res.append(info["norms"])
    # e_2 ~ P^2, e_3 ~ e_2^2 ~ P^4 under exact Newton
    assert res[1][1] / res[0][1] == pytest.approx(100.0, rel=0.1)
    assert res[1][2] / res[0][2] == pytest.approx(1e4, rel=0.2)


def test_ldu_identity_schur_and_scaling():
    prob = _problem("gibbs")
    dt = 1e-3
    am, af, gam = S.gen_alpha(0.5)
    yn, ydn, y1, yd1 = _random_newton_iterate(prob, 41, dt, gam)
    st = S.stage_values(yn, ydn, y1, yd1, am, af)
    K = S.assemble_matrix(prob, st, (am, af, gam, dt))
    rhs = np.ones(K.shape[0])
    K, _ = S.apply_dirichlet(K, rhs, S.dirichlet_dofs(prob))
    N = prob.N
    w = S.diag_scaling(K)
    Ks = sp.diags(w) @ K @ sp.diags(w)
    assert np.allclose(np.abs(Ks.diagonal()), 1.0, rtol=1e-14)
    A, B, C, D = (b.toarray() for b in S.split_blocks(Ks, N))
    Sx = S.explicit_schur(Ks, N)
    Ai = np.linalg.inv(A)
    L = np.block([[np.eye(3 * N), np.zeros((3 * N, N))], [C @ Ai, np.eye(N)]])
    Dg = np.block([[A, np.zeros((3 * N, N))], [np.zeros((N, 3 * N)), Sx]])
    U = np.block([[np.eye(3 * N), Ai @ B], [np.zeros((N, 3 * N)), np.eye(N)]])
    Kd = Ks.toarray()
    assert np.max(np.abs(L @ Dg @ U - Kd)) <= 1e-12 * np.max(np.abs(Kd))
    shat = S.schur_hat_diag(Ks, N)
    ref = np.diag(D) - np.einsum("ik,k,ki->i", C, 1.0 / np.diag(A), B)
    assert np.max(np.abs(shat - ref)) <= 1e-13 * np.max(np.abs(ref))
    bj = S.block_jacobi_inverse(Ks, N)
    for a in range(N):
        blk = A[3 * a:3 * a + 3, 3 * a:3 * a + 3]
        assert np.allclose(bj[a] @ blk, np.eye(3), atol=1e-12)


# ------------------------------------------------------------ block preconditioners

@pytest.mark.parametrize("kind", S.BLOCK_KINDS)
def test_block_preconditioner_steps_invert_the_printed_matrix(kind):
    """The block steps (Algorithm 1 and its DU / D / SIMPLE variants) invert
    the preconditioner matrix as printed in expanded form (§4.3: SIMPLE =
    [[A, A diag(A)^-1 B], [C, D]]; the DU and D parts of the LDU
    factorization of eq. a_ldu_block_factorization)."""
    rng = np.random.default_rng(40)
    N = 6
    n = 4 * N
    K = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.6)
    K[np.arange(n), np.arange(n)] += 6.0
    K = sp.csr_matrix(K)
    P = S.block_precond_matrix(K, N, kind)
    x = rng.standard_normal(n)
    assert np.allclose(S.block_precond_apply(K, N, kind, P @ x), x, rtol=1e-10, atol=1e-10)


def test_block_preconditioner_structure():
    """LDU is the matrix itself; DU is block upper triangular with the Schur
    complement in the corner; SIMPLE keeps C and D and perturbs the upper right
    block by A diag(A)^-1 B - B."""
    rng = np.random.default_rng(41)
    N = 5
    n = 4 * N
    K = rng.standard_normal((n, n))
    K[np.arange(n), np.arange(n)] += 8.0
    K = sp.csr_matrix(K)
    A, B, C, D = (m.toarray() for m in S.split_blocks(K, N))
    assert np.array_equal(S.block_precond_matrix(K, N, "LDU"), K.toarray())
    Pdu = S.block_precond_matrix(K, N, "DU")
    assert np.allclose(Pdu[3 * N:, :3 * N], 0) and np.allclose(Pdu[3 * N:, 3 * N:], D - C @ np.linalg.solve(A, B))
    Ps = S.block_precond_matrix(K, N, "SIMPLE")
    assert np.array_equal(Ps[3 * N:], K.toarray()[3 * N:])
    assert np.allclose(Ps[:3 * N, 3 * N:], A @ np.diag(1 / np.diag(A)) @ B)
    # with A diagonal, SIMPLE is exact
    K2 = K.toarray()
    K2[:3 * N, :3 * N] = np.diag(np.diag(A))
    K2 = sp.csr_matrix(K2)
    assert np.allclose(S.block_precond_matrix(K2, N, "SIMPLE"), K2.toarray())


# ------------------------------------------------------------ symmetrized inner solve

def test_symmetrized_schur_equals_schur_for_symmetric_A():
    rng = np.random.default_rng(60)
    N = 5
    n = 4 * N
    K = rng.standard_normal((n, n))
    A = K[:3 * N, :3 * N]
    A[:] = A @ A.T + 3 * N * np.eye(3 * N)
    Ks = sp.csr_matrix(K)
    assert np.allclose(S.symmetrized_schur(Ks, N), S.explicit_schur(Ks, N), rtol=1e-11, atol=1e-11)
    # a skew part changes it; the symmetric part alone decides
    K2 = K.copy()
    Sk = rng.standard_normal((3 * N, 3 * N))
    K2[:3 * N, :3 * N] += Sk - Sk.T
    K2 = sp.csr_matrix(K2)
    assert np.allclose(S.symmetrized_schur(K2, N), S.symmetrized_schur(Ks, N), rtol=1e-11, atol=1e-11)
    assert not np.allclose(S.explicit_schur(K2, N), S.explicit_schur(Ks, N), rtol=1e-6)


def test_block_jacobi_pcg():
    """PCG solves an SPD system; with M = A (block-diagonal A) it takes one
    iteration; in exact arithmetic it ends within n iterations."""
    rng = np.random.default_rng(61)
    N = 10
    n = 3 * N
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    blocks = np.array([A[3 * i:3 * i + 3, 3 * i:3 * i + 3] for i in range(N)])
    Minv = np.linalg.inv(blocks)
    b = rng.standard_normal(n)
    x, k = S.block_jacobi_pcg(A, Minv, b, 1e-12)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9) and k <= n + 5
    Ab = np.zeros((n, n))
    for i in range(N):
        Ab[3 * i:3 * i + 3, 3 * i:3 * i + 3] = blocks[i]
    x1, k1 = S.block_jacobi_pcg(Ab, Minv, b, 1e-12)
    assert k1 == 1 and np.allclose(x1, np.linalg.solve(Ab, b), rtol=1e-12)


def test_direct_solve_is_stable():
    """The oracle's direct solve (SuperLU on the 12^3-hex cube's Newton
    system, n = 8,788, at a random state with non-zero rates) is backward
    stable: relative residual at rounding level, and a 1e-16 relative change
    of the matrix entries moves the solution by rounding only (well
    conditioned after the §4.1 scaling)."""
    n, DT = 12, 1e-3
    m = inputs.cube_mesh(n)
    prob = S.Problem(m, inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, 0.3), 1e3),
                     load={"p_max": 2e4, "t_ramp": 10 * DT})
    N = prob.N
    st = inputs.random_state(N, seed=23, u_scale=0.02 / n, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    rhs, _, _, _ = S.newton_rhs(prob, st, 3 * DT + af * DT, ga)
    Kd, r = S.apply_dirichlet(S.assemble_matrix(prob, st, ga), rhs, S.dirichlet_dofs(prob))
    x = S.direct_solve(Kd, r)
    assert np.linalg.norm(Kd @ x - r) <= 1e-14 * np.linalg.norm(r)
    Kp = Kd.copy()
    Kp.data = Kp.data * (1 + 1e-16 * np.random.default_rng(0).standard_normal(Kp.data.size))
    xp = S.direct_solve(Kp, r)
    assert np.linalg.norm(xp - x) <= 1e-13 * np.linalg.norm(x)
