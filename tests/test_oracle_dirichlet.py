"""Pins of the oracle's non-homogeneous Dirichlet data: the ramped targets
g(t), dg/dt(t), the predictor that imposes them (§3.3, predictor stage) and
the Newton step that carries them (multi-corrector stage, steps 1-7).

* A rigid translation driven through the boundary is an exact solution of the
  discrete problem: with every boundary node prescribed u = c s(t),
  s(t) = min(t / T, 1), and a consistent start (u = c t0 / T,
  v = udot = c / T, vdot = 0, p = pdot = 0) the free interior nodes must
  follow u = c t / T, v = udot = c / T, vdot = 0, p = 0 while t < T: F = I
  gives no stress, vdot = 0 no inertia, udot = v no kinematic residual, and
  the generalized-alpha relations (§3.2) integrate motion that is linear in
  time exactly.
* Started from rest, the prescribed boundary velocity jumps to c / T at
  t = 0+. The generalized-alpha rates of the prescribed components then
  relax to the exact rates with the amplification -rho_inf per step (the
  high-frequency spectral radius of the scheme, §3.2): udot_k = c/T
  (1 - (-rho_inf)^k) and vdot_k = c / (T gamma dt) (-rho_inf)^(k-1).
* Across the end of the ramp the prescribed values hold at c and the
  prescribed velocity drops to 0.
* On every prescribed component the predicted pair (y, ydot) satisfies
  eq. gen_alpha_def_y_n_plus_1 (read with the stray comma removed).
"""
import numpy as np
import pytest

from paper_1809_06350_gb300 import inputs
from oracle import newton as Nw
from oracle import system as S

DT = 1e-3
C_TRANS = np.array([2e-3, -1e-3, 3e-3])


def _all_boundary_translation(n, T, rho0=1e3, seed=4):
    """Jittered cube whose boundary nodes are prescribed in all three
    components to the translation c s(t)."""
    m = inputs.cube_mesh(n, jitter=0.05, seed=seed)
    X = m["X"]
    tol = 1e-12
    bnd = np.flatnonzero(np.any((X < tol) | (X > 1.0 - tol), axis=1))
    dn = np.repeat(bnd, 3)
    dc = np.tile(np.arange(3), bnd.size)
    m = dict(m)
    m["dirichlet"] = np.ascontiguousarray(np.stack([dn, dc], 1), dtype=np.int32)
    m["dirichlet_values"] = C_TRANS[dc].astype(np.float64)
    prob = S.Problem(m, inputs.material_nh(1e5, 1e6, rho0), load={"p_max": 0.0, "t_ramp": T})
    return prob, bnd


def _state(N, u, v, ud, vd):
    yn = {"u": np.tile(u, (N, 1)), "p": np.zeros(N), "v": np.tile(v, (N, 1))}
    ydn = {"udot": np.tile(ud, (N, 1)), "pdot": np.zeros(N), "vdot": np.tile(vd, (N, 1))}
    return yn, ydn


def test_dirichlet_targets_ramp():
    prob, _ = _all_boundary_translation(2, T=2.5 * DT)
    T = 2.5 * DT
    m = prob.dir_mask
    for t, s, sd in ((0.0, 0.0, 1.0 / T), (DT, 0.4, 1.0 / T), (2 * DT, 0.8, 1.0 / T),
                     (3 * DT, 1.0, 0.0), (7 * DT, 1.0, 0.0)):
        g, gd = Nw.dirichlet_targets(prob, t)
        want = np.broadcast_to(C_TRANS, g.shape)
        assert np.allclose(g[m], (s * want)[m], rtol=1e-15, atol=0)
        assert np.allclose(gd[m], (sd * want)[m], rtol=1e-15, atol=0)
        assert not np.any(g[~m]) and not np.any(gd[~m])


def test_rigid_translation_through_boundary_is_exact():
    T = 10 * DT
    prob, bnd = _all_boundary_translation(3, T=T)
    N = prob.N
    interior = np.setdiff1d(np.arange(N), bnd)
    assert interior.size == 8
    t = 2 * DT
    vel = C_TRANS / T
    yn, ydn = _state(N, C_TRANS * t / T, vel, vel, np.zeros(3))
    scale = np.max(np.abs(C_TRANS))
    for _step in range(3):
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, t, DT, rho_inf=0.5, tol_r=1e-14, tol_a=1e-20, l_max=8)
        t += DT
        u_ex = C_TRANS * t / T
        for name, arr, ex, sc in (("u", y1["u"], u_ex, scale), ("v", y1["v"], vel, scale / T),
                                  ("udot", yd1["udot"], vel, scale / T), ("vdot", yd1["vdot"], 0 * vel, scale / T)):
            err = np.max(np.abs(arr - ex[None, :]))
            assert err <= 1e-12 * sc, (name, err)
        assert np.max(np.abs(y1["p"])) <= 1e-12 * 1e5 and np.max(np.abs(yd1["pdot"])) <= 1e-12 * 1e5 / T
        yn, ydn = y1, yd1


def test_prescribed_rates_from_rest_relax_by_rho_inf():
    rho_inf = 0.5
    am, af, gam = S.gen_alpha(rho_inf)
    T = 3.5 * DT
    prob, bnd = _all_boundary_translation(2, T=T, rho0=1e3)
    N = prob.N
    yn, ydn = _state(N, np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3))
    m = prob.dir_mask
    c = np.broadcast_to(C_TRANS, (N, 3))
    t = 0.0
    for k in range(1, 6):
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, t, DT, rho_inf=rho_inf, tol_r=1e-12, tol_a=1e-20, l_max=8)
        assert info["converged"]
        t_new = t + DT
        # eq. gen_alpha_def_y_n_plus_1 on every prescribed component
        for yk, ydk in (("u", "udot"), ("v", "vdot")):
            lhs = y1[yk][m]
            rhs = yn[yk][m] + DT * ydn[ydk][m] + gam * DT * (yd1[ydk][m] - ydn[ydk][m])
            assert np.max(np.abs(lhs - rhs)) <= 1e-15 * max(1.0, np.max(np.abs(lhs)))
        if t_new < T:
            assert np.allclose(y1["u"][m], (c * t_new / T)[m], rtol=1e-14, atol=0)
            assert np.allclose(y1["v"][m], (c / T)[m], rtol=1e-14, atol=0)
            ud_ex = (c / T) * (1.0 - (-rho_inf) ** k)
            vd_ex = (c / (T * gam * DT)) * (-rho_inf) ** (k - 1)
            assert np.allclose(yd1["udot"][m], ud_ex[m], rtol=1e-12, atol=0)
            assert np.allclose(yd1["vdot"][m], vd_ex[m], rtol=1e-12, atol=0)
        else:
            assert np.array_equal(y1["u"][m], c[m])
            assert not np.any(y1["v"][m])
        yn, ydn, t = y1, yd1, t_new
    assert t > T  # the run crossed the end of the ramp


def test_tube_stretch_predictor_sets_top_face():
    """The config-3 stretch: u_z on z = L ramps to 0.2 L; z = 0 and the pins
    stay at zero; the predicted rates obey eq. gen_alpha_def_y_n_plus_1 with a
    non-zero ydot_n."""
    m = inputs.tube_mesh(1, 8, 2)
    T = 4 * DT
    prob = S.Problem(m, inputs.material_hgo(), load={"p_max": 0.0, "t_ramp": T})
    N = prob.N
    am, af, gam = S.gen_alpha(0.5)
    rng = np.random.default_rng(5)
    yn = {"u": 1e-4 * rng.standard_normal((N, 3)), "p": rng.standard_normal(N),
          "v": 1e-2 * rng.standard_normal((N, 3))}
    ydn = {"udot": 1e-2 * rng.standard_normal((N, 3)), "pdot": rng.standard_normal(N),
           "vdot": rng.standard_normal((N, 3))}
    t_np1 = 2 * DT
    y1, yd1 = Nw.predictor(prob, yn, ydn, t_np1, DT, gam)
    top = np.flatnonzero(np.abs(prob.X[:, 2] - 0.05) < 1e-12)
    bot = np.flatnonzero(np.abs(prob.X[:, 2]) < 1e-12)
    assert np.allclose(y1["u"][top, 2], 0.2 * 0.05 * 0.5, rtol=1e-15)
    assert np.allclose(y1["v"][top, 2], 0.2 * 0.05 / T, rtol=1e-15)
    assert not np.any(y1["u"][bot, 2]) and not np.any(y1["v"][bot, 2])
    mk = prob.dir_mask
    for yk, ydk in (("u", "udot"), ("v", "vdot")):
        rhs = yn[yk] + DT * ydn[ydk] + gam * DT * (yd1[ydk] - ydn[ydk])
        assert np.max(np.abs(y1[yk][mk] - rhs[mk])) <= 1e-15 * max(1.0, np.max(np.abs(y1[yk])))
        # free components take the plain predictor
        assert np.array_equal(y1[yk][~mk], yn[yk][~mk])
        assert np.allclose(yd1[ydk][~mk], ((gam - 1) / gam * ydn[ydk])[~mk], rtol=1e-15, atol=0)
