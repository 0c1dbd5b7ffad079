"""Pins of the oracle's element residual (Appendix A residual formulas).

* reference geometry: partition of unity of gradients, reproduction of X,
  volumes summing to the cube volume;
* patch test: an affine displacement with constant pressure and zero rates
  gives zero interior residual on a jittered mesh;
* rigid motion: u = (Q - I) X + c, p = 0 gives zero residual everywhere, and
  a superposed rotation rotates R_m and leaves R_p unchanged;
* homogeneous uniaxial compression (closed form of the neo-Hookean cube under
  a dead load P0 with rollers): the assembled residual, traction included,
  vanishes on every free dof; compressible and incompressible.
"""
import numpy as np
import pytest
from scipy.optimize import fsolve

from paper_1809_06350_gb300 import inputs
from oracle import element as el
from oracle import system as S


def _rotation(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def _boundary_nodes(mesh):
    X = mesh["X"]
    L = X.max()
    on = np.any((np.abs(X) < 1e-12) | (np.abs(X - L) < 1e-12), axis=1)
    return on


def test_reference_geometry():
    m = inputs.cube_mesh(4, jitter=0.05, seed=0)
    X, t = m["X"], m["tets"].astype(np.int64)
    geo = el.reference_geometry(X, t)
    assert np.all(geo["V"] > 0)
    assert geo["V"].sum() == pytest.approx(1.0, rel=1e-13)
    assert np.max(np.abs(geo["G"].sum(axis=1))) < 1e-12 / 0.25
    # sum_A X_A (x) grad N_A = I  (P1 reproduces linear fields)
    R = np.einsum("eAi,eAI->eiI", X[t], geo["G"])
    assert np.max(np.abs(R - np.eye(3))) < 1e-12
    # barycentric gradients by an independent route: rows of inv([1 X])
    M = np.concatenate([np.ones((t.shape[0], 4, 1)), X[t]], axis=2)
    Minv = np.linalg.inv(M)  # columns: coefficients of N_A = c0 + c . X
    assert np.max(np.abs(np.swapaxes(Minv[:, 1:, :], 1, 2) - geo["G"])) < 1e-9


@pytest.mark.parametrize("vol", ["gibbs", "incompressible"])
def test_patch_test_affine(vol):
    m = inputs.cube_mesh(4, jitter=0.05, seed=0)
    kappa = 1e6 if vol == "gibbs" else np.inf
    mat = inputs.material_nh(1e5, kappa, 1e3)
    prob = S.Problem(m, mat)
    rng = np.random.default_rng(3)
    H = 0.05 * rng.standard_normal((3, 3))
    X = m["X"]
    st = inputs.zero_state(prob.N)
    st["u"] = X @ H.T + np.array([0.01, -0.02, 0.005])
    J = np.linalg.det(np.eye(3) + H)
    st["p"][:] = 0.5 * 1e6 * (1 / J - J)
    Rm, Rp = S.assemble_residual(prob, st, 0.0)
    interior = ~_boundary_nodes(m)
    scale = np.abs(Rm[~interior]).max()
    assert scale > 0
    assert np.abs(Rm[interior]).max() < 1e-11 * scale
    pscale = prob.tau.max() * prob.geo["V"].max() * abs(st["p"][0]) * np.abs(prob.geo["G"]).max()
    assert np.abs(Rp).max() < 1e-12 * pscale


@pytest.mark.parametrize("fibres", [False, True])
def test_rigid_motion_zero_residual_and_invariance(fibres):
    rng = np.random.default_rng(9)
    if fibres:
        m = inputs.tube_mesh(2, 12, 3)
        mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.1)
    else:
        m = inputs.cube_mesh(3, jitter=0.05, seed=1)
        mat = inputs.material_nh(1e5, 1e6, 1e3)
    prob = S.Problem(m, mat)
    X = m["X"]
    Q = _rotation(rng)
    st = inputs.zero_state(prob.N)
    st["u"] = X @ (Q - np.eye(3)).T + np.array([0.3, -0.1, 0.2])
    Rm, Rp = S.assemble_residual(prob, st, 0.0)
    h = np.cbrt(prob.geo["V"].mean())
    assert np.abs(Rm).max() < 1e-10 * mat["mu"] * h * h
    assert np.abs(Rp).max() < 1e-14
    # superposed rotation of a general state
    st = inputs.random_state(prob.N, seed=4, u_scale=0.02 * h, v_scale=0.1, p_scale=2e3)
    Rm1, Rp1 = S.assemble_residual(prob, st, 0.0)
    st2 = dict(st)
    st2["u"] = (X + st["u"]) @ Q.T - X
    st2["v"] = st["v"] @ Q.T
    st2["vdot"] = st["vdot"] @ Q.T
    Rm2, Rp2 = S.assemble_residual(prob, st2, 0.0)
    assert np.abs(Rm2 - Rm1 @ Q.T).max() < 1e-10 * np.abs(Rm1).max()
    assert np.abs(Rp2 - Rp1).max() < 1e-10 * np.abs(Rp1).max()


def _uniaxial(mu, kappa, P0, incompressible):
    if incompressible:
        c = fsolve(lambda c: mu * (c - c ** -2) + P0, 0.9, xtol=1e-15)[0]
        a = c ** -0.5
        p = mu * (a * a - c * c) / 3.0
        return a, c, p

    def f(z):
        a, c = z
        J = a * a * c
        return [mu * J ** (-5 / 3) * (c * c - a * a) + P0 / (a * a),
                mu * J ** (-5 / 3) * (a * a - c * c) / 3.0 - 0.5 * kappa * (1 / J - J)]

    a, c = fsolve(f, [1.01, 0.95], xtol=1e-14)
    J = a * a * c
    return a, c, mu * J ** (-5 / 3) * (a * a - c * c) / 3.0


@pytest.mark.parametrize("incompressible", [False, True])
def test_uniaxial_compression_closed_form(incompressible):
    """Static homogeneous solution F = diag(a, a, c) of the dead-loaded cube
    with rollers: lateral faces traction-free, P_zz = -P0 on top."""
    mu, kappa, P0 = 1e5, 1e6, 2e4
    a, c, p = _uniaxial(mu, kappa, P0, incompressible)
    m = inputs.cube_mesh(4, jitter=0.05, seed=2)
    mat = inputs.material_nh(mu, np.inf if incompressible else kappa, 1e3)
    prob = S.Problem(m, mat, load={"p_max": P0, "t_ramp": 1e-9})
    st = inputs.zero_state(prob.N)
    st["u"] = m["X"] * np.array([a - 1.0, a - 1.0, c - 1.0])
    st["p"][:] = p
    Rm, Rp = S.assemble_residual(prob, st, 1.0)
    free = ~prob.dir_mask
    fscale = P0 * m["h"] ** 2
    assert np.abs(Rm[free]).max() < 1e-9 * fscale
    # R_p holds only tau J p_,i terms that cancel for constant p
    pscale = prob.tau.max() * prob.geo["V"].max() * abs(p) * np.abs(prob.geo["G"]).max()
    assert np.abs(Rp).max() < 1e-12 * pscale
    # the bottom supports carry the load: their internal force sums to +P0 * area
    bottom = np.abs(m["X"][:, 2]) < 1e-12
    assert Rm[bottom, 2].sum() == pytest.approx(P0 * 1.0, rel=1e-10)
