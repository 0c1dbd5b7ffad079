"""Pin of the oracle's dense discrete adjoint: dJ/d(mu_e, kappa_e) of the mean
top-face displacement after three generalized-alpha steps equals central
finite differences of the oracle's own forward runs (direct solves)."""
import numpy as np
import pytest

from oracle import adjoint as Ad
from oracle import system as S
from paper_1809_06350_gb300 import inputs

DT = 1e-3


def _problem(mu_e, kappa_e):
    m = inputs.cube_mesh(2, jitter=0.05, seed=0)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    return m, S.Problem(m, mat, fields={"mu_e": mu_e, "kappa_e": kappa_e},
                        load={"p_max": 2e4, "t_ramp": 3 * DT})


def _J(mu_e, kappa_e, nsteps=3):
    m, prob = _problem(mu_e, kappa_e)
    st = Ad.forward(prob, nsteps, DT, tol=1e-12)
    return Ad.top_uz_weights(m) @ st[-1][0]


def test_dense_adjoint_matches_central_differences():
    E = 48
    f = inputs.element_fields(E, inputs.material_nh(1e5, 1e6, 1e3), seed=4)
    mu, ka = f["mu_e"], f["kappa_e"]
    m, prob = _problem(mu, ka)
    states = Ad.forward(prob, 3, DT, tol=1e-12)
    grad = Ad.gradient(prob, states, Ad.top_uz_weights(m), DT)
    scale = np.abs(grad).max(axis=0)
    for e in (0, 17, 40):
        for k, base in ((0, mu), (1, ka)):
            h = 1e-4 * base[e]
            p, q = base.copy(), base.copy()
            p[e] += h
            q[e] -= h
            args_p = (p, ka) if k == 0 else (mu, p)
            args_q = (q, ka) if k == 0 else (mu, q)
            fd = (_J(*args_p) - _J(*args_q)) / (2 * h)
            assert abs(grad[e, k] - fd) <= 1e-6 * scale[k] + 1e-6 * abs(fd), (e, k, grad[e, k], fd)
