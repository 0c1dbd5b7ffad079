"""Pins of the oracle's constitutive relations against the paper's definitions.

* rho(p), beta(p) closed forms vs the definitions rho = (dG_vol/dp)^-1,
  beta = -G_vol''/G_vol' (§2) applied to the §5.1 Gibbs energy, differentiated
  symbolically by SymPy from the energy as printed.
* P~ (paper route S~ -> P:S~ -> sigma_dev -> J sigma_dev F^-T) vs the
  complex-step derivative of the isochoric energy Psi_iso(F) = rho0 G_iso(C~(F)).
* sigma_dev symmetric and traceless; objectivity P~(QF) = Q P~(F); P~(I) = 0.
"""
import numpy as np
import pytest

from oracle import constitutive as cm

sympy = pytest.importorskip("sympy")


def test_rho_beta_match_gibbs_energy_definitions():
    p, k, r0 = sympy.symbols("p kappa rho0", positive=True)
    s = sympy.sqrt(p ** 2 + k ** 2)
    # §5.1 volumetric Gibbs energy, as printed
    G = (p * s - p ** 2) / (2 * k * r0) - k / (2 * r0) * sympy.log((s - p) / k)
    dG = sympy.diff(G, p)
    d2G = sympy.diff(G, p, 2)
    rho_def = 1 / dG
    beta_def = -d2G / dG
    for pv in (-3e5, -1e4, 0.0, 2.5e3, 7e5):
        for kv in (2.1667e5, 1e6, 4.9967e7):
            sub = {p: pv, k: kv, r0: 1e3}
            rho, beta, drho, dbeta = cm.rho_beta(np.array(pv), kv, 1e3, "gibbs")
            assert rho == pytest.approx(float(rho_def.subs(sub).evalf(30)), rel=1e-12)
            assert beta == pytest.approx(float(beta_def.subs(sub).evalf(30)), rel=1e-12)
            assert drho == pytest.approx(float(sympy.diff(rho_def, p).subs(sub).evalf(30)), rel=1e-10)
            assert dbeta == pytest.approx(float(sympy.diff(beta_def, p).subs(sub).evalf(30)), rel=1e-10)


def test_g_vol_matches_printed_energy_numerically():
    # the oracle's energy is the printed one: FD of it gives 1/rho
    for pv in (-2e5, 0.0, 3e5):
        h = 1.0
        d = (cm.g_vol_gibbs(pv + h, 1e6, 1e3) - cm.g_vol_gibbs(pv - h, 1e6, 1e3)) / (2 * h)
        rho = cm.rho_beta(np.array(pv), 1e6, 1e3, "gibbs")[0]
        assert d == pytest.approx(1.0 / rho, rel=1e-8)


def test_mass_conservation_state():
    # p = (kappa/2)(1/J - J) is the pressure at which rho(p) J = rho0
    for J in (0.8, 0.97, 1.0, 1.05, 1.3):
        p = 0.5 * 1e6 * (1.0 / J - J)
        rho = cm.rho_beta(np.array(p), 1e6, 1e3, "gibbs")[0]
        assert rho * J == pytest.approx(1e3, rel=1e-13)


def test_incompressible_volumetric():
    rho, beta, drho, dbeta = cm.rho_beta(np.array([1.0, -5e4]), 0.0, 1e3, "incompressible")
    assert np.all(rho == 1e3) and np.all(beta == 0) and np.all(drho == 0) and np.all(dbeta == 0)


def _random_F(rng, n, amp=0.25):
    F = np.eye(3) + amp * rng.standard_normal((n, 3, 3))
    d = np.linalg.det(F)
    F[d < 0] *= -1.0
    return F


def _fibres(rng, n, kd):
    a1 = rng.standard_normal((n, 3))
    a1 /= np.linalg.norm(a1, axis=1, keepdims=True)
    a2 = rng.standard_normal((n, 3))
    a2 /= np.linalg.norm(a2, axis=1, keepdims=True)
    H1, H2 = cm.structure_tensors(a1, a2, kd)
    return (np.full(n, 2e5), np.full(n, 5.0), H1, H2)


@pytest.mark.parametrize("fibres", [False, True])
def test_piola_is_energy_derivative(fibres):
    rng = np.random.default_rng(11)
    n = 64
    F = _random_F(rng, n)
    mu = np.full(n, 1e5)
    fib = _fibres(rng, n, 0.1) if fibres else None
    P, J, Fi = cm.piola_dev(F, mu, fib)
    h = 1e-30
    Pcs = np.zeros_like(P)
    for i in range(3):
        for I in range(3):
            Fc = F.astype(np.complex128)
            Fc[:, i, I] += 1j * h
            Pcs[:, i, I] = cm.psi_iso(Fc, mu, fib).imag / h
    scale = np.abs(Pcs).max(axis=(1, 2), keepdims=True)
    assert np.max(np.abs(P - Pcs) / scale) < 1e-12


def test_sigma_dev_symmetric_traceless_objective():
    rng = np.random.default_rng(5)
    n = 32
    F = _random_F(rng, n)
    mu = np.full(n, 8e4)
    fib = _fibres(rng, n, 0.2)
    s = cm.sigma_dev(F, mu, fib)
    sc = np.abs(s).max()
    assert np.max(np.abs(s - np.swapaxes(s, 1, 2))) < 1e-12 * sc
    assert np.max(np.abs(np.trace(s, axis1=1, axis2=2))) < 1e-11 * sc
    # objectivity: P~(QF) = Q P~(F) for a rotation Q
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    P1, _, _ = cm.piola_dev(F, mu, fib)
    P2, _, _ = cm.piola_dev(np.einsum("ij,ejk->eik", q, F), mu, fib)
    assert np.max(np.abs(P2 - np.einsum("ij,ejk->eik", q, P1))) < 1e-11 * np.abs(P1).max()


def test_stress_free_reference_and_rotation():
    rng = np.random.default_rng(2)
    n = 8
    mu = np.full(n, 1e5)
    fib = _fibres(rng, n, 0.15)
    P, J, _ = cm.piola_dev(np.tile(np.eye(3), (n, 1, 1)), mu, fib)
    assert np.max(np.abs(P)) < 1e-9
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    P, _, _ = cm.piola_dev(np.tile(q, (n, 1, 1)), mu, None)
    assert np.max(np.abs(P)) < 1e-9
