"""Constitutive relations of the Gibbs-energy continuum model (oracle; test
infrastructure only).

All functions accept real or complex arrays (complex-step differentiation runs
through them), so nothing here uses abs(), conj() or real().

Sources:
* §2, constitutive relations: rho = (dG_vol/dp)^-1, beta = (1/rho) drho/dp,
  sigma_dev = J^-1 F~ (P : S~) F~^T with S~ = 2 d(rho0 G_iso)/dC~.
* §5.1: compressible neo-Hookean Gibbs energy
  G = mu/(2 rho0)(tr C~ - 3) + [p sqrt(p^2+k^2) - p^2]/(2 k rho0)
      - k/(2 rho0) ln((sqrt(p^2+k^2) - p)/k).
* §5.2: fully incompressible G_vol = p/rho0 and the HGO isochoric part with
  fibres G_f = k1/(2 k2 rho0)(exp(k2 E^2) - 1), E = H : C~ - 1,
  H = k_d I + (1 - 3 k_d) a (x) a.
* Appendix A: P~_iI = J sigma_dev_ij F^-1_Ij.
"""
from __future__ import annotations

import numpy as np


def det3(M):
    return (M[..., 0, 0] * (M[..., 1, 1] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 1])
            - M[..., 0, 1] * (M[..., 1, 0] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 0])
            + M[..., 0, 2] * (M[..., 1, 0] * M[..., 2, 1] - M[..., 1, 1] * M[..., 2, 0]))


def inv3(M):
    """Inverse of [...,3,3] matrices by the adjugate (analytic, complex-safe)."""
    d = det3(M)
    a = M
    inv = np.empty_like(M)
    inv[..., 0, 0] = a[..., 1, 1] * a[..., 2, 2] - a[..., 1, 2] * a[..., 2, 1]
    inv[..., 0, 1] = a[..., 0, 2] * a[..., 2, 1] - a[..., 0, 1] * a[..., 2, 2]
    inv[..., 0, 2] = a[..., 0, 1] * a[..., 1, 2] - a[..., 0, 2] * a[..., 1, 1]
    inv[..., 1, 0] = a[..., 1, 2] * a[..., 2, 0] - a[..., 1, 0] * a[..., 2, 2]
    inv[..., 1, 1] = a[..., 0, 0] * a[..., 2, 2] - a[..., 0, 2] * a[..., 2, 0]
    inv[..., 1, 2] = a[..., 0, 2] * a[..., 1, 0] - a[..., 0, 0] * a[..., 1, 2]
    inv[..., 2, 0] = a[..., 1, 0] * a[..., 2, 1] - a[..., 1, 1] * a[..., 2, 0]
    inv[..., 2, 1] = a[..., 0, 1] * a[..., 2, 0] - a[..., 0, 0] * a[..., 2, 1]
    inv[..., 2, 2] = a[..., 0, 0] * a[..., 1, 1] - a[..., 0, 1] * a[..., 1, 0]
    return inv / d[..., None, None]


# ---------------------------------------------------------------- volumetric

def g_vol_gibbs(p, kappa, rho0):
    """G_vol(p) of the compressible neo-Hookean Gibbs energy (§5.1)."""
    s = np.sqrt(p * p + kappa * kappa)
    return (p * s - p * p) / (2.0 * kappa * rho0) - kappa / (2.0 * rho0) * np.log((s - p) / kappa)


def rho_beta(p, kappa, rho0, vol):
    """rho(p), beta(p), drho/dp, dbeta/dp.

    Gibbs model: dG_vol/dp = (sqrt(p^2+k^2) - p)/(k rho0), hence
    rho = rho0 (p + sqrt(p^2+k^2))/k, beta = 1/sqrt(p^2+k^2),
    drho/dp = rho beta, dbeta/dp = -p/(p^2+k^2)^(3/2)  (§2 definitions applied
    to the §5.1 energy). Incompressible (§5.2, G_vol = p/rho0): rho = rho0,
    beta = 0.
    """
    if vol == "incompressible":
        one = np.ones_like(p)
        return rho0 * one, 0.0 * p, 0.0 * p, 0.0 * p
    s = np.sqrt(p * p + kappa * kappa)
    rho = rho0 * (p + s) / kappa
    beta = 1.0 / s
    return rho, beta, rho * beta, -p / (s * s * s)


# ---------------------------------------------------------------- isochoric

def structure_tensors(a1, a2, kd):
    """H_i = k_d I + (1 - 3 k_d) a_i (x) a_i for the two fibre families (§5.2)."""
    I = np.eye(3)
    H1 = kd * I + (1.0 - 3.0 * kd) * np.einsum("ei,ej->eij", a1, a1)
    H2 = kd * I + (1.0 - 3.0 * kd) * np.einsum("ei,ej->eij", a2, a2)
    return H1, H2


def psi_iso(F, mu, fib=None):
    """rho0 G_iso(C~(F)): the isochoric energy per unit reference volume.

    ``fib`` is None or a tuple (k1, k2, H1, H2) with per-element arrays.
    """
    J = det3(F)
    C = np.einsum("...kI,...kJ->...IJ", F, F)
    Ct = J[..., None, None] ** (-2.0 / 3.0) * C
    tr = Ct[..., 0, 0] + Ct[..., 1, 1] + Ct[..., 2, 2]
    psi = 0.5 * mu * (tr - 3.0)
    if fib is not None:
        k1, k2, H1, H2 = fib
        for H in (H1, H2):
            E = np.einsum("...IJ,...IJ->...", H, Ct) - 1.0
            psi = psi + k1 / (2.0 * k2) * (np.exp(k2 * E * E) - 1.0)
    return psi


def fictitious_pk2(Ct, mu, fib=None):
    """S~ = 2 d(rho0 G_iso)/dC~ (§2): mu I for the ground matrix, plus
    2 k1 E exp(k2 E^2) H_i per fibre family (§5.2)."""
    I = np.eye(3)
    St = mu[..., None, None] * I * np.ones_like(Ct)
    if fib is not None:
        k1, k2, H1, H2 = fib
        for H in (H1, H2):
            E = np.einsum("...IJ,...IJ->...", H, Ct) - 1.0
            St = St + (2.0 * k1 * E * np.exp(k2 * E * E))[..., None, None] * H
    return St


def piola_dev(F, mu, fib=None):
    """Deviatoric first Piola stress P~ = J sigma_dev F^-T by the paper's route.

    C~ = J^{-2/3} F^T F; S~ as above; P : S~ = S~ - (1/3)(S~ : C~) C~^-1;
    sigma_dev = J^-1 F~ (P : S~) F~^T with F~ = J^{-1/3} F (§2);
    P~_iI = J sigma_dev_ij F^-1_Ij (Appendix A notation).
    Returns (P~, J, F^-1).
    """
    J = det3(F)
    Fi = inv3(F)
    C = np.einsum("...kI,...kJ->...IJ", F, F)
    Ct = J[..., None, None] ** (-2.0 / 3.0) * C
    St = fictitious_pk2(Ct, mu, fib)
    Cti = inv3(Ct)
    SC = np.einsum("...IJ,...IJ->...", St, Ct)
    PS = St - (SC / 3.0)[..., None, None] * Cti
    Ft = J[..., None, None] ** (-1.0 / 3.0) * F
    sig = np.einsum("...iI,...IJ,...jJ->...ij", Ft, PS, Ft) / J[..., None, None]
    P = J[..., None, None] * np.einsum("...ij,...Ij->...iI", sig, Fi)
    return P, J, Fi


def sigma_dev(F, mu, fib=None):
    """Cauchy deviatoric stress (for invariant checks: symmetric, traceless)."""
    J = det3(F)
    C = np.einsum("...kI,...kJ->...IJ", F, F)
    Ct = J[..., None, None] ** (-2.0 / 3.0) * C
    St = fictitious_pk2(Ct, mu, fib)
    Cti = inv3(Ct)
    SC = np.einsum("...IJ,...IJ->...", St, Ct)
    PS = St - (SC / 3.0)[..., None, None] * Cti
    Ft = J[..., None, None] ** (-1.0 / 3.0) * F
    return np.einsum("...iI,...IJ,...jJ->...ij", Ft, PS, Ft) / J[..., None, None]


def wave_speed(mu, kappa, rho0, vol):
    """Maximum wave speed c for tau_M (§3.1): bulk speed sqrt((lambda+2mu)/rho0)
    with lambda = kappa - 2mu/3 when compressible, shear speed sqrt(mu/rho0)
    when incompressible."""
    if vol == "incompressible":
        return np.sqrt(mu / rho0)
    return np.sqrt((kappa + 4.0 * mu / 3.0) / rho0)
