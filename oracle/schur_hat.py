"""Explicit sparse Schur-complement approximation and a polynomial
preconditioner built on it (oracle; test infrastructure only).

Plain definitions, in float64:

* ``schur_hat``      -- S^ = D - C diag(A)^-1 B (§4.2), diag(A) the scalar
  diagonal of the (scaled) velocity block, as a sparse matrix. Its pattern is
  the distance-2 node graph of the mesh.
* ``splitmix64`` / ``power_start`` -- the counter-based generator SplitMix64
  (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014) and the start vector of the power method drawn from it; the
  CUDA side implements the same published generator on its own.
* ``lmax_estimate``  -- a fixed number of power-method steps on M^-1 S^,
  M = diag(S^), times a safety factor: an estimate of the largest eigenvalue.
* ``chebyshev_apply`` -- z = p(M^-1 S^) M^-1 v: a fixed number of steps of the
  Chebyshev iteration for S^ z = v, zero start, Jacobi-preconditioned, on the
  interval [lmax / ratio, lmax] (the three-term recurrence of the classical
  Chebyshev semi-iteration, e.g. Saad, Iterative Methods for Sparse Linear
  Systems, 2nd ed., §12.3). The paper applies algebraic multigrid built from
  S^ as the preconditioner of the Schur-complement solve (§5); this is the
  polynomial stand-in, a fixed linear operator in S^ for given (lmax, ratio,
  degree).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .system import split_blocks

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15
POWER_STEPS = 10        # power-method steps for the bound
POWER_SAFETY = 1.1      # the bound is POWER_SAFETY times the last estimate
DIAG_EPS = 1e-300       # |diag| at or below this is treated as 1


def schur_hat(K, N):
    """S^ = D - C diag(A)^-1 B (§4.2) as a CSR matrix (N x N)."""
    A, B, C, D = split_blocks(K, N)
    return (D - C @ sp.diags(1.0 / A.diagonal()) @ B).tocsr()


def splitmix64(k):
    """Output k (k = 0, 1, ...) of SplitMix64 seeded with 0: the state after
    k + 1 increments by the golden gamma, passed through the variant-13 mixer
    (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31)."""
    z = ((k + 1) * GOLDEN64) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def power_start(N):
    """x0_i = 2 u_i - 1 with u_i the top 53 bits of splitmix64(i) over 2^53."""
    return np.array([2.0 * ((splitmix64(i) >> 11) * 2.0 ** -53) - 1.0 for i in range(N)])


def jacobi_inverse(Sh):
    d = Sh.diagonal()
    out = np.ones_like(d)
    big = np.abs(d) > DIAG_EPS
    out[big] = 1.0 / d[big]
    return out


def lmax_estimate(Sh, steps=POWER_STEPS, safety=POWER_SAFETY):
    """safety * ||y_k|| after k power steps y_j = M^-1 S^ x_{j-1} / ||x_{j-1}||,
    x_j = y_j, from x_0 = power_start(N); M = diag(S^)."""
    dinv = jacobi_inverse(Sh)
    x = power_start(Sh.shape[0])
    nx = np.linalg.norm(x)
    lam = 0.0
    for _ in range(steps):
        y = dinv * (Sh @ x) / nx
        lam = np.linalg.norm(y)
        x, nx = y, lam
    return safety * lam


def chebyshev_apply(Sh, lmax, ratio, degree, v):
    """degree steps of the Chebyshev iteration for S^ z = v from z = 0 with the
    Jacobi preconditioner M = diag(S^), on [lmax / ratio, lmax]:
        theta = (lmax + lmin) / 2, delta = (lmax - lmin) / 2, sigma = theta / delta,
        r_0 = v, rho_0 = 1 / sigma, d_0 = M^-1 r_0 / theta;
        z_{k+1} = z_k + d_k;  r_{k+1} = r_k - S^ d_k;
        rho_{k+1} = 1 / (2 sigma - rho_k);
        d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) M^-1 r_{k+1}.
    The residual after `degree` steps is T_degree((theta - M^-1 S^) / delta) /
    T_degree(sigma) applied to v in the M^-1-preconditioned sense."""
    dinv = jacobi_inverse(Sh)
    lmin = lmax / ratio
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    z = np.zeros_like(v)
    r = v.astype(np.float64).copy()
    rho = 1.0 / sigma
    d = dinv * r / theta
    for k in range(degree):
        z = z + d
        if k == degree - 1:
            break
        r = r - Sh @ d
        rho_n = 1.0 / (2.0 * sigma - rho)
        d = rho_n * rho * d + (2.0 * rho_n / delta) * (dinv * r)
        rho = rho_n
    return z
