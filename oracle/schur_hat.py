"""Explicit sparse Schur-complement approximation and a polynomial
preconditioner built on it (oracle; test infrastructure only).

Plain definitions, in float64:

* ``schur_hat``      -- S^ = D - C diag(A)^-1 B (§4.2), diag(A) the scalar
  diagonal of the (scaled) velocity block, as a sparse matrix. Its pattern is
  the distance-2 node graph of the mesh.
* ``splitmix64`` / ``power_start`` -- the counter-based generator SplitMix64
  (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014) and the Krylov start vector drawn from it; the CUDA side
  implements the same published generator on its own.
* ``ritz_bounds``    -- k steps of Arnoldi (classical Gram-Schmidt, two
  passes) on |M|^-1/2 S^ |M|^-1/2 (similar to M^-1 S^ when diag(S^) > 0) from
  the normalised power_start vector; the extreme eigenvalues of the symmetric
  part of the k x k Hessenberg matrix (Ritz values; for a symmetric operator
  they interlace the spectrum, the Lanczos bounds) give the interval of the
  Chebyshev preconditioner: [theta_min / RITZ_LOW, RITZ_SAFETY theta_max]
  (``cheb_interval`` clamps it, or fixes lmin = lmax / ratio on request).
* ``arnoldi_hessenberg_m`` / ``ritz_bounds_m`` / ``chebyshev_apply_block`` --
  the same interval and polynomial for the velocity block A with the 3x3
  block-Jacobi M (A's diagonal blocks): Arnoldi on M^-1 A in the M-inner
  product (H symmetric when A is), z = p(M^-1 A) M^-1 v.
* ``chebyshev_apply`` -- z = p(M^-1 S^) M^-1 v: a fixed number of steps of the
  Chebyshev iteration for S^ z = v, zero start, Jacobi-preconditioned, on the
  interval [lmin, lmax] (the three-term recurrence of the classical
  Chebyshev semi-iteration, e.g. Saad, Iterative Methods for Sparse Linear
  Systems, 2nd ed., §12.3). The paper applies algebraic multigrid built from
  S^ as the preconditioner of the Schur-complement solve (§5); this is the
  polynomial stand-in, a fixed linear operator in S^ for a given interval and
  degree.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .system import split_blocks

MASK64 = (1 << 64) - 1
GOLDEN64 = 0x9E3779B97F4A7C15
RITZ_STEPS = 12         # Arnoldi steps of ritz_bounds
RITZ_SAFETY = 1.05      # lmax = RITZ_SAFETY x the largest Ritz value
RITZ_LOW = 2.0          # lmin = the smallest Ritz value / RITZ_LOW
CHEB_MAX_RATIO = 1000.0  # the interval's lmax / lmin is clamped to [CHEB_MIN_RATIO, CHEB_MAX_RATIO]
CHEB_MIN_RATIO = 1.5
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


def float32_values(Sh):
    """S^ with every entry rounded to FP32 (the copy the CUDA preconditioner
    reads); M = diag(S^) stays FP64 wherever it appears."""
    out = Sh.copy()
    out.data = out.data.astype(np.float32).astype(np.float64)
    return out


def arnoldi_hessenberg(Sh, k=RITZ_STEPS, Sv=None):
    """H (k+1 x k) of k Arnoldi steps on |M|^-1/2 Sv |M|^-1/2 from power_start
    (Sv = S^ unless given, M = diag(S^)), each new direction orthogonalised
    twice against the basis (classical Gram-Schmidt); stops early (returning
    the leading block) if a direction vanishes."""
    Sv = Sh if Sv is None else Sv
    s = np.sqrt(np.abs(jacobi_inverse(Sh)))
    N = Sh.shape[0]
    x = power_start(N)
    V = np.zeros((k + 1, N))
    H = np.zeros((k + 1, k))
    V[0] = x / np.linalg.norm(x)
    for j in range(k):
        w = s * (Sv @ (s * V[j]))
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return H[:j + 2, :j + 1]
        V[j + 1] = w / H[j + 1, j]
    return H


def ritz_bounds(Sh, k=RITZ_STEPS, Sv=None):
    """(lmin, lmax) for the Chebyshev interval from the Ritz values of
    arnoldi_hessenberg: the eigenvalues of (H_k + H_k^T) / 2, H_k the square
    leading block."""
    H = arnoldi_hessenberg(Sh, k, Sv)
    kk = H.shape[1]
    Hk = H[:kk, :kk]
    theta = np.linalg.eigvalsh(0.5 * (Hk + Hk.T))
    return theta[0] / RITZ_LOW, RITZ_SAFETY * theta[-1]


def cheb_interval(bounds, ratio=0.0):
    """The Chebyshev interval from (lmin, lmax) = ritz_bounds(...): ratio > 0
    fixes lmin = lmax / ratio; ratio = 0 keeps the estimated lmin, clamped to
    [lmax / CHEB_MAX_RATIO, lmax / CHEB_MIN_RATIO]."""
    lmin, lmax = bounds
    if ratio > 0:
        return lmax / ratio, lmax
    return min(max(lmin, lmax / CHEB_MAX_RATIO), lmax / CHEB_MIN_RATIO), lmax


def block_diag_inverse(A, N):
    """Inverses [N, 3, 3] of the 3x3 diagonal blocks of A (3N x 3N)."""
    A = A.tocsr()
    blocks = np.array([A[3 * i:3 * i + 3, 3 * i:3 * i + 3].toarray() for i in range(N)])
    return blocks, np.linalg.inv(blocks)


def arnoldi_hessenberg_m(A, N, k=RITZ_STEPS):
    """H (k+1 x k) of k Arnoldi steps on T = M^-1 A (M the 3x3 block diagonal
    of A) in the M-inner product <x, y> = x^T M y, from the normalised
    power_start(3N) vector, each new direction orthogonalised twice (classical
    Gram-Schmidt). For symmetric A and SPD M, T is self-adjoint in this inner
    product and H is symmetric."""
    A = A.tocsr()
    Mb, Mi = block_diag_inverse(A, N)
    M = lambda v: np.einsum("nij,nj->ni", Mb, v.reshape(N, 3)).ravel()
    Minv = lambda v: np.einsum("nij,nj->ni", Mi, v.reshape(N, 3)).ravel()
    x = power_start(3 * N)
    V = np.zeros((k + 1, 3 * N))
    H = np.zeros((k + 1, k))
    V[0] = x / np.sqrt(x @ M(x))
    for j in range(k):
        w = Minv(A @ V[j])
        for _ in range(2):
            h = V[:j + 1] @ M(w)
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.sqrt(max(w @ M(w), 0.0))
        if H[j + 1, j] == 0.0:
            return H[:j + 2, :j + 1]
        V[j + 1] = w / H[j + 1, j]
    return H


def ritz_bounds_m(A, N, k=RITZ_STEPS, Av=None):
    """(lmin, lmax) for the Chebyshev interval of M^-1 A from the Ritz values of
    arnoldi_hessenberg_m (eigenvalues of the symmetric part of H_k), with the
    same safety factors as ritz_bounds. Av, if given, replaces A in the
    products (M stays the block diagonal of A)."""
    H = arnoldi_hessenberg_m(A if Av is None else _with_diag_blocks(Av, A, N), N, k)
    kk = H.shape[1]
    Hk = H[:kk, :kk]
    theta = np.linalg.eigvalsh(0.5 * (Hk + Hk.T))
    return theta[0] / RITZ_LOW, RITZ_SAFETY * theta[-1]


def _with_diag_blocks(Av, A, N):
    """Av with A's exact 3x3 diagonal blocks (so that M is A's block diagonal)."""
    out = Av.tolil()
    A = A.tocsr()
    for i in range(N):
        out[3 * i:3 * i + 3, 3 * i:3 * i + 3] = A[3 * i:3 * i + 3, 3 * i:3 * i + 3].toarray()
    return out.tocsr()


def chebyshev_apply(Sh, lmin, lmax, degree, v, Sv=None):
    """degree steps of the Chebyshev iteration for S^ z = v from z = 0 with the
    Jacobi preconditioner M = diag(S^), on [lmin, lmax]:
        theta = (lmax + lmin) / 2, delta = (lmax - lmin) / 2, sigma = theta / delta,
        r_0 = v, rho_0 = 1 / sigma, d_0 = M^-1 r_0 / theta;
        z_{k+1} = z_k + d_k;  r_{k+1} = r_k - S^ d_k;
        rho_{k+1} = 1 / (2 sigma - rho_k);
        d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) M^-1 r_{k+1}.
    The residual after `degree` steps is T_degree((theta - M^-1 S^) / delta) /
    T_degree(sigma) applied to v in the M^-1-preconditioned sense. Sv, if
    given, replaces S^ in the products (M stays diag(S^))."""
    dinv = jacobi_inverse(Sh)
    return chebyshev_iteration(Sh if Sv is None else Sv, lambda r: dinv * r, lmin, lmax, degree, v)


def chebyshev_apply_block(A, N, lmin, lmax, degree, v, Av=None):
    """The same Chebyshev iteration for A z = v with the 3x3 block-Jacobi
    preconditioner M (A's diagonal blocks): z = p(M^-1 A) M^-1 v. Av, if given,
    replaces A in the products."""
    _, Mi = block_diag_inverse(A, N)
    minv = lambda r: np.einsum("nij,nj->ni", Mi, r.reshape(N, 3)).ravel()
    return chebyshev_iteration(A if Av is None else Av, minv, lmin, lmax, degree, v)


def chebyshev_iteration(Op, minv, lmin, lmax, degree, v):
    """degree steps of the Chebyshev iteration for Op z = v from z = 0 with the
    preconditioner minv (the recurrence of chebyshev_apply)."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    z = np.zeros_like(v)
    r = v.astype(np.float64).copy()
    rho = 1.0 / sigma
    d = minv(r) / theta
    for k in range(degree):
        z = z + d
        if k == degree - 1:
            break
        r = r - Op @ d
        rho_n = 1.0 / (2.0 * sigma - rho)
        d = rho_n * rho * d + (2.0 * rho_n / delta) * minv(r)
        rho = rho_n
    return z
