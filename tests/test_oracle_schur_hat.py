"""Pins of the explicit S^ = D - C diag(A)^-1 B, the power-method bound and
the Chebyshev polynomial preconditioner (oracle/schur_hat.py).

* SplitMix64 reproduces the generator's published output sequence;
* S^ equals a brute-force triple loop on a tiny random block system, equals
  the exact dense Schur complement when A is diagonal, and its pattern on a
  mesh lies inside the distance-2 node graph;
* the Arnoldi basis behind the Ritz bounds is orthonormal and satisfies the
  Arnoldi relation; on a 1D Laplacian the Ritz values interlace the known
  spectrum and, after n steps, are that spectrum;
* the Chebyshev residual equals T_k((theta - M^-1 S^)/delta) / T_k(sigma)
  applied to M^-1 v (Chebyshev polynomial theory), degree 1 is scaled
  Jacobi, and a high degree reaches the exact solve.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb

from oracle import schur_hat as SH
from oracle import system as S
from oracle import newton as Nw
from paper_1809_06350_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_published_sequence():
    vals = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert [SH.splitmix64(k) for k in range(len(vals))] == vals


def test_power_start_range_and_spread():
    x = SH.power_start(4096)
    assert np.all(x >= -1.0) and np.all(x < 1.0)
    assert abs(x.mean()) < 0.05 and abs(np.mean(x * x) - 1.0 / 3.0) < 0.03


def _random_block_system(N, rng, diagonal_A=False):
    n = 4 * N
    K = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.5)
    A = K[:3 * N, :3 * N]
    if diagonal_A:
        A[:] = np.diag(rng.uniform(1.0, 2.0, 3 * N))
    else:
        A[np.arange(3 * N), np.arange(3 * N)] = rng.uniform(1.0, 2.0, 3 * N) * rng.choice([-1, 1], 3 * N)
    return sp.csr_matrix(K)


def test_schur_hat_brute_force():
    rng = np.random.default_rng(3)
    N = 4
    K = _random_block_system(N, rng)
    Kd = K.toarray()
    ref = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            s = Kd[3 * N + i, 3 * N + j]
            for m in range(3 * N):
                s -= Kd[3 * N + i, m] * Kd[m, 3 * N + j] / Kd[m, m]
            ref[i, j] = s
    assert np.allclose(SH.schur_hat(K, N).toarray(), ref, rtol=1e-13, atol=1e-13)


def test_schur_hat_exact_for_diagonal_A():
    rng = np.random.default_rng(4)
    N = 5
    K = _random_block_system(N, rng, diagonal_A=True)
    assert np.allclose(SH.schur_hat(K, N).toarray(), S.explicit_schur(K, N), rtol=1e-12, atol=1e-12)


@pytest.fixture(scope="module")
def mesh_system():
    DT = 1e-3
    mesh = inputs.cube_mesh(4)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, 0.5), 1e3)
    prob = S.Problem(mesh, mat, load={"p_max": 2e4, "t_ramp": 10 * DT})
    N = prob.N
    z3, z1 = np.zeros((N, 3)), np.zeros(N)
    rec = []
    Nw.newton_step(prob, {"u": z3, "p": z1, "v": z3}, {"udot": z3, "pdot": z1, "vdot": z3}, 0.0, DT,
                   l_max=1, record=rec)
    K = rec[0][0].tocsr()
    w = S.diag_scaling(K)
    return mesh, N, (sp.diags(w) @ K @ sp.diags(w)).tocsr()


def test_schur_hat_pattern_is_distance_two(mesh_system):
    mesh, N, K = mesh_system
    tets = np.asarray(mesh["tets"])
    adj = np.zeros((N, N), dtype=bool)
    for e in tets:
        adj[np.ix_(e, e)] = True
    d2 = (adj.astype(np.int64) @ adj.astype(np.int64)) > 0
    Sh = SH.schur_hat(K, N).toarray()
    assert not np.any((Sh != 0) & ~d2)
    assert np.count_nonzero(Sh) > np.count_nonzero(adj)
    # its diagonal is the diagonal used by the point-Jacobi S-preconditioner
    assert np.allclose(np.diag(Sh), S.schur_hat_diag(K, N), rtol=1e-13)


def _spd_unit(n, rng):
    Q = rng.standard_normal((n, n))
    Sd = Q @ Q.T + n * np.eye(n)
    return sp.csr_matrix(Sd)


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 6])
def test_chebyshev_residual_polynomial(degree):
    rng = np.random.default_rng(10 + degree)
    n = 15
    Sh = _spd_unit(n, rng)
    d = Sh.diagonal()
    # M^-1 S^ is similar to the symmetric D^-1/2 S^ D^-1/2
    Ssym = (Sh.toarray() / np.sqrt(d)[:, None]) / np.sqrt(d)[None, :]
    lam, Q = np.linalg.eigh(Ssym)
    lmax, ratio = 1.05 * lam.max(), 7.0
    lmin = lmax / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    v = rng.standard_normal(n)
    z = SH.chebyshev_apply(Sh, lmax / ratio, lmax, degree, v)
    c = np.zeros(degree + 1)
    c[degree] = 1.0
    poly = npcheb.chebval((theta - lam) / delta, c) / npcheb.chebval(theta / delta, c)
    # M^-1 r = D^-1/2 Q poly(Lambda) Q^T D^1/2 (M^-1 v)
    mv = v / d
    ref = (Q @ (poly * (Q.T @ (np.sqrt(d) * mv)))) / np.sqrt(d)
    got = (v - Sh @ z) / d
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(mv).max())


def test_chebyshev_degree_one_is_scaled_jacobi():
    rng = np.random.default_rng(5)
    Sh = _spd_unit(9, rng)
    v = rng.standard_normal(9)
    z = SH.chebyshev_apply(Sh, 0.3, 3.0, 1, v)
    theta = 0.5 * (3.0 + 0.3)
    assert np.allclose(z, v / Sh.diagonal() / theta, rtol=1e-14)


def test_chebyshev_high_degree_solves():
    rng = np.random.default_rng(6)
    Sh = _spd_unit(12, rng)
    d = Sh.diagonal()
    lam = np.linalg.eigvalsh((Sh.toarray() / np.sqrt(d)[:, None]) / np.sqrt(d)[None, :])
    lmax = 1.01 * lam.max()
    ratio = lmax / (0.99 * lam.min())
    v = rng.standard_normal(12)
    z = SH.chebyshev_apply(Sh, lmax / ratio, lmax, 60, v)
    assert np.allclose(z, np.linalg.solve(Sh.toarray(), v), rtol=1e-9, atol=1e-12)


def test_arnoldi_relation_and_orthonormal_basis(mesh_system):
    """H from ritz_bounds' Arnoldi satisfies T V_k = V_{k+1} H with T the
    symmetrically scaled S^; rebuilt here from H alone by the Arnoldi relation
    column by column (each column of V_{k+1} follows from the previous ones)."""
    _, N, K = mesh_system
    Sh = SH.schur_hat(K, N)
    s = np.sqrt(np.abs(1.0 / Sh.diagonal()))
    T = sp.diags(s) @ Sh @ sp.diags(s)
    H = SH.arnoldi_hessenberg(Sh, 8)
    x0 = SH.power_start(N)
    V = [x0 / np.linalg.norm(x0)]
    for j in range(8):
        w = T @ V[j] - sum(H[i, j] * V[i] for i in range(j + 1))
        V.append(w / H[j + 1, j])
    Vm = np.array(V)
    assert np.allclose(Vm @ Vm.T, np.eye(9), atol=1e-10)


def test_ritz_values_of_symmetric_operator():
    """1D Laplacian tridiag(-1/2, 2, -1/2), n = 60: M^-1 S^ = I - T/4 has the
    eigenvalues 1 - cos(k pi / 61) / 2. Ritz values lie inside the spectrum
    (Cauchy interlacing), the extreme ones approach its ends, and with k = n
    steps they are the spectrum."""
    n = 60
    L = sp.diags([-0.5 * np.ones(n - 1), 2.0 * np.ones(n), -0.5 * np.ones(n - 1)], [-1, 0, 1]).tocsr()
    ev = 1.0 - 0.5 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    lmin, lmax = SH.ritz_bounds(L, 12)
    tmin, tmax = lmin * SH.RITZ_LOW, lmax / SH.RITZ_SAFETY
    assert ev.min() - 1e-12 <= tmin and tmax <= ev.max() + 1e-12
    assert tmax > ev.max() - 0.02 and tmin < ev.min() + 0.1
    H = SH.arnoldi_hessenberg(L, n)
    kk = H.shape[1]
    theta = np.linalg.eigvalsh(0.5 * (H[:kk, :kk] + H[:kk, :kk].T))
    assert kk == n and np.allclose(theta, np.sort(ev), atol=1e-9)


def test_cheb_interval_clamps():
    assert SH.cheb_interval((0.5, 3.0), 20.0) == (3.0 / 20.0, 3.0)
    assert SH.cheb_interval((0.5, 3.0)) == (0.5, 3.0)
    assert SH.cheb_interval((2.9, 3.0)) == (2.0, 3.0)
    assert SH.cheb_interval((-1.0, 3.0)) == (3.0 / SH.CHEB_MAX_RATIO, 3.0)


def test_float32_values_keep_pattern_and_round_entries():
    rng = np.random.default_rng(8)
    Sh = _spd_unit(10, rng)
    S32 = SH.float32_values(Sh)
    assert np.array_equal(S32.indices, Sh.indices) and np.array_equal(S32.indptr, Sh.indptr)
    assert np.array_equal(S32.data, Sh.data.astype(np.float32).astype(np.float64))
    # Sv replaces S^ in the products only: with Sv = S^ nothing changes
    v = rng.standard_normal(10)
    assert np.array_equal(SH.chebyshev_apply(Sh, 0.5, 3.0, 4, v), SH.chebyshev_apply(Sh, 0.5, 3.0, 4, v, Sv=Sh))


def _spd_block_system(N, rng):
    n = 3 * N
    Q = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.3)
    A = Q @ Q.T + n * np.eye(n) * 0.2
    return sp.csr_matrix(A)


def test_m_inner_product_arnoldi_symmetric_and_interlacing():
    """For SPD A the M-inner-product Arnoldi on M^-1 A gives a symmetric H
    (M^-1 A is self-adjoint in <x, y> = x^T M y) whose eigenvalues interlace
    the spectrum of M^-1 A; with k = n steps they are that spectrum."""
    rng = np.random.default_rng(90)
    N = 8
    A = _spd_block_system(N, rng)
    Mb, Mi = SH.block_diag_inverse(A, N)
    Mfull = np.zeros((3 * N, 3 * N))
    for i in range(N):
        Mfull[3 * i:3 * i + 3, 3 * i:3 * i + 3] = Mb[i]
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(Mfull, A.toarray())).real)
    H = SH.arnoldi_hessenberg_m(A, N, 10)
    Hk = H[:10, :10]
    assert np.allclose(Hk, Hk.T, atol=1e-10 * np.abs(Hk).max())
    theta = np.linalg.eigvalsh(0.5 * (Hk + Hk.T))
    assert ev[0] - 1e-10 <= theta[0] and theta[-1] <= ev[-1] + 1e-10
    Hn = SH.arnoldi_hessenberg_m(A, N, 3 * N)
    kk = Hn.shape[1]
    assert kk == 3 * N
    Hs = Hn[:kk, :kk]
    assert np.allclose(np.linalg.eigvalsh(0.5 * (Hs + Hs.T)), ev, atol=1e-8 * ev[-1])


@pytest.mark.parametrize("degree", [1, 3, 5])
def test_block_chebyshev_residual_polynomial(degree):
    """z = p(M^-1 A) M^-1 v with M the 3x3 block diagonal: the residual
    M^-1 (v - A z) is T_k((theta - M^-1 A)/delta) / T_k(sigma) M^-1 v."""
    rng = np.random.default_rng(91 + degree)
    N = 6
    A = _spd_block_system(N, rng)
    _, Mi = SH.block_diag_inverse(A, N)
    Minv = np.zeros((3 * N, 3 * N))
    for i in range(N):
        Minv[3 * i:3 * i + 3, 3 * i:3 * i + 3] = Mi[i]
    T = Minv @ A.toarray()
    lam, X = np.linalg.eig(T)
    lam, X = lam.real, X.real
    lmin, lmax = 0.9 * lam.min(), 1.05 * lam.max()
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    v = rng.standard_normal(3 * N)
    z = SH.chebyshev_apply_block(A, N, lmin, lmax, degree, v)
    c = np.zeros(degree + 1)
    c[degree] = 1.0
    poly = npcheb.chebval((theta - lam) / delta, c) / npcheb.chebval(theta / delta, c)
    ref = X @ (poly * np.linalg.solve(X, Minv @ v))
    assert np.allclose(Minv @ (v - A @ z), ref, rtol=1e-9, atol=1e-11 * np.abs(Minv @ v).max())
