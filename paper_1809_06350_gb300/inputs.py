"""Seeded synthetic inputs: meshes, boundary sets, material parameters and states.

This module is the only code shared by the CUDA path and the CPU oracle. It
generates *inputs* (node coordinates, tetrahedra, boundary sets, material
parameters, random states) and holds none of the method's arithmetic: no
residual, no tangent, no time-integration constant, no solver step.

Workloads (all seeded, all synthetic; the paper's Gmsh meshes are not
available, so structured meshes of the same shape stand in for them):

* ``cube``: the compressed-block benchmark of §5.1 on a unit cube, an
  ``n x n x n`` hex grid with every hex split into 6 tetrahedra along one
  consistent main diagonal (a conforming Kuhn/Freudenthal split). Interior
  nodes are jittered uniformly by +-5% of the grid spacing per component.
  Bottom face: u_z = 0; faces x = 0 and y = 0: symmetry rollers (u_x = 0,
  u_y = 0); top face: dead nominal traction -P(t) e_z.
* ``tube``: the thick-walled arterial tube standing in for the §5.2 strip,
  swept in (r, theta, z) with theta periodic, HGO fibres at +-40 degrees.
"""
from __future__ import annotations

import numpy as np

# Local corner offsets of a hex cell, indexed by bit pattern (x | y<<1 | z<<2).
_CORNERS = np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])

# The 6 tetrahedra of the Kuhn split: each is the path 0 -> e_a -> e_a+e_b -> 7
# for a permutation (a, b, c) of the three axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _kuhn_local_tets():
    tets = []
    for a, b, _c in _PERMS:
        c0 = 0
        c1 = c0 | (1 << a)
        c2 = c1 | (1 << b)
        c3 = 7
        tets.append((c0, c1, c2, c3))
    return np.array(tets, dtype=np.int64)


def _signed_volumes(X, tets):
    d1 = X[tets[:, 1]] - X[tets[:, 0]]
    d2 = X[tets[:, 2]] - X[tets[:, 0]]
    d3 = X[tets[:, 3]] - X[tets[:, 0]]
    return np.einsum("ei,ei->e", d1, np.cross(d2, d3)) / 6.0


def _orient_positive(X, tets):
    """Swap two vertices of every tetrahedron whose signed volume is negative."""
    vol = _signed_volumes(X, tets)
    neg = vol < 0
    t = tets.copy()
    t[neg, 1], t[neg, 2] = tets[neg, 2], tets[neg, 1]
    return t


def structured_tets(nx, ny, nz, periodic_y=False):
    """Connectivity of a Kuhn-split structured grid with (nx+1)(ny+1)(nz+1) nodes.

    With ``periodic_y`` the y index wraps (ny distinct node layers), which the
    tube uses for its periodic theta direction.
    """
    nyn = ny if periodic_y else ny + 1
    loc = _kuhn_local_tets()
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    cells = []
    for t in loc:
        verts = []
        for c in t:
            ci = i + _CORNERS[c, 0]
            cj = j + _CORNERS[c, 1]
            ck = k + _CORNERS[c, 2]
            if periodic_y:
                cj = cj % ny
            verts.append(ci + (nx + 1) * (cj + nyn * ck))
        cells.append(np.stack(verts, axis=1))
    tets = np.stack(cells, axis=1).reshape(-1, 4)
    return tets


def cube_mesh(n=8, L=1.0, jitter=0.05, seed=0):
    """Unit-cube compression mesh (the §5.1 block benchmark's geometry).

    Returns a dict with node coordinates ``X`` [N,3] (float64), positively
    oriented tetrahedra ``tets`` [E,4] (int32), outward top-face triangles
    ``traction_tris`` [T,3] (int32), the Dirichlet list ``dirichlet`` [K,2]
    (node, component) with prescribed values ``dirichlet_values`` [K] (zero:
    rollers and the fixed bottom), and the grid size.
    """
    h = L / n
    g = np.arange(n + 1) * h
    Xi, Yi, Zi = np.meshgrid(g, g, g, indexing="ij")
    # lexicographic node order: x fastest
    X = np.stack([Xi.transpose(2, 1, 0).ravel(), Yi.transpose(2, 1, 0).ravel(),
                  Zi.transpose(2, 1, 0).ravel()], axis=1)
    idx = np.arange(X.shape[0])
    ix = idx % (n + 1)
    iy = (idx // (n + 1)) % (n + 1)
    iz = idx // ((n + 1) ** 2)
    interior = (ix > 0) & (ix < n) & (iy > 0) & (iy < n) & (iz > 0) & (iz < n)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=X.shape)
        X = X + d * interior[:, None]
    tets = _orient_positive(X, structured_tets(n, n, n))
    # top face (z = L) triangles: split each top quad along the same diagonal
    # as the Kuhn split (corner 0 -> corner 3 of the quad in x,y)
    qi, qj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    qi, qj = qi.ravel(), qj.ravel()
    base = n * (n + 1) ** 2

    def nid(a, b):
        return base + a + (n + 1) * b

    n00, n10, n01, n11 = nid(qi, qj), nid(qi + 1, qj), nid(qi, qj + 1), nid(qi + 1, qj + 1)
    # outward normal +z: counter-clockwise seen from above
    tris = np.concatenate([np.stack([n00, n10, n11], 1), np.stack([n00, n11, n01], 1)], 0)
    dir_nodes, dir_comps = [], []
    for comp, sel in ((0, ix == 0), (1, iy == 0), (2, iz == 0)):
        nodes = idx[sel]
        dir_nodes.append(nodes)
        dir_comps.append(np.full(nodes.shape, comp))
    dirichlet = np.stack([np.concatenate(dir_nodes), np.concatenate(dir_comps)], 1)
    order = np.lexsort((dirichlet[:, 1], dirichlet[:, 0]))
    dirichlet = dirichlet[order]
    return {
        "name": f"cube{n}",
        "X": np.ascontiguousarray(X, dtype=np.float64),
        "tets": np.ascontiguousarray(tets, dtype=np.int32),
        "traction_tris": np.ascontiguousarray(tris, dtype=np.int32),
        "traction_dir": np.array([0.0, 0.0, -1.0]),
        "dirichlet": np.ascontiguousarray(dirichlet, dtype=np.int32),
        "dirichlet_values": np.zeros(dirichlet.shape[0]),
        "n": n,
        "h": h,
    }


def tube_mesh(nr=10, nth=200, nz=100, r_in=0.01, wall=0.002, L=0.05, stretch=0.2):
    """Thick-walled tube (arterial-wall stand-in), theta periodic.

    z = 0: u_z = 0; z = L: u_z = stretch * L * s(t) (the ramp s is applied by
    the caller's load schedule); one node on z = 0 pinned in x and y, and a
    second one pinned in y, to remove rigid translation and rotation.
    Fibre directions per element: a_{1,2} = cos(40 deg) e_theta +- sin(40 deg)
    e_z at the element centroid (angle from the circumferential direction).
    """
    r = r_in + np.arange(nr + 1) * (wall / nr)
    th = np.arange(nth) * (2 * np.pi / nth)
    z = np.arange(nz + 1) * (L / nz)
    R, T, Z = np.meshgrid(r, th, z, indexing="ij")
    # node order: r fastest, then theta, then z (matches structured_tets)
    R = R.transpose(2, 1, 0).ravel()
    T = T.transpose(2, 1, 0).ravel()
    Z = Z.transpose(2, 1, 0).ravel()
    X = np.stack([R * np.cos(T), R * np.sin(T), Z], 1)
    tets = _orient_positive(X, structured_tets(nr, nth, nz, periodic_y=True))
    idx = np.arange(X.shape[0])
    iz = idx // ((nr + 1) * nth)
    bottom = idx[iz == 0]
    top = idx[iz == nz]
    dn = [bottom, top]
    dc = [np.full(bottom.shape, 2), np.full(top.shape, 2)]
    dv = [np.zeros(bottom.shape), np.full(top.shape, stretch * L)]
    # pin node (r_in, theta=0, z=0) in x and y, node (r_in, theta=pi/2, z=0) in x
    n0 = 0
    n1 = (nr + 1) * (nth // 4)
    dn += [np.array([n0, n0, n1])]
    dc += [np.array([0, 1, 0])]
    dv += [np.zeros(3)]
    dirichlet = np.stack([np.concatenate(dn), np.concatenate(dc)], 1)
    vals = np.concatenate(dv)
    order = np.lexsort((dirichlet[:, 1], dirichlet[:, 0]))
    cen = X[tets].mean(axis=1)
    thc = np.arctan2(cen[:, 1], cen[:, 0])
    e_th = np.stack([-np.sin(thc), np.cos(thc), np.zeros_like(thc)], 1)
    e_z = np.array([0.0, 0.0, 1.0])
    ang = np.deg2rad(40.0)
    a1 = np.cos(ang) * e_th + np.sin(ang) * e_z
    a2 = np.cos(ang) * e_th - np.sin(ang) * e_z
    return {
        "name": f"tube{nr}x{nth}x{nz}",
        "X": np.ascontiguousarray(X, dtype=np.float64),
        "tets": np.ascontiguousarray(tets, dtype=np.int32),
        "traction_tris": np.zeros((0, 3), dtype=np.int32),
        "traction_dir": np.array([0.0, 0.0, -1.0]),
        "dirichlet": np.ascontiguousarray(dirichlet[order], dtype=np.int32),
        "dirichlet_values": np.ascontiguousarray(vals[order]),
        "fibre_a1": np.ascontiguousarray(a1),
        "fibre_a2": np.ascontiguousarray(a2),
    }


def kappa_from_nu(mu, nu):
    """Bulk modulus from shear modulus and Poisson ratio (isotropic elasticity)."""
    if nu >= 0.5:
        return np.inf
    return 2.0 * mu * (1.0 + nu) / (3.0 * (1.0 - 2.0 * nu))


def material_nh(mu=1e5, kappa=1e6, rho0=1e3, body=(0.0, 0.0, 0.0)):
    """Compressible neo-Hookean Gibbs material (§5.1); kappa = inf means incompressible."""
    vol = "incompressible" if not np.isfinite(kappa) else "gibbs"
    return {"vol": vol, "mu": float(mu), "kappa": float(kappa) if np.isfinite(kappa) else 0.0,
            "rho0": float(rho0), "body": np.array(body, dtype=np.float64), "fibres": 0,
            "k1": 0.0, "k2": 0.0, "kd": 0.0, "c_m": 1e-3}


def material_hgo(mu=3e4, k1=2e5, k2=5.0, kd=0.0, rho0=1e3):
    """Fully incompressible HGO material with two fibre families (§5.2)."""
    return {"vol": "incompressible", "mu": float(mu), "kappa": 0.0, "rho0": float(rho0),
            "body": np.zeros(3), "fibres": 2, "k1": float(k1), "k2": float(k2),
            "kd": float(kd), "c_m": 1e-3}


def element_fields(n_tets, mat, seed=1, sigma=0.3, with_fibres=False):
    """Per-element log-normal random fields: mu_e = mu exp(sigma xi),
    kappa_e = kappa exp(sigma zeta), xi, zeta iid N(0,1) (seeded)."""
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(n_tets)
    zeta = rng.standard_normal(n_tets)
    out = {"mu_e": mat["mu"] * np.exp(sigma * xi)}
    if mat["vol"] == "gibbs":
        out["kappa_e"] = mat["kappa"] * np.exp(sigma * zeta)
    if with_fibres:
        eta = rng.standard_normal(n_tets)
        out["k1_e"] = mat["k1"] * np.exp(sigma * eta)
        out["k2_e"] = mat["k2"] * np.exp(0.1 * sigma * rng.standard_normal(n_tets))
    return out


def random_state(n_nodes, seed=3, u_scale=1e-3, v_scale=1e-2, p_scale=1e3,
                 rate_scale=1.0):
    """A seeded random (y, ydot) state used to exercise every term of the
    residual and tangent in parity tests. Returns dict of float64 arrays:
    u, v [N,3], p [N], udot, vdot [N,3], pdot [N]."""
    rng = np.random.default_rng(seed)
    return {
        "u": u_scale * rng.standard_normal((n_nodes, 3)),
        "v": v_scale * rng.standard_normal((n_nodes, 3)),
        "p": p_scale * rng.standard_normal(n_nodes),
        "udot": v_scale * rng.standard_normal((n_nodes, 3)),
        "vdot": rate_scale * rng.standard_normal((n_nodes, 3)),
        "pdot": p_scale * rate_scale * rng.standard_normal(n_nodes),
    }


def zero_state(n_nodes):
    z3 = np.zeros((n_nodes, 3))
    z1 = np.zeros(n_nodes)
    return {"u": z3.copy(), "v": z3.copy(), "p": z1.copy(),
            "udot": z3.copy(), "vdot": z3.copy(), "pdot": z1.copy()}


def load_schedule(p_max=2e4, n_steps=1, dt=1e-3):
    """Dead-load ramp: P(t) = p_max * min(t / (n_steps * dt), 1)."""
    return {"p_max": float(p_max), "t_ramp": float(n_steps * dt)}


def random_vector(n, seed=7):
    return np.random.default_rng(seed).standard_normal(n)
