"""Shared helpers of the GPU parity tests: build/load the CUDA library, upload
seeded inputs, and express oracle matrices in the library's block-CSR order."""
from __future__ import annotations

import numpy as np
import torch

from paper_1809_06350_gb300 import build, hyel as H, inputs
from oracle import system as S

_BUILT = False


def ensure_built():
    global _BUILT
    if not _BUILT:
        build.build()
        _BUILT = True


class GpuProblem:
    """A mesh uploaded to the CUDA library plus the matching oracle problem."""

    def __init__(self, mesh, mat, fields=None, load=None, with_oracle=True):
        ensure_built()
        self.mesh, self.mat, self.fields = mesh, mat, fields
        self.load = load or {"p_max": 0.0, "t_ramp": 1.0}
        self.stream = torch.cuda.current_stream().cuda_stream
        self.ctx = H.hyel_create(0, self.stream)
        self.inp = H.MeshInputs(mesh, mat, fields, self.load)
        H.hyel_mesh_upload(self.ctx, self.inp.X, self.inp.tets, self.inp.bc, self.inp.mat)
        self.info = H.hyel_mesh_info(self.ctx)
        self.N = self.info["N"]
        self.prob = S.Problem(mesh, mat, fields=fields, load=self.load) if with_oracle else None

    def close(self):
        if self.ctx is not None:
            H.hyel_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- device state helpers
    @staticmethod
    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")

    def stage(self, st):
        t = {k: self.dev(st[k]) for k in ("u", "p", "v", "udot", "pdot", "vdot")}
        return t, H.state_struct(t["u"], t["p"], t["v"], t["udot"], t["pdot"], t["vdot"])

    def download(self):
        rp, col, A, B, C, D = H.hyel_matrix_download(self.ctx, self.N, self.info["nnzb"])
        return rp, col, A, B, C, D


def oracle_blocks(K, N, rp, col):
    """Blocks of an oracle 4N x 4N matrix at the library's block-CSR positions."""
    Kd = K.toarray() if hasattr(K, "toarray") else K
    rows = np.repeat(np.arange(N), np.diff(rp))
    r3 = 3 * rows[:, None] + np.arange(3)
    c3 = 3 * col[:, None] + np.arange(3)
    A = Kd[r3[:, :, None], c3[:, None, :]]
    B = Kd[r3, 3 * N + col[:, None]]
    C = Kd[3 * N + rows[:, None], c3]
    D = Kd[3 * N + rows, 3 * N + col]
    return A, B, C, D


def row_scaled_error(gpu, orc, rows, nrows):
    """max over entries of |gpu - orc| / max|orc over the same block row| (X16 reading)."""
    g = gpu.reshape(gpu.shape[0], -1)
    o = orc.reshape(orc.shape[0], -1)
    scale = np.zeros(nrows)
    np.maximum.at(scale, rows, np.abs(o).max(axis=1))
    s = scale[rows][:, None]
    s = np.where(s > 0, s, 1.0)
    return np.max(np.abs(g - o) / s)


def gen_alpha(rho_inf):
    return S.gen_alpha(rho_inf)


def oracle_blocks_sparse(K, N, rows, cols):
    """Blocks (rows[k], cols[k]) of a sparse oracle 4N x 4N matrix, vectorized."""
    K = K.tocsr()
    r3 = (3 * rows[:, None] + np.arange(3)).astype(np.int64)
    c3 = (3 * cols[:, None] + np.arange(3)).astype(np.int64)
    A = np.asarray(K[np.repeat(r3, 3, axis=1).ravel(), np.tile(c3, (1, 3)).ravel()]).reshape(-1, 3, 3)
    B = np.asarray(K[r3.ravel(), np.repeat(3 * N + cols, 3)]).reshape(-1, 3)
    C = np.asarray(K[np.repeat(3 * N + rows, 3), c3.ravel()]).reshape(-1, 3)
    D = np.asarray(K[3 * N + rows, 3 * N + cols]).ravel()
    return A, B, C, D
