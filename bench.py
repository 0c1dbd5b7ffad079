#!/usr/bin/env python
"""Benchmark: Newton linear-solve throughput of the nested block-preconditioned
Newton step on one GB300 (FP64; FP32 preconditioner levels; FP32 levels with
A read as BF16 entries times a per-block FP32 scale), plus BSR SpMV bandwidth.

Workload (one bench step = one generalized-alpha time step, every part of the
hot path: stage values, element assembly, Dirichlet elimination, diagonal
scaling, outer FGMRES with the SCR preconditioner to 1e-10, Newton update):
the 48^3-hex cube (663,552 P1 tets, 117,649 nodes, 470,596 linear unknowns),
compressible neo-Hookean Gibbs material mu = 1e5 Pa, nu = 0.3 (kappa from
nu), rho0 = 1e3, dead load 2e4 Pa on the top face ramped over 10 steps,
dt = 1e-3, rho_inf = 0.5, sub-solver tolerances 1e-2. K timed steps run
t = 0, dt, ..., (K-1) dt from rest (K = 10 is the whole 10-step run). The
S-solve is preconditioned by the degree-8 Chebyshev polynomial in the explicit
S^ = D - C diag(A)^-1 B (its values and interval rebuilt every Newton
iteration, inside the timed region); --s-precond jacobi selects diag(S^)^-1.

metric value = linear unknowns x Newton linear solves per second over all
ranks (replicas: every rank solves its own copy; no collective in the path).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hyel|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton linear-solve time & BSR SpMV GB/s on 1 GB300, FP64 vs mixed at 1e-9 rel"
UNIT = "unknowns*solves/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="hyel", choices=["hyel", "reference"])
    p.add_argument("--n", type=int, default=48, help="hexes per cube edge")
    p.add_argument("--nu", type=float, default=0.3)
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the Poisson-ratio sweep keys")
    p.add_argument("--no-tube", action="store_true", help="skip the full-size tube (config 3) step")
    p.add_argument("--tube-dt", type=float, default=1e-5, help="time step of the full-size tube step")
    p.add_argument("--tube-only", action="store_true",
                   help="instead of the benchmark: only the full-size tube step (--tube-dt, solver options as given)")
    p.add_argument("--stiff-only", action="store_true",
                   help="instead of the benchmark: only the stiff full-size tube solve with the multigrid A-solves")
    p.add_argument("--compare-a-precond", action="store_true",
                   help="instead of the benchmark: one nested solve of a stiffness-dominated tube system per "
                        "A-preconditioner (block-Jacobi, multigrid, Chebyshev), iteration counts and times")
    p.add_argument("--host-loops", action="store_true",
                   help="drive the Krylov loops from the host (for per-kernel ncu launch lists)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16s"],
                   help="preconditioner-level precision of the main timed run (fp64 is the headline; "
                        "the mixed forms are also timed beside it unless --no-mixed)")
    p.add_argument("--s-precond", default="cheb", choices=["jacobi", "cheb"],
                   help="S-solve preconditioner: the Chebyshev polynomial in the explicit S^ (default), "
                        "or diag(S^)^-1")
    p.add_argument("--cheb-degree", type=int, default=8)
    p.add_argument("--a-precond", default="bjacobi", choices=["bjacobi", "cheb", "amg"],
                   help="A-solve preconditioner: 3x3 block-Jacobi (default), the Chebyshev polynomial in "
                        "M^-1 A, or aggregation multigrid")
    p.add_argument("--dt", type=float, default=1e-3, help="time step (the paper's cube runs 1e-1 and 1e-5)")
    p.add_argument("--inner", default="gmres", choices=["gmres", "cg"],
                   help="inner A-solve of the S product: GMRES on A (default) or CG on (A + A^T)/2")
    p.add_argument("--block", default="ldu", choices=["ldu", "du", "d", "simple"],
                   help="block preconditioner of the outer FGMRES: Algorithm 1 (ldu, default), its DU and D "
                        "parts, or SIMPLE (the paper's comparison baseline)")
    p.add_argument("--cheb-ratio", type=float, default=0.0,
                   help="0: interval from Ritz estimates; > 1: fixed lmax / lmin")
    return p.parse_args()


def workload(args):
    from paper_1809_06350_gb300 import inputs
    dt = args.dt
    mesh = inputs.cube_mesh(args.n, jitter=0.05, seed=0)
    mu = 1e5
    mat = inputs.material_nh(mu, inputs.kappa_from_nu(mu, args.nu), 1e3)
    load = {"p_max": 2e4, "t_ramp": 10 * dt}
    return mesh, mat, load, dt


def config_dict(args, mesh):
    N = mesh["X"].shape[0]
    sprec = "diag(S^)" if args.s_precond == "jacobi" else \
        f"chebyshev(S^), degree {args.cheb_degree}, " + \
        (f"lmax/lmin {args.cheb_ratio:g}" if args.cheb_ratio > 0 else "interval from Ritz values")
    return {"workload": f"cube{args.n}^3 compression, nu={args.nu}", "levels": args.precision,
            "s_precond": sprec, "block_precond": args.block.upper(),
            "inner_solver": "CG on (A + A^T)/2" if args.inner == "cg" else "GMRES on A",
            "a_precond": args.a_precond,
            "tets": int(mesh["tets"].shape[0]),
            "nodes": int(N), "unknowns": int(4 * N), "dt": args.dt, "rho_inf": 0.5, "outer_rtol": 1e-10,
            "sub_rtol": 1e-2, "steps_per_run": "t = 0..K-1 from rest, load ramp over 10 steps",
            "l2": "working set larger than L2 (FP64 blocks 218 MB, Krylov bases > 1 GB); no flush",
            "parallelism": "replicas"}


# ------------------------------------------------------------------ clocks

class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                r = [x.strip() for x in r]
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(kernel, source="sparse.cu", field="dram_bytes_per_launch_full_size"):
    """DRAM bytes (per launch, or per unit named by `field`) from the committed
    ncu summary, if it was taken on the current source of the kernel; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}.md")
    src = os.path.join(ROOT, "paper_1809_06350_gb300", "csrc", source)
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith("- ") and ":" in line)
        fields = {k.strip("- ").strip(): v.strip() for k, v in fields.items()}
        if fields.get("source_sha256_16") != sha:
            return None
        return float(fields[field])
    except Exception:
        return None


def cpu_sample(n_sample=12, steps=2, args=None):
    """The oracle (complex-step assembly + SuperLU direct solves) on a
    bounded sample: the same cube workload at n_sample^3 hexes."""
    import numpy as np
    from oracle import newton as Nw
    from oracle import system as S
    from paper_1809_06350_gb300 import inputs
    mesh = inputs.cube_mesh(n_sample, jitter=0.05, seed=0)
    mu = 1e5
    nu = args.nu if args else 0.3
    mat = inputs.material_nh(mu, inputs.kappa_from_nu(mu, nu), 1e3)
    dt = args.dt if args else 1e-3
    prob = S.Problem(mesh, mat, load={"p_max": 2e4, "t_ramp": 10 * dt})
    z = inputs.zero_state(prob.N)
    yn = {k: z[k] for k in ("u", "p", "v")}
    ydn = {k: z[k] for k in ("udot", "pdot", "vdot")}
    solves = 0
    t0 = time.perf_counter()
    for k in range(steps):
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, k * dt, dt)
        solves += info["iterations"]
        yn = {kk: y1[kk] for kk in ("u", "p", "v")}
        ydn = {kk: yd1[kk] for kk in ("udot", "pdot", "vdot")}
    sec = time.perf_counter() - t0
    n = 4 * prob.N
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return {"value": n * solves / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle Newton steps t=0..{steps - 1} on the {n_sample}^3-hex cube "
                      f"(n={n} unknowns, {solves} direct solves, {sec:.1f} s); rate in unknowns*solves/s"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def cpu_plan(args):
    """The CPU side of the measurement plan, on the host cores of the GPU machine:
    (1) the oracle's element assembly (the complex-step residual Jacobian of
    the Appendix A element routine, vectorized numpy over elements, one
    thread) timed on a 16^3-hex sample (24,576 tets) of the workload's cube
    and scaled to one pass over the 48^3 cube's 663,552 tets; (2) the
    oracle's direct solve (SuperLU, COLAMD) of one Newton system of the
    16^3-hex cube (n = 19,652). The 48^3 direct solve is not attempted: its
    banded storage alone is about 74 GB."""
    from oracle import system as S
    from paper_1809_06350_gb300 import inputs
    n = 16
    mesh = inputs.cube_mesh(n, jitter=0.05, seed=0)
    mu = 1e5
    mat = inputs.material_nh(mu, inputs.kappa_from_nu(mu, args.nu), 1e3)
    prob = S.Problem(mesh, mat, load={"p_max": 2e4, "t_ramp": 10 * args.dt})
    st = inputs.random_state(prob.N, seed=17, u_scale=0.02 / n, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, args.dt)
    t0 = time.perf_counter()
    K = S.assemble_matrix(prob, st, ga)
    t_asm = time.perf_counter() - t0
    rhs, _, _, _ = S.newton_rhs(prob, st, af * args.dt, ga)
    Kd, r = S.apply_dirichlet(K, rhs, S.dirichlet_dofs(prob))
    t0 = time.perf_counter()
    S.direct_solve(Kd, r)
    t_lu = time.perf_counter() - t0
    E48 = 6 * 48 ** 3
    return {"cpu_model": cpu_model(),
            "oracle_assembly_pass_s_cube48": t_asm * E48 / prob.E,
            "oracle_assembly_sample": f"tangent assembly of the {n}^3-hex cube ({prob.E} tets, {t_asm:.2f} s, one "
                                      f"thread), scaled by 663,552 / {prob.E}",
            "oracle_direct_solve_s_cube16": t_lu,
            "oracle_direct_solve_sample": f"SuperLU (COLAMD) factor + solve of one Newton system, n = {4 * prob.N}",
            "oracle_direct_solve_cube48": "not attempted: banded storage about 74 GB"}


# ------------------------------------------------------------------ arms

def run_reference(args, rank, world):
    if rank != 0:
        return
    base = cpu_sample(args=args)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        cpu_sample(n_sample=8, steps=1, args=args)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_sample(n_sample=10, steps=1, args=args)["value"])
    sec = time.perf_counter() - t0
    v = statistics.mean(vals)
    mesh, _, _, _ = workload(args)
    cfg = config_dict(args, mesh)
    cfg["workload"] += " (oracle timed on a 10^3-hex sample of it)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(1, args.steps + args.warmup),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": "each step: oracle Newton step t=0 on the 10^3-hex cube (direct solve)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def nu_sweep(ctx, H, torch, stream, args, names, sizes, dev, state, sprec_kw, graph, steps=5):
    """The Poisson-ratio sweep of the cube workload (nu = 0.45, 0.499 and the
    incompressible model nu = 0.5), same mesh, load and solver options as the
    headline run: `steps` time steps from rest with FP64 levels and with FP32
    levels, each timed with CUDA events on the library's stream after one
    warm-up step, and the relative difference of the FP32-level state from the
    FP64-level state after every step (untimed rerun)."""
    from paper_1809_06350_gb300 import inputs
    out = {}
    mu = 1e5
    mesh = inputs.cube_mesh(args.n, jitter=0.05, seed=0)
    load = {"p_max": 2e4, "t_ramp": 10 * args.dt}
    for nu in (0.45, 0.499, 0.5):
        mat = inputs.material_nh(mu, inputs.kappa_from_nu(mu, nu), 1e3)
        inp = H.MeshInputs(mesh, mat, None, load)
        H.hyel_mesh_upload(ctx, inp.X, inp.tets, inp.bc, inp.mat)
        row = {}
        states = {}
        for lab, prec in (("fp64", H.HYEL_PREC_FP64), ("fp32", H.HYEL_PREC_FP32)):
            sp = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=prec, graph=graph, **sprec_kw)
            for t in dev.values():
                t.zero_()
            H.hyel_newton_step(ctx, H.time_params(dt=args.dt, t_n=0.0), sp, state, raise_on_error=False)
            for t in dev.values():
                t.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            its = 0
            e0.record(stream)
            for k in range(steps):
                st, rc = H.hyel_newton_step(ctx, H.time_params(dt=args.dt, t_n=k * args.dt), sp, state,
                                            raise_on_error=False)
                if rc not in (H.HYEL_OK, H.HYEL_ENOCONV):
                    raise H.HyelError(rc, H.hyel_last_error(ctx))
                its += st.iterations
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[lab + "_ms_per_step"] = ms / steps
            row[lab + "_newton_solves"] = its
            for t in dev.values():
                t.zero_()
            seq = []
            for k in range(steps):
                H.hyel_newton_step(ctx, H.time_params(dt=args.dt, t_n=k * args.dt), sp, state, raise_on_error=False)
                seq.append(torch.cat([dev[nm] for nm in names]).clone())
            states[lab] = seq
        row["fp32_per_step_rel_diff_vs_fp64"] = [
            float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(states["fp32"], states["fp64"])]
        row["speedup_fp32_vs_fp64"] = row["fp64_ms_per_step"] / row["fp32_ms_per_step"]
        out[f"nu={nu}"] = row
    out["note"] = (f"{steps} time steps from rest per run after one warm-up step, 48^3 cube, dead load ramped over 10 "
                   "steps, headline solver options; nu = 0.5 is the incompressible model")
    return out


def tube_step(ctx, H, torch, stream, graph, sprec_kw, dt=1e-5, precisions=None):
    """Config 3 at full size: the thick-walled HGO tube (10 x 200 x 100 hexes,
    1.2M tets, 222,200 nodes, fully incompressible, fibres at +-40 degrees),
    the first time step of the 20 % stretch ramp (10 steps) from rest at the
    paper's small HGO time step dt = 1e-5, FP64 and FP32 levels: one untimed
    step (builds the workspaces and graphs), then the same step from rest
    timed with CUDA events on the library's stream."""
    from paper_1809_06350_gb300 import inputs
    m = inputs.tube_mesh()
    mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.0)
    inp = H.MeshInputs(m, mat, None, {"p_max": 0.0, "t_ramp": 10 * dt})
    H.hyel_mesh_upload(ctx, inp.X, inp.tets, inp.bc, inp.mat)
    N = m["X"].shape[0]
    z = {k: torch.zeros(3 * N if k in ("u", "v", "udot", "vdot") else N, dtype=torch.float64, device="cuda")
         for k in ("u", "p", "v", "udot", "pdot", "vdot")}
    state = H.state_struct(z["u"], z["p"], z["v"], z["udot"], z["pdot"], z["vdot"])
    out = {"workload": f"tube 10x200x100 HGO (N={N}, E={m['tets'].shape[0]}, n={4 * N}), dt={dt:g}, "
                       "first step of a 10-step stretch ramp to 20 %, from rest"}
    for lab, prec in (precisions or (("fp64", H.HYEL_PREC_FP64), ("fp32", H.HYEL_PREC_FP32))):
        sp = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=prec, graph=graph, **sprec_kw)
        tp = H.time_params(dt=dt, t_n=0.0, l_max=8)
        for rep in range(1 if len(precisions or ()) else 2):
            for t in z.values():
                t.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, rc = H.hyel_newton_step(ctx, tp, sp, state, raise_on_error=False)
            e1.record(stream)
            torch.cuda.synchronize()
        out[lab] = {"ms_per_step": e0.elapsed_time(e1), "newton_its": st.iterations, "converged": bool(st.converged),
                    "rel_residual": st.res_norm / st.res_norm0 if st.res_norm0 else None, "outer_its": st.outer_its,
                    "a_its": st.a_its, "s_its": st.s_its, "inner_its": st.inner_its, "status": rc,
                    "unknowns_solves_per_s": 4 * N * st.iterations / (e0.elapsed_time(e1) * 1e-3)}
    if precisions is None:
        out["stiff_solve_multigrid"] = stiff_tube_solve(ctx, H, torch, stream, N, graph)
    return out


def stiff_tube_solve(ctx, H, torch, stream, N, graph=1, dt=1e-3):
    """The same tube where A is stiffness-dominated (dt = 1e-3: c2 K about
    10^3 alpha_m M on the wall): the tangent at rest, one nested solve of a
    seeded random right-hand side (outer 1e-10, sub-solvers 1e-2) with the
    smoothed-aggregation multigrid A-solves and point-Jacobi on diag(S^),
    FP32 levels. The first solve builds the hierarchy and its operators; the
    second is timed with CUDA events on the library's stream."""
    from paper_1809_06350_gb300 import inputs
    z = [torch.zeros(3 * N if k in (0, 2, 3, 5) else N, dtype=torch.float64, device="cuda") for k in range(6)]
    H.hyel_assemble(ctx, H.time_params(dt=dt), H.state_struct(*z), 0, 0)
    rhs = torch.as_tensor(inputs.random_vector(4 * N, seed=1), device="cuda")
    sp = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=H.HYEL_PREC_FP32, graph=graph,
                         a_precond=H.HYEL_APREC_AMG, s_precond=H.HYEL_SPREC_JACOBI)
    for rep in range(2):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, rc = H.hyel_solve_nested(ctx, sp, rhs.data_ptr(), x.data_ptr(), raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
    return {"workload": f"tube 10x200x100 HGO (n={4 * N}), dt={dt:g}, tangent at rest, random right-hand side",
            "solver": "multigrid A-solves (smoothed aggregation, rigid-body modes), diag(S^), FP32 levels",
            "ms": e0.elapsed_time(e1), "status": rc, "outer_its": st.outer_its,
            "a_its_per_a_solve": st.a_its / max(1, st.a_solves),
            "inner_its_per_s_product": st.inner_its / max(1, st.inner_solves),
            "s_its_per_s_solve": st.s_its / max(1, st.s_solves), "rel_residual": st.rel_residual,
            "levels_block_nodes": [n for n, _ in H.hyel_amg_info(ctx)]}


def compare_a_precond(args):
    """The A-preconditioners on a stiffness-dominated system: the 10 x 100 x 50
    HGO tube (56,100 nodes) at dt = 1e-3 (c2 K about 10^3 alpha_m M on the thin
    wall), the tangent at rest, one nested solve (outer 1e-10, sub-solvers
    1e-2) of a seeded random right-hand side per case; block-Jacobi runs with
    FP64 levels only (with FP32 levels it reaches the 200-iteration outer cap)."""
    import torch
    from paper_1809_06350_gb300 import build as bld
    from paper_1809_06350_gb300 import hyel as H
    from paper_1809_06350_gb300 import inputs
    bld.build()
    dt = 1e-3
    m = inputs.tube_mesh(10, 100, 50)
    N = m["X"].shape[0]
    ctx = H.hyel_create(0, torch.cuda.current_stream().cuda_stream)
    inp = H.MeshInputs(m, inputs.material_hgo(3e4, 2e5, 5.0, 0.0), None, {"p_max": 0.0, "t_ramp": 10 * dt})
    H.hyel_mesh_upload(ctx, inp.X, inp.tets, inp.bc, inp.mat)
    z = {k: torch.zeros(3 * N if k in ("u", "v", "udot", "vdot") else N, dtype=torch.float64, device="cuda")
         for k in ("u", "p", "v", "udot", "pdot", "vdot")}
    H.hyel_assemble(ctx, H.time_params(dt=dt), H.state_struct(*(z[k] for k in ("u", "p", "v", "udot", "pdot",
                                                                                 "vdot"))), 0, 0)
    rhs = torch.as_tensor(inputs.random_vector(4 * N, seed=1), device="cuda")
    cases = [("block-Jacobi, diag(S^)", H.HYEL_PREC_FP64, H.HYEL_APREC_BJACOBI, H.HYEL_SPREC_JACOBI),
             ("block-Jacobi, Chebyshev-8 on S^", H.HYEL_PREC_FP64, H.HYEL_APREC_BJACOBI, H.HYEL_SPREC_CHEB),
             ("multigrid, diag(S^)", H.HYEL_PREC_FP64, H.HYEL_APREC_AMG, H.HYEL_SPREC_JACOBI),
             ("multigrid, diag(S^)", H.HYEL_PREC_FP32, H.HYEL_APREC_AMG, H.HYEL_SPREC_JACOBI),
             ("Chebyshev-8 on A, Chebyshev-8 on S^", H.HYEL_PREC_FP64, H.HYEL_APREC_CHEB, H.HYEL_SPREC_CHEB),
             ("Chebyshev-8 on A, Chebyshev-8 on S^", H.HYEL_PREC_FP32, H.HYEL_APREC_CHEB, H.HYEL_SPREC_CHEB)]
    out = []
    for name, prec, ap, sp_ in cases:
        sp = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=prec, graph=1, a_precond=ap, s_precond=sp_,
                             s_cheb_degree=8, a_cheb_degree=8)
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rc = H.hyel_solve_nested(ctx, sp, rhs.data_ptr(), x.data_ptr(), raise_on_error=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out.append({"case": name, "levels": "fp64" if prec == H.HYEL_PREC_FP64 else "fp32", "status": rc,
                    "seconds": sec, "outer_its": st.outer_its, "a_its_per_solve": st.a_its / max(1, st.a_solves),
                    "inner_its_per_solve": st.inner_its / max(1, st.inner_solves),
                    "s_its_per_solve": st.s_its / max(1, st.s_solves), "rel_residual": st.rel_residual})
    H.hyel_destroy(ctx)
    print(json.dumps({"compare_a_precond": out, "workload": "tube 10x100x50 HGO (N=%d), dt=1e-3, tangent at rest, "
                                                            "random right-hand side (seed 1)" % N}), flush=True)


def run_hyel(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1809_06350_gb300 import build as bld
    from paper_1809_06350_gb300 import hyel as H
    from paper_1809_06350_gb300 import replicas

    bld.build()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    mesh, mat, load, dt = workload(args)
    N = mesh["X"].shape[0]
    n_unk = 4 * N
    ctx = H.hyel_create(local_rank, stream.cuda_stream)
    inp = H.MeshInputs(mesh, mat, None, load)
    H.hyel_mesh_upload(ctx, inp.X, inp.tets, inp.bc, inp.mat)
    names = ("u", "p", "v", "udot", "pdot", "vdot")
    sizes = {"u": 3 * N, "p": N, "v": 3 * N, "udot": 3 * N, "pdot": N, "vdot": 3 * N}
    dev = {k: torch.zeros(sizes[k], dtype=torch.float64, device="cuda") for k in names}
    state = H.state_struct(*(dev[k] for k in names))

    def reset():
        for t in dev.values():
            t.zero_()

    acc = {"ms_solve": 0.0, "ms_assemble": 0.0}

    def run_steps(K, sp, t_offset=0, host=None):
        its = 0
        for k in range(K):
            if host is not None:
                for nm in names:
                    dev[nm].copy_(host[nm], non_blocking=True)
            tp = H.time_params(dt=dt, t_n=(t_offset + k) * dt)
            st, rc = H.hyel_newton_step(ctx, tp, sp, state, raise_on_error=False)
            if rc not in (H.HYEL_OK, H.HYEL_ENOCONV):
                raise H.HyelError(rc, H.hyel_last_error(ctx))
            its += st.iterations
            acc["ms_solve"] += st.ms_solve
            acc["ms_assemble"] += st.ms_assemble
            if host is not None:
                for nm in names:
                    host[nm].copy_(dev[nm], non_blocking=True)
        return its

    def barrier():
        replicas.barrier()

    def timed(K, sp, host=None, profile=False):
        reset()
        if host is not None:
            for t in host.values():
                t.zero_()
        barrier()
        torch.cuda.synchronize()
        if profile:
            H.hyel_profile(ctx, 1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = H.hyel_launch_count()
        e0.record(stream)
        its = run_steps(K, sp, host=host)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        launches = H.hyel_launch_count() - l0
        prof = H.hyel_profile_read(ctx) if profile else None
        if profile:
            H.hyel_profile(ctx, 0)
        ms, its_total = replicas.reduce_timing(ms, its, device="cuda")
        return ms, its, its_total, launches, prof

    graph = 0 if args.host_loops else 1
    sprec_kw = {"s_precond": H.HYEL_SPREC_JACOBI if args.s_precond == "jacobi" else H.HYEL_SPREC_CHEB,
                "s_cheb_degree": args.cheb_degree, "s_cheb_ratio": args.cheb_ratio,
                "block_precond": {"ldu": H.HYEL_BLOCK_LDU, "du": H.HYEL_BLOCK_DU, "d": H.HYEL_BLOCK_D,
                                  "simple": H.HYEL_BLOCK_SIMPLE}[args.block],
                "inner_solver": H.HYEL_INNER_CG_SYM if args.inner == "cg" else H.HYEL_INNER_GMRES,
                "a_precond": {"bjacobi": H.HYEL_APREC_BJACOBI, "cheb": H.HYEL_APREC_CHEB,
                              "amg": H.HYEL_APREC_AMG}[args.a_precond]}
    main_prec = {"fp64": H.HYEL_PREC_FP64, "fp32": H.HYEL_PREC_FP32, "bf16s": H.HYEL_PREC_BF16S}[args.precision]
    if args.stiff_only:
        from paper_1809_06350_gb300 import inputs
        tm = inputs.tube_mesh()
        tin = H.MeshInputs(tm, inputs.material_hgo(3e4, 2e5, 5.0, 0.0), None, {"p_max": 0.0, "t_ramp": 1e-2})
        H.hyel_mesh_upload(ctx, tin.X, tin.tets, tin.bc, tin.mat)
        res = stiff_tube_solve(ctx, H, torch, stream, tm["X"].shape[0], graph)
        H.hyel_destroy(ctx)
        if rank == 0:
            print(json.dumps({"stiff_solve_multigrid": res}), flush=True)
        return
    if args.tube_only:
        # one timed step per run, no warm-up: the step itself takes seconds
        res = tube_step(ctx, H, torch, stream, graph, sprec_kw, dt=args.tube_dt,
                        precisions=((args.precision, main_prec),))
        H.hyel_destroy(ctx)
        if rank == 0:
            cfg = config_dict(args, mesh)
            res["solver"] = {k: cfg[k] for k in ("levels", "s_precond", "block_precond", "inner_solver", "a_precond")}
            print(json.dumps({"config3_tube": res}), flush=True)
        return
    sp64 = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=main_prec, graph=graph, **sprec_kw)
    sp32 = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=H.HYEL_PREC_FP32, graph=graph, **sprec_kw)
    sp16 = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=H.HYEL_PREC_BF16S, graph=graph, **sprec_kw)
    # warm-up (also builds the Krylov workspaces)
    reset()
    run_steps(args.warmup, sp64)
    if not args.no_mixed and args.precision == "fp64":
        for spm in (sp32, sp16):
            reset()
            run_steps(1, spm)
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    clocks.start()
    acc["ms_solve"] = acc["ms_assemble"] = 0.0
    ms, its, its_total, launches, _ = timed(args.steps, sp64)
    ck = clocks.stop()
    solve_ms = acc["ms_solve"] / max(1, its)
    asm_ms = acc["ms_assemble"] / max(1, args.steps)  # per time step: tangent passes + residual-only checks

    final64 = torch.cat([dev[k] for k in names])

    def mixed_run(spm, cls):
        msm, itsm, itsm_total, _, _ = timed(args.steps, spm)
        fin = torch.cat([dev[k] for k in names])
        return {"value": n_unk * itsm_total / (msm / 1e3), "unit": UNIT, "ms_per_step": msm / args.steps,
                "newton_solves": itsm, "speedup_vs_fp64": ms / msm,
                "state_rel_diff_vs_fp64": float(torch.linalg.norm(fin - final64) / torch.linalg.norm(final64))}

    def per_step_states(spm):
        # untimed: the state after every time step of the same run from rest
        reset()
        out = []
        for k in range(args.steps):
            tp = H.time_params(dt=dt, t_n=k * dt)
            H.hyel_newton_step(ctx, tp, spm, state, raise_on_error=False)
            out.append(torch.cat([dev[nm] for nm in names]).clone())
        return out

    mixed = mixed16 = None
    if not args.no_mixed and args.precision == "fp64":
        mixed = mixed_run(sp32, "spmv_A32")
        mixed16 = mixed_run(sp16, "spmv_A16")
        ref_states = per_step_states(sp64)
        for md, spm in ((mixed, sp32), (mixed16, sp16)):
            st_m = per_step_states(spm)
            md["per_step_rel_diff_vs_fp64"] = [
                float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(st_m, ref_states)]
        del ref_states
    e2e = None
    if not args.no_e2e:
        host = {k: torch.zeros(sizes[k], dtype=torch.float64, pin_memory=True) for k in names}
        mse, itse, itse_total, _, _ = timed(args.steps, sp64, host=host)
        per = 8 * sum(sizes.values())
        e2e = {"value": n_unk * itse_total / (mse / 1e3), "unit": UNIT, "h2d_bytes_per_step": per,
               "d2h_bytes_per_step": per}

    value = n_unk * its_total / (ms / 1e3)
    peak, peak_kind = peaks()

    def spmv_timed(matrix, dtype, cls, reps=25):
        """The A-block SpMV of the scaled system timed alone: CUDA events on
        the library's stream around each launch, L2 flushed before each; and,
        after the same flush, a plain streaming read of the same byte count
        (hyel_stream_read_probe): the rate a kernel that reads that many bytes
        once can reach."""
        x = torch.randn(3 * N, dtype=dtype, device="cuda")
        y = torch.empty(3 * N, dtype=dtype, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        clean = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
        src = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")

        def l2_flush():
            # write 256 MB, then read another 256 MB so that the flush's dirty
            # lines are written back before the timed launch
            flush.zero_()
            clean.sum()

        H.hyel_profile(ctx, 1)
        for _ in range(reps):
            l2_flush()
            H.hyel_spmv(ctx, H.HYEL_OP_A, matrix, x.data_ptr(), y.data_ptr())
        pr = H.hyel_profile_read(ctx)[cls]
        H.hyel_profile(ctx, 0)
        us = 1e3 * pr["ms"] / pr["launches"]
        by = pr["bytes"] / pr["launches"]
        nb = int(by) // 16 * 16
        tr = 0.0
        for _ in range(reps):
            l2_flush()
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            H.hyel_stream_read_probe(ctx, src.data_ptr(), nb, sink.data_ptr())
            r1.record(stream)
            torch.cuda.synchronize()
            tr += r0.elapsed_time(r1)
        read_gbs = nb / (tr / reps * 1e-3) / 1e9
        return by / (us * 1e-6) / 1e9, us, by, read_gbs

    # per-launch CUDA events need host-launched kernels: replay the same K
    # steps with host-driven Krylov loops (same kernels, same order, same
    # iterates) and time every launch of the profiled classes on the stream
    sp_prof = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=main_prec, graph=0, **sprec_kw)
    _, _, _, _, prof_host = timed(args.steps, sp_prof, profile=True)
    dom = max(("gmres_A", "gmres_S"), key=lambda k: prof_host[k]["ms"])  # the dominant persistent kernel
    pl = prof_host[dom]
    us_live = 1e3 * pl["ms"] / max(1, pl["launches"])
    by_live = pl["bytes"] / max(1, pl["launches"])
    gbs_live = by_live / (us_live * 1e-6) / 1e9 if pl["launches"] else None

    def fp64_peak(reps=5):
        """FP64 FMA rate of this GPU, measured now by the library's probe
        kernel (independent FMA chains, no memory traffic), best of reps."""
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")
        H.hyel_fp64_fma_probe(ctx, 1 << 10, sink.data_ptr())
        best = 0.0
        for _ in range(reps):
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fl = H.hyel_fp64_fma_probe(ctx, 1 << 14, sink.data_ptr())
            a1.record(stream)
            torch.cuda.synchronize()
            best = max(best, fl / (a0.elapsed_time(a1) * 1e-3) / 1e12)
        return best

    fp64_tflops = fp64_peak()

    H.hyel_solve_setup(ctx)
    gbs64, us64, by64, rd64 = spmv_timed(H.HYEL_MAT_SCALED64, torch.float64, "spmv_A64")
    gbs32, us32, by32, rd32 = spmv_timed(H.HYEL_MAT_SCALED32, torch.float32, "spmv_A32")
    gbs16, us16, by16, rd16 = spmv_timed(H.HYEL_MAT_SCALED_BF16S, torch.float32, "spmv_A16")
    tname = {"fp64": "<double>", "fp32": "<float>", "bf16s": "<float, bf16>"}[args.precision]
    kdesc = {"gmres_A": "k_gmres_a" + tname + " (persistent A-solve, one cooperative launch per intermediate "
                        "A-solve: SELL-32 SpMV of A M^-1, Gram-Schmidt, Givens, solution update)",
             "gmres_S": "k_gmres_s" + tname + " (persistent S-solve, one cooperative launch per S-solve: "
                        "Schur products with their inner A-solves, Gram-Schmidt, Givens" +
                        (", Chebyshev polynomial in S^" if args.s_precond == "cheb" else "") + ")"}
    prof_name = "gmres_" + dom[-1].lower() + ("_cheb" if dom == "gmres_S" and args.s_precond == "cheb" else "")
    traffic_ratio = profile_traffic(prof_name + "_cube48", "solver.cu", "dram_over_algorithmic")
    roof = {"kernel": kdesc[dom],
            "bound": "hbm", "achieved": gbs_live, "peak": peak, "unit": "GB/s",
            "frac": gbs_live / peak if gbs_live else None,
            "traffic": (traffic_ratio * by_live if traffic_ratio is not None and args.precision == "fp64"
                        else None),
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy burst)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "bytes_per_launch": by_live, "avg_launch_us": us_live, "launches": pl["launches"],
            "algorithmic_bytes": ("per A-iteration j: A M^-1 values + indices + 4(N+1), and 2(j+1)+6 passes "
                                  "over 3N-vectors (4(j+1)+10 with a second Gram-Schmidt pass); per S-iteration: "
                                  "B, C, D values + indices twice, the Chebyshev S^ products (FP32 values + "
                                  "indices) and vector passes, and its inner A-solve's bytes (counted on the "
                                  "device, summed over the launch's iterations)"),
            "measured": "CUDA events around every launch on the library stream, in a host-driven replay of the "
                        "timed K steps (the graph-mode run has no per-kernel events)",
            "fp64_pipe_note": "9 DFMA per 76-byte block: GB300's 1.2 TFLOP/s FP64 pipe caps the SpMV phase near "
                              "5.1 TB/s",
            "alone_l2_flushed": {
                "note": "one launch between two events after an L2 flush (256 MB written, then 256 MB of another buffer read, so that no dirty line of the flush is written back during the launch)",
                "same_size_read": "read_gbs: hyel_stream_read_probe reading the same byte count after the same "
                                  "flush; frac_of_same_size_read = achieved / read_gbs",
                "spmv_A64": {"achieved": gbs64, "frac": gbs64 / peak, "bytes_per_launch": by64, "avg_launch_us": us64,
                             "read_gbs": rd64, "frac_of_same_size_read": gbs64 / rd64},
                "spmv_A32": {"achieved": gbs32, "frac": gbs32 / peak, "bytes_per_launch": by32, "avg_launch_us": us32,
                             "read_gbs": rd32, "frac_of_same_size_read": gbs32 / rd32},
                "spmv_A16": {"achieved": gbs16, "frac": gbs16 / peak, "bytes_per_launch": by16,
                             "avg_launch_us": us16, "read_gbs": rd16, "frac_of_same_size_read": gbs16 / rd16}}}
    # the element pass: FP64-arithmetic bound (its FP64 instructions per tet
    # come from the committed ncu counters of the same source)
    E = int(mesh["tets"].shape[0])

    def elem_entry(parts, desc):
        """parts: (kernel class, profile field of its FP64 flops per tet)."""
        ms = sum(prof_host[c]["ms"] for c, _ in parts)
        n = sum(prof_host[c]["launches"] for c, _ in parts)
        fl, dram, ok = 0.0, 0.0, True
        for c, field in parts:
            fpt = profile_traffic("element_cube48", "assemble.cu", field)
            dpt = profile_traffic("element_cube48", "assemble.cu", field.replace("fp64_flops", "dram_bytes"))
            if fpt is None or dpt is None:
                ok = False
                break
            fl += fpt * E * prof_host[c]["launches"]
            dram += dpt * E * prof_host[c]["launches"]
        us = 1e3 * ms / max(1, n)
        ach = fl / (ms * 1e-3) / 1e12 if (ok and ms > 0) else None
        return {"kernel": desc, "bound": "alu", "achieved": ach, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": ach / fp64_tflops if ach else None,
                "traffic": dram / n if (ok and n) else None,
                "peak_source": "measured in this run: FP64 FMA-chain probe kernel (hyel_fp64_fma_probe), best of 5; "
                               "nominal GB300 FP64 1.25 TFLOP/s",
                "flops_per_launch": fl / n if (ok and n) else None, "tets": E, "avg_launch_us": us, "launches": n,
                "algorithmic_flops": "FP64 flops per tet (2 per DFMA, 1 per DADD or DMUL) counted by ncu on the "
                                     "same kernel source (profiles/element_cube48.md), x tets, per launch",
                "measured": "CUDA events around every launch on the library stream (host-driven replay)"}

    roof_k = {
        dom: roof,
        "assemble_elem": elem_entry((("assemble_elem", "fp64_flops_per_tet_tangent"),
                                     ("assemble_corr", "fp64_flops_per_tet_tangent_corr")),
                                    "k_element<true, *> (element residual and tangent blocks, one thread per tet; "
                                    "<true, true> also forms the K_{.,udot} R_k terms)"),
        "assemble_res": elem_entry((("assemble_res", "fp64_flops_per_tet_residual"),),
                                   "k_element<false, false> (residual-only element pass)")}
    other = "gmres_A" if dom == "gmres_S" else "gmres_S"
    po = prof_host[other]
    if po["launches"]:
        us_o = 1e3 * po["ms"] / po["launches"]
        by_o = po["bytes"] / po["launches"]
        pn_o = "gmres_" + other[-1].lower() + ("_cheb" if other == "gmres_S" and args.s_precond == "cheb" else "")
        ratio_o = profile_traffic(pn_o + "_cube48", "solver.cu", "dram_over_algorithmic")
        roof_k[other] = {"kernel": kdesc[other], "bound": "hbm", "achieved": by_o / (us_o * 1e-6) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": by_o / (us_o * 1e-6) / 1e9 / peak,
                         "traffic": (ratio_o * by_o if ratio_o is not None and args.precision == "fp64" else None),
                         "bytes_per_launch": by_o, "avg_launch_us": us_o, "launches": po["launches"]}
    for k in ("gmres_A", "gmres_S"):
        if k in roof_k and roof_k[k].get("achieved"):
            pn = "gmres_" + k[-1].lower() + ("_cheb" if k == "gmres_S" and args.s_precond == "cheb" else "")
            ratio = profile_traffic(pn + "_cube48", "solver.cu", "dram_over_algorithmic")
            roof_k[k]["dram_frac"] = (ratio * roof_k[k]["achieved"] / peak) if (ratio and args.precision == "fp64") \
                else None
            roof_k[k]["dram_note"] = ("DRAM bytes = the committed ncu capture's DRAM / algorithmic ratio x the "
                                      "algorithmic bytes; where it is below 1 the rest is served from L2")
    # the dominant kernel by replay time takes the top-level roofline
    tms = {"gmres_S": prof_host["gmres_S"]["ms"], "gmres_A": prof_host["gmres_A"]["ms"],
           "assemble_elem": prof_host["assemble_elem"]["ms"] + prof_host["assemble_corr"]["ms"]}
    top = max((k for k in tms if k in roof_k), key=lambda k: tms[k])
    roof = dict(roof_k[top])
    roof["dominant_by_replay_ms"] = {k: prof_host[k]["ms"] for k in ("gmres_S", "gmres_A", "assemble_elem",
                                                                     "assemble_corr", "assemble_res", "gather",
                                                                     "schur_hat")}

    kclass = {k: {"ms": v["ms"], "launches": v["launches"],
                  "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else None)}
              for k, v in prof_host.items()}
    sweep = None if args.no_sweep else nu_sweep(ctx, H, torch, stream, args, names, sizes, dev, state, sprec_kw,
                                                graph)
    tube = None if args.no_tube else tube_step(ctx, H, torch, stream, graph, sprec_kw, dt=args.tube_dt)
    H.hyel_destroy(ctx)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_sample(args=args)
        cpu.update(cpu_plan(args))
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f64 outer / f32 levels",
                                             "bf16s": "f64 outer / f32 levels, bf16 A"}[args.precision], "data": "synthetic (seeded jittered cube, no dataset)",
            "config": config_dict(args, mesh), "clocks": ck, "e2e": e2e, "gpu_launches": launches,
            "roofline": roof, "roofline_kernels": roof_k, "cpu_baseline": cpu, "nu_sweep": sweep,
            "config3_tube": tube,
            "newton_solves": its, "solve_ms_per_newton_it": solve_ms, "assembly_ms_per_step": asm_ms,
            "mixed_fp32_preconditioner": mixed, "mixed_bf16s_preconditioner": mixed16,
            "kernel_classes_host_replay": kclass}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.compare_a_precond:
            if rank == 0:
                compare_a_precond(args)
        elif args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_hyel(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
