"""bench.py's command line on the host: --help works, and the solver options
(Poisson ratio, time step, S- and A-preconditioners, block preconditioner,
inner solver) reach the reported config. Runs the reference arm (the oracle on
the host cores), so no GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def test_help():
    r = subprocess.run([sys.executable, BENCH, "--help"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    for opt in ("--s-precond", "--cheb-degree", "--a-precond", "--block", "--inner", "--dt", "--nu", "--no-sweep",
                "--no-tube", "--no-mixed", "--no-e2e", "--no-cpu", "--tube-only", "--tube-dt", "--stiff-only",
                "--compare-a-precond", "--host-loops"):
        assert opt in r.stdout, opt


def test_options_reach_the_config(tmp_path):
    cmd = [sys.executable, BENCH, "--impl", "reference", "--steps", "1", "--warmup", "0", "--nu", "0.45",
           "--dt", "0.002", "--s-precond", "jacobi", "--block", "simple", "--inner", "cg", "--a-precond", "cheb"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    c = d["config"]
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert "nu=0.45" in c["workload"] and c["dt"] == 0.002
    assert c["s_precond"] == "diag(S^)" and c["block_precond"] == "SIMPLE"
    assert c["inner_solver"].startswith("CG") and c["a_precond"] == "cheb"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # the reference arm names the sample it actually times
    assert "sample" in c["workload"] and "10^3" in c["workload"]
