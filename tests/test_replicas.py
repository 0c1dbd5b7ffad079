"""The multi-GPU mode is replicas only (each rank solves its own copy of the
workload). Its host-side logic runs here on world_size-2 gloo process groups:
the job time is the slowest rank's, the work is summed, one rank is the
identity, and the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1809_06350_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier()
        ms, work = replicas.reduce_timing(10.0 + 5.0 * rank, 3 + rank, device="cpu")
        out[rank] = (ms, work)
    finally:
        dist.destroy_process_group()


def test_reduce_timing_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == (15.0, 7) and res[1] == (15.0, 7)


def test_reduce_timing_single_process_is_identity():
    sys.path.insert(0, ROOT)
    from paper_1809_06350_gb300 import replicas
    assert replicas.reduce_timing(12.5, 4) == (12.5, 4)


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    """bench.py --impl reference under a 2-rank gloo launch: one JSON line
    (rank 0), every rank exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
