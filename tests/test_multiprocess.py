"""The N > 1 path of bench.py on the CPU, with two gloo ranks on 127.0.0.1: the rendezvous
and the max-over-ranks timing reduction that the GPU arm uses, and the reference arm
under torch.distributed.run (rank 0 alone runs the oracle and prints the one JSON line,
the other rank exits 0 without work). The library's own runs are replicas with no
data-path collective, so this host logic is the whole multi-process path."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    a = argparse.Namespace(gpus=world)
    r, w, dist = bench.dist_setup(a)
    got = bench.max_over_ranks(1.5 + r, dist)  # per-rank elapsed times; the line takes the max
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump({"rank": r, "world": w, "max": got}, f)
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert sorted(x["rank"] for x in res) == [0, 1]
    assert all(x["world"] == 2 and x["max"] == 2.5 for x in res)


def test_reference_arm_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--L", "4", "--N", "64", "--n-mcmc", "2",
           "--cpu-sample", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_hmc_workload():
    # the HMC workload's reference arm: the oracle's HMC transitions on a bounded sample
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--sampler", "hmc", "--precision", "fp32", "--steps",
           "1", "--warmup", "0", "--L", "4", "--N", "64", "--n-mcmc", "2", "--cpu-sample", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["config"]["sampler"] == "hmc" and line["value"] > 0
    assert "HMC transitions" in line["cpu_baseline"]["sample"]
