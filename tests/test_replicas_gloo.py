"""The bench's multi-rank path on CPU (world size 2, gloo): process-group
setup from the torchrun environment, the barrier, and the max-over-ranks
timing reduction; and the reference arm printing from rank 0 only."""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_setup(None)
    bench.barrier(ws)
    m = bench.max_over_ranks(ws, 10.0 * (r + 1))
    with open(os.path.join(out, f"rank{r}.txt"), "w") as f:
        f.write(f"{ws} {r} {local} {m}")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_barrier(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ws, rank, local, m = open(tmp_path / f"rank{r}.txt").read().split()
        assert (int(ws), int(rank), int(local)) == (2, r, r)
        assert float(m) == 20.0          # every rank reports the slowest rank's time


def test_reference_arm_prints_from_rank_zero_only():
    """Under torchrun with two ranks the reference arm prints one JSON line
    (rank 0) and the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and '"impl": "reference"' in lines[0]
