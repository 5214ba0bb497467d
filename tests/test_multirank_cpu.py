"""The multi-GPU path of bench.py on CPU: world_size 2 with gloo.  Every rank
serves its own regions (weak scaling, no collective on the data path); the
ranks meet only in the barrier and the max-over-ranks of the timed interval.
The reference arm launched the same way prints its line from rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(10.0 * (rank + 1), world)
        origins = [bench.query_origin(rank, i) for i in range(8)]
        q.put((rank, m, origins))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(m == 20.0 for _, m, _ in res)
    # 4096^2 regions of every (rank, step) are pairwise disjoint, with room
    # for the decode halo and the 20-step cone
    boxes = [(x, y) for _, _, o in res for (x, y) in o]
    span = 4096 + 2 * (128 + 20 * 64 + 64)
    for i in range(len(boxes)):
        for j in range(i + 1, len(boxes)):
            (x1, y1), (x2, y2) = boxes[i], boxes[j]
            assert abs(x1 - x2) >= span or abs(y1 - y2) >= span


def test_reference_arm_under_torchrun_prints_once():
    # launched as the multi-GPU run is (torchrun, two ranks, gloo here): rank
    # 0 alone times the oracle and prints the line, the other rank exits 0
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
