"""The multi-process path of bench.py on the CPU (gloo, two ranks): one
replica per rank, no data-path collective, the job time is the maximum over
ranks, and only rank 0 prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out[rank] = bench.max_over_ranks(float(rank + 1) * 0.5, world, "cpu")
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_max_worker, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 1.0, 1: 1.0}


def test_reference_arm_two_ranks():
    """bench.py --impl reference under torchrun with two gloo ranks: exit 0,
    exactly one JSON line (rank 0), n_gpus = 2."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def _oracle_columns(w):
    """Columns j0..j1-1 of C by the dense oracle, each conductor solved on
    its own (so a column is the same computation whoever asks for it)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle as O
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    A = O.dense_matrix(ps, rtol=1e-10)
    B = O.rhs_unit_potentials(ps)
    Wt = O.charge_weights(ps).T

    def solve(j0, j1):
        cols = [O.EPS0 * w.voxel_size * (Wt @ np.linalg.solve(A, B[:, j])) for j in range(j0, j1)]
        return np.stack(cols, 1) if cols else np.zeros((Wt.shape[0], 0))
    return solve, ps.n_conductors


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2004_02609_gb300 import shard
    from paper_2004_02609_gb300 import workloads as W
    w = W.random_structure((5, 4, 4), 6, n_cond=3, n_diel=1)
    solve, m = _oracle_columns(w)
    out[rank] = shard.capacitance_sharded(solve, m).tolist()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_capacitance_equals_single_rank(world):
    """The conductors' solves split over gloo ranks (3 conductors over 2 or
    3 ranks), the column blocks all-gathered: every rank holds the matrix a
    single process computes, bit for bit."""
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2004_02609_gb300 import shard
    from paper_2004_02609_gb300 import workloads as W
    w = W.random_structure((5, 4, 4), 6, n_cond=3, n_diel=1)
    solve, m = _oracle_columns(w)
    full = solve(0, m)
    assert [shard.column_range(m, r, world) for r in range(world)][-1][1] == m
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        for r in range(world):
            assert np.array_equal(np.asarray(out[r]), full)
