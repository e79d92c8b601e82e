"""Multi-rank host logic on the CPU: world_size 2 over gloo.

* The row-sharded step (nb_set_shard): the library's partition of target
  rows (nb_shard_rows, a host function), the exchange the binding hands to
  torch.distributed (rank-ordered blocks), and the block layout the library's
  pack/unpack kernels use (a 4-int header, count, status, unclipped count, 0,
  then the pairs, padded to the pair capacity; the force rows as three blocks
  of ceil(n / world) doubles). The oracle's forces_targets stands in for each
  rank's kick; the joined force and flag set must equal the oracle's whole
  kick bit for bit.
* bench.py's timing under torchrun: the max over ranks of the timed region
  and the whole-job rate, and the reference arm (rank 0 alone prints).
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    m = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.job_rate(1e9, 10, m)
    out.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 150.0  # the slowest rank's time on every rank
        assert rate == pytest.approx(1e9 * 10 / 0.150)  # one job, the slowest rank's time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(30500 + os.getpid() % 1000),
           "bench.py", "--impl", "reference", "--gpus", "2", "--workload", "toy_disk_256",
           "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


# ------------------------------------------------------------------ row sharding
def _shard_worker(rank, world, port, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import nbref
    from paper_2604_09184_b300 import ics, shard
    d = ics.make_disk(301, 2.0, 0.98, 1.02, 0.02, 0.01, 6.0, seed=77, f_radius=1.0)
    p = nbref.params(dt_rcrit=d.dt)
    rc = 8.0 * np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(d.n)])
    r0, r1 = shard.rows(d.n, rank, world)
    # this rank's kick rows (the oracle stands in for the library's kick)
    a_rows, pairs = nbref.forces_targets(d.x, d.m, rc, np.arange(r0, r1, dtype=np.int32))
    # the library's kick emits a pair (i < j) from its lower row only
    pairs = pairs[(pairs[:, 0] >= r0) & (pairs[:, 0] < r1)]
    cap = 4096
    # exchange 1: [count, status, unclipped count, 0] + cap pairs
    blk = np.zeros(4 + 2 * cap, dtype=np.int32)
    blk[0], blk[1], blk[2] = len(pairs), 0, len(pairs)
    blk[4:4 + 2 * len(pairs)] = np.asarray(pairs, dtype=np.int32).reshape(-1)
    send = torch.from_numpy(blk.view(np.uint8).copy())
    recv = torch.empty(world * send.numel(), dtype=torch.uint8)
    shard.allgather_into(recv, send)
    got = recv.numpy().view(np.int32).reshape(world, 4 + 2 * cap)
    all_pairs = np.concatenate([got[q, 4:4 + 2 * got[q, 0]].reshape(-1, 2) for q in range(world)])
    # exchange 2: three blocks of `chunk` doubles, zero beyond the last row
    chunk = -(-d.n // world)
    ablk = np.zeros((3, chunk))
    ablk[:, :r1 - r0] = a_rows.T
    send = torch.from_numpy(ablk.reshape(-1).view(np.uint8).copy())
    recv = torch.empty(world * send.numel(), dtype=torch.uint8)
    shard.allgather_into(recv, send)
    g = recv.numpy().view(np.float64).reshape(world, 3, chunk)
    a = np.concatenate([g[q, :, :min(chunk, d.n - q * chunk)].T for q in range(world)])
    a_full, p_full = nbref.forces(d.x, d.m, rc)
    out.put((rank, (r0, r1), bool(np.array_equal(a, a_full)),
             sorted(map(tuple, all_pairs.tolist())) == sorted(map(tuple, p_full.tolist())),
             len(p_full)))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_kick_joins_to_the_whole_kick_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0a, r1a), (r0b, r1b) = res[0][1], res[1][1]
    assert (r0a, r1a, r0b, r1b) == (0, 151, 151, 301)
    for rank, _, same_a, same_pairs, npairs in res:
        assert same_a and same_pairs and npairs > 0, rank


def test_shard_partition_covers_every_row():
    from paper_2604_09184_b300 import shard
    for n in (1, 2, 7, 256, 65538):
        for world in (1, 2, 3, 8):
            b = [shard.rows(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
            assert all(r1 - r0 <= -(-n // world) for r0, r1 in b)


def test_state_error_splits_encounter_and_quiet_bodies():
    """The accuracy report's error of a state against the oracle's: common ids
    only, and with the oracle's encounter log the bodies that entered an
    encounter apart from the quiet rest (the 1e-12 bar applies to those)."""
    import numpy as np
    import bench
    b = {"ids": np.array([0, 1, 2, 3, 4]), "x": np.ones((5, 3))}
    a = {"ids": np.array([0, 1, 2, 4]), "x": np.ones((4, 3))}  # body 3 absorbed on one side
    a["x"][2] *= 1 + 1e-10   # id 2: an encounter body
    a["x"][3] *= 1 + 5e-13   # id 4: quiet
    log = np.array([[0, 2, 3], [7, 1, 2]], np.int32)  # (step, id_i, id_j)
    e = bench._state_err(a, b, log)
    assert e["bodies"] == 4 and not e["ids_identical"]
    assert e["bodies_above_1e-12"] == 1 and e["encounter_bodies"] == 2
    assert e["encounter_bodies_above_1e-12"] == 1
    assert abs(e["max"] - 1e-10) < 1e-16 and 4e-13 < e["quiet_max"] < 6e-13
    q = bench._state_err(a, b, np.zeros((0, 3), np.int32))
    assert q["encounter_bodies"] == 0 and q["quiet_max"] == q["max"]
    assert "quiet_max" not in bench._state_err(a, b)
