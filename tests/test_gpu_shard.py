"""Row-sharded step (nb_set_shard) on one GPU.

A sharded run joins the ranks' row blocks with two all-gathers per step. On
one GPU the ranks are emulated by host threads, each with its own system on
its own stream; the all-gather waits for the calling rank's stream, copies
its block to the host, meets the other ranks at a host barrier and copies the
gathered blocks back. No kernel ever waits on another rank's kernel: the only
synchronisation is between host threads, after each rank's own stream has
drained. Every rank must end bit-identical to the unsharded nb_step (the kick
rows of a block are bit-identical to the whole kick's), for uneven blocks,
encounter groups and mergers.
"""
import ctypes as C
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import nbref  # noqa: E402
from paper_2604_09184_b300 import build, ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2604_09184_b300 import nb
    nb.lib()


def mods():
    from paper_2604_09184_b300 import nb, shard
    return nb, shard


class HostExchange:
    """All-gather between host threads standing in for ranks."""

    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.blocks = [None] * world
        self.calls = [0] * world

    def fn_for(self, rank):
        nb, shard = mods()

        def fn(user, send, recv, nbytes, stream):
            try:
                st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                st.synchronize()  # the packing kernel of this rank is done
                with torch.cuda.stream(st):
                    self.blocks[rank] = shard.device_bytes(send, nbytes).cpu()
                self.barrier.wait(timeout=120)
                gathered = torch.cat(self.blocks)  # rank order
                with torch.cuda.stream(st):
                    shard.device_bytes(recv, nbytes * self.world).copy_(gathered)
                st.synchronize()
                self.barrier.wait(timeout=120)  # all read before the next exchange
                self.calls[rank] += 1
                return 0
            except Exception:  # noqa: BLE001
                self.barrier.abort()
                return -1

        return shard.ALLGATHER_FN(fn)


def run_sharded(d, rc, world, steps, **kw):
    """Each rank in its own thread and stream: returns per-rank (state,
    encounter list, stats, status) after `steps` steps."""
    nb, shard = mods()
    ex = HostExchange(world)
    out = [None] * world

    def rank_main(r):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = nb.NBodySystem(nb.params(dt_rcrit=d.dt, **kw), d.x, d.v, d.m, d.R, rc=rc)
            keep = shard.Shard(s, r, world, fn=ex.fn_for(r))
            code = s.step_status(steps, d.dt)
            out[r] = (s.state(), s.encounter_list(), s.stats(), code, keep.row0, keep.row1)
            del keep, s

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    return out, ex


def reference(d, rc, steps, **kw):
    nb, _ = mods()
    s = nb.NBodySystem(nb.params(dt_rcrit=d.dt, **kw), d.x, d.v, d.m, d.R, rc=rc)
    s.step(steps, d.dt)
    return s.state(), s.encounter_list(), s.stats()


def oracle_rc(d):
    p = nbref.params(dt_rcrit=d.dt)
    return np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(d.n)])


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_step_equals_nb_step_bit_for_bit(world):
    """The 2049-body adjoint workload (a close-encounter group nearly every
    step), 20 steps, 1-3 emulated ranks with uneven row blocks."""
    d = ics.workload("adjoint_2k_j")
    rc = oracle_rc(d)
    sr, er, str_ = reference(d, rc, 20)
    assert str_["groups"] > 0
    out, ex = run_sharded(d, rc, world, 20)
    blocks = []
    for r, (sg, eg, stg, code, r0, r1) in enumerate(out):
        assert code == 0, (r, code)
        for k in ("ids", "x", "v", "m", "R", "rc"):
            assert np.array_equal(sg[k], sr[k]), (world, r, k)
        assert np.array_equal(eg, er), (world, r)
        for k in ("groups", "bs_substeps", "bs_halvings", "merges", "encounter_pairs"):
            assert stg[k] == str_[k], (world, r, k)
        blocks.append((r0, r1))
    # the blocks partition the rows in rank order
    assert blocks[0][0] == 0 and blocks[-1][1] == d.n
    assert all(blocks[k][1] == blocks[k + 1][0] for k in range(world - 1))
    if world > 1:
        assert ex.calls == [2 * 20] * world  # two exchanges per step


def test_sharded_double_single_step_equals_nb_step_bit_for_bit():
    """The double-single kick sets its coordinate grid from all positions, so
    a rank's block of rows is bit-identical to those rows of the whole kick:
    the sharded double-single step equals the unsharded one bit for bit
    (2049 bodies with Jupiter, 3 ranks, 10 steps with encounter groups)."""
    nb, _ = mods()
    d = ics.workload("adjoint_2k_j")
    rc = oracle_rc(d)
    kw = dict(precision=nb.NB_PREC_DS)
    sr, er, str_ = reference(d, rc, 10, **kw)
    assert str_["groups"] > 0
    out, _ = run_sharded(d, rc, 3, 10, **kw)
    for sg, eg, stg, code, r0, r1 in out:
        assert code == 0
        for k in ("ids", "x", "v", "m"):
            assert np.array_equal(sg[k], sr[k]), k
        assert np.array_equal(eg, er)


def test_sharded_step_with_mergers_and_uneven_blocks():
    """A merging disk (radii inflated 400x) on 3 ranks over 60 steps: mergers
    change masses and positions inside the direct solver, identically on
    every rank."""
    d = ics.workload("toy_disk_256", f_radius=400.0)
    rc = oracle_rc(d)
    sr, er, str_ = reference(d, rc, 60)
    assert str_["merges"] > 0
    out, _ = run_sharded(d, rc, 3, 60)
    for r, (sg, eg, stg, code, r0, r1) in enumerate(out):
        assert code == 0
        for k in ("ids", "x", "v", "m"):
            assert np.array_equal(sg[k], sr[k]), (r, k)
        assert np.array_equal(eg, er)
        assert stg["merges"] == str_["merges"]


def test_sharded_step_full_size_two_ranks():
    """The 64k disk with Jupiter and Saturn on 2 emulated ranks, 2 steps."""
    d = ics.workload("mmsn_64k_js")
    rc = oracle_rc(d)
    sr, er, _ = reference(d, rc, 2, kick_symmetric=-1)  # ranks run the row kick
    out, _ = run_sharded(d, rc, 2, 2, kick_symmetric=-1)
    for sg, eg, stg, code, r0, r1 in out:
        assert code == 0
        assert np.array_equal(sg["x"], sr["x"]) and np.array_equal(sg["v"], sr["v"])
        assert np.array_equal(eg, er)


def test_shard_rejects_unsharded_options_and_a_failed_exchange_rolls_back():
    """rcrit_refresh (and gas, ejection) are not sharded: NB_E_INVALID. An
    exchange that fails fails the step on that rank and restores its state."""
    nb, shard = mods()
    d = ics.workload("toy_disk_256", n=64)
    s = nb.NBodySystem(nb.params(dt_rcrit=d.dt, rcrit_refresh=1), d.x, d.v, d.m, d.R)
    with pytest.raises(nb.NbError):
        shard.Shard(s, 0, 2, fn=shard.ALLGATHER_FN(lambda *a: 0))
    s2 = nb.NBodySystem(nb.params(dt_rcrit=d.dt), d.x, d.v, d.m, d.R)
    x0 = s2.state()["x"]
    keep = shard.Shard(s2, 0, 2, fn=shard.ALLGATHER_FN(lambda *a: 1))  # always fails
    code = s2.step_status(3, d.dt)
    assert code == nb.NB_E_CUDA
    assert np.array_equal(s2.state()["x"], x0)
    keep.release()
    s2.step(1, d.dt)  # unsharded again
