"""Batched ensembles on the GPU against the CPU oracle, system by system.

Each system of a batch is integrated by the oracle on its own; the batched
kernel must give the same states (relative position error <= 1e-12 after the
run, or the conditioning bound of the parity suite), the same survivors and
masses, and per-system energy consistent with the oracle's.
"""
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


def nbm():
    from paper_2604_09184_b300 import nb
    return nb


def oracle_run(d, steps, dt, **kw):
    p = nbref.params(dt_rcrit=dt, **kw)
    rc = np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(d.n)])
    s = nbref.RefSystem(p, d.x, d.v, d.m, d.R, rc=rc)
    assert s.step(steps, dt) == 0
    return s, rc


def batch_of(disks, dt, rcs=None, **kw):
    nb = nbm()
    rc = None if rcs is None else np.concatenate(rcs)
    return nb.NBodyBatch(nb.params(dt_rcrit=dt, **kw), disks, rc=rc)


@pytest.mark.parametrize("sym", [0, -1])
def test_batch_matches_oracle_per_system(sym):
    """The unordered-pair kick (32-body block pairs, default) and the row kick
    (kick_symmetric = -1), each system against its own oracle run."""
    disks = ics.ensemble(n_systems=24, seed=ics.SEED_BASE + 33)
    dt, steps = 3.0, 40
    refs, rcs = [], []
    for d in disks:
        s, rc = oracle_run(d, steps, dt)
        refs.append(s)
        rcs.append(rc)
    b = batch_of(disks, dt, rcs, kick_symmetric=sym)
    b.step(steps, dt)
    st = b.state()
    for k, (d, ref) in enumerate(zip(disks, refs)):
        sg, sr = b.system_state(k, st), ref.state()
        assert np.array_equal(sg["ids"], sr["ids"])
        assert np.array_equal(b.encounter_list(k), ref.encounter_list()), k
        rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
        assert rel.max() <= 1e-12, (k, d.n, rel.max())
        assert np.allclose(sg["m"], sr["m"], rtol=1e-15, atol=0)


@pytest.mark.parametrize("sym", [0, -1])
def test_batch_with_encounters_and_mergers(sym):
    disks = [ics.make_disk(n, 2.0, 0.7, 1.3, 0.01, 0.005, 6.0, seed=900 + n, f_radius=400.0)
             for n in (64, 128, 200)]
    dt, steps = 6.0, 60
    refs, rcs = [], []
    for d in disks:
        s, rc = oracle_run(d, steps, dt)
        refs.append(s)
        rcs.append(rc)
    assert sum(r.stats()["merges"] for r in refs) > 0
    b = batch_of(disks, dt, rcs, kick_symmetric=sym)
    b.step(steps, dt)
    st = b.state()
    assert b.stats()["merges"] == sum(r.stats()["merges"] for r in refs)
    assert b.stats()["groups"] == sum(r.stats()["groups"] for r in refs)
    E, El = b.energy()
    for k, ref in enumerate(refs):
        sg, sr = b.system_state(k, st), ref.state()
        assert np.array_equal(sg["ids"], sr["ids"])
        assert np.array_equal(b.encounter_list(k), ref.encounter_list()), k
        rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
        assert rel.max() <= 1e-11, (k, rel.max())
        em = ref.energy_momentum()
        assert abs(E[k] - em["E"]) <= 1e-12 * abs(em["E"])
        assert abs(El[k] - em["E_lost"]) <= 1e-9 * abs(em["E_lost"]) + 1e-24


def test_batch_force_update_after_encounters_both_branches():
    """After the direct solver the batch updates the force from the trial one
    (the members' new minus trial terms) unless the group members are more
    than a third of the system, where it evaluates the force in full. Five-body
    systems whose one encounter ends in a merger take the full branch; a
    12-body system with three merging pairs and a 64-body one take the
    incremental branch. All against the oracle over 40 steps."""
    w = 0.05
    disks = [ics.make_disk(5, 2.0, 1.0 - w / 2, 1.0 + w / 2, 0.02, 0.01, 6.0, seed=3000 + k,
                           f_radius=300.0) for k in (0, 9, 19, 28)]
    disks.append(ics.make_disk(12, 2.0, 1.0 - w / 2, 1.0 + w / 2, 0.02, 0.01, 6.0, seed=3103,
                               f_radius=300.0))
    disks.append(ics.make_disk(64, 2.0, 0.7, 1.3, 0.01, 0.005, 6.0, seed=964, f_radius=400.0))
    dt, steps = 6.0, 40
    refs, rcs = [], []
    for d in disks:
        s, rc = oracle_run(d, steps, dt)
        refs.append(s)
        rcs.append(rc)
    for r in refs[:5]:
        assert r.stats()["groups"] >= 1 and r.stats()["merges"] >= 1
    b = batch_of(disks, dt, rcs)
    b.step(steps, dt)
    st = b.state()
    assert b.stats()["merges"] == sum(r.stats()["merges"] for r in refs)
    assert b.stats()["groups"] == sum(r.stats()["groups"] for r in refs)
    for k, ref in enumerate(refs):
        sg, sr = b.system_state(k, st), ref.state()
        assert np.array_equal(sg["ids"], sr["ids"])
        assert np.array_equal(b.encounter_list(k), ref.encounter_list()), k
        rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
        assert rel.max() <= 1e-11, (k, rel.max())
        relv = np.linalg.norm(sg["v"] - sr["v"], axis=1) / np.linalg.norm(sr["v"], axis=1)
        assert relv.max() <= 1e-11, (k, relv.max())


def test_batch_chunking_and_autotune_are_transparent():
    """Graph replay of chunks, a direct remainder launch and one-step calls give
    the same bits; autotuning leaves the state unchanged."""
    disks = ics.ensemble(n_systems=40, seed=ics.SEED_BASE + 34)
    dt = 3.0
    a = batch_of(disks, dt)
    b = batch_of(disks, dt)
    a.set_shape(128, 7)
    a.step(23, dt)  # 3 graph replays + remainder of 2
    b.set_shape(128, 1)
    for _ in range(23):
        b.step(1, dt)
    sa, sb = a.state(), b.state()
    assert np.array_equal(sa["x"], sb["x"]) and np.array_equal(sa["v"], sb["v"])
    before = a.state()
    threads, ms = a.autotune(dt)
    assert threads in (64, 128, 256) and ms > 0
    after = a.state()
    assert np.array_equal(before["x"], after["x"]) and np.array_equal(before["v"], after["v"])


@pytest.mark.parametrize("threads", [64, 256])
def test_batch_thread_shapes_agree(threads):
    disks = ics.ensemble(n_systems=12, seed=ics.SEED_BASE + 35)
    dt = 3.0
    a = batch_of(disks, dt)
    b = batch_of(disks, dt)
    a.set_shape(threads, 10)
    b.set_shape(128, 10)
    a.step(10, dt)
    b.step(10, dt)
    # the per-system momentum sum is a block reduction whose order follows the
    # thread count; everything else is identical
    xa, xb = a.state()["x"], b.state()["x"]
    assert np.max(np.linalg.norm(xa - xb, axis=1) / np.linalg.norm(xb, axis=1)) <= 1e-13


def test_batch_energy_tracks_oracle():
    """Energy after 200 steps (mergers off): the batched systems carry the same
    energy error as the oracle's runs of the same systems (the error itself is
    the method's, ~1e-10 to ~1e-7 with close encounters)."""
    disks = ics.ensemble(n_systems=8, seed=ics.SEED_BASE + 36)
    dt, steps = 3.0, 200
    rcs, refs = [], []
    for d in disks:
        s, rc = oracle_run(d, steps, dt, merge=0)
        refs.append(s)
        rcs.append(rc)
    b = batch_of(disks, dt, rcs, merge=0)
    E0, _ = b.energy()
    b.step(steps, dt)
    E1, _ = b.energy()
    for k, ref in enumerate(refs):
        er = ref.energy_momentum()["E"]
        assert abs(E1[k] - er) <= 1e-12 * abs(er), (k, E1[k], er)
    assert np.max(np.abs(E1 / E0 - 1)) < 1e-6


def test_batch_rejects_oversize_system():
    nb = nbm()
    big = ics.make_disk(nb.NB_BATCH_MAX_N + 1, 1.0, 0.5, 2.0, 0.02, 0.01, 3.0, seed=1)
    with pytest.raises(nb.NbError):
        nb.NBodyBatch(nb.params(dt_rcrit=3.0), [big])


def test_batch_time_budget_rolls_back():
    """A per-launch time budget far below one system's step: the call fails
    with NB_E_TIMEOUT and leaves the state as it was; without the budget the
    same call succeeds."""
    nb = nbm()
    disks = ics.ensemble(n_systems=64, seed=ics.SEED_BASE + 37)
    dt = 3.0
    b = batch_of(disks, dt)
    b.step(2, dt)
    before = b.state()
    b.set_budget(1e-6)
    with pytest.raises(nb.NbError) as e:
        b.step(5, dt)
    assert e.value.code == nb.NB_E_TIMEOUT
    after = b.state()
    assert np.array_equal(before["x"], after["x"]) and np.array_equal(before["v"], after["v"])
    b.set_budget(0.0)
    b.step(5, dt)
    ref = batch_of(disks, dt)
    ref.step(7, dt)
    assert np.array_equal(b.state()["x"], ref.state()["x"])


def test_batch_load_balance_report():
    disks = ics.ensemble(n_systems=256, seed=ics.SEED_BASE + 38)
    b = batch_of(disks, 3.0)
    b.step(3, 3.0)
    bal = b.balance()
    assert bal["ctas"] >= 1 and bal["max_cta_ms"] > 0
    assert 0.0 < bal["efficiency"] <= 1.0


def test_batch_speculative_half_steps_are_bit_identical():
    """bs_speculate on (default) and off: identical states and direct-solver
    counters on systems with encounters, halvings and mergers."""
    disks = [ics.make_disk(n, 2.0, 0.7, 1.3, 0.01, 0.005, 6.0, seed=900 + n, f_radius=400.0)
             for n in (64, 128, 200)] + ics.ensemble(n_systems=16, seed=ics.SEED_BASE + 35)
    dt, steps = 6.0, 40
    out = []
    for sp in (0, 1):
        b = batch_of(disks, dt, bs_speculate=sp)
        b.step(steps, dt)
        out.append((b.state(), b.stats()))
    (s0, t0), (s1, t1) = out
    for k in s0:
        assert np.array_equal(np.asarray(s0[k]), np.asarray(s1[k])), k
    for k in ("groups", "bs_derivs", "bs_substeps", "bs_halvings", "merges"):
        assert t0[k] == t1[k], (k, t0[k], t1[k])
    assert t0["bs_halvings"] > 0 and t0["merges"] > 0


def test_batch_kick_awkward_coordinates():
    """The batched kick's fixed-point differences on coordinates they do not
    hold exactly (|x| < 2^-36 AU), exact zeros (a flat disk) and close pairs
    straddling an axis, against the oracle over 20 steps."""
    d = ics.make_disk(40, 2.0, 0.8, 1.2, 0.02, 0.01, 6.0, seed=4242)
    x = d.x.copy()
    x[:12, 2] = 0.0
    x[12:20, 2] = np.linspace(-3e-13, 3e-13, 8)
    v = d.v.copy()
    x[20] = [1e-12, 1.0, 0.0]                      # on a circular orbit across the y axis
    v[20] = [-np.sqrt(ics.G_GAUSS), 0.0, 0.0]
    x[21] = x[20] + np.array([-3e-12, 2e-4, 1e-14])
    v[21] = v[20]                                  # a co-moving close pair
    d2 = ics.Disk(x=x, v=v, m=d.m, R=d.R, dt=d.dt)
    dt, steps = 6.0, 20
    ref, rc = oracle_run(d2, steps, dt)
    b = batch_of([d2], dt, [rc])
    b.step(steps, dt)
    sg, sr = b.system_state(0), ref.state()
    assert np.array_equal(sg["ids"], sr["ids"])
    rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
    assert rel.max() <= 1e-12, rel.max()


def test_batch_size_extremes_match_oracle():
    """Systems at the batch's limits in one launch: N = NB_BATCH_MAX_N (512,
    the most a CTA holds in shared memory), 511, 16, 2 and a lone body, each
    against its own oracle run over 30 steps."""
    nb = nbm()
    sizes = [nb.NB_BATCH_MAX_N, 16, 2, 1, nb.NB_BATCH_MAX_N - 1]
    disks = [ics.make_disk(n, 2.0, 0.5, 2.0, 0.02, 0.01, 3.0, seed=4100 + n) for n in sizes]
    dt, steps = 3.0, 30
    refs, rcs = [], []
    for d in disks:
        s, rc = oracle_run(d, steps, dt)
        refs.append(s)
        rcs.append(rc)
    b = batch_of(disks, dt, rcs)
    b.step(steps, dt)
    st = b.state()
    assert b.stats()["groups"] == sum(r.stats()["groups"] for r in refs)
    for k, (d, ref) in enumerate(zip(disks, refs)):
        sg, sr = b.system_state(k, st), ref.state()
        assert np.array_equal(sg["ids"], sr["ids"]), k
        rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
        assert rel.max() <= 1e-12, (k, d.n, rel.max())
        relv = np.linalg.norm(sg["v"] - sr["v"], axis=1) / np.linalg.norm(sr["v"], axis=1)
        assert relv.max() <= 1e-11, (k, d.n, relv.max())


@pytest.mark.parametrize("sym", [0, -1])
def test_batch_schedules_are_bit_identical(sym):
    """Kick tile rows (32, 64, 128; the row kick's), buckets of independent
    launch chains (1, 3, 8) and threads per CTA change where and when each
    system's work runs, never its arithmetic: identical states, encounter
    lists and counters after 30 steps with encounters and mergers, for the
    unordered-pair kick and the row kick."""
    disks = [ics.make_disk(n, 2.0, 0.7, 1.3, 0.01, 0.005, 6.0, seed=900 + n, f_radius=400.0)
             for n in (64, 128, 200)] + ics.ensemble(n_systems=40, seed=ics.SEED_BASE + 36)
    dt, steps = 6.0, 30
    runs = []
    for rows, buckets, threads in ((128, 1, 128), (32, 3, 256), (64, 8, 64)):
        b = batch_of(disks, dt, kick_symmetric=sym)
        b.set_shape(threads, 7)
        b.set_schedule(rows, buckets)
        b.step(steps, dt)
        runs.append((b.state(), [b.encounter_list(k) for k in range(len(disks))], b.stats()))
    s0, e0, t0 = runs[0]
    assert t0["merges"] > 0 and t0["groups"] > 0
    for s1, e1, t1 in runs[1:]:
        for k in s0:
            assert np.array_equal(np.asarray(s0[k]), np.asarray(s1[k])), k
        assert all(np.array_equal(a, c) for a, c in zip(e0, e1))
        for k in ("groups", "bs_derivs", "bs_substeps", "bs_halvings", "merges"):
            assert t0[k] == t1[k], k
