"""Full-size multi-step FP64 parity: the CUDA library against the oracle on the
benchmark workloads themselves, not subsets.

  - the 16k disk with Jupiter and Saturn (16386 bodies), 100 steps;
  - the adjoint workload (2048 planetesimals + Jupiter), 100 steps, through
    nb_step and through the adjoint's checkpointed forward;
  - the 64k disk with Jupiter and Saturn (65538 bodies), 10 steps.

Each compares, element by element: ids and masses, encounter lists, group
and merger counts (all exactly), the direct solver's accepted-substep and
halving counts, and positions. The bar is a relative position error of 1e-12.

The direct solver accepts a substep, or halves it, by comparing an
extrapolation error estimate with bs_tol. Both sides compute that estimate
from the same formula with different rounding (the GPU's reciprocal roots
and exponential are its own, within 1-2 ulp), so a group whose estimate sits
within rounding of bs_tol can take the other branch. Either branch converges
to the tolerance, and the group's state differs by about bs_tol (1e-14), but
each flip changes the accepted-substep count by one or two and the halving
count by one. Over thousands of substeps such flips occur: the counts are
held to within max(2, 0.1 %), the test prints the difference, and it also
prints the oracle's own counts under 1-ulp input perturbations (the same
decisions flipping on the oracle alone).

These disks have close encounters every step, and a Bulirsch-Stoer
integration through an encounter amplifies rounding: the oracle disagrees with itself by more than 1e-12 on some
encounter bodies when its inputs move by one ulp. Bodies that never entered
an encounter are therefore held to 1e-12 flat, encounter bodies to
max(1e-12, 3 x the largest spread of the oracle's own positions under 1-ulp
input perturbations; a flipped direct-solver decision moves other bodies than
a perturbation does, so the bound is over the whole run, not body by body), and
the test prints how many bodies that wider bound applies to and the spread
it measured.
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
    from paper_2604_09184_b300 import nb
    nb.lib()


def nbmod():
    from paper_2604_09184_b300 import nb
    return nb


def oracle_rc(d, p):
    return np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(d.n)])


_SPREAD = {}


def oracle_spread(d, rc, steps, xb, trials, **kw):
    """Largest relative position spread of the oracle against its own run xb
    when every input coordinate moves by one ulp (the run's conditioning),
    and the oracle's direct-solver counts in those runs."""
    key = (d.name, d.n, steps, trials, tuple(sorted(kw.items())))
    if key in _SPREAD:
        return _SPREAD[key]
    rp = nbref.params(dt_rcrit=d.dt, **kw)
    rng = np.random.default_rng(1)
    worst = np.zeros(len(xb))
    counts = []
    for _ in range(trials):
        x = d.x * (1 + rng.choice([-1, 1], d.x.shape) * 2.0 ** -53)
        v = d.v * (1 + rng.choice([-1, 1], d.v.shape) * 2.0 ** -53)
        s = nbref.RefSystem(rp, x, v, d.m, d.R, rc=rc)
        assert s.step(steps, d.dt) == 0
        st = s.state()
        counts.append((s.stats()["bs_substeps"], s.stats()["bs_halvings"]))
        if st["x"].shape != xb.shape:
            worst = np.full(len(xb), np.inf)  # a merger moved: the run is not conditioned at all
            continue
        worst = np.maximum(worst, np.linalg.norm(st["x"] - xb, axis=1) / np.linalg.norm(xb, axis=1))
    _SPREAD[key] = (worst, counts)
    return _SPREAD[key]


def check_run(d, steps, sr_sys, sg, enc_list_g, stats_g, trials, label, **kw):
    """Compare one GPU result (state sg, encounter list, stats) with the oracle
    system sr_sys after `steps` steps."""
    sr = sr_sys.state()
    er = sr_sys.encounter_list()
    assert np.array_equal(sr["ids"], sg["ids"]), label
    assert np.array_equal(sr["m"], sg["m"]), label
    assert np.array_equal(er, enc_list_g), (label, len(er), len(enc_list_g))
    counts_note = ""
    if stats_g is not None:
        rs = sr_sys.stats()
        for k in ("groups", "merges", "encounter_pairs"):
            assert rs[k] == stats_g[k], (label, k, rs[k], stats_g[k])
        dsub = stats_g["bs_substeps"] - rs["bs_substeps"]
        dhalv = stats_g["bs_halvings"] - rs["bs_halvings"]
        counts_note = "; BS substeps %d vs oracle %d, halvings %d vs %d" % (
            stats_g["bs_substeps"], rs["bs_substeps"], stats_g["bs_halvings"], rs["bs_halvings"])
        if dsub or dhalv:
            _, counts = oracle_spread(d, sr_sys._rc_init, steps, sr["x"], trials, **kw)
            counts_note += " (oracle under 1-ulp input perturbations: %s)" % counts
        assert abs(dsub) <= max(2, 1e-3 * rs["bs_substeps"]), (label, counts_note)
        assert abs(dhalv) <= max(2, 1e-3 * rs["bs_substeps"]), (label, counts_note)
    rel = np.linalg.norm(sg["x"] - sr["x"], axis=1) / np.linalg.norm(sr["x"], axis=1)
    relv = np.linalg.norm(sg["v"] - sr["v"], axis=1) / np.linalg.norm(sr["v"], axis=1)
    enc = np.isin(sr["ids"], er[:, 1:].reshape(-1)) if len(er) else np.zeros(len(rel), bool)
    quiet_max = rel[~enc].max() if (~enc).any() else 0.0
    assert quiet_max <= 1e-12, (label, quiet_max)
    assert relv[~enc].max() <= 1e-11 if (~enc).any() else True
    over = rel > 1e-12
    spread_max = 0.0
    if over.any():
        rc = sr_sys._rc_init
        spread, _ = oracle_spread(d, rc, steps, sr["x"], trials, **kw)
        spread_max = float(np.max(spread))
        bound = max(1e-12, 3.0 * spread_max)
        assert rel.max() <= bound, (label, rel.max(), spread_max)
    print("%s: %d bodies, %d encounter bodies, %d above 1e-12 (max %.2e; oracle 1-ulp spread "
          "%.2e), quiet bodies max %.2e, %d encounter pairs%s" % (
              label, len(rel), int(enc.sum()), int(over.sum()), rel.max(), spread_max, quiet_max,
              len(er), counts_note))
    return rel


def run_pair(d, steps, gpu_kw=None, **kw):
    nb = nbmod()
    rp = nbref.params(dt_rcrit=d.dt, **kw)
    rc = oracle_rc(d, rp)
    ref = nbref.RefSystem(rp, d.x, d.v, d.m, d.R, rc=rc)
    ref._rc_init = rc
    assert ref.step(steps, d.dt) == 0
    gpu = nb.NBodySystem(nb.params(dt_rcrit=d.dt, **kw, **(gpu_kw or {})), d.x, d.v, d.m, d.R,
                         rc=rc)
    gpu.step(steps, d.dt)
    return ref, gpu, rc


def test_fullsize_mmsn_16k_100_steps():
    d = ics.workload("mmsn_16k_js")
    assert d.n == 16386
    ref, gpu, _ = run_pair(d, 100)
    st = gpu.stats()
    assert st["steps"] == 100 and st["groups"] > 0
    check_run(d, 100, ref, gpu.state(), gpu.encounter_list(), st, 2, "mmsn_16k_js x 100")


def test_fullsize_adjoint_workload_100_steps():
    """The adjoint workload's forward, both through nb_step and through the
    adjoint's checkpointed forward pass (nb_adjoint_forward), against the
    oracle."""
    nb = nbmod()
    d = ics.workload("adjoint_2k_j")
    assert d.n == 2049
    ref, gpu, rc = run_pair(d, 100)
    st = gpu.stats()
    assert st["groups"] > 0
    check_run(d, 100, ref, gpu.state(), gpu.encounter_list(), st, 2, "adjoint_2k_j x 100")
    adj = nb.NBodyAdjoint(nb.params(dt_rcrit=d.dt), d.x, d.v, d.m, d.R, rc, 100, 10)
    adj.forward(d.dt)
    sa = adj.state()
    alive = sa["alive"] != 0
    sg = {"ids": np.nonzero(alive)[0].astype(np.int32), "x": sa["x"][alive], "v": sa["v"][alive],
          "m": sa["m"][alive]}
    check_run(d, 100, ref, sg, ref.encounter_list(), None, 2, "adjoint forward x 100")
    # the adjoint forward is the same map as nb_step, bit for bit
    sgs = gpu.state()
    assert np.array_equal(sg["x"], sgs["x"]) and np.array_equal(sg["v"], sgs["v"])


def test_fullsize_mmsn_64k_10_steps():
    d = ics.workload("mmsn_64k_js")
    assert d.n == 65538
    ref, gpu, _ = run_pair(d, 10)
    st = gpu.stats()
    assert st["steps"] == 10 and st["groups"] > 0
    check_run(d, 10, ref, gpu.state(), gpu.encounter_list(), st, 1, "mmsn_64k_js x 10")


def test_large_groups_on_the_cluster_solver_5_steps():
    """The 16k disk family at N = 4098 under the literal velocity reading of
    Eq. rcrit (vel_mode 1): every step forms one group of ~280 bodies and
    hundreds of small ones. Groups of 64 or more bodies run on a thread-block
    cluster (k_bs_cluster); the run is checked against the oracle over 5 steps
    like the other full-size runs, and the GPU step time is printed."""
    import networkx as nx
    nb = nbmod()
    d = ics.workload("mmsn_16k_js", n=4096)
    ref, gpu, rc = run_pair(d, 5, gpu_kw={"bs_cluster_min": 64}, vel_mode=1)
    el = ref.encounter_list()
    g = nx.Graph()
    g.add_edges_from((int(i), int(j)) for s, i, j in el if s == 0)
    largest = max(len(c) for c in nx.connected_components(g))
    assert largest >= 100, largest
    check_run(d, 5, ref, gpu.state(), gpu.encounter_list(), gpu.stats(), 2,
              "mmsn_16k_js n=4096 vel_mode=1 x 5 (largest group %d)" % largest, vel_mode=1)
    # the step time with the cluster solver (events on the library's stream)
    g2 = nb.NBodySystem(nb.params(dt_rcrit=d.dt, vel_mode=1, bs_cluster_min=64), d.x, d.v, d.m,
                        d.R, rc=rc)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    g2.step(3, d.dt)
    e1.record(st)
    torch.cuda.synchronize()
    print("large-group step: %.1f ms per step (3 steps from the initial state)" % (
        e0.elapsed_time(e1) / 3))
