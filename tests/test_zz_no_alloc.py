"""nb_kick_noalloc: the kick for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a framework's allocator owns the device,
allocation is forbidden once the host is running, or a plug-in must never
touch the CUDA allocator). nb_kick_noalloc takes only inputs and outputs and
keeps its scratch in a static device array of the library, so it handles at
most NB_NOALLOC_MAX_N bodies. This file checks it through the C ABI against
nb_kick (which takes caller scratch) with the kick tolerance of the parity
suite, on two calls in a row (the shared array keeps the previous call's
contents, so the second call also checks that it is cleared properly).
It is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09184_b300 import build
    build.build()
    from paper_2604_09184_b300 import nb as nbm
    nbm.lib()
    return nbm


def _case(n, seed, rc_scale):
    from paper_2604_09184_b300 import ics
    from oracle import nbref
    d = ics.workload("mmsn_16k_js", n=n, seed_offset=seed)
    p = nbref.params(dt_rcrit=d.dt)
    rc = rc_scale * np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(d.n)])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    return dev(d.x), dev(d.m), dev(rc)


def _pairset(p):
    return sorted(tuple(int(v) for v in q) for q in p.cpu().numpy().reshape(-1, 2))


# Per-body tolerance against nb_kick in the same precision: the two add their
# partial sums in a different order (this variant uses at most 4 source
# chunks), so they agree to rounding. FP64 and mixed accumulate in FP64; the
# double-single kick accumulates its chunks in float pairs and is held to the
# bound the parity suite gives it.
_TOL = {0: (1e-13, 1e-15), 1: (1e-13, 1e-15), 2: (1e-10, 1e-13)}


def _check_against_nb_kick(nb, x, m, rc, precision):
    a_ref, p_ref, code = nb.kick(x, m, rc, precision=precision)
    assert code == nb.NB_OK
    nbod = x.shape[0]
    a = torch.full((nbod, 3), float("nan"), dtype=torch.float64, device="cuda")
    pairs = torch.full((16 * nbod + 64, 2), -1, dtype=torch.int32, device="cuda")
    cnt, code = nb.kick_noalloc(x, m, rc, a, pairs, precision=precision)
    assert code == nb.NB_OK
    ar = a_ref.cpu().numpy()
    rel, absf = _TOL[precision]
    err = np.linalg.norm(a.cpu().numpy() - ar, axis=1)
    assert np.all(err <= rel * np.linalg.norm(ar, axis=1) + absf * np.abs(ar).max())
    assert cnt == p_ref.shape[0]
    assert _pairset(pairs[:cnt]) == _pairset(p_ref)


def test_noalloc_kick_matches_nb_kick_twice(nb):
    for n, seed, rc_scale in [(3000, 1, 6.0), (1200, 2, 1.0)]:
        x, m, rc = _case(n, seed, rc_scale)
        _check_against_nb_kick(nb, x, m, rc, nb.NB_PREC_FP64)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_noalloc_kick_every_precision_odd_n(nb, precision):
    """An odd body count (the partial-sum block then starts off a 256-byte
    boundary) in every kick precision, twice in a row."""
    for n, seed in [(1001, 3), (257, 4)]:
        x, m, rc = _case(n, seed, 4.0)
        _check_against_nb_kick(nb, x, m, rc, precision)


def test_noalloc_kick_at_size_limit(nb):
    """n = NB_NOALLOC_MAX_N fills the static array exactly (positions, rc^2
    and 4 j-chunks of partial sums), in FP64 and in double-single."""
    x, m, rc = _case(nb.NB_NOALLOC_MAX_N - 2, 5, 2.0)
    assert x.shape[0] == nb.NB_NOALLOC_MAX_N
    _check_against_nb_kick(nb, x, m, rc, nb.NB_PREC_FP64)
    _check_against_nb_kick(nb, x, m, rc, nb.NB_PREC_DS)


def test_noalloc_overflow_reports_true_count(nb):
    """A pair buffer smaller than the flagged set: NB_E_OVERFLOW, the true count,
    and only pairs of the true set written."""
    x, m, rc = _case(3000, 1, 6.0)
    _, p_ref, code = nb.kick(x, m, rc)
    assert code == nb.NB_OK and p_ref.shape[0] > 8
    nbod = x.shape[0]
    a = torch.empty((nbod, 3), dtype=torch.float64, device="cuda")
    pairs = torch.full((8, 2), -1, dtype=torch.int32, device="cuda")
    cnt, code = nb.kick_noalloc(x, m, rc, a, pairs)
    assert code == nb.NB_E_OVERFLOW
    assert cnt == p_ref.shape[0]
    assert set(_pairset(pairs)) <= set(_pairset(p_ref))


def test_noalloc_binding_rejects_bad_buffers(nb):
    """The binding refuses buffers the kernel would write past."""
    x, m, rc = _case(200, 6, 1.0)
    nbod = x.shape[0]
    good_a = torch.empty((nbod, 3), dtype=torch.float64, device="cuda")
    good_p = torch.empty((64, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        nb.kick_noalloc(x, m, rc, good_a[:-1], good_p)
    with pytest.raises(ValueError):
        nb.kick_noalloc(x, m, rc, good_a, good_p.reshape(-1))
    with pytest.raises(ValueError):
        nb.kick_noalloc(x, m, rc, good_a, good_p.to(torch.int64))
    with pytest.raises(ValueError):
        nb.kick_noalloc(x, m, rc[:-1], good_a, good_p)
    with pytest.raises(ValueError):
        nb.kick_noalloc(x.t().contiguous().t(), m, rc, good_a, good_p)
    with pytest.raises(ValueError):
        nb.kick_noalloc(x.cpu(), m, rc, good_a, good_p)


def test_noalloc_rejects_oversize(nb):
    n = nb.NB_NOALLOC_MAX_N + 1
    x = torch.ones((n, 3), dtype=torch.float64, device="cuda")
    m = torch.ones(n, dtype=torch.float64, device="cuda")
    a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pairs = torch.empty((4, 2), dtype=torch.int32, device="cuda")
    cnt, code = nb.kick_noalloc(x, m, m, a, pairs)
    assert code == nb.NB_E_INVALID
