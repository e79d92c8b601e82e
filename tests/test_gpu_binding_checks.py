"""The binding refuses buffers that a kernel would read or write past.

Every entry point of nb.py passes raw pointers to libnb. A host tensor where a
device pointer is expected, a tensor of the wrong dtype or a short one would
make a kernel read or write outside its buffer, so the binding checks
device, dtype, layout and shape first and raises ValueError; nothing reaches
the GPU. Each case below plants one such mistake in otherwise good arguments
and checks the refusal; a correct call follows each group, so the checks do
not refuse good buffers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_09184_b300 import build, ics  # noqa: E402


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2604_09184_b300 import nb as nbm
    nbm.lib()
    return nbm


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype)


def _disk(n=64):
    return ics.make_disk(n, 2.0, 0.8, 2.5, 0.02, 0.01, 8.0, seed=9001)


def test_system_init_refuses_mismatched_inputs(nb):
    d = _disk()
    p = nb.params(dt_rcrit=d.dt)
    x, v, m, R = _dev(d.x), _dev(d.v), _dev(d.m), _dev(d.R)
    for bad in ((x[:-1], v, m, R), (x, v.reshape(-1), m, R), (x, v, m.cpu(), R),
                (x, v, m, R[:-1])):
        with pytest.raises(ValueError):
            nb.NBodySystem(p, *bad)
    with pytest.raises(ValueError):
        nb.NBodySystem(p, x, v, m, R, rc=_dev(np.ones(d.n - 1)))
    with pytest.raises(ValueError):
        nb.NBodySystem(p, x, v, m, R, ids=_dev(np.arange(d.n + 1), torch.int32))
    with pytest.raises(ValueError):  # host arrays of the wrong length
        nb.NBodySystem(p, d.x[:-1], d.v, d.m, d.R)
    s = nb.NBodySystem(p, x, v, m, R)
    s.step(2, d.dt)
    g = nb.NBodySystem(p, d.x, d.v, d.m, d.R)
    g.step(2, d.dt)
    assert np.array_equal(s.state()["x"], g.state()["x"])


def test_state_device_and_set_state_refuse_short_buffers(nb):
    d = _disk()
    s = nb.NBodySystem(nb.params(dt_rcrit=d.dt), d.x, d.v, d.m, d.R)
    n = d.n
    f = lambda *sh: torch.zeros(sh, dtype=torch.float64, device="cuda")  # noqa: E731
    out = dict(x=f(n, 3), v=f(n, 3), m=f(n), R=f(n), rc=f(n),
               ids=torch.zeros(n, dtype=torch.int32, device="cuda"))
    for k, bad in (("x", f(n - 1, 3)), ("ids", torch.zeros(n, dtype=torch.int64, device="cuda")),
                   ("v", f(n, 3).t()), ("rc", torch.zeros(n, dtype=torch.float64))):
        with pytest.raises(ValueError):
            s.state_device(dict(out, **{k: bad}))
    k = s.state_device(out)
    assert k == n
    assert np.array_equal(out["x"].cpu().numpy(), s.state()["x"])
    a, pairs = s.fsal()
    st = s.state()
    with pytest.raises(ValueError):
        s.set_state(st["x"], st["v"], st["m"], st["R"], st["rc"], st["ids"], a[:-1], pairs)
    with pytest.raises(ValueError):
        s.set_fsal(a[:-1], pairs)
    s.set_state(st["x"], st["v"], st["m"], st["R"], st["rc"], st["ids"], a, pairs)


def test_single_kernel_entry_points_refuse_bad_buffers(nb):
    d = _disk(200)
    x, m = _dev(d.x), _dev(d.m)
    rc = torch.full((d.n,), 1e-3, dtype=torch.float64, device="cuda")
    for args in ((x, m[:-1], rc), (x, m, rc[:-1]), (x.reshape(-1), m, rc), (x.cpu(), m, rc)):
        with pytest.raises(ValueError):
            nb.kick(*args)
    a, _, code = nb.kick(x, m, rc)
    assert code == nb.NB_OK and a.shape == (d.n, 3)
    v = _dev(d.v)
    al = torch.ones(d.n, dtype=torch.int32, device="cuda")
    for args in ((x, v[:-1], m), (x, v, m[:-2]), (x.cpu(), v, m)):
        with pytest.raises(ValueError):
            nb.energy_grad(*args)
    with pytest.raises(ValueError):
        nb.energy_grad(x, v, m, al[:-1])
    nb.energy_grad(x, v, m, al)
    xk, vk = x.clone(), v.clone()
    for bad in ((xk, vk[:-1]), (xk, vk.to(torch.float32)), (xk.t(), vk), (xk.cpu(), vk)):
        with pytest.raises(ValueError):
            nb.kepler_drift(*bad, 2.959122082855911e-4, 1.0)
    assert nb.kepler_drift(xk, vk, 2.959122082855911e-4, 1.0) == nb.NB_OK
    with pytest.raises(ValueError):
        nb.math_eval(nb.NB_MATH_EXP, torch.zeros(8, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        nb.ratio_le(m, m[:-1], m)


def test_adjoint_and_batch_refuse_mismatched_inputs(nb):
    d = _disk(48)
    p = nb.params(dt_rcrit=d.dt)
    rc = np.full(d.n, 1e-3)
    with pytest.raises(ValueError):
        nb.NBodyAdjoint(p, d.x, d.v, d.m, d.R, rc[:-1], 4, 2)
    with pytest.raises(ValueError):
        nb.NBodyAdjoint(p, _dev(d.x), _dev(d.v), _dev(d.m), _dev(d.R), rc, 4, 2)  # host rc
    adj = nb.NBodyAdjoint(p, d.x, d.v, d.m, d.R, rc, 4, 2)
    adj.forward(d.dt)
    g = (np.zeros((d.n, 3)), np.zeros((d.n, 3)), np.zeros(d.n))
    with pytest.raises(ValueError):
        adj.backward(g[0][:-1], g[1], g[2])
    adj.backward(*g)
    with pytest.raises(ValueError):
        nb.NBodyBatch(p, [d, d], rc=np.full(d.n, 1e-3))
