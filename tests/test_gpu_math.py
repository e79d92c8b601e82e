"""The device arithmetic helpers one by one (nb_math_eval) against exact
references: the table-driven exponential against Decimal, the seeded
reciprocal, reciprocal root and r^-3 against correctly rounded values, and
the direct solver's changeover weight 1 - w against the oracle's changeover
(the paragraph after Eq. Hc)."""
import math
import os
import sys
from decimal import Decimal, getcontext

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import nbref  # noqa: E402
from paper_2604_09184_b300 import build  # noqa: E402

U = 2.0 ** -52  # one ulp of 1


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    from paper_2604_09184_b300 import nb as m
    m.lib()
    return m


def evaluate(nb, fn, x):
    t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")
    return nb.math_eval(fn, t).cpu().numpy()


def exact(fn, xs, prec=40):
    getcontext().prec = prec
    return np.array([float(fn(Decimal(float(v)))) for v in xs])


def ulps(got, ref):
    """|got - ref| in units of ref's own ulp."""
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_exp_table_driven(nb):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-80, 80, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                        [0.0, -0.0, 1e-300, -1e-300, 2.0 ** -9, -2.0 ** -9, 80.0, -80.0, 700.0,
                         -700.0, math.log(2.0) / 256, 0.5, -0.5],
                        rng.uniform(-700, 700, 2000)])
    got = evaluate(nb, nb.NB_MATH_EXP, x)
    ref = exact(lambda d: d.exp(), x)
    err = ulps(got, ref)
    assert err.max() <= 1.5, (x[err.argmax()], err.max())
    assert np.mean(err) < 0.3
    assert got[x == 0.0].tolist() == [1.0, 1.0]


def test_reciprocal_and_reciprocal_root(nb):
    rng = np.random.default_rng(2)
    x = np.concatenate([10.0 ** rng.uniform(-37, 37, 20000), [1.0, 2.0, 0.75, 3.0, 1e-30]])
    got = evaluate(nb, nb.NB_MATH_RCP, x)
    assert ulps(got, 1.0 / x).max() <= 1.0
    got = evaluate(nb, nb.NB_MATH_RSQRT, x)
    ref = exact(lambda d: 1 / d.sqrt(), x)
    assert ulps(got, ref).max() <= 1.0


@pytest.mark.parametrize("fn_name,bound", [("NB_MATH_RPOW32", 2.0), ("NB_MATH_RPOW32_M", 2.0),
                                           ("NB_MATH_RINV3", 2.0),
                                           ("NB_MATH_RPOW32_MIXED", 1e-11 / U)])
def test_r_minus_three(nb, fn_name, bound):
    """x^(-3/2) from x = r^2 as the kicks form m / r^3 (m = 1): the FP64
    forms within 2 ulp (the unordered-pair kick's r^-3 with its residual and
    series on the integer pipe too), the single-Newton-step (mixed) form
    within 1e-11."""
    rng = np.random.default_rng(3)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 20000), [1.0, 4.0, 2.0, 1e-20]])
    got = evaluate(nb, getattr(nb, fn_name), x)
    ref = exact(lambda d: 1 / (d * d.sqrt()), x)
    err = ulps(got, ref)
    assert err.max() <= bound, err.max()


def test_close_weight_matches_oracle_changeover(nb):
    """1 - w with w = K - r dK/dr for rc = 1 over the whole changeover
    (0.1 < r < 1) and outside it, against the oracle's K and dK/dr."""
    rng = np.random.default_rng(4)
    r = np.concatenate([rng.uniform(0.0, 1.2, 20000), np.linspace(0.099, 0.102, 301),
                        np.linspace(0.995, 1.001, 301), [0.0, 0.1, 0.55, 1.0, 2.0]])
    got = evaluate(nb, nb.NB_MATH_CLOSE_WEIGHT, r)
    ref = np.empty_like(r)
    for i, v in enumerate(r):
        K, dK = nbref.changeover(float(v), 1.0)
        ref[i] = 1.0 - (K - v * dK)
    err = np.abs(got - ref)
    assert err.max() <= 2e-14, (r[err.argmax()], err.max())
    inside = (r > 0.15) & (r < 0.7)  # where 1 - w is not a cancellation near 0
    assert (np.abs(got - ref)[inside] / np.abs(ref[inside])).max() <= 1e-13
    assert np.all(got[r >= 1.0] == 0.0)
    assert np.all(got[r <= 0.1] == 1.0)


def test_mass_coefficients(nb):
    """1.5 m (significand sum, truncated) and 1.875 m (through a float) as the
    two-argument r^-3 builds them: relative errors below 2^-52 and 2^-18, zero
    for zero (the polynomial multiplies them by e < 2^-19 and e^2)."""
    rng = np.random.default_rng(5)
    m = np.concatenate([10.0 ** rng.uniform(-30, 30, 20000), [0.0, 1.0, 2.0 - 2.0 ** -52, 1e-10,
                                                              2.29e-10, 9.5e-4, 2.0 ** -126]])
    m15 = evaluate(nb, nb.NB_MATH_MASS15, m)
    m1875 = evaluate(nb, nb.NB_MATH_MASS1875, m)
    nz = m > 0
    getcontext().prec = 40
    ref15 = np.array([float(Decimal(float(v)) * Decimal("1.5")) for v in m])
    assert np.all(np.abs(m15[nz] - ref15[nz]) <= 2.0 ** -52 * ref15[nz])
    assert np.all(np.abs(m1875[nz] - 1.875 * m[nz]) <= 2.0 ** -18 * 1.875 * m[nz])
    assert m15[~nz].tolist() == [0.0] and m1875[~nz].tolist() == [0.0]


def test_neville_weights_are_the_correctly_rounded_quotients(nb):
    """The direct solver's Neville weights 1 / ((n_j / n_{j-q})^2 - 1) for
    n_k = 2k, read from its table, equal the IEEE quotients (j - q)^2 /
    (q (2j - q)) bit for bit (the values the division gave at run time)."""
    x = np.array([16 * j + q for j in range(13) for q in range(16)], dtype=np.float64)
    got = evaluate(nb, nb.NB_MATH_NEVILLE, x)
    want = np.array([((j - q) ** 2 / (q * (2 * j - q))) if 1 <= q < j else 0.0
                     for j in range(13) for q in range(16)])
    assert np.array_equal(got, want)
    assert got[16 * 2 + 1] == 1.0 / 3.0  # (n_2 / n_1)^2 - 1 = 3


def test_acceptance_test_equals_the_division(nb):
    """The solver's division-free acceptance test decides fl(a / b) <= tol
    exactly as the IEEE division does: random quotients, quotients within a
    few ulps of tol on either side, exact ones (b a power of two) at tol and
    its neighbours, and non-finite values (a NaN or inf / inf rejects)."""
    rng = np.random.default_rng(11)
    n = 20000
    tol = 10.0 ** rng.uniform(-16, -6, n)
    b = 10.0 ** rng.uniform(-3, 3, n)
    a_rand = b * tol * 10.0 ** rng.uniform(-1, 1, n)
    near = [b * tol]
    for k in (1, 2, 3):
        near.append(np.nextafter(near[-1], np.inf))
    lo = [b * tol]
    for k in (1, 2, 3):
        lo.append(np.nextafter(lo[-1], -np.inf))
    b2 = 2.0 ** rng.integers(-20, 20, n).astype(np.float64)
    exact_q = [tol * b2, np.nextafter(tol, np.inf) * b2, np.nextafter(tol, 0.0) * b2]
    A = np.concatenate([a_rand] + near + lo + exact_q + [np.zeros(4)])
    B = np.concatenate([b] * 9 + [b2] * 3 + [np.ones(4)])
    T = np.concatenate([tol] * 12 + [np.full(4, 1e-14)])
    A = np.concatenate([A, [np.inf, 1.0, np.nan, np.inf, 0.0]])
    B = np.concatenate([B, [1.0, np.inf, 1.0, np.inf, 1e-300]])
    T = np.concatenate([T, [1e-14, 1e-14, 1e-14, 1e-14, 0.0]])
    with np.errstate(invalid="ignore"):
        want = (A / B <= T).astype(np.float64)
    got = nb.ratio_le(*(torch.as_tensor(v, device="cuda") for v in (A, B, T))).cpu().numpy()
    assert np.array_equal(got, want)
    assert 0 < want.sum() < len(want)


def test_invalid_function_rejected(nb):
    L = nb.lib()
    assert L.nb_math_eval(99, 0, None, None, None) == nb.NB_E_INVALID
    assert L.nb_math_eval(0, -1, None, None, None) == nb.NB_E_INVALID
    assert L.nb_math_eval(0, 4, None, None, None) == nb.NB_E_INVALID
    assert L.nb_math_eval(0, 0, None, None, None) == nb.NB_OK
