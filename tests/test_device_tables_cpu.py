"""Constants that the CUDA kernels carry as literals, checked on the CPU
against their definitions computed independently to 60 digits: the
table-driven exponential's 2^(j/128) table and its ln2/128 split, and the
host-callable integer construction of a float seed's square and cube."""
import os
import re
import subprocess
from decimal import Decimal, getcontext

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2604_09184_b300", "csrc", "nb_internal.cuh")


def _body(name):
    src = open(HDR).read()
    i = src.index(name)
    return src[i:src.index("}", i)]


def test_exp_table_is_two_to_the_j_over_128_rounded():
    getcontext().prec = 60
    tab = _body("kExp2Tab[128] = {")
    vals = [float.fromhex(t) for t in re.findall(r"0x[0-9a-f.]+p[+-]\d+", tab)]
    assert len(vals) == 128
    for j, v in enumerate(vals):
        assert v == float(Decimal(2) ** (Decimal(j) / Decimal(128))), j


def test_ln2_over_128_split():
    getcontext().prec = 60
    src = open(HDR).read()
    hi, lo = [float.fromhex(h) for h in re.findall(
        r"__fma_rn\(-kd, (0x[0-9a-f.]+p[+-]\d+), [rx]\)", src)]
    L = Decimal(2).ln() / 128
    assert hi == float(L)
    assert lo == float(L - Decimal(hi))
    assert abs(Decimal(hi) + Decimal(lo) - L) < Decimal(2) ** -115  # 2^-107 relative
    k = re.search(r"xf \* ([0-9.]+)f\)", src).group(1)  # 128 / ln2 in FP32 (only picks k)
    assert abs(float(k) - float(128 / Decimal(2).ln())) < 1e-9


def test_seed_powers_bit_construction(tmp_path):
    """seed_powers (host-callable) against exact integer products for every
    significand pattern class: y0^2 exact, y0^3 within half an ulp."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "sp.cu"
    src.write_text(r'''
#include "nb_internal.cuh"
#include <cstdio>
#include <cstring>
#include <cmath>
int main() {
  unsigned long long state = 88172645463325252ull;
  long bad = 0;
  for (long it = 0; it < 2000000; ++it) {
    state ^= state << 13; state ^= state >> 7; state ^= state << 17;
    unsigned e = 63 + (unsigned)(state % 128), mant = (unsigned)((state >> 8) & 0x7fffff);
    if (it < 3) mant = it == 0 ? 0u : (it == 1 ? 0x7fffffu : 1u);
    unsigned yb = (e << 23) | mant;
    float yf; memcpy(&yf, &yb, 4);
    nb::SeedPow sp = nb::seed_powers(yb);
    long double y = yf;
    if ((long double)sp.t != y * y) ++bad;
    unsigned __int128 s = mant | 0x800000u, s3 = s * s * s;
    // |y3 - y0^3| <= half an ulp of y3 (exact value from the 72-bit integer)
    int L = 127 - __builtin_clzll((unsigned long long)(s3 >> 64));
    unsigned __int128 q = s3 >> (L - 52), rem = s3 - (q << (L - 52));
    unsigned __int128 half = (unsigned __int128)1 << (L - 53);
    unsigned __int128 qr = q + (rem >= half ? 1 : 0);
    double want_lo = ldexp((double)(unsigned long long)q, L - 52 + 3 * ((int)e - 127) - 69);
    double want_hi = ldexp((double)(unsigned long long)qr, L - 52 + 3 * ((int)e - 127) - 69);
    bool tie = rem == half;
    if (!(sp.y3 == want_hi || (tie && sp.y3 == want_lo))) ++bad;
  }
  printf("%ld\n", bad);
  return bad != 0;
}
''')
    exe = tmp_path / "sp"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + os.path.dirname(HDR),
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "0", out.stdout + out.stderr


def test_sep2_int_against_long_double(tmp_path):
    """The integer-arithmetic r^2 of the kick's pair loop (host-callable, the
    same code): within half an ulp plus 2^-58 relative of the sum computed in
    long double (64-bit significands) for components spread over 2^-60..2^20,
    with zeros, signs and near-cancelling magnitudes."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "r2.cu"
    src.write_text(r"""
#include "nb_internal.cuh"
#include <cstdio>
#include <cmath>
int main() {
  unsigned long long st = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; };
  long bad = 0;
  for (long it = 0; it < 3000000; ++it) {
    double c[3];
    const int e0 = (int)(rnd() % 81) - 60;
    for (int k = 0; k < 3; ++k) {
      const unsigned long long r = rnd();
      const int mode = (int)(r % 8);
      double v = ldexp(1.0 + (double)(rnd() >> 12) * 0x1p-52, e0 - (int)(rnd() % (mode < 4 ? 4 : 70)));
      if (mode == 7) v = 0.0;
      c[k] = (r & 256) ? -v : v;
    }
    const double got = nb::sep2_int(c[0], c[1], c[2]);
    long double ex = (long double)c[0] * c[0] + (long double)c[1] * c[1] + (long double)c[2] * c[2];
    if (ex == 0.0L) { if (got != 0.0) ++bad; continue; }
    const long double ulp = (long double)(nextafter((double)ex, INFINITY) - (double)ex);
    const long double err = fabsl((long double)got - ex);
    if (err > 0.5L * ulp + ldexpl(ex, -58)) {
      if (bad < 5) printf("bad %.20Lg %.20g\n", ex, got);
      ++bad;
    }
  }
  printf("%ld\n", bad);
  return bad != 0;
}
""")
    exe = tmp_path / "r2"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + os.path.dirname(HDR),
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("0"), out.stdout + out.stderr


def test_fixed_point_differences(tmp_path):
    """The kick's integer dx (128-bit fixed-point positions, exact difference,
    rounded to a double): for coordinates in the exact range (2^-36..1e8 AU,
    both signs, coincident and nearly coincident pairs) it equals the FP64
    subtraction except on exact ties (rounded upward, so within half an ulp)
    and, for a negative difference, one unit of 2^-88 AU;
    for smaller coordinates its error stays below 2^-86 AU plus half an ulp;
    r^2 is within half an ulp plus 2^-57 of the long-double sum of the exact
    differences."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "fx.cu"
    src.write_text(r"""
#include "nb_internal.cuh"
#include <cstdio>
#include <cmath>
int main() {
  unsigned long long st = 0x2545F4914F6CDD1Dull;
  auto rnd = [&]() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; };
  auto uni = [&]() { return (double)((rnd() >> 11) | 1ull) * 0x1p-53; };
  long bad = 0, ties = 0, n = 0;
  // magnitudes whose top 54 bits are all ones (rounding carries out of 64
  // bits) and exact powers of two, both signs: X = 2^k units - 1 unit
  for (int k = 40; k <= 120; ++k) {
    const double a = ldexp(1.0, k - 88), b = ldexp(1.0, -88);
    const double cases[4][2] = {{a, b}, {b, a}, {a, 0.0}, {0.0, a}};
    for (auto& c : cases) {
      const nb::FixDiff f = nb::fix_diff(nb::fix_of(c[0]), nb::fix_of(c[1]));
      const long double dl = (long double)c[0] - (long double)c[1];
      const double u = fabs(nextafter((double)dl, INFINITY) - (double)dl);
      if (fabsl((long double)f.d - dl) > 0.5L * u + ldexpl(1.0L, -88)) {
        if (bad < 5) printf("edge k=%d %.17g %.17g: %.17g\n", k, c[0], c[1], f.d);
        ++bad;
      }
    }
  }
  for (long it = 0; it < 2000000; ++it) {
    const bool tiny = (it % 10) == 0;
    double a[3], b[3];
    for (int k = 0; k < 3; ++k) {
      const int mode = (int)(rnd() % 6);
      const double lo = tiny ? -16.0 : -10.8, span = tiny ? 8.0 : 18.8;  // log10 range
      const double sa = pow(10.0, lo + span * uni()), sb = pow(10.0, lo + span * uni());
      a[k] = (rnd() & 1 ? -1.0 : 1.0) * sa;
      if (mode == 0) b[k] = a[k];                                        // coincident
      else if (mode == 1) b[k] = a[k] * (1.0 + 1e-12 * (uni() - 0.5));   // nearly
      else if (mode == 2) b[k] = -a[k];
      else b[k] = (rnd() & 1 ? -1.0 : 1.0) * sb;
    }
    nb::FixDiff f[3];
    long double ex = 0.0L;
    for (int k = 0; k < 3; ++k) {
      f[k] = nb::fix_diff(nb::fix_of(a[k]), nb::fix_of(b[k]));
      const double want = a[k] - b[k];
      const long double dl = (long double)a[k] - (long double)b[k];
      ex += dl * dl;
      if (tiny) {  // truncation of each coordinate (< 2^-88) plus the rounding of dx
        const long double u = (long double)fabs(nextafter(want, INFINITY) - want);
        if (fabsl((long double)f[k].d - dl) > ldexpl(1.0L, -86) + 0.5L * u) ++bad;
        continue;
      }
      ++n;
      if (f[k].d != want) {
        // ties round upward; a negative difference is taken one unit (2^-88 AU) small
        const double u = fabs(nextafter(want, INFINITY) - want);
        const long double err = fabsl((long double)f[k].d - dl);
        if (err > 0.5L * u + ldexpl(1.0L, -88)) { if (bad < 5) printf("dx %.17g %.17g: %.17g vs %.17g\n", a[k], b[k], f[k].d, want); ++bad; }
        else ++ties;
      }
    }
    const double r2 = nb::sep2_fix(f[0], f[1], f[2]);
    if (ex == 0.0L) { if (r2 != 0.0) ++bad; continue; }
    const long double ulp = (long double)(nextafter((double)ex, INFINITY) - (double)ex);
    // tiny: each difference is off by e < 2^-87 (plus its rounding), so r^2 by
    // at most 3 (2 |d| e + e^2)
    // (a negative difference is taken one unit, 2^-88 AU, small: 2 |d| 2^-88 per component)
    const long double tol = tiny ? ldexpl(ex, -50) + 3.0L * (ldexpl(sqrtl(ex), -83) + ldexpl(1.0L, -170))
                                 : 0.5L * ulp + ldexpl(ex, -57) + 3.0L * ldexpl(sqrtl(ex), -87);
    if (fabsl((long double)r2 - ex) > tol) { if (bad < 10) printf("r2 %.20Lg %.20g\n", ex, r2); ++bad; }
  }
  printf("ties %ld of %ld\n%ld\n", ties, n, bad);
  return bad != 0;
}
""")
    exe = tmp_path / "fx"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + os.path.dirname(HDR),
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr


def test_integer_pipe_rinv3_against_long_double(tmp_path):
    """r^-3 from a float seed with the residual and the (1 - e)^(-3/2) series
    on the integer pipe and one FP64 product (host-callable, the same code the
    unordered-pair kick runs): within 1.7 ulp of 1 / (r^2 sqrt(r^2)) in long
    double, for r^2 over 2^-100..2^100 with extreme significands and seeds
    off by up to 1e-6 relative either way (|e| up to ~2e-6; the kick's seed,
    rsqrtf of r^2 truncated to a float, is off by at most ~2^-20)."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "r3.cu"
    src.write_text(r"""
#include "nb_internal.cuh"
#include <cstdio>
#include <cstring>
#include <cmath>
int main() {
  unsigned long long st = 0x2545F4914F6CDD1Dull;
  auto rnd = [&]() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; };
  long bad = 0;
  long double worst = 0.0L;
  for (long it = 0; it < 3000000; ++it) {
    const int E = (int)(rnd() % 201) - 100;
    unsigned long long mant = rnd() >> 12;
    const int mode = (int)(it % 16);
    if (mode == 0) mant = 0ull;
    if (mode == 1) mant = 0xfffffffffffffull;
    if (mode == 2) mant = 1ull;
    const double r2 = ldexp(1.0 + (double)mant * 0x1p-52, E);
    const long double y = 1.0L / sqrtl((long double)r2);
    // seed: the exact root moved by up to 1e-6 relative (or the kick's own
    // construction: rsqrt of r^2 truncated to a float), rounded to a float
    float yf;
    if (mode == 3) {
      unsigned hr = (unsigned)(nb::nb_dbits(r2) >> 32);
      unsigned fb = (hr << 3) + 0x40000000u;
      float r2f; memcpy(&r2f, &fb, 4);
      yf = 1.0f / sqrtf(r2f);
    } else {
      const long double u = ((long double)(rnd() >> 11) * 0x1p-53L * 2.0L - 1.0L) * 1e-6L;
      yf = (float)(y * (1.0L + u));
    }
    unsigned yb; memcpy(&yb, &yf, 4);
    const double got = nb::rinv3_from_seed(r2, yb);
    const long double ex = y * y * y;
    const long double rel = fabsl((long double)got - ex) / ex;
    if (rel > worst) worst = rel;
    if (rel > 1.7L * 0x1p-52L) {
      if (bad < 5) printf("bad r2=%a yb=%08x got=%a ex=%La\n", r2, yb, got, ex);
      ++bad;
    }
  }
  printf("worst %.3Lg ulp\n%ld\n", worst / 0x1p-52L, bad);
  return bad != 0;
}
""")
    exe = tmp_path / "r3"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + os.path.dirname(HDR),
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("\n0"), out.stdout + out.stderr
