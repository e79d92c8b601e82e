// Universal-variable Kepler drift (the first sum of Eq. Ha: Kepler motion
// about mu = G m0, "solved analytically"), shared by the single-system drift
// kernel, the batched kernel and the adjoint. The solver is written once,
// templated on its scalar type: double for the integrator, Dual<1> (value
// and one partial derivative) for the adjoint's Jacobian of the drift map.
#pragma once

#include "nb_internal.cuh"

namespace nb {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers with ND partials: ND = 6 carries the whole
// Jacobian of (x, v) -> (x', v'), ND = 1 one of its columns (one input
// direction per thread). They live in their own namespace so that their
// sqrt/log/fabs/copysign are found only by argument-dependent lookup and
// never hide the double versions.
// ---------------------------------------------------------------------------
namespace ad {
template <int ND>
struct Dual {
  double v;
  double d[ND];
};

template <int ND>
__device__ __forceinline__ double val(const Dual<ND>& a) { return a.v; }

template <int ND>
__device__ __forceinline__ Dual<ND> mkd(double v) {
  Dual<ND> r;
  r.v = v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = 0.0;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator+(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator-(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator-(const Dual<ND>& a) {
  Dual<ND> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator*(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator/(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator+(const Dual<ND>& a, double b) {
  Dual<ND> r = a;
  r.v += b;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator+(double b, const Dual<ND>& a) { return a + b; }
template <int ND>
__device__ __forceinline__ Dual<ND> operator-(const Dual<ND>& a, double b) {
  Dual<ND> r = a;
  r.v -= b;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator-(double b, const Dual<ND>& a) { return -(a - b); }
template <int ND>
__device__ __forceinline__ Dual<ND> operator*(const Dual<ND>& a, double b) {
  Dual<ND> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> operator*(double b, const Dual<ND>& a) { return a * b; }
template <int ND>
__device__ __forceinline__ Dual<ND> operator/(const Dual<ND>& a, double b) { return a * (1.0 / b); }
template <int ND>
__device__ __forceinline__ Dual<ND> operator/(double a, const Dual<ND>& b) { return mkd<ND>(a) / b; }
template <int ND>
__device__ __forceinline__ Dual<ND> sqrt(const Dual<ND>& a) {
  Dual<ND> r;
  r.v = ::sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> log(const Dual<ND>& a) {
  Dual<ND> r;
  r.v = ::log(a.v);
#pragma unroll
  for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] / a.v;
  return r;
}
template <int ND>
__device__ __forceinline__ Dual<ND> fabs(const Dual<ND>& a) { return a.v < 0.0 ? -a : a; }
template <int ND>
__device__ __forceinline__ Dual<ND> copysign(const Dual<ND>& a, const Dual<ND>& s) {
  return (a.v < 0.0) != (s.v < 0.0) ? -a : a;
}
}  // namespace ad

using ad::Dual;
using ad::mkd;
__device__ __forceinline__ double val(double a) { return a; }
using ad::val;

// ---------------------------------------------------------------------------
// Stumpff functions c0..c3 (Danby's method): quarter z until |z| <= 0.1,
// sum the c2, c3 series there, rebuild c0 = 1 - z c2 and c1 = 1 - z c3, then
// undo each quartering with the argument-quadrupling identities
//   c0(4z) = 2 c0^2 - 1,  c1(4z) = c0 c1,  c2(4z) = c1^2 / 2,
//   c3(4z) = (c2 + c0 c3) / 4.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stumpff(T z, T& c0, T& c1, T& c2, T& c3) {
  int nq = 0;
  while (::fabs(val(z)) > 0.1 && nq < 64) {
    z = z * 0.25;
    ++nq;
  }
  // c2 = sum_k (-z)^k / (2k+2)!, k = 0..6, and c3 = sum_k (-z)^k / (2k+3)!,
  // k = 0..5: at |z| <= 0.1 the first terms left out are below 1e-20 and
  // 5e-18 of the sums (2e-4 and 0.05 ulp)
  c2 = 1.0 / 2.0 -
       z * (1.0 / 24.0 -
            z * (1.0 / 720.0 -
                 z * (1.0 / 40320.0 -
                      z * (1.0 / 3628800.0 -
                           z * (1.0 / 479001600.0 - z * (1.0 / 87178291200.0))))));
  c3 = 1.0 / 6.0 -
       z * (1.0 / 120.0 -
            z * (1.0 / 5040.0 -
                 z * (1.0 / 362880.0 - z * (1.0 / 39916800.0 - z * (1.0 / 6227020800.0)))));
  c1 = 1.0 - z * c3;
  c0 = 1.0 - z * c2;
  for (; nq > 0; --nq) {
    c3 = (c2 + c0 * c3) * 0.25;
    c2 = c1 * c1 * 0.5;
    c1 = c0 * c1;
    c0 = 2.0 * c0 * c0 - 1.0;
  }
}

// Reciprocals and the radius of the solver. For doubles (the integrator) a
// lone warp issues one FP64 instruction per 64 cycles, so the radius and its
// reciprocal come from the seeded reciprocal root of r^2 (r^2 on the integer
// pipe) and the positive denominators from the seeded reciprocal: 5 and 3
// FP64 instructions against ~11 for sqrt and ~9 for a division, each within
// about an ulp. The dual types (the adjoint's Jacobian, whose values are not
// fed back) keep the plain quotient and root.
__device__ __forceinline__ void radius_and_inverse(double x, double y, double z, double& r,
                                                   double& ir) {
  const double r2 = sep2_int(x, y, z);
  ir = rinv_fast(r2);
  r = r2 * ir;
}
template <int ND>
__device__ __forceinline__ void radius_and_inverse(const Dual<ND>& x, const Dual<ND>& y,
                                                   const Dual<ND>& z, Dual<ND>& r, Dual<ND>& ir) {
  r = sqrt(x * x + y * y + z * z);
  ir = 1.0 / r;
}
__device__ __forceinline__ double pos_rcp(double x) { return rcp_fast(x); }
template <int ND>
__device__ __forceinline__ Dual<ND> pos_rcp(const Dual<ND>& x) {
  return 1.0 / x;
}

// Universal Kepler equation t(s) = r0 G1(s) + eta G2(s) + mu G3(s) = h with
// G_k = s^k c_k(beta s^2). Newton's method from the second-order start (or,
// for an unbound orbit deep in the exponential regime, the asymptotic
// inverse), Laguerre-Conway (n = 5) if Newton has not converged after 10
// updates. An update below 1e-10 |s| is followed by one last update (for the
// dual type that last update also carries the implicit derivative of s).
// Returns 0 or NB_E_NOCONV; on return G[0..3] hold the G_k at the final s.
template <typename T>
static __device__ int kepler_solve(double mu, const T& r0, const T& ir0, const T& eta,
                                   const T& beta, double h, int max_iter, T G[4], int* iters) {
  T s0 = h * ir0 - eta * (0.5 * h * h) * (ir0 * ir0 * ir0);
  if (val(beta) < 0.0) {
    const T g = sqrt(-beta);
    if (val(g) * ::fabs(val(s0)) > 2.0) {
      const double sg = h > 0.0 ? 1.0 : -1.0;
      const T c = r0 + sg * eta / g + mu / (g * g);
      const T arg = 2.0 * ::fabs(h) * g / c;
      if (val(c) > 0.0 && val(arg) > 1.0) {
        const T sa = sg * log(arg) / g;
        if (::fabs(val(sa)) < ::fabs(val(s0))) s0 = sa;
      }
    }
  }
  int it = 0;
  for (int method = 0; method < 2; ++method) {
    T s = s0;
    bool last = false;
    const int cap = method == 0 ? 10 : max_iter;
    for (int k = 0; k < cap && it < max_iter; ++k, ++it) {
      T c0, c1, c2, c3;
      stumpff(beta * s * s, c0, c1, c2, c3);
      const T G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
      const T F = r0 * G1 + eta * G2 + mu * G3 - h;
      const T Fp = r0 * c0 + eta * G1 + mu * G2;
      T ds;
      if (method == 0) {
        ds = F * pos_rcp(Fp);  // Fp = r(s) > 0
      } else {
        const T Fpp = eta * c0 + (mu - beta * r0) * G1;
        const T disc = fabs(16.0 * Fp * Fp - 20.0 * F * Fpp);
        ds = 5.0 * F / (Fp + copysign(sqrt(disc), Fp));
      }
      s = s - ds;
      if (!isfinite(val(s))) break;
      if (last) {
        T d0, d1, d2, d3;
        stumpff(beta * s * s, d0, d1, d2, d3);
        G[0] = d0;
        G[1] = s * d1;
        G[2] = s * s * d2;
        G[3] = s * s * s * d3;
        *iters = it + 1;
        return 0;
      }
      if (::fabs(val(ds)) <= 1e-10 * ::fabs(val(s))) last = true;
    }
    if (it >= max_iter) break;
  }
  *iters = it;
  return NB_E_NOCONV;
}

// Gauss f and g drift of one body by h; returns 0 or NB_E_NOCONV.
template <typename T>
__device__ __forceinline__ int kepler_drift(double mu, T& x, T& y, T& z, T& vx, T& vy, T& vz,
                                            double h, int max_iter, int* iters) {
  *iters = 0;
  if (h == 0.0) return 0;
  T r0, ir0;
  radius_and_inverse(x, y, z, r0, ir0);
  const T v2 = vx * vx + vy * vy + vz * vz;
  const T eta = x * vx + y * vy + z * vz;
  const T beta = (2.0 * mu) * ir0 - v2;
  T G[4];
  const int st = kepler_solve(mu, r0, ir0, eta, beta, h, max_iter, G, iters);
  if (st) return st;
  const T r = r0 * G[0] + eta * G[1] + mu * G[2];
  const T ir = pos_rcp(r);
  const T fm1 = -mu * G[2] * ir0;        // f - 1
  const T g = r0 * G[1] + eta * G[2];    // g
  const T fd = -mu * G[1] * (ir * ir0);  // fdot
  const T gdm1 = -mu * G[2] * ir;        // gdot - 1
  const T nx = x + (fm1 * x + g * vx), ny = y + (fm1 * y + g * vy), nz = z + (fm1 * z + g * vz);
  const T nvx = vx + (fd * x + gdm1 * vx), nvy = vy + (fd * y + gdm1 * vy),
          nvz = vz + (fd * z + gdm1 * vz);
  x = nx; y = ny; z = nz;
  vx = nvx; vy = nvy; vz = nvz;
  return 0;
}

}  // namespace nb
