// Universal-variable Kepler drift (the first sum of Eq. Ha: Kepler motion
// about mu = G m0, "solved analytically"), shared by the single-system drift
// kernel and the batched kernel.
#pragma once

#include "nb_internal.cuh"

namespace nb {

// ---------------------------------------------------------------------------
// Stumpff functions c0..c3 (Danby's method): quarter z until |z| <= 0.1,
// sum the c2, c3 series there, rebuild c0 = 1 - z c2 and c1 = 1 - z c3, then
// undo each quartering with the argument-quadrupling identities
//   c0(4z) = 2 c0^2 - 1,  c1(4z) = c0 c1,  c2(4z) = c1^2 / 2,
//   c3(4z) = (c2 + c0 c3) / 4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stumpff(double z, double& c0, double& c1, double& c2,
                                        double& c3) {
  int nq = 0;
  while (fabs(z) > 0.1 && nq < 64) {
    z *= 0.25;
    ++nq;
  }
  // c2 = sum_k (-z)^k / (2k+2)!,  c3 = sum_k (-z)^k / (2k+3)!,  k = 0..7
  c2 = 1.0 / 2.0 -
       z * (1.0 / 24.0 -
            z * (1.0 / 720.0 -
                 z * (1.0 / 40320.0 -
                      z * (1.0 / 3628800.0 -
                           z * (1.0 / 479001600.0 -
                                z * (1.0 / 87178291200.0 - z * (1.0 / 20922789888000.0)))))));
  c3 = 1.0 / 6.0 -
       z * (1.0 / 120.0 -
            z * (1.0 / 5040.0 -
                 z * (1.0 / 362880.0 -
                      z * (1.0 / 39916800.0 -
                           z * (1.0 / 6227020800.0 -
                                z * (1.0 / 1307674368000.0 - z * (1.0 / 355687428096000.0)))))));
  c1 = 1.0 - z * c3;
  c0 = 1.0 - z * c2;
  for (; nq > 0; --nq) {
    c3 = (c2 + c0 * c3) * 0.25;
    c2 = c1 * c1 * 0.5;
    c1 = c0 * c1;
    c0 = 2.0 * c0 * c0 - 1.0;
  }
}

// Universal Kepler equation t(s) = r0 G1(s) + eta G2(s) + mu G3(s) = h with
// G_k = s^k c_k(beta s^2). Newton's method from the second-order start (or,
// for an unbound orbit deep in the exponential regime, the asymptotic
// inverse), Laguerre-Conway (n = 5) if Newton has not converged after 10
// updates. An update below 1e-10 |s| is followed by one last update.
// Returns 0 or NB_E_NOCONV; on return G[0..3] hold the G_k at the final s.
static __device__ int kepler_solve(double mu, double r0, double eta, double beta, double h,
                            int max_iter, double G[4], int* iters) {
  double s0 = h / r0 - eta * h * h / (2.0 * r0 * r0 * r0);
  if (beta < 0.0) {
    const double g = sqrt(-beta);
    if (g * fabs(s0) > 2.0) {
      const double sg = h > 0.0 ? 1.0 : -1.0;
      const double c = r0 + sg * eta / g + mu / (g * g);
      const double arg = 2.0 * g * fabs(h) / c;
      if (c > 0.0 && arg > 1.0) {
        const double sa = sg * log(arg) / g;
        if (fabs(sa) < fabs(s0)) s0 = sa;
      }
    }
  }
  int it = 0;
  for (int method = 0; method < 2; ++method) {
    double s = s0;
    bool last = false;
    const int cap = method == 0 ? 10 : max_iter;
    for (int k = 0; k < cap && it < max_iter; ++k, ++it) {
      double c0, c1, c2, c3;
      stumpff(beta * s * s, c0, c1, c2, c3);
      const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
      const double F = r0 * G1 + eta * G2 + mu * G3 - h;
      const double Fp = r0 * c0 + eta * G1 + mu * G2;
      double ds;
      if (method == 0) {
        ds = F / Fp;
      } else {
        const double Fpp = eta * c0 + (mu - beta * r0) * G1;
        const double disc = fabs(16.0 * Fp * Fp - 20.0 * F * Fpp);
        ds = 5.0 * F / (Fp + copysign(sqrt(disc), Fp));
      }
      s -= ds;
      if (!isfinite(s)) break;
      if (last) {
        double d0, d1, d2, d3;
        stumpff(beta * s * s, d0, d1, d2, d3);
        G[0] = d0;
        G[1] = s * d1;
        G[2] = s * s * d2;
        G[3] = s * s * s * d3;
        *iters = it + 1;
        return 0;
      }
      if (fabs(ds) <= 1e-10 * fabs(s)) last = true;
    }
    if (it >= max_iter) break;
  }
  *iters = it;
  return NB_E_NOCONV;
}

// Gauss f and g drift of one body by h; returns 0 or NB_E_NOCONV.
__device__ __forceinline__ int kepler_drift(double mu, double& x, double& y, double& z,
                                            double& vx, double& vy, double& vz, double h,
                                            int max_iter, int* iters) {
  *iters = 0;
  if (h == 0.0) return 0;
  const double r0 = sqrt(x * x + y * y + z * z);
  const double v2 = vx * vx + vy * vy + vz * vz;
  const double eta = x * vx + y * vy + z * vz;
  const double beta = 2.0 * mu / r0 - v2;
  double G[4];
  const int st = kepler_solve(mu, r0, eta, beta, h, max_iter, G, iters);
  if (st) return st;
  const double r = r0 * G[0] + eta * G[1] + mu * G[2];
  const double fm1 = -mu * G[2] / r0;           // f - 1
  const double g = r0 * G[1] + eta * G[2];      // g
  const double fd = -mu * G[1] / (r * r0);      // fdot
  const double gdm1 = -mu * G[2] / r;           // gdot - 1
  const double nx = x + (fm1 * x + g * vx), ny = y + (fm1 * y + g * vy), nz = z + (fm1 * z + g * vz);
  const double nvx = vx + (fd * x + gdm1 * vx), nvy = vy + (fd * y + gdm1 * vy),
               nvz = vz + (fd * z + gdm1 * vz);
  x = nx; y = ny; z = nz;
  vx = nvx; vy = nvy; vz = nvz;
  return 0;
}

}  // namespace nb
