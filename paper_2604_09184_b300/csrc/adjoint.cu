// Discrete adjoint of the hybrid symplectic step: gradients of a loss on the
// final state with respect to the initial positions, velocities and masses.
//
// The step is B(h/2) C(h/2) A(h) C(h/2) B(h/2) (Eqs. H, Ha, Hb, Hc); its
// adjoint runs the same maps in reverse with their transposed Jacobians:
//   B (kick, Eq. Hb):   lambda_x += J_a^T mu with mu = (h/2) lambda_v, where
//                        J_a is the tidal tensor of the changeover-weighted
//                        pair force, and lambda_m += (da/dm)^T mu;
//   C (Eq. Hc):          lambda_v_i += (h/2) (m_i/m0) sum_k lambda_x_k and
//                        lambda_m_i += (h/2) v_i . sum_k lambda_x_k / m0;
//   A (Kepler, Eq. Ha):  per body, the transposed 6x6 Jacobian of the f/g map
//                        (forward-mode dual numbers through the universal-
//                        variable solve); bodies of a close-encounter group
//                        take the adjoint of the recorded Bulirsch-Stoer
//                        substeps: Neville extrapolation is linear in the
//                        modified-midpoint results, each midpoint sequence is
//                        reversed with the Jacobian of the group's equations
//                        of motion, mergers with the Jacobian of the merge map.
// All discrete events (flags, groups, BS substep sizes and columns, mergers)
// and the critical radii are held at their forward values. The forward pass
// keeps a checkpoint every `every` steps; the backward pass replays each
// segment from its checkpoint (the forward is deterministic, so the replay
// reproduces every decision) while recording the per-step states it needs.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bs.cuh"
#include "kepler.cuh"
#include "nb_internal.cuh"

namespace nb {

constexpr int ANT = 256;     // threads of the O(N) adjoint kernels
constexpr int VNT = 128;     // threads of the kick VJP (targets per CTA)
constexpr int ABNT = 64;     // threads of the BS adjoint CTA
constexpr int kSubCap = 256; // recorded BS substeps per group and step
constexpr int kMrgCap = 16;  // recorded mergers per group and step

// K, dK/dy, d2K/dy2 of the infinitely smooth switch K = f(y) / (f(y) + f(1-y)),
// f(y) = exp(-1/y), with one exponential and one reciprocal: u = 1 - y,
// w = 1 / (y u), E = exp(1/y - 1/u) = exp((u - y) w), K = 1/(1+E),
// A = 1/y^2 + 1/u^2 = (y^2 + u^2) w^2, A' = 2/u^3 - 2/y^3 = 2 (y^3 - u^3) w^3,
// K' = E K^2 A, K'' = E K^2 (2 K E A^2 + A' - A^2). Where |1/y - 1/u| > 80
// K is within 2e-35 of 0 or 1 and its derivatives vanish to double precision.
// The range tests compare bit patterns.
__device__ void changeover_y(double y, double& K, double& K1, double& K2) {
  K1 = 0.0;
  K2 = 0.0;
  const long long by = __double_as_longlong(y);
  if (by <= 0ll) {  // y <= 0 (either zero)
    K = 0.0;
    return;
  }
  if (by >= __double_as_longlong(1.0)) {
    K = 1.0;
    return;
  }
  const double u = 1.0 - y;
  const double yu = y * u;
  const double iw = rcp_fast(yu);
  const double dd = (u - y) * iw;
  const long long bd = __double_as_longlong(dd);
  if ((bd & 0x7fffffffffffffffll) > __double_as_longlong(80.0)) {
    K = bd > 0 ? 0.0 : 1.0;
    return;
  }
  const double E = exp_fast(dd);
  K = rcp_fast(1.0 + E);
  const double s2 = __fma_rn(y, y, u * u);
  const double iw2 = iw * iw;
  const double A = s2 * iw2;
  const double A1 = 2.0 * ((y - u) * (s2 + yu)) * (iw2 * iw);
  const double EK2 = E * K * K;
  K1 = EK2 * A;
  K2 = EK2 * (2.0 * K * E * A * A + A1 - A * A);
}

// Radial profile of a pair term and its derivative divided by r:
// kick (close = 0): phi = w / r^3, w = K - r K_r (w = 1 beyond rc);
// close force (close = 1): psi = (1 - w) / r^3 (0 beyond rc).
__device__ void pair_profile(double r2, double rc, int close, double& p, double& dp_r) {
  const double ir = rinv_fast(r2);
  const double r = r2 * ir;
  const double ir3 = ir * ir * ir;
  double w = 1.0, wp = 0.0;
  if (r2 < rc * rc) {
    const double L = 0.9 * rc;
    const double iL = rcp_fast(L);
    double K, K1, K2;
    changeover_y((r - 0.1 * rc) * iL, K, K1, K2);
    const double Kr = K1 * iL, Krr = K2 * iL * iL;
    w = K - r * Kr;
    wp = -r * Krr;
  }
  if (close) {
    p = (1.0 - w) * ir3;
    dp_r = (-wp - 3.0 * (1.0 - w) * ir) * ir3 * ir;
  } else {
    p = w * ir3;
    dp_r = (wp - 3.0 * w * ir) * ir3 * ir;
  }
}

struct Vjp {
  const double *x, *y, *z, *m, *rc;
  const int* alive;
  const double *mux, *muy, *muz;  // (h/2) lambda_v
  double* part;                   // S x 4 x n partial sums (x, y, z, m)
  int n, chunk;
};

// Partial sums over the j-chunk blockIdx.y of
//   lambda_x_k += G sum_j T_kj (m_k mu_j - m_j mu_k), T = phi I + (phi'/r) d d^T,
//   lambda_m_k += G sum_j phi mu_j . (x_k - x_j),
// phi = w / r^3. Beyond rc (w = 1, the common case) phi = r^-3 and
// phi'/r = -3 r^-5, with 1/r from the seeded reciprocal root.
__global__ void __launch_bounds__(VNT) k_kick_vjp(Vjp V) {
  __shared__ double sx[VNT], sy[VNT], sz[VNT], sm[VNT], src2[VNT], su[VNT], sv[VNT], sw[VNT];
  __shared__ double srcv[VNT];
  const int k = blockIdx.x * VNT + threadIdx.x;
  const bool act = k < V.n && V.alive[k];
  const double xk = act ? V.x[k] : 0.0, yk = act ? V.y[k] : 0.0, zk = act ? V.z[k] : 0.0;
  const double mk = act ? V.m[k] : 0.0, rck = act ? V.rc[k] : 0.0;
  const double rck2 = rck * rck;
  const double mxk = act ? V.mux[k] : 0.0, myk = act ? V.muy[k] : 0.0, mzk = act ? V.muz[k] : 0.0;
  double ax = 0.0, ay = 0.0, az = 0.0, am = 0.0;
  const int j0 = blockIdx.y * V.chunk;
  const int j1 = min(V.n, j0 + V.chunk);
  for (int jt = j0; jt < j1; jt += VNT) {
    __syncthreads();
    const int j = jt + threadIdx.x;
    if (j < j1) {
      const bool aj = V.alive[j] != 0;
      sx[threadIdx.x] = V.x[j]; sy[threadIdx.x] = V.y[j]; sz[threadIdx.x] = V.z[j];
      // absorbed bodies: zero mass and cotangent, so every term vanishes
      sm[threadIdx.x] = aj ? V.m[j] : 0.0;
      srcv[threadIdx.x] = V.rc[j];
      src2[threadIdx.x] = V.rc[j] * V.rc[j];
      su[threadIdx.x] = aj ? V.mux[j] : 0.0;
      sv[threadIdx.x] = aj ? V.muy[j] : 0.0;
      sw[threadIdx.x] = aj ? V.muz[j] : 0.0;
    }
    __syncthreads();
    if (!act) continue;
    const int cnt = min(VNT, j1 - jt);
    for (int q = 0; q < cnt; ++q) {
      const double dx = sx[q] - xk, dy = sy[q] - yk, dz = sz[q] - zk;
      // r^2 on the integer pipe; a pair within one high-word unit of its
      // threshold, or coincident, is decided on the FP64 expression (as the
      // forward kick decides it)
      double r2 = sep2_int(dx, dy, dz);
      bool inside = false;
      if (__double2hiint(r2) <= max(__double2hiint(rck2), __double2hiint(src2[q])) + 1) {
        r2 = sep2(dx, dy, dz);
        if (__double_as_longlong(r2) == 0ll) continue;  // the target itself (and coincident bodies)
        inside = nn_less(r2, rck2) || nn_less(r2, src2[q]);
      }
      double p, dp_r;
      if (!inside) {
        const double ri = rinv_fast(r2);
        const double ir2 = ri * ri;
        p = ri * ir2;
        dp_r = -3.0 * p * ir2;
      } else {
        pair_profile(r2, fmax(rck, srcv[q]), 0, p, dp_r);
      }
      const double ux = __fma_rn(mk, su[q], -sm[q] * mxk);
      const double uy = __fma_rn(mk, sv[q], -sm[q] * myk);
      const double uz = __fma_rn(mk, sw[q], -sm[q] * mzk);
      const double t = dp_r * (dx * ux + dy * uy + dz * uz);
      ax = __fma_rn(t, dx, __fma_rn(p, ux, ax));
      ay = __fma_rn(t, dy, __fma_rn(p, uy, ay));
      az = __fma_rn(t, dz, __fma_rn(p, uz, az));
      am = __fma_rn(-p, su[q] * dx + sv[q] * dy + sw[q] * dz, am);
    }
  }
  if (k < V.n) {
    double* o = V.part + (size_t)blockIdx.y * 4 * V.n;
    o[k] = ax;
    o[V.n + k] = ay;
    o[2 * V.n + k] = az;
    o[3 * V.n + k] = am;
  }
}

// lambda += G sum_s part[s] in a fixed order (deterministic).
__global__ void __launch_bounds__(ANT) k_kick_vjp_sum(int n, int S, const double* part, double G,
                                                     const int* alive, double* lx, double* ly,
                                                     double* lz, double* lm) {
  const int k = blockIdx.x * ANT + threadIdx.x;
  if (k >= n || !alive[k]) return;
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int q = 0; q < S; ++q) {
    const double* o = part + (size_t)q * 4 * n;
    a += o[k];
    b += o[n + k];
    c += o[2 * n + k];
    d += o[3 * n + k];
  }
  lx[k] += G * a;
  ly[k] += G * b;
  lz[k] += G * c;
  lm[k] += G * d;
}

// Per-block sums of lambda_x over the bodies with alive != 0 (fixed order).
__global__ void __launch_bounds__(ANT) k_sum3(int n, const int* alive, const double* a,
                                             const double* b, const double* c, double* parts) {
  __shared__ double red[3 * 32 + 3];
  const int i = blockIdx.x * ANT + threadIdx.x;
  double x = 0.0, y = 0.0, z = 0.0;
  if (i < n && alive[i]) {
    x = a[i]; y = b[i]; z = c[i];
  }
  block_sum3(x, y, z, red);
  if (threadIdx.x == 0) {
    parts[3 * blockIdx.x] = x;
    parts[3 * blockIdx.x + 1] = y;
    parts[3 * blockIdx.x + 2] = z;
  }
}

// Adjoint of C(h/2): x' = x + (h/2) P / m0 with P = sum m v.
__global__ void __launch_bounds__(ANT) k_cdrift_vjp(int n, int nparts, const double* parts,
                                                   const int* alive, const double* m,
                                                   const double* vx, const double* vy,
                                                   const double* vz, double hh, double m0,
                                                   double* lvx, double* lvy, double* lvz,
                                                   double* lm) {
  __shared__ double red[3 * 32 + 3];
  double S[3];
  reduce_parts3(parts, nparts, red, S);
  const int i = blockIdx.x * ANT + threadIdx.x;
  if (i >= n || !alive[i]) return;
  const double c = hh * m[i] / m0;
  lvx[i] += c * S[0];
  lvy[i] += c * S[1];
  lvz[i] += c * S[2];
  lm[i] += hh * (vx[i] * S[0] + vy[i] * S[1] + vz[i] * S[2]) / m0;
}

// Transposed Jacobian of the Kepler drift for bodies outside the step's
// groups. Six threads per body: thread c carries the derivative along input
// c (one column of the 6x6 Jacobian, forward mode, one partial), so that
// lambda_in[c] = sum_o lambda_out[o] dout_o / din_c is its own dot product;
// the six take the same iteration path (it depends on the values only). Five
// bodies per warp: each thread's FP64 work is about twice the drift's instead
// of seven times with all six partials in one thread.
constexpr int kKvBodies = 5;
__global__ void __launch_bounds__(ANT) k_kepler_vjp(int n, const double* xs6, const int* alive,
                                                   const int* ingrp, double mu, double h,
                                                   int max_iter, double* lx, double* ly,
                                                   double* lz, double* lvx, double* lvy,
                                                   double* lvz, int* status) {
  const int lane = threadIdx.x & 31;
  const int slot = lane / 6, c = lane - 6 * slot;
  const int i = ((blockIdx.x * ANT + threadIdx.x) >> 5) * kKvBodies + slot;
  const bool act = slot < kKvBodies && i < n && alive[i] && !ingrp[i];
  bool ok = false;
  double li = 0.0;
  if (act) {
    Dual<1> q[6];
    for (int a = 0; a < 6; ++a) {
      q[a] = mkd<1>(xs6[(size_t)a * n + i]);
      q[a].d[0] = a == c ? 1.0 : 0.0;
    }
    int it;
    ok = kepler_drift(mu, q[0], q[1], q[2], q[3], q[4], q[5], h, max_iter, &it) == 0;
    if (ok) {
      const double lo[6] = {lx[i], ly[i], lz[i], lvx[i], lvy[i], lvz[i]};
      for (int a = 0; a < 6; ++a) li += lo[a] * q[a].d[0];
    } else if (c == 0) {
      atomicCAS(status, 0, NB_E_NOCONV);
    }
  }
  __syncwarp();  // the body's six threads have read lambda before any of them writes
  if (act && ok) {
    double* o = c == 0 ? lx : c == 1 ? ly : c == 2 ? lz : c == 3 ? lvx : c == 4 ? lvy : lvz;
    o[i] = li;
  }
}

// ---------------------------------------------------------------------------
// Bulirsch-Stoer adjoint: one CTA per group.
// ---------------------------------------------------------------------------
// Midpoint states of one substep: column j keeps z_0..z_2j at state index
// j^2 - 1 + t, kmax^2 + 2 kmax states in all.
__host__ __device__ constexpr int adj_nstates(int kmax) { return kmax * kmax + 2 * kmax; }
__host__ __device__ constexpr int adj_sidx(int j, int t) { return j * j - 1 + t; }

// Per-member record of a step's direct-solver replay (doubles): the starts
// of the accepted substeps (kSubCap x (6 + 4)).
__host__ __device__ constexpr int adj_rec_stride() { return kSubCap * 10; }
// Per-member scratch of the reverse (doubles): the midpoint states of one
// substep and their adjoints, a derivative buffer per column, f0 and its
// adjoint, the running adjoint (6 state + 1 mass), an accumulator (6) and a
// mass accumulator per column.
__host__ __device__ inline int adj_work_stride(int kmax) {
  return 12 * adj_nstates(kmax) + 7 * kmax + 25;
}

// Weights of the extrapolated value: T_kk = sum_j c_kj T_j1, the Neville
// recursion being linear in the column results. [k][j] for 1 <= j <= k <=
// kMaxBsK, the recursion applied to unit vectors, evaluated by the compiler.
struct ExtrapTab {
  double c[kMaxBsK + 1][kMaxBsK + 1];
};
__host__ __device__ constexpr ExtrapTab extrap_tab() {
  ExtrapTab t{};
  for (int k = 1; k <= kMaxBsK; ++k)
    for (int j0 = 1; j0 <= k; ++j0) {
      double Tn[kMaxBsK + 1][kMaxBsK + 1] = {};
      for (int j = 1; j <= k; ++j) {
        Tn[j][1] = (j == j0) ? 1.0 : 0.0;
        for (int q = 1; q < j; ++q) {
          const double inv = (double)((j - q) * (j - q)) / (double)(q * (2 * j - q));
          Tn[j][q + 1] = Tn[j][q] + (Tn[j][q] - Tn[j - 1][q]) * inv;
        }
      }
      t.c[k][j0] = Tn[k][k];
    }
  return t;
}
static __constant__ ExtrapTab kExtrap = extrap_tab();
// the Lagrange weights at h = 0 of n = 2, 4, 6 in h^2: 1/24, -16/15, 81/40
static_assert(extrap_tab().c[3][1] - 1.0 / 24.0 < 1e-15 && 1.0 / 24.0 - extrap_tab().c[3][1] < 1e-15 &&
                  extrap_tab().c[3][2] + 16.0 / 15.0 < 1e-15 && -16.0 / 15.0 - extrap_tab().c[3][2] < 1e-15 &&
                  extrap_tab().c[3][3] - 81.0 / 40.0 < 1e-15 && 81.0 / 40.0 - extrap_tab().c[3][3] < 1e-15,
              "extrapolation weights");

// H / h for a substep H = h 2^-level (both normal): the power of two from
// the exponent fields.
__device__ __forceinline__ double pow2_ratio(double H, double h) {
  const long long eH = (__double_as_longlong(H) >> 52) & 0x7ff;
  const long long eh = (__double_as_longlong(h) >> 52) & 0x7ff;
  return __longlong_as_double((1023ll + eH - eh) << 52);
}

struct AdjGroupArgs {
  int n, kmax, bs_stride, work_stride;
  const int* grp;  // [0] ngroups [1] nmembers [2..] off[ng+1] then members
  const double* xs6;
  const double *m0, *R0, *rc0;
  double* lx[3];
  double* lv[3];
  double* lm;
  double* gscr;    // the record pass's scratch for groups of more than 8 bodies
  // the step's record buffer: written by the record pass, read by the reverse
  double* rslot;   // n * adj_rec_stride()
  double* gend;    // n * 10: the record pass's working copies, left at the end state
  double* H;       // n * kSubCap
  int* kk;         // n * kSubCap
  int* counts;     // n * 4: substeps, mergers, overflow, the record's status
  int* mrg;        // n * kMrgCap * 3
  double* mst;     // n * kMrgCap * 14
  // the reverse's own scratch
  double* work;    // n * work_stride
  double* gwork;   // n * 10
  int* status;
};

// Right-hand side of the group's equations of motion (Eq. Ha restricted to
// the group) for member b: f_b = (v_b, -mu x_b / r_b^3 + G sum_q m_q psi d_bq),
// psi = (1 - w) / r^3 inside rc. z: states of all M members (6 each). Uses
// the members' masses, critical radii and alive flags in the working copies.
__device__ void grp_f(const BsCtx& c, const double* z, int b, double* fb) {
  if (!bs_alive(c, b)) {
    for (int k = 0; k < 6; ++k) fb[k] = 0.0;
    return;
  }
  const double* zb = z + 6 * b;
  fb[0] = zb[3]; fb[1] = zb[4]; fb[2] = zb[5];
  const double r2 = zb[0] * zb[0] + zb[1] * zb[1] + zb[2] * zb[2];
  const double ir = rinv_fast(r2);
  const double ks = -c.mu * (ir * ir * ir);
  double ax = ks * zb[0], ay = ks * zb[1], az = ks * zb[2];
  for (int q = 0; q < c.M; ++q) {
    if (q == b || !bs_alive(c, q)) continue;
    const double* zq = z + 6 * q;
    const double dx = zq[0] - zb[0], dy = zq[1] - zb[1], dz = zq[2] - zb[2];
    const double q2 = sep2(dx, dy, dz);
    const double rc = fmax(c.g[10 * b + 8], c.g[10 * q + 8]);
    if (q2 == 0.0 || !(q2 < rc * rc)) continue;
    double p, dp_r;
    pair_profile(q2, rc, 1, p, dp_r);
    const double f = c.G * c.g[10 * q + 6] * p;
    ax += f * dx; ay += f * dy; az += f * dz;
  }
  fb[3] = ax; fb[4] = ay; fb[5] = az;
}

// out_b += scale (J^T w)_b and lm_b += scale (dF/dm_b)^T w for member b, J the
// Jacobian of grp_f at the states z, w = (w_x, w_v) per member:
//   (J^T w)_x,b = -mu (I / r^3 - 3 x x^T / r^5) w_v,b
//                 + G sum_q T_bq (m_b w_v,q - m_q w_v,b),  T = psi I + (psi'/r) d d^T,
//   (J^T w)_v,b = w_x,b,   dF/dm_b . w = G sum_q psi w_v,q . (x_b - x_q).
__device__ void grp_vjp(const BsCtx& c, const double* z, const double* w, int b, double* ob,
                        double* lmb, double scale) {
  if (!bs_alive(c, b)) return;
  const double* zb = z + 6 * b;
  const double* wb = w + 6 * b;
  double o[3];
  const double r2 = zb[0] * zb[0] + zb[1] * zb[1] + zb[2] * zb[2];
  const double ir = rinv_fast(r2);
  const double ir3 = ir * ir * ir;
  const double ir5 = ir3 * ir * ir;
  const double xw = zb[0] * wb[3] + zb[1] * wb[4] + zb[2] * wb[5];
  for (int k = 0; k < 3; ++k) o[k] = -c.mu * (wb[3 + k] * ir3 - 3.0 * zb[k] * xw * ir5);
  double am = 0.0;
  const double mb = c.g[10 * b + 6], rcb = c.g[10 * b + 8];
  for (int q = 0; q < c.M; ++q) {
    if (q == b || !bs_alive(c, q)) continue;
    const double* zq = z + 6 * q;
    const double* wq = w + 6 * q;
    const double dx = zq[0] - zb[0], dy = zq[1] - zb[1], dz = zq[2] - zb[2];
    const double q2 = sep2(dx, dy, dz);
    const double rc = fmax(rcb, c.g[10 * q + 8]);
    if (q2 == 0.0 || !(q2 < rc * rc)) continue;
    double p, dp_r;
    pair_profile(q2, rc, 1, p, dp_r);
    const double mq = c.g[10 * q + 6];
    const double ux = mb * wq[3] - mq * wb[3], uy = mb * wq[4] - mq * wb[4],
                 uz = mb * wq[5] - mq * wb[5];
    const double du = dx * ux + dy * uy + dz * uz;
    o[0] += c.G * (p * ux + dp_r * du * dx);
    o[1] += c.G * (p * uy + dp_r * du * dy);
    o[2] += c.G * (p * uz + dp_r * du * dz);
    am -= c.G * p * (wq[3] * dx + wq[4] * dy + wq[5] * dz);
  }
  for (int k = 0; k < 3; ++k) {
    ob[k] += scale * o[k];
    ob[3 + k] += scale * wb[k];
  }
  *lmb += scale * am;
}

// One CTA per group: replay the group's integration from the saved state,
// recording every accepted substep (bs_integrate_group with a BsRec), then
// pull the adjoint back through the substeps, last first. Per substep: undo
// the mergers that followed it (merge map x' = (m_a x_a + m_b x_b) / M,
// M = m_a + m_b), replay the midpoint sequences of columns 1..k (k the
// accepted column) keeping every state, and reverse them as a wave over the
// columns; the Neville extrapolation is linear in the column results, with
// weights c_j from the same recursion applied to unit vectors.
// The adjoint of one group's integration by a team (one warp or one CTA):
// cw is the team's shared scratch for the extrapolation weights.
// scr: the team's direct-solver scratch (M slots of bs_stride doubles;
// nslots >= 2 M lets the replay speculate on half-size attempts).
// The record pass of one group's adjoint by a team (one warp or one CTA):
// replay the group's integration from the step's saved state with the
// direct solver, recording every accepted substep's start, size and column
// and every merger into the step's record buffer (counts[3] = the status).
// scr: the team's direct-solver scratch (M slots of bs_stride doubles;
// nslots >= 2 M lets the replay speculate on half-size attempts).
template <class Team>
__device__ void bs_record_group(const AdjGroupArgs& A, const Phys& P, double h, int grp,
                                Team& team, double* scr, int nslots) {
  const int ng = A.grp[0];
  const int* goff = A.grp + 2;
  const int* gmem = A.grp + 2 + ng + 1;
  const int n = A.n;
  const int tid = team.tid(), NT = team.nthreads();
  const int off = goff[grp];
  BsCtx c;
  c.M = goff[grp + 1] - off;
  c.stride = A.bs_stride;
  c.base = scr;
  c.g = A.gend + (size_t)off * 10;
  c.kmax = A.kmax;
  c.G = P.G;
  c.mu = P.mu;
  c.mu15 = 1.5 * P.mu;
  c.mu1875 = 1.875 * P.mu;
  const int M = c.M;
  // the group's contiguous record block, arrays of M members each
  double* r_ys = A.rslot + (size_t)off * adj_rec_stride();
  BsRec rec;
  rec.cap = kSubCap;
  rec.mcap = kMrgCap;
  rec.counts = A.counts + 4 * (size_t)grp;
  rec.H = A.H + (size_t)grp * kSubCap;
  rec.k = A.kk + (size_t)grp * kSubCap;
  rec.ys = r_ys;
  rec.ms = r_ys + (size_t)kSubCap * M * 6;
  rec.Rs = rec.ms + (size_t)kSubCap * M;
  rec.rcs = rec.Rs + (size_t)kSubCap * M;
  rec.alv = rec.rcs + (size_t)kSubCap * M;
  rec.mrg = A.mrg + (size_t)grp * kMrgCap * 3;
  rec.mst = A.mst + (size_t)grp * kMrgCap * 14;
  for (int b = tid; b < M; b += NT) {
    const int body = gmem[off + b];
    double* y = c.base + (size_t)b * c.stride + OY;
    for (int k = 0; k < 6; ++k) y[k] = A.xs6[(size_t)k * n + body];
    double* g = c.g + 10 * b;
    g[6] = A.m0[body]; g[7] = A.R0[body]; g[8] = A.rc0[body]; g[9] = 1.0;
    bs_set_aux(c, b, P.G, g[6], g[8]);
  }
  if (tid == 0) {
    rec.counts[0] = 0; rec.counts[1] = 0; rec.counts[2] = 0; rec.counts[3] = 0;
  }
  team.sync();
  BsTally tally{0, 0, 0, 0};
  double El = 0.0;
  int st = bs_integrate(c, P, h, team, tally, &El, &rec,
                        P.bs_speculate && 2 * M <= nslots ? scr + (size_t)M * c.stride : nullptr);
  team.sync();
  if (!st && rec.counts[2]) st = NB_E_OVERFLOW;
  if (st && tid == 0) {
    rec.counts[3] = st;
    atomicCAS(A.status, 0, st);
  }
  team.sync();
}

// The reverse of one group's integration by a team, from the record pass's
// buffer: pull the adjoint back through the recorded substeps, last first.
// Per substep: undo the mergers that followed it (merge map x' = (m_a x_a +
// m_b x_b) / M, M = m_a + m_b), replay the midpoint sequences of columns
// 1..k (k the accepted column) keeping every state, and reverse them as a
// wave over the columns; the Neville extrapolation is linear in the column
// results, with weights c_j from the same recursion applied to unit vectors.
// cw is the team's shared scratch for the extrapolation weights. A group
// whose record pass failed is left alone (its status fails the pass).
template <class Team>
__device__ void bs_reverse_group(const AdjGroupArgs& A, const Phys& P, double h, int grp,
                                 Team& team, double* cw) {
  const int ng = A.grp[0];
  const int* goff = A.grp + 2;
  const int* gmem = A.grp + 2 + ng + 1;
  const int tid = team.tid(), NT = team.nthreads();
  const int NS = adj_nstates(A.kmax);
  double hj[kMaxBsK + 1];  // h / n_j
  for (int j = 1; j <= A.kmax; ++j) hj[j] = h / (2 * j);
  {
    const int off = goff[grp];
    if (A.counts[4 * (size_t)grp + 3]) return;
    BsCtx c;
    c.M = goff[grp + 1] - off;
    c.stride = A.bs_stride;
    c.base = nullptr;
    c.g = A.gwork + (size_t)off * 10;
    c.kmax = A.kmax;
    c.G = P.G;
    c.mu = P.mu;
    c.mu15 = 1.5 * P.mu;
    c.mu1875 = 1.875 * P.mu;
    const int M = c.M;
    const double* r_ys = A.rslot + (size_t)off * adj_rec_stride();
    const double* r_ms = r_ys + (size_t)kSubCap * M * 6;
    const double* r_Rs = r_ms + (size_t)kSubCap * M;
    const double* r_rcs = r_Rs + (size_t)kSubCap * M;
    const double* r_alv = r_rcs + (size_t)kSubCap * M;
    // the group's contiguous work block, arrays of M members each
    double* zst = A.work + (size_t)off * A.work_stride;  // NS states x 6M
    double* lzst = zst + (size_t)NS * 6 * M;        // NS states x 6M
    double* fcol = lzst + (size_t)NS * 6 * M;       // kmax x 6M
    double* f0 = fcol + (size_t)A.kmax * 6 * M;     // 6M
    double* lf0 = f0 + 6 * M;                       // 6M
    double* ly = lf0 + 6 * M;                       // 6M
    double* lin = ly + 6 * M;                       // 6M
    double* lmv = lin + 6 * M;                      // M
    double* lmc = lmv + M;                          // kmax x M
    BsRec rec;
    rec.counts = A.counts + 4 * (size_t)grp;
    rec.H = A.H + (size_t)grp * kSubCap;
    rec.k = A.kk + (size_t)grp * kSubCap;
    rec.mrg = A.mrg + (size_t)grp * kMrgCap * 3;
    rec.mst = A.mst + (size_t)grp * kMrgCap * 14;
    const int nsub = rec.counts[0], nmrg = rec.counts[1];
    // adjoint at the end of the BS: members alive at the end take the step's
    // lambda; absorbed members start from zero
    for (int b = tid; b < M; b += NT) {
      const int body = gmem[off + b];
      const bool live = A.gend[(size_t)(off + b) * 10 + 9] != 0.0;
      for (int k = 0; k < 3; ++k) {
        ly[6 * b + k] = live ? A.lx[k][body] : 0.0;
        ly[6 * b + 3 + k] = live ? A.lv[k][body] : 0.0;
      }
      lmv[b] = live ? A.lm[body] : 0.0;
    }
    team.sync();
    int mq = nmrg - 1;
    for (int s = nsub - 1; s >= 0; --s) {
      // undo the mergers that followed substep s (last first)
      for (; mq >= 0 && rec.mrg[3 * mq] == s; --mq) {
        if (tid == 0) {
          const int a = rec.mrg[3 * mq + 1], b = rec.mrg[3 * mq + 2];
          const double* ya = rec.mst + 14 * mq;
          const double* yb = ya + 6;
          const double ma = ya[12], mb = ya[13], Mt = ma + mb;
          double lyn[6], dot_a = 0.0, dot_b = 0.0;
          for (int k = 0; k < 6; ++k) {
            lyn[k] = ly[6 * a + k];
            const double yn = (ma * ya[k] + mb * yb[k]) / Mt;
            dot_a += lyn[k] * (ya[k] - yn) / Mt;
            dot_b += lyn[k] * (yb[k] - yn) / Mt;
          }
          const double lM = lmv[a];
          for (int k = 0; k < 6; ++k) {
            ly[6 * a + k] = (ma / Mt) * lyn[k];
            ly[6 * b + k] = (mb / Mt) * lyn[k];
          }
          lmv[a] = lM + dot_a;
          lmv[b] = lM + dot_b;
        }
        team.sync();
      }
      const int kacc = rec.k[s];
      const double H = rec.H[s];
      // working copies at the substep's start; clear the adjoint buffers
      for (int b = tid; b < M; b += NT) {
        const size_t o = (size_t)s * M + b;
        double* g = c.g + 10 * b;
        g[6] = r_ms[o]; g[7] = r_Rs[o]; g[8] = r_rcs[o]; g[9] = r_alv[o];
        for (int k = 0; k < 6; ++k) {
          zst[6 * b + k] = r_ys[6 * o + k];  // state (1, 0) doubles as y
          lf0[6 * b + k] = 0.0;
        }
        for (int j = 1; j <= kacc; ++j) lmc[(j - 1) * M + b] = 0.0;
      }
      for (int e = tid; e < adj_nstates(kacc) * 6 * M; e += NT) lzst[e] = 0.0;
      // extrapolation weights: T_kk = sum_j cw[j] T_j1; the column sizes
      // H / n_j = hj[j] (H / h), the power of two exact
      for (int j = 1 + tid; j <= kacc; j += NT) cw[j] = kExtrap.c[kacc][j];
      const double sc = pow2_ratio(H, h);
      team.sync();
      const double* y = zst;  // M states
      for (int b = tid; b < M; b += NT) grp_f(c, y, b, f0 + 6 * b);
      team.sync();
      // replay: z_0 = y, z_1 = y + hs f0, z_{t+1} = z_{t-1} + 2 hs f(z_t)
      for (int it = tid; it < kacc * M; it += NT) {
        const int j = 1 + it / M, b = it % M;
        const double hs = hj[j] * sc;
        double* z0 = zst + (size_t)adj_sidx(j, 0) * 6 * M + 6 * b;
        double* z1 = zst + (size_t)adj_sidx(j, 1) * 6 * M + 6 * b;
        for (int k = 0; k < 6; ++k) {
          if (j > 1) z0[k] = y[6 * b + k];  // column 1's z_0 is y itself
          z1[k] = y[6 * b + k] + hs * f0[6 * b + k];
        }
      }
      team.sync();
      for (int t = 1; t < 2 * kacc; ++t) {
        const int j0 = t / 2 + 1;  // columns with t < 2j
        const int ncol = kacc - j0 + 1;
        for (int it = tid; it < ncol * M; it += NT) {
          const int j = j0 + it / M, b = it % M;
          grp_f(c, zst + (size_t)adj_sidx(j, t) * 6 * M, b, fcol + (size_t)(j - 1) * 6 * M + 6 * b);
        }
        team.sync();
        for (int it = tid; it < ncol * M; it += NT) {
          const int j = j0 + it / M, b = it % M;
          const double hs = hj[j] * sc;
          const double* zm = zst + (size_t)adj_sidx(j, t - 1) * 6 * M + 6 * b;
          double* zn = zst + (size_t)adj_sidx(j, t + 1) * 6 * M + 6 * b;
          const double* f = fcol + (size_t)(j - 1) * 6 * M + 6 * b;
          for (int k = 0; k < 6; ++k) zn[k] = zm[k] + 2.0 * hs * f[k];
        }
        team.sync();
      }
      // reverse, tau = 0: T_j = (z_2j + z_2j-1 + hs f(z_2j)) / 2 with
      // lambda_T = cw_j lambda_Y
      for (int it = tid; it < kacc * M; it += NT) {
        const int j = 1 + it / M, b = it % M;
        double* lzn = lzst + (size_t)adj_sidx(j, 2 * j) * 6 * M;
        double* lzp = lzst + (size_t)adj_sidx(j, 2 * j - 1) * 6 * M;
        for (int k = 0; k < 6; ++k) {
          const double lT = cw[j] * ly[6 * b + k];
          lzn[6 * b + k] += 0.5 * lT;
          lzp[6 * b + k] += 0.5 * lT;
        }
      }
      team.sync();
      // the f-term of T: w = cw_j lambda_Y for every member; staged in fcol
      for (int it = tid; it < kacc * M; it += NT) {
        const int j = 1 + it / M, b = it % M;
        for (int k = 0; k < 6; ++k) fcol[(size_t)(j - 1) * 6 * M + 6 * b + k] = cw[j] * ly[6 * b + k];
      }
      team.sync();
      for (int it = tid; it < kacc * M; it += NT) {
        const int j = 1 + it / M, b = it % M;
        const double hs = hj[j] * sc;
        grp_vjp(c, zst + (size_t)adj_sidx(j, 2 * j) * 6 * M, fcol + (size_t)(j - 1) * 6 * M, b,
                lzst + (size_t)adj_sidx(j, 2 * j) * 6 * M + 6 * b, lmc + (j - 1) * M + b,
                0.5 * hs);
      }
      team.sync();
      // tau = 1 .. 2k - 1: column j reverses z_{m+1} = z_{m-1} + 2 hs f(z_m) at m = 2j - tau
      for (int tau = 1; tau < 2 * kacc; ++tau) {
        const int j0 = (tau + 2) / 2;  // columns with m = 2j - tau >= 1
        const int ncol = kacc - j0 + 1;
        for (int it = tid; it < ncol * M; it += NT) {
          const int j = j0 + it / M, b = it % M;
          const int m = 2 * j - tau;
          const double hs = hj[j] * sc;
          const double* lnext = lzst + (size_t)adj_sidx(j, m + 1) * 6 * M;
          double* lprev = lzst + (size_t)adj_sidx(j, m - 1) * 6 * M + 6 * b;
          for (int k = 0; k < 6; ++k) lprev[k] += lnext[6 * b + k];
          grp_vjp(c, zst + (size_t)adj_sidx(j, m) * 6 * M, lnext, b,
                  lzst + (size_t)adj_sidx(j, m) * 6 * M + 6 * b, lmc + (j - 1) * M + b,
                  2.0 * hs);
        }
        team.sync();
      }
      // z_1 = z_0 + hs f0 and z_0 = y: lambda_y = sum_j (lambda_z0 + lambda_z1),
      // lambda_f0 = sum_j hs_j lambda_z1 (columns in ascending order)
      for (int b = tid; b < M; b += NT) {
        double acc[6] = {0, 0, 0, 0, 0, 0}, af[6] = {0, 0, 0, 0, 0, 0};
        double am = 0.0;
        for (int j = 1; j <= kacc; ++j) {
          const double hs = hj[j] * sc;
          const double* l0 = lzst + (size_t)adj_sidx(j, 0) * 6 * M + 6 * b;
          const double* l1 = lzst + (size_t)adj_sidx(j, 1) * 6 * M + 6 * b;
          for (int k = 0; k < 6; ++k) {
            acc[k] += l0[k] + l1[k];
            af[k] += hs * l1[k];
          }
          am += lmc[(j - 1) * M + b];
        }
        for (int k = 0; k < 6; ++k) {
          lin[6 * b + k] = acc[k];
          lf0[6 * b + k] = af[k];
        }
        lmv[b] += am;
      }
      team.sync();
      for (int b = tid; b < M; b += NT) grp_vjp(c, y, lf0, b, lin + 6 * b, lmv + b, 1.0);
      team.sync();
      for (int b = tid; b < M; b += NT)
        for (int k = 0; k < 6; ++k) ly[6 * b + k] = lin[6 * b + k];
      team.sync();
    }
    // lambda at the saved state of the members
    for (int b = tid; b < M; b += NT) {
      const int body = gmem[off + b];
      for (int k = 0; k < 3; ++k) {
        A.lx[k][body] = ly[6 * b + k];
        A.lv[k][body] = ly[6 * b + 3 + k];
      }
      A.lm[body] = lmv[b];
    }
    team.sync();
  }
}


// Record pass of a step's groups: groups of up to 8 bodies one per warp (the
// warp's direct-solver scratch in dynamic shared memory), larger ones one per
// CTA (scratch in gscr).
__global__ void __maxnreg__(128) k_bs_record(AdjGroupArgs A, Phys P, double h) {
  __shared__ double s_red[ABNT];
  __shared__ int s_flags[4];
  __shared__ int s_wflags[ABNT / 32][4];
  extern __shared__ double s_bscr[];  // the warp teams' scratch, 8 slots each
  const int ng = A.grp[0];
  const int* goff = A.grp + 2;
  const int warp = threadIdx.x >> 5;
  WarpTeam wt{s_wflags[warp]};
  for (int grp = blockIdx.x * (ABNT / 32) + warp; grp < ng; grp += gridDim.x * (ABNT / 32)) {
    if (goff[grp + 1] - goff[grp] > 8) continue;
    bs_record_group(A, P, h, grp, wt, s_bscr + (size_t)warp * 8 * A.bs_stride, 8);
  }
  __syncthreads();
  BlockTeam bt{s_red, s_flags};
  for (int grp = blockIdx.x; grp < ng; grp += gridDim.x) {
    if (goff[grp + 1] - goff[grp] <= 8) continue;
    bs_record_group(A, P, h, grp, bt, A.gscr + (size_t)goff[grp] * A.bs_stride, 0);
  }
}

// Reverse of a step's groups from the record buffer: groups of up to 8
// bodies one per warp, larger ones one per CTA.
__global__ void __maxnreg__(168) k_bs_reverse(AdjGroupArgs A, Phys P, double h) {
  __shared__ double s_red[ABNT];
  __shared__ int s_flags[4];
  __shared__ double cw[ABNT / 32][kMaxBsK + 2];
  __shared__ int s_wflags[ABNT / 32][4];
  const int ng = A.grp[0];
  const int* goff = A.grp + 2;
  const int warp = threadIdx.x >> 5;
  WarpTeam wt{s_wflags[warp]};
  for (int grp = blockIdx.x * (ABNT / 32) + warp; grp < ng; grp += gridDim.x * (ABNT / 32)) {
    if (goff[grp + 1] - goff[grp] > 8) continue;
    bs_reverse_group(A, P, h, grp, wt, cw[warp]);
  }
  __syncthreads();
  BlockTeam bt{s_red, s_flags};
  for (int grp = blockIdx.x; grp < ng; grp += gridDim.x) {
    if (goff[grp + 1] - goff[grp] <= 8) continue;
    bs_reverse_group(A, P, h, grp, bt, cw[0]);
  }
}

// ---------------------------------------------------------------------------
// Recording of one step of the replay.
// ---------------------------------------------------------------------------
struct StepRec {
  double* xs6;    // 6n saved state (after C(h/2)): x y z vx vy vz
  double* st0;    // 4n at the saved point: m, R, rc, (alive as double)
  double* x26;    // 6n after A (before the closing C(h/2))
  double* st1;    // 3n after A: m, rc, (alive as double)
  int* ingrp;     // n
  int* grp;       // 2 + (n + 1) + n: ngroups, nmembers, offsets, members
};

__global__ void k_rec_saved(Dev d, StepRec r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.n;
  if (i >= n) return;
  r.xs6[i] = d.xs[i]; r.xs6[n + i] = d.ys[i]; r.xs6[2 * n + i] = d.zs[i];
  r.xs6[3 * n + i] = d.vxs[i]; r.xs6[4 * n + i] = d.vys[i]; r.xs6[5 * n + i] = d.vzs[i];
  r.st0[i] = d.m[i]; r.st0[n + i] = d.R[i]; r.st0[2 * n + i] = d.rc[i];
  r.st0[3 * n + i] = d.alive[i] ? 1.0 : 0.0;
}

__global__ void k_rec_after(Dev d, StepRec r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.n;
  const int ng = d.ctrl->n_groups, nm = ng > 0 ? d.ctrl->n_members : 0;
  if (i == 0) {
    r.grp[0] = ng;
    r.grp[1] = nm;
  }
  if (i <= ng) r.grp[2 + i] = ng > 0 ? d.grp_off[i] : 0;
  if (i < nm) r.grp[2 + ng + 1 + i] = d.grp_mem[i];
  if (i >= n) return;
  r.x26[i] = d.x[i]; r.x26[n + i] = d.y[i]; r.x26[2 * n + i] = d.z[i];
  r.x26[3 * n + i] = d.vx[i]; r.x26[4 * n + i] = d.vy[i]; r.x26[5 * n + i] = d.vz[i];
  r.st1[i] = d.m[i]; r.st1[n + i] = d.rc[i]; r.st1[2 * n + i] = d.alive[i] ? 1.0 : 0.0;
  r.ingrp[i] = (ng > 0 && d.member_slot[i] >= 0) ? 1 : 0;
}

__global__ void k_alive_from(int n, const double* a, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] != 0.0 ? 1 : 0;
}

__global__ void k_scale3(int n, double s, const double* a, const double* b, const double* c,
                         double* oa, double* ob, double* oc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  oa[i] = s * a[i];
  ob[i] = s * b[i];
  oc[i] = s * c[i];
}

__global__ void k_aos_to_soa(int n, const double* a3, double* x, double* y, double* z, int add) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (add) {
    x[i] += a3[3 * i]; y[i] += a3[3 * i + 1]; z[i] += a3[3 * i + 2];
  } else {
    x[i] = a3[3 * i]; y[i] = a3[3 * i + 1]; z[i] = a3[3 * i + 2];
  }
}

__global__ void k_soa_to_aos(int n, const double* x, const double* y, const double* z, double* a3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  a3[3 * i] = x[i]; a3[3 * i + 1] = y[i]; a3[3 * i + 2] = z[i];
}

__global__ void k_mask(int n, const int* alive, double* a, double* b, double* c, double* d2,
                       double* e, double* f, double* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || alive[i]) return;
  a[i] = b[i] = c[i] = d2[i] = e[i] = f[i] = g[i] = 0.0;
}

}  // namespace nb

using namespace nb;

struct nb_adjoint {
  nb_system* sys;
  cudaStream_t st;
  int n, every, max_ckpt, nsteps_done;
  double dt;
  // checkpoints: per checkpoint 13n doubles, n alive ints, fprev pairs, ctrl
  double* ck_d;
  int* ck_i;
  Ctrl* ck_c;
  int n_ckpt;
  // step records of two segments: the backward pass reverses one segment
  // while the replay of the one before it fills the other buffer
  StepRec* recs[2];  // host arrays of device pointers
  int rec_cap;
  cudaStream_t st2;  // the replays' stream
  cudaEvent_t ev_rep;
  // adjoint vectors and scratch
  double *lx, *ly, *lz, *lvx, *lvy, *lvz, *lm, *mux, *muy, *muz, *parts;
  int* alive0;
  int* alive1;
  int* status;
  double* gscr;  // the record pass's direct-solver scratch (groups of more than 8 bodies)
  // the records of two steps' direct-solver replays: the record pass of step
  // t - 1 fills one on its own stream while the reverse of step t reads the other
  struct RecBuf {
    double *rslot, *gend, *H, *mst;
    int *kk, *counts, *mrg;
  } rb[2];
  double *work, *gwork;  // the reverse's scratch
  int work_stride;
  cudaStream_t st3;  // the record passes' stream
  cudaEvent_t ev_rec[2], ev_free[2], ev_seg;
  cudaStream_t st4;  // the Kepler transpose, beside the direct solver's reverse
  cudaEvent_t ev_kf, ev_kj;
  double* vpart;  // kick VJP partial sums, vjp_S x 4 x n
  int vjp_S;
  char err[256];
};

namespace {

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct ACarver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = al256(off);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int kmax_of(const nb_params& p) {
  return p.bs_kmax < 3 ? 3 : (p.bs_kmax > kMaxBsK ? kMaxBsK : p.bs_kmax);
}

// Source chunks of the kick VJP: about 8 CTAs per SM over the launch (at
// N = 2049 whole 128-body chunks gave 289 CTAs, two per SM, and the dependent
// FP64 chain of each pair went unhidden), chunks of at least 16 sources.
int vjp_split(int n) {
  const int tiles = (n + VNT - 1) / VNT;
  int S = (148 * 8 + tiles - 1) / tiles;
  const int maxS = (n + 15) / 16;
  if (S > maxS) S = maxS;
  return S < 1 ? 1 : S;
}

size_t adj_layout(const nb_params& p, int n, int nsteps, int every, char* base, nb_adjoint* a) {
  const size_t sys_bytes = nb_workspace_bytes(&p, n);
  ACarver c{base, 0};
  char* sysws = c.take<char>(sys_bytes);
  const int nck = nsteps / every + 2;
  int pair_cap = 1;
  {
    const int cap = p.pair_capacity > 0 ? p.pair_capacity : (4 * n > 4096 ? 4 * n : 4096);
    while (pair_cap < cap) pair_cap <<= 1;
  }
  double* ck_d = c.take<double>((size_t)nck * 13 * n);
  int* ck_i = c.take<int>((size_t)nck * (n + 2 * (size_t)pair_cap));
  Ctrl* ck_c = c.take<Ctrl>(nck);
  const int kmax = kmax_of(p);
  const int stride = adj_work_stride(kmax);
  std::vector<StepRec> recs(2 * (size_t)every);
  for (int t = 0; t < 2 * every; ++t) {
    recs[t].xs6 = c.take<double>(6 * (size_t)n);
    recs[t].st0 = c.take<double>(4 * (size_t)n);
    recs[t].x26 = c.take<double>(6 * (size_t)n);
    recs[t].st1 = c.take<double>(3 * (size_t)n);
    recs[t].ingrp = c.take<int>(n);
    recs[t].grp = c.take<int>(2 * (size_t)n + 3);
  }
  double* vec = c.take<double>(10 * (size_t)n);
  const int nparts = (n + ANT - 1) / ANT;
  double* parts = c.take<double>(3 * (size_t)nparts);
  int* alive0 = c.take<int>(n);
  int* alive1 = c.take<int>(n);
  int* status = c.take<int>(4);
  double* gscr = c.take<double>((size_t)n * bs_stride_for_kmax(kmax));
  nb_adjoint::RecBuf rb[2];
  for (int q = 0; q < 2; ++q) {
    rb[q].rslot = c.take<double>((size_t)n * adj_rec_stride());
    rb[q].gend = c.take<double>((size_t)n * 10);
    rb[q].H = c.take<double>((size_t)n * kSubCap);
    rb[q].kk = c.take<int>((size_t)n * kSubCap);
    rb[q].counts = c.take<int>((size_t)n * 4);
    rb[q].mrg = c.take<int>((size_t)n * kMrgCap * 3);
    rb[q].mst = c.take<double>((size_t)n * kMrgCap * 14);
  }
  double* work = c.take<double>((size_t)n * stride);
  double* gwork = c.take<double>((size_t)n * 10);
  const int vS = vjp_split(n);
  double* vpart = c.take<double>((size_t)vS * 4 * n);
  if (a && base) {
    a->vpart = vpart;
    a->vjp_S = vS;
    a->sys = (nb_system*)sysws;  // placeholder; replaced by the real handle in init
    a->ck_d = ck_d; a->ck_i = ck_i; a->ck_c = ck_c;
    a->max_ckpt = nck;
    a->rec_cap = every;
    for (int b = 0; b < 2; ++b) {
      a->recs[b] = (StepRec*)malloc(sizeof(StepRec) * every);
      for (int t = 0; t < every; ++t) a->recs[b][t] = recs[(size_t)b * every + t];
    }
    a->lx = vec; a->ly = vec + n; a->lz = vec + 2 * n;
    a->lvx = vec + 3 * n; a->lvy = vec + 4 * n; a->lvz = vec + 5 * n;
    a->lm = vec + 6 * n; a->mux = vec + 7 * n; a->muy = vec + 8 * n; a->muz = vec + 9 * n;
    a->parts = parts; a->alive0 = alive0; a->alive1 = alive1; a->status = status;
    a->gscr = gscr;
    a->rb[0] = rb[0];
    a->rb[1] = rb[1];
    a->work = work; a->gwork = gwork; a->work_stride = stride;
  }
  (void)sysws;
  return al256(c.off);
}

#define NB_ACU(call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      snprintf(a->err, sizeof(a->err), "%s: %s", #call, cudaGetErrorString(e_));        \
      return NB_E_CUDA;                                                                 \
    }                                                                                   \
  } while (0)

// Bit comparison of the replayed state (x, v, m) with a checkpoint: a replay
// that does not reproduce the forward would give the gradient of another
// trajectory, so the backward pass reports it instead.
__global__ void k_replay_check(Dev d, const double* cd, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.n;
  if (i >= n) return;
  const double* arr[7] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.m};
  bool same = true;
  for (int q = 0; q < 7; ++q)
    same = same && __double_as_longlong(arr[q][i]) == __double_as_longlong(cd[(size_t)q * n + i]);
  if (!same) atomicExch(bad, 1);
}

// Copy the system's full state to (dir 0) or from (dir 1) checkpoint k, on
// stream st (the adjoint's own stream unless given).
int checkpoint(nb_adjoint* a, int k, int dir, cudaStream_t st = nullptr) {
  if (!st) st = a->st;
  const Dev& d = a->sys->d;
  const int n = d.n;
  double* arr[] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.m, d.R, d.rc, d.rc2, d.ax, d.ay, d.az};
  double* cd = a->ck_d + (size_t)k * 13 * n;
  int* ci = a->ck_i + (size_t)k * (n + 2 * (size_t)d.pair_cap);
  const cudaMemcpyKind K = cudaMemcpyDeviceToDevice;
  for (int q = 0; q < 13; ++q)
    NB_ACU(cudaMemcpyAsync(dir ? arr[q] : cd + (size_t)q * n, dir ? cd + (size_t)q * n : arr[q],
                           sizeof(double) * n, K, st));
  NB_ACU(cudaMemcpyAsync(dir ? d.alive : ci, dir ? ci : d.alive, sizeof(int) * n, K, st));
  NB_ACU(cudaMemcpyAsync(dir ? (void*)d.fprev : (void*)(ci + n), dir ? (void*)(ci + n) : (void*)d.fprev,
                         sizeof(int2) * d.pair_cap, K, st));
  NB_ACU(cudaMemcpyAsync(dir ? d.ctrl : a->ck_c + k, dir ? a->ck_c + k : d.ctrl, sizeof(Ctrl), K, st));
  if (dir) {
    NB_ACU(cudaMemsetAsync(d.member_slot, 0xff, sizeof(int) * n, st));
    // forget the previous step's members (their slots were just cleared)
    NB_ACU(cudaMemsetAsync(&d.ctrl->n_prev_members, 0, sizeof(int), st));
  }
  return NB_OK;
}

// One step of the replay with the recording kernels around the BS phase
// (the same kernels as nb_step(1)).
void replay_step(nb_adjoint* a, double dt, const StepRec& r, cudaStream_t st) {
  nb_system* s = a->sys;
  const Dev& d = s->d;
  const int g = (d.n + 255) / 256;
  launch_open_h(d, dt, st);
  launch_drift_h(d, s->P, dt, st);
  k_rec_saved<<<g, 256, 0, st>>>(d, r);
  launch_kick(d, s->P, 0, st);
  launch_encounter(d, s->P, st);
  // the force update in the two halves nb_step uses (same arithmetic, so the
  // replay reproduces the forward bit for bit; here on one stream)
  launch_finish_part(d, s->P, 1, st);
  launch_bs(d, s->P, dt, st);
  launch_finish_part(d, s->P, 2, st);
  launch_scatter(d, s->P, st);
  launch_member_kick(d, s->P, st);
  k_rec_after<<<g + 1, 256, 0, st>>>(d, r);
  launch_close_h(d, s->P, dt, 1, st);
}

// Replay of segment seg from its checkpoint into the records `recs` on
// stream st, and the bit comparison of its end with the next checkpoint
// (flag status[2 + slot]).
int replay_segment(nb_adjoint* a, int seg, StepRec* recs, cudaStream_t st, int slot) {
  const int start = seg * a->every;
  const int len = a->nsteps_done - start < a->every ? a->nsteps_done - start : a->every;
  int rc = checkpoint(a, seg, 1, st);
  if (rc) return rc;
  for (int t = 0; t < len; ++t) replay_step(a, a->dt, recs[t], st);
  const int n = a->n;
  k_replay_check<<<(n + 255) / 256, 256, 0, st>>>(a->sys->d, a->ck_d + (size_t)(seg + 1) * 13 * n,
                                                  a->status + 2 + slot);
  return NB_OK;
}

void kick_vjp(nb_adjoint* a, const double* x6, const double* m, const double* rc,
              const int* alive, double hh) {
  const int n = a->n;
  const int g = (n + ANT - 1) / ANT;
  k_scale3<<<g, ANT, 0, a->st>>>(n, hh, a->lvx, a->lvy, a->lvz, a->mux, a->muy, a->muz);
  const int S = a->vjp_S;
  const int tiles = (n + VNT - 1) / VNT;
  Vjp V;
  V.x = x6; V.y = x6 + n; V.z = x6 + 2 * n; V.m = m; V.rc = rc; V.alive = alive;
  V.mux = a->mux; V.muy = a->muy; V.muz = a->muz;
  V.part = a->vpart;
  V.n = n;
  V.chunk = (n + S - 1) / S;  // the last chunks may be short or empty (zero partials)
  k_kick_vjp<<<dim3(tiles, S), VNT, 0, a->st>>>(V);
  k_kick_vjp_sum<<<g, ANT, 0, a->st>>>(n, S, a->vpart, a->sys->P.G, alive, a->lx, a->ly, a->lz,
                                       a->lm);
}

void cdrift_vjp(nb_adjoint* a, const int* alive, const double* m, const double* v6, double hh) {
  const int n = a->n;
  const int g = (n + ANT - 1) / ANT;
  k_sum3<<<g, ANT, 0, a->st>>>(n, alive, a->lx, a->ly, a->lz, a->parts);
  k_cdrift_vjp<<<g, ANT, 0, a->st>>>(n, g, a->parts, alive, m, v6 + 3 * n, v6 + 4 * n,
                                     v6 + 5 * n, hh, a->sys->P.m0, a->lvx, a->lvy, a->lvz,
                                     a->lm);
}

// The reverse of one step. The closing B(h/2) of a step and the opening
// B(h/2) of the next act at the same positions, masses and critical radii,
// with nothing in between, and the kick's transpose is linear in lambda_v:
// the two are one kick_vjp of weight h, taken with the earlier step's closing
// kick (close_w = h), and the later step skips its opening one (open = false).
// The last step closes with h/2 and the first step opens with h/2.
// The direct solver's arguments of a step: its groups and saved state, the
// record buffer buf, the adjoint vectors and the reverse's scratch.
AdjGroupArgs group_args(nb_adjoint* a, const StepRec& r, int buf) {
  const int n = a->n;
  const Phys& P = a->sys->P;
  AdjGroupArgs A;
  A.n = n;
  A.kmax = P.bs_kmax;
  A.bs_stride = bs_stride_for_kmax(P.bs_kmax);
  A.work_stride = a->work_stride;
  A.grp = r.grp;
  A.xs6 = r.xs6;
  A.m0 = r.st0; A.R0 = r.st0 + n; A.rc0 = r.st0 + 2 * n;
  A.lx[0] = a->lx; A.lx[1] = a->ly; A.lx[2] = a->lz;
  A.lv[0] = a->lvx; A.lv[1] = a->lvy; A.lv[2] = a->lvz;
  A.lm = a->lm;
  A.gscr = a->gscr;
  const nb_adjoint::RecBuf& b = a->rb[buf];
  A.rslot = b.rslot; A.gend = b.gend; A.H = b.H; A.kk = b.kk; A.counts = b.counts;
  A.mrg = b.mrg; A.mst = b.mst;
  A.work = a->work; A.gwork = a->gwork;
  A.status = a->status;
  return A;
}

int group_grid(int n) { return n < 2 * 148 ? n : 2 * 148; }

// The record pass of a step (the direct solver's replay of its groups with
// recording) into buffer buf, on stream st.
void record_step(nb_adjoint* a, double dt, const StepRec& r, int buf, cudaStream_t st) {
  const AdjGroupArgs A = group_args(a, r, buf);
  const size_t wsm = (size_t)(ABNT / 32) * 8 * A.bs_stride * sizeof(double);  // <= 48.1 KB
  if (wsm > 40 * 1024)  // with the static shared memory beyond the 48 KB default
    cudaFuncSetAttribute(k_bs_record, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
  k_bs_record<<<group_grid(a->n), ABNT, wsm, st>>>(A, a->sys->P, dt);
}

// The reverse of one step, its direct-solver records in buffer buf. The
// closing B(h/2) of a step and the opening B(h/2) of the next act at the same
// positions, masses and critical radii, with nothing in between, and the
// kick's transpose is linear in lambda_v: the two are one kick_vjp of weight
// h, taken with the earlier step's closing kick (close_w = h), and the later
// step skips its opening one (open = false). The last step closes with h/2
// and the first step opens with h/2.
void backward_step(nb_adjoint* a, double dt, const StepRec& r, double close_w, bool open,
                   int buf) {
  const int n = a->n;
  const int g = (n + ANT - 1) / ANT;
  const double hh = 0.5 * dt;
  k_alive_from<<<g, ANT, 0, a->st>>>(n, r.st1 + 2 * n, a->alive1);
  k_alive_from<<<g, ANT, 0, a->st>>>(n, r.st0 + 3 * n, a->alive0);
  // closing B(h/2) at the final positions (with the next step's opening
  // B(h/2)), then the closing C(h/2)
  kick_vjp(a, r.x26, r.st1, r.st1 + n, a->alive1, close_w);
  cdrift_vjp(a, a->alive1, r.st1, r.x26, hh);
  // A(h): Kepler outside the groups, Bulirsch-Stoer inside; the two touch
  // disjoint bodies' lambda, so the Kepler transpose runs on its own stream
  // beside the direct solver's reverse
  const Phys& P = a->sys->P;
  const int gk = (((n + kKvBodies - 1) / kKvBodies) * 32 + ANT - 1) / ANT;
  cudaEventRecord(a->ev_kf, a->st);
  cudaStreamWaitEvent(a->st4, a->ev_kf, 0);
  k_kepler_vjp<<<gk, ANT, 0, a->st4>>>(n, r.xs6, a->alive0, r.ingrp, P.mu, dt, P.kepler_max_iter,
                                       a->lx, a->ly, a->lz, a->lvx, a->lvy, a->lvz, a->status);
  cudaEventRecord(a->ev_kj, a->st4);
  k_bs_reverse<<<group_grid(n), ABNT, 0, a->st>>>(group_args(a, r, buf), P, dt);
  cudaStreamWaitEvent(a->st, a->ev_kj, 0);
  // the record buffer is free for the record pass two steps back
  cudaEventRecord(a->ev_free[buf], a->st);
  // opening C(h/2), then the opening B(h/2) at the step's start positions
  // (for the first step; the others' went with the step before)
  cdrift_vjp(a, a->alive0, r.st0, r.xs6, hh);
  if (open) kick_vjp(a, r.xs6, r.st0, r.st0 + 2 * n, a->alive0, hh);
}

}  // namespace

extern "C" {

size_t nb_adjoint_workspace_bytes(const nb_params* p, int n, int nsteps, int checkpoint_every) {
  if (!p || n < 1 || nsteps < 1 || checkpoint_every < 1 || nb_workspace_bytes(p, n) == 0 ||
      p->rcrit_refresh != 0 || p->gas != 0 || p->eject_r != 0.0 || p->ml_levels != 0)
    return 0;
  return adj_layout(*p, n, nsteps, checkpoint_every, nullptr, nullptr);
}

int nb_adjoint_init(nb_adjoint** out, const nb_params* p, int n, const double* x,
                    const double* v, const double* m, const double* R, const double* rc,
                    int nsteps, int checkpoint_every, void* workspace, size_t ws_bytes,
                    void* stream, int inputs_on_device) {
  if (!out || !rc) return NB_E_INVALID;
  *out = nullptr;
  if (p && p->precision != NB_PREC_FP64) return NB_E_INVALID;
  const size_t need = nb_adjoint_workspace_bytes(p, n, nsteps, checkpoint_every);
  if (need == 0) return NB_E_INVALID;
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return NB_E_WORKSPACE;
  nb_adjoint* a = (nb_adjoint*)calloc(1, sizeof(nb_adjoint));
  if (!a) return NB_E_INVALID;
  adj_layout(*p, n, nsteps, checkpoint_every, (char*)workspace, a);
  a->n = n;
  a->every = checkpoint_every;
  a->st = (cudaStream_t)stream;
  nb_system* s = nullptr;
  const int rc0 = nb_init_system(&s, p, n, x, v, m, R, rc, nullptr, workspace,
                                 nb_workspace_bytes(p, n), stream, inputs_on_device);
  bool ok = rc0 == NB_OK &&
            cudaStreamCreateWithFlags(&a->st2, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&a->st3, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&a->st4, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&a->ev_kf, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&a->ev_kj, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&a->ev_rep, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&a->ev_seg, cudaEventDisableTiming) == cudaSuccess;
  for (int q = 0; q < 2 && ok; ++q)
    ok = cudaEventCreateWithFlags(&a->ev_rec[q], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&a->ev_free[q], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    a->sys = s;
    nb_adjoint_destroy(a);
    return rc0 != NB_OK ? rc0 : NB_E_CUDA;
  }
  a->sys = s;
  *out = a;
  return NB_OK;
}

int nb_adjoint_forward(nb_adjoint* a, int nsteps, double dt) {
  if (!a || nsteps < 1 || !std::isfinite(dt)) return NB_E_INVALID;
  // segments plus one slot for the final state
  const int nseg = (nsteps + a->every - 1) / a->every;
  if (nseg + 1 > a->max_ckpt) return NB_E_OVERFLOW;
  if (a->n_ckpt > 0) {  // back to the initial state of an earlier call
    const int rc = checkpoint(a, 0, 1);
    if (rc) return rc;
  }
  NvtxRange range("nb_adjoint_forward");
  a->dt = dt;
  a->n_ckpt = 0;
  a->nsteps_done = 0;
  for (int done = 0; done < nsteps;) {
    int rc = checkpoint(a, a->n_ckpt++, 0);
    if (rc) return rc;
    const int k = nsteps - done < a->every ? nsteps - done : a->every;
    rc = nb_step(a->sys, k, dt);
    if (rc) {
      snprintf(a->err, sizeof(a->err), "forward: %s", nb_last_error(a->sys));
      return rc;
    }
    done += k;
  }
  const int rc = checkpoint(a, a->n_ckpt, 0);  // final state
  if (rc) return rc;
  a->nsteps_done = nsteps;
  return NB_OK;
}

int nb_adjoint_state(nb_adjoint* a, double* x, double* v, double* m, int* alive,
                     int out_on_device) {
  if (!a) return NB_E_INVALID;
  const Dev& d = a->sys->d;
  const int n = d.n;
  double* tmp = d.snap;
  const int g = (n + 255) / 256;
  const cudaMemcpyKind K = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (x) {
    k_soa_to_aos<<<g, 256, 0, a->st>>>(n, d.x, d.y, d.z, tmp);
    NB_ACU(cudaMemcpyAsync(x, tmp, sizeof(double) * 3 * n, K, a->st));
  }
  if (v) {
    k_soa_to_aos<<<g, 256, 0, a->st>>>(n, d.vx, d.vy, d.vz, tmp + 3 * n);
    NB_ACU(cudaMemcpyAsync(v, tmp + 3 * n, sizeof(double) * 3 * n, K, a->st));
  }
  if (m) NB_ACU(cudaMemcpyAsync(m, d.m, sizeof(double) * n, K, a->st));
  if (alive) NB_ACU(cudaMemcpyAsync(alive, d.alive, sizeof(int) * n, K, a->st));
  NB_ACU(cudaStreamSynchronize(a->st));
  return NB_OK;
}

int nb_adjoint_backward(nb_adjoint* a, const double* gx, const double* gv, const double* gm,
                        double* dx0, double* dv0, double* dm0, int on_device) {
  if (!a || !gx || !gv || !gm || a->nsteps_done < 1) return NB_E_INVALID;
  const int n = a->n;
  const int g = (n + 255) / 256;
  const Dev& d = a->sys->d;
  double* tmp = d.snap;  // staging (16 n doubles)
  const cudaMemcpyKind Kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  NB_ACU(cudaMemcpyAsync(tmp, gx, sizeof(double) * 3 * n, Kin, a->st));
  NB_ACU(cudaMemcpyAsync(tmp + 3 * n, gv, sizeof(double) * 3 * n, Kin, a->st));
  NB_ACU(cudaMemcpyAsync(a->lm, gm, sizeof(double) * n, Kin, a->st));
  k_aos_to_soa<<<g, 256, 0, a->st>>>(n, tmp, a->lx, a->ly, a->lz, 0);
  k_aos_to_soa<<<g, 256, 0, a->st>>>(n, tmp + 3 * n, a->lvx, a->lvy, a->lvz, 0);
  // absorbed bodies' final states are constants
  k_mask<<<g, 256, 0, a->st>>>(n, d.alive, a->lx, a->ly, a->lz, a->lvx, a->lvy, a->lvz, a->lm);
  NB_ACU(cudaMemsetAsync(a->status, 0, 4 * sizeof(int), a->st));
  const int total = a->nsteps_done;
  // Segments from the last to the first. A segment's replay (forward with
  // recording, the system's arrays) and the reverse of the segment after it
  // (its records and the adjoint's own arrays) touch disjoint memory, so the
  // replay of segment seg - 1 runs on the second stream beside the reverse of
  // segment seg; both are latency-bound (the direct solver's groups) and
  // leave most of the GPU idle. Buffers alternate; the streams join after
  // every segment, when the host checks the status words.
  NB_ACU(cudaEventRecord(a->ev_rep, a->st));
  NB_ACU(cudaStreamWaitEvent(a->st2, a->ev_rep, 0));
  int cur = 0;
  {
    NvtxRange r("adjoint: replay the last segment");
    int rc = replay_segment(a, a->n_ckpt - 1, a->recs[cur], a->st2, cur);
    if (rc) return rc;
  }
  for (int seg = a->n_ckpt - 1; seg >= 0; --seg) {
    const int start = seg * a->every;
    const int len = total - start < a->every ? total - start : a->every;
    NB_ACU(cudaEventRecord(a->ev_rep, a->st2));  // segment seg's records are complete
    NB_ACU(cudaStreamWaitEvent(a->st, a->ev_rep, 0));
    if (seg > 0) {
      NvtxRange r("adjoint: replay the segment before, beside the reverse");
      int rc = replay_segment(a, seg - 1, a->recs[1 - cur], a->st2, 1 - cur);
      if (rc) return rc;
    }
    {
      // the reverse of the segment's steps, last first; the record pass of
      // step t - 1 (its own stream, its own buffer) runs beside the reverse
      // of step t, and waits for the reverse that last read its buffer
      NvtxRange r("adjoint: reverse segment");
      NB_ACU(cudaEventRecord(a->ev_seg, a->st));
      NB_ACU(cudaStreamWaitEvent(a->st3, a->ev_seg, 0));
      record_step(a, a->dt, a->recs[cur][len - 1], (len - 1) & 1, a->st3);
      NB_ACU(cudaEventRecord(a->ev_rec[(len - 1) & 1], a->st3));
      for (int t = len - 1; t >= 0; --t) {
        NB_ACU(cudaStreamWaitEvent(a->st, a->ev_rec[t & 1], 0));
        if (t > 0) {
          if (t + 1 <= len - 1) NB_ACU(cudaStreamWaitEvent(a->st3, a->ev_free[(t - 1) & 1], 0));
          record_step(a, a->dt, a->recs[cur][t - 1], (t - 1) & 1, a->st3);
          NB_ACU(cudaEventRecord(a->ev_rec[(t - 1) & 1], a->st3));
        }
        backward_step(a, a->dt, a->recs[cur][t], start + t == total - 1 ? 0.5 * a->dt : a->dt,
                      start + t == 0, t & 1);
      }
    }
    NB_ACU(cudaEventRecord(a->ev_rep, a->st2));
    NB_ACU(cudaStreamWaitEvent(a->st, a->ev_rep, 0));
    int st[4] = {0, 0, 0, 0};
    NB_ACU(cudaMemcpyAsync(st, a->status, sizeof(st), cudaMemcpyDeviceToHost, a->st));
    Ctrl c;
    NB_ACU(cudaMemcpyAsync(&c, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, a->st));
    NB_ACU(cudaStreamSynchronize(a->st));
    NB_ACU(cudaGetLastError());
    if (c.status || st[0]) {
      snprintf(a->err, sizeof(a->err), "backward: %s", nb_status_string(c.status ? c.status : st[0]));
      return c.status ? c.status : st[0];
    }
    if (st[2 + cur] || (seg > 0 && st[2 + (1 - cur)])) {
      snprintf(a->err, sizeof(a->err),
               "backward: the replay of segment %d did not reproduce the forward state",
               st[2 + cur] ? seg : seg - 1);
      return NB_E_INVALID;
    }
    cur = 1 - cur;
  }
  // leave the system at its final state again
  int rc = checkpoint(a, a->n_ckpt, 1);
  if (rc) return rc;
  const cudaMemcpyKind Kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  k_soa_to_aos<<<g, 256, 0, a->st>>>(n, a->lx, a->ly, a->lz, tmp);
  k_soa_to_aos<<<g, 256, 0, a->st>>>(n, a->lvx, a->lvy, a->lvz, tmp + 3 * n);
  if (dx0) NB_ACU(cudaMemcpyAsync(dx0, tmp, sizeof(double) * 3 * n, Kout, a->st));
  if (dv0) NB_ACU(cudaMemcpyAsync(dv0, tmp + 3 * n, sizeof(double) * 3 * n, Kout, a->st));
  if (dm0) NB_ACU(cudaMemcpyAsync(dm0, a->lm, sizeof(double) * n, Kout, a->st));
  NB_ACU(cudaStreamSynchronize(a->st));
  return NB_OK;
}

const char* nb_adjoint_last_error(const nb_adjoint* a) { return a ? a->err : "no adjoint"; }

void nb_adjoint_destroy(nb_adjoint* a) {
  if (!a) return;
  if (a->sys) nb_destroy(a->sys);
  if (a->st2) cudaStreamDestroy(a->st2);
  if (a->st3) cudaStreamDestroy(a->st3);
  if (a->st4) cudaStreamDestroy(a->st4);
  if (a->ev_kf) cudaEventDestroy(a->ev_kf);
  if (a->ev_kj) cudaEventDestroy(a->ev_kj);
  if (a->ev_rep) cudaEventDestroy(a->ev_rep);
  if (a->ev_seg) cudaEventDestroy(a->ev_seg);
  for (int q = 0; q < 2; ++q) {
    if (a->ev_rec[q]) cudaEventDestroy(a->ev_rec[q]);
    if (a->ev_free[q]) cudaEventDestroy(a->ev_free[q]);
  }
  free(a->recs[0]);
  free(a->recs[1]);
  free(a);
}

}  // extern "C"
