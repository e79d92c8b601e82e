// Direct solver for close-encounter groups (the paper's "direct solver" for
// H_A when bodies are in a close encounter, section "The hybrid symplectic
// integrator"; perfect mergers per "Detailing the outcomes of collisions").
// Shared by the single-system kernel (one CTA per group) and the batched
// kernel (each system's CTA integrates its own groups).
#pragma once

#include "nb_internal.cuh"

namespace nb {

// ---------------------------------------------------------------------------
// Bulirsch-Stoer for one group per CTA.
// Scratch per member slot (bs_stride_for_kmax(kmax) doubles):
//   y[6] | f0[6] | per extrapolation column j = 1..kmax: zm[6] zc[6] f[6] |
//   T[2][kmax][6] | aux[4] = (G m, 1 / (0.9 rc), rc^2, 0.1 rc).
// Working copies of m, R, rc, alive live in gnew[slot*10+6..9].
//
// A group of two bodies keeps only two lanes of its CTA busy, and every FP64
// warp instruction holds the B300 FP64 pipe for the full warp, so the solver's
// speed is its count of dependent FP64 warp instructions. Two consequences:
// the right-hand side uses the seeded reciprocal roots and reciprocals of
// nb_internal.cuh and precomputed per-member constants, and the modified-
// midpoint sequences of the extrapolation columns, which are independent of
// one another, advance together in separate lanes (a "wave" over columns):
// an attempt that converges at column J takes 2J + 1 dependent derivative
// evaluations instead of J^2 + 2J. Each column's arithmetic, the Neville
// table and the acceptance test are the same as column-after-column, so the
// result does not depend on how many columns run at once.
// ---------------------------------------------------------------------------
constexpr int OY = 0, OF0 = 6;
constexpr int CZM = 0, CZC = 6, CF = 12;  // fields of a column block


struct BsCtx {
  double* base;  // scratch of the group's first slot
  double* g;     // gnew of the group's first slot
  int stride, M, kmax;
  double G, mu;
  double mu15, mu1875;  // 1.5 mu and 1.875 mu (the star term's refinement polynomial)
  double rc_scale = 1.0;  // changeover radii r_crit * rc_scale (multi-level changeover)
};

__device__ __forceinline__ bool bs_alive(const BsCtx& c, int b) { return c.g[10 * b + 9] != 0.0; }

__device__ __forceinline__ double* bs_aux(const BsCtx& c, int b) {
  return c.base + (size_t)b * c.stride + bs_off_T(c.kmax) + 12 * c.kmax;
}

__device__ __forceinline__ void bs_set_aux(const BsCtx& c, int b, double G, double m, double rc) {
  double* a = bs_aux(c, b);
  a[0] = G * m;
  a[1] = 1.0 / (0.9 * rc);
  a[2] = rc * rc;
  a[3] = 0.1 * rc;
}


// 1 - w for a pair inside rc (w = K - r dK/dr, K the infinitely smooth switch
// K = f(y) / (f(y) + f(1 - y)), f(y) = exp(-1/y)), from r = qq, rc01 =
// 0.1 rc and inv09 = 1 / (0.9 rc). One exponential and two reciprocals: with
// E = exp(1/y - 1/(1-y)) = exp((u - y) / (y u)), u = 1 - y, K = 1 / (1 + E)
// and dK/dy = K (1 - K) (1/y^2 + 1/u^2) = E K^2 (y^2 + u^2) / (y u)^2. Where
// |1/y - 1/u| > 80, K is within 2e-35 of 0 or 1 and w is 0 or 1 to double
// precision. The range tests compare bit patterns.
__device__ __forceinline__ double close_weight(double qq, double rc01, double inv09) {
  const double y = (qq - rc01) * inv09;
  if (__double_as_longlong(y) < __double_as_longlong(1.0 / 746.0)) return 1.0;  // also y < 0
  const double u = 1.0 - y;
  if (__double_as_longlong(u) < __double_as_longlong(1.0 / 746.0)) return 0.0;
  const double iw = rcp_fast(y * u);
  const double dd = (u - y) * iw;
  const long long bd = __double_as_longlong(dd);
  if ((bd & 0x7fffffffffffffffll) > __double_as_longlong(80.0)) return bd > 0 ? 1.0 : 0.0;
  const double E = exp_fast(dd);
  const double K = rcp_fast(1.0 + E);
  const double dKdy = (E * K) * K * (__fma_rn(y, y, u * u) * (iw * iw));
  return 1.0 - (K - qq * dKdy * inv09);
}

// Neville weights 1 / ((n_j / n_{j-q})^2 - 1) = (j - q)^2 / (q (2j - q)) for
// the substep counts n_k = 2k, [j][q] for 1 <= q < j <= kMaxBsK: each the
// correctly rounded quotient, as the division gives it at run time, folded
// by the compiler.
struct NevilleTab {
  double w[kMaxBsK + 1][kMaxBsK + 1];
};
__host__ __device__ constexpr NevilleTab neville_tab() {
  NevilleTab t{};
  for (int j = 2; j <= kMaxBsK; ++j)
    for (int q = 1; q < j; ++q)
      t.w[j][q] = (double)((j - q) * (j - q)) / (double)(q * (2 * j - q));
  return t;
}
static __constant__ NevilleTab kNeville = neville_tab();

// fmax(m, |v|) for m >= 0 (a NaN v leaves m), on bit patterns: the integer
// pipe instead of the FP64 one.
__device__ __forceinline__ double nn_max_abs(double m, double v) {
  const long long b = __double_as_longlong(v) & 0x7fffffffffffffffll;
  return (b > 0x7ff0000000000000ll || b <= __double_as_longlong(m)) ? m : __longlong_as_double(b);
}

// fl(a / b) <= tol for b > 0, with tol_up the next double above tol, almost
// always without the division: the FMA residual a - t b is rounded once, so
// its sign is that of the exact value; a < tol b accepts (a / b < tol) and
// a > tol_up b rejects (a / b > tol_up). Only a quotient strictly between
// tol and tol_up, or a non-finite one, goes through the division, which
// rejects a NaN.
__device__ __forceinline__ bool ratio_le(double a, double b, double tol, double tol_up) {
  if (__fma_rn(-tol, b, a) < 0.0) return true;
  if (__fma_rn(-tol_up, b, a) > 0.0) return false;
  return a / b <= tol;
}

// The next double above tol (tol >= 0).
__device__ __forceinline__ double next_up(double tol) {
  return __longlong_as_double(__double_as_longlong(tol) + 1ll);
}

// The acceptance test of column j >= 3 for one member: the position and the
// velocity parts of the change between the two highest extrapolations A and
// B, each in the max-norm relative to the part's own max-norm, within tol.
__device__ __forceinline__ bool bs_member_ok(const double* A, const double* B, double tol,
                                             double tol_up) {
  bool ok = true;
  for (int part = 0; part < 2; ++part) {
    double dm = 0.0, ym = 0.0;
    for (int k = 3 * part; k < 3 * part + 3; ++k) {
      dm = nn_max_abs(dm, A[k] - B[k]);
      ym = nn_max_abs(ym, A[k]);
    }
    ok = ok && ratio_le(dm, ym + 1e-300, tol, tol_up);
  }
  return ok;
}

// Field fout of member b = d/dt of field fo (Eq. Ha restricted to the group).
static __device__ void bs_deriv(const BsCtx& c, int fo, int fout, int b) {
  const double* yb = c.base + (size_t)b * c.stride + fo;
  double* fb = c.base + (size_t)b * c.stride + fout;
  if (!bs_alive(c, b)) {
    for (int k = 0; k < 6; ++k) fb[k] = 0.0;
    return;
  }
  fb[0] = yb[3];
  fb[1] = yb[4];
  fb[2] = yb[5];
  const double r2 = sep2_int(yb[0], yb[1], yb[2]);  // r^2 on the integer pipe
  const double ks = -scale_fast<NB_PREC_FP64>(r2, c.mu, c.mu15, c.mu1875);  // -mu / r^3
  double ax = ks * yb[0], ay = ks * yb[1], az = ks * yb[2];
  const double* ab = bs_aux(c, b);
  for (int q = 0; q < c.M; ++q) {
    if (q == b || !bs_alive(c, q)) continue;
    const double* yq = c.base + (size_t)q * c.stride + fo;
    const double dx = yq[0] - yb[0], dy = yq[1] - yb[1], dz = yq[2] - yb[2];
    const double q2 = sep2_int(dx, dy, dz);
    if (__double_as_longlong(q2) == 0ll) continue;
    const double* aq = bs_aux(c, q);
    if (!(nn_less(q2, ab[2]) || nn_less(q2, aq[2]))) continue;  // 1 - w = 0 beyond rc
    const double ri = rinv_fast(q2);
    const double omw = close_weight(q2 * ri, nn_max(ab[3], aq[3]), nn_min(ab[1], aq[1]));
    const double f = aq[0] * omw * (ri * ri * ri);
    ax = __fma_rn(f, dx, ax);
    ay = __fma_rn(f, dy, ay);
    az = __fma_rn(f, dz, az);
  }
  fb[3] = ax;
  fb[4] = ay;
  fb[5] = az;
}

static __device__ double pair_energy(const Phys& P, const double* a, double ma, const double* b,
                              double mb) {
  const double va2 = a[3] * a[3] + a[4] * a[4] + a[5] * a[5];
  const double vb2 = b[3] * b[3] + b[4] * b[4] + b[5] * b[5];
  const double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  const double rab = sqrt(dx * dx + dy * dy + dz * dz);
  return 0.5 * ma * va2 + 0.5 * mb * vb2 - P.G * P.m0 * ma / ra - P.G * P.m0 * mb / rb -
         P.G * ma * mb / rab;
}

// Record of one group's integration for the adjoint's replay: the state,
// masses, radii, critical radii and alive flags at the start of every
// accepted substep, its size H and extrapolation column k, and every merger
// with the pre-merger states. Slots are per member (stride 6 for states).
struct BsRec {
  int cap, mcap;                      // substep and merger capacities
  int* counts;                        // [0] substeps, [1] mergers, [2] overflow
  double* H;                          // cap
  int* k;                             // cap
  double *ys, *ms, *Rs, *rcs, *alv;   // cap * M * 6, cap * M (x4)
  int* mrg;                           // mcap * 3: (substep, a, b)
  double* mst;                        // mcap * 14: y_a, y_b, m_a, m_b before the merger
};

// Perfect merging on contact, scanned in ascending slot (= body) order.
static __device__ void bs_merge_scan(const BsCtx& c, const Phys& P, double* El, int* merges,
                                     BsRec* rec = nullptr, int sub = 0) {
  for (int a = 0; a < c.M; ++a) {
    for (int b = a + 1; b < c.M; ++b) {
      if (!bs_alive(c, a) || !bs_alive(c, b)) continue;
      double* ya = c.base + (size_t)a * c.stride + OY;
      double* yb = c.base + (size_t)b * c.stride + OY;
      const double dx = yb[0] - ya[0], dy = yb[1] - ya[1], dz = yb[2] - ya[2];
      const double rab = sqrt(dx * dx + dy * dy + dz * dz);
      double* ga = c.g + 10 * a;
      double* gb = c.g + 10 * b;
      if (!(rab < ga[7] + gb[7])) continue;
      const double ma = ga[6], mb = gb[6];
      if (rec) {
        const int q = rec->counts[1];
        if (q < rec->mcap) {
          rec->mrg[3 * q] = sub;
          rec->mrg[3 * q + 1] = a;
          rec->mrg[3 * q + 2] = b;
          for (int k = 0; k < 6; ++k) {
            rec->mst[14 * q + k] = ya[k];
            rec->mst[14 * q + 6 + k] = yb[k];
          }
          rec->mst[14 * q + 12] = ma;
          rec->mst[14 * q + 13] = mb;
        } else {
          rec->counts[2] = 1;
        }
        rec->counts[1] = q + 1;
      }
      const double e0 = pair_energy(P, ya, ma, yb, mb);
      const double M = ma + mb;
      for (int k = 0; k < 6; ++k) ya[k] = (ma * ya[k] + mb * yb[k]) / M;
      const double Rn = cbrt(ga[7] * ga[7] * ga[7] + gb[7] * gb[7] * gb[7]);
      ga[6] = M;
      ga[7] = Rn;
      gb[9] = 0.0;
      const double v2 = ya[3] * ya[3] + ya[4] * ya[4] + ya[5] * ya[5];
      const double r = sqrt(ya[0] * ya[0] + ya[1] * ya[1] + ya[2] * ya[2]);
      const double e1 = 0.5 * M * v2 - P.G * P.m0 * M / r;
      *El += e0 - e1;
      ga[8] = rcrit(P, ya[0], ya[1], ya[2], ya[3], ya[4], ya[5], M);
      bs_set_aux(c, a, P.G, M, ga[8] * c.rc_scale);
      *merges += 1;
    }
  }
}


// Counters of the direct solver (summed over the groups a CTA integrates).
struct BsTally {
  long long derivs, substeps, halvings, merges;
  long long ml_substeps = 0, ml_groups = 0;  // multi-level changeover
};

// One speculative attempt pair (see bs_integrate): the attempt of size H
// from y (slots of c) and, in the other lanes, the attempt of size H/2 from
// the same y (column and Neville scratch in the slots of cs; it reads y, f0
// and the masses and radii from c's slots and its own copy of the members'
// aux words). Both columns sets advance in one wave over the kmax columns;
// f0 = f(y) is shared (the half-size attempt would compute the same values).
// Flags: [0], [1] = the H attempt accepted at column [1]; [2], [3] = the H/2
// attempt accepted at column [3]. After its acceptance the H/2 attempt's
// Neville rows stop, so its accepted row stays in place. Returns the number
// of derivative evaluations the H/2 attempt would have taken on its own
// (its f0 included), up to its acceptance or its last column.
template <class Sy>
static __device__ long long bs_attempt_pair(const BsCtx& c, const BsCtx& cs, const Phys& P,
                                            const double* hj, double sc, Sy& sy,
                                            BsTally& tally) {
  const int kmax = c.kmax, M = c.M;
  const int NT = sy.nthreads(), tid = sy.tid();
  int* s_flags = sy.flags();
  const int offT = bs_off_T(kmax);
  const int KM = kmax * M;
  const double tol_up = next_up(P.bs_tol);
  // start both column sets: z0 = y, z1 = y + hs f0
  for (int it = tid; it < 2 * KM; it += NT) {
    const int half = it >= KM, r = it - half * KM;
    const int j = 1 + r / M, b = r % M;
    const double* s = c.base + (size_t)b * c.stride;
    double* col = (half ? cs.base : c.base) + (size_t)b * c.stride + bs_off_col(j);
    const double hs = hj[j] * (half ? 0.5 * sc : sc);
    for (int k = 0; k < 6; ++k) {
      col[CZM + k] = s[OY + k];
      col[CZC + k] = s[OY + k] + hs * s[OF0 + k];
    }
  }
  sy.sync();
  long long sd = 1;  // the H/2 attempt's own f0
  for (int t = 1; t <= 2 * kmax; ++t) {
    const int j0 = max(1, (t + 1) / 2);
    const int ncol = kmax - j0 + 1, NI = ncol * M;
    const bool sdone = s_flags[2] != 0;
    for (int it = tid; it < 2 * NI; it += NT) {
      const int half = it >= NI, r = it - half * NI;
      const int j = j0 + r / M, b = r % M;
      bs_deriv(half ? cs : c, bs_off_col(j) + CZC, bs_off_col(j) + CF, b);
    }
    sy.sync();
    tally.derivs += ncol;
    if (!sdone) sd += ncol;
    for (int it = tid; it < 2 * NI; it += NT) {
      const int half = it >= NI, r = it - half * NI;
      const int j = j0 + r / M, b = r % M;
      double* sl = (half ? cs.base : c.base) + (size_t)b * c.stride;
      double* col = sl + bs_off_col(j);
      const double hs = hj[j] * (half ? 0.5 * sc : sc);
      if (t < 2 * j) {
        for (int k = 0; k < 6; ++k) {
          const double zn = col[CZM + k] + 2.0 * hs * col[CF + k];
          col[CZM + k] = col[CZC + k];
          col[CZC + k] = zn;
        }
      } else if (!(half && sdone)) {  // t == 2j: the column's result T_j1
        double* Tc = sl + offT + (j & 1) * kmax * 6;
        for (int k = 0; k < 6; ++k) Tc[k] = 0.5 * (col[CZC + k] + col[CZM + k] + hs * col[CF + k]);
      }
    }
    sy.sync();
    if (t & 1) continue;
    const int j = t / 2;  // column j of both attempts is complete: Neville rows and tests
    bool fm = false, fs = false;  // a member of the H (H/2) attempt fails the test
    for (int it = tid; it < 2 * M; it += NT) {
      const int half = it >= M, b = it - half * M;
      if (half && sdone) continue;
      double* sl = (half ? cs.base : c.base) + (size_t)b * c.stride;
      double* Tc = sl + offT + (j & 1) * kmax * 6;
      double* Tp = sl + offT + ((j - 1) & 1) * kmax * 6;
      for (int q = 1; q < j; ++q) {
        const double inv = kNeville.w[j][q];
        for (int k = 0; k < 6; ++k) {
          const double tq = Tc[6 * (q - 1) + k];
          Tc[6 * q + k] = __fma_rn(tq - Tp[6 * (q - 1) + k], inv, tq);
        }
      }
      if (j >= 3 && bs_alive(c, b) &&
          !bs_member_ok(Tc + 6 * (j - 1), Tc + 6 * (j - 2), P.bs_tol, tol_up)) {
        if (half) fs = true; else fm = true;
      }
    }
    if (j < 3) {
      sy.sync();
      continue;
    }
    const bool Fm = sy.any_to_first(fm);
    sy.sync();  // the team's reduction scratch is reused
    const bool Fs = sy.any_to_first(fs);
    if (tid == 0) {
      if (!Fm) {
        s_flags[0] = 1;
        s_flags[1] = j;
      }
      if (!sdone && !Fs) {
        s_flags[2] = 1;
        s_flags[3] = j;
      }
    }
    sy.sync();
    if (s_flags[0]) {
      for (int b = tid; b < M; b += NT) {
        double* sl = c.base + (size_t)b * c.stride;
        const double* Tc = sl + offT + (j & 1) * kmax * 6 + 6 * (j - 1);
        for (int k = 0; k < 6; ++k) sl[OY + k] = Tc[k];
      }
      sy.sync();
      break;
    }
  }
  return sd;
}

// Integrate H_A restricted to one group over h with all threads of the
// calling CTA (any blockDim): Gragg modified midpoint with n_j = 2j substeps,
// Neville extrapolation in the substep squared, acceptance at j >= 3 when
// every live body's position and velocity changes between the two highest
// columns are within bs_tol of its own max-norm; halving on failure at k_max,
// doubling back after an early success on an aligned boundary; perfect
// merging scan after every accepted substep. Columns run in windows of W
// (all of them for small groups): within a window every column advances one
// midpoint substep per wave step, and column j completes at wave step 2j,
// when its Neville row is built and tested. The group state starts in the y
// fields and ends there. Sy is the team that runs it: one CTA (BlockTeam)
// or a thread-block cluster (ClusterTeam, in encounter.cu); it provides the
// thread index and count, the barrier, a max-reduction and four flag words.
// Every team member takes the same branches. Returns 0, NB_E_NOCONV or
// NB_E_TIMEOUT (the same in every thread); *El (tid 0) receives the energy
// removed by mergers.
//
// Speculation (spec: M more slots of scratch after the group's, or null):
// when the team has lanes for both (2 kmax M <= its threads), every attempt
// of size H also runs, in the spare lanes, the attempt of size H/2 that a
// failure would lead to (bs_attempt_pair). If the H attempt fails and the
// H/2 one was accepted, the H/2 result is taken, with the same state updates,
// counters and records as running the two attempts one after the other; the
// arithmetic of each attempt is unchanged, so the result is the same bit for
// bit, and a failure costs no wave steps of its own.
template <class Sy>
static __device__ int bs_integrate(const BsCtx& c, const Phys& P, double h, Sy& sy,
                                   BsTally& tally, double* El, BsRec* rec,
                                   double* spec = nullptr) {
  int rec_n = 0;  // accepted substeps recorded (the same in every thread)
  const int kmax = c.kmax;
  const int M = c.M;
  const int NT = sy.nthreads();
  const int tid = sy.tid();
  int* s_flags = sy.flags();
  const int offT = bs_off_T(kmax);
  // columns per window: enough (column, member) items to fill about two
  // passes of the CTA, never fewer than one column
  int W = (2 * NT) / (M > 0 ? M : 1);
  W = W < 1 ? 1 : (W > kmax ? kmax : W);
  const bool can_spec = spec != nullptr && 2 * kmax * M <= NT;
  // h / n_j for the columns; an attempt of size H = h 2^-level takes
  // hj[j] 2^-level, the same double as H / n_j (scaling by a power of two is
  // exact), so no attempt divides
  double hj[kMaxBsK + 1];
  for (int j = 1; j <= kmax; ++j) hj[j] = h / (2 * j);
  const double tol_up = next_up(P.bs_tol);
  BsCtx cs = c;
  if (can_spec) cs.base = spec;
  int level = 0;
  long long done = 0;
  int status = 0;
  long long attempts = 0;
  int merges = 0;
  while (done < (1ll << level)) {
    const double H = ldexp(h, -level);
    const double sc = ldexp(1.0, -level);
    const bool sp = can_spec && level + 1 <= P.bs_max_halvings;
    if (rec && rec_n < rec->cap) {  // stage the substep's start (kept if it is accepted)
      for (int b = tid; b < M; b += NT) {
        const double* y = c.base + (size_t)b * c.stride + OY;
        const double* g = c.g + 10 * b;
        const size_t o = (size_t)rec_n * M + b;
        for (int k = 0; k < 6; ++k) rec->ys[6 * o + k] = y[k];
        rec->ms[o] = g[6];
        rec->Rs[o] = g[7];
        rec->rcs[o] = g[8];
        rec->alv[o] = g[9];
      }
    }
    if (tid == 0) {
      s_flags[0] = 0;
      s_flags[1] = 0;
      if (sp) {
        s_flags[2] = 0;
        s_flags[3] = 0;
      }
    }
    // f0 = f(y), shared by every column (and by the speculative attempt)
    for (int b = tid; b < M; b += NT) {
      bs_deriv(c, OY, OF0, b);
      if (sp) {  // the speculative slots' copy of the aux words
        const double* a = bs_aux(c, b);
        double* as = bs_aux(cs, b);
        for (int k = 0; k < 4; ++k) as[k] = a[k];
      }
    }
    sy.sync();
    tally.derivs += 1;
    long long sderivs = 0;
    if (sp) {
      sderivs = bs_attempt_pair(c, cs, P, hj, sc, sy, tally);
    } else {
      for (int ja = 1; ja <= kmax && !s_flags[0]; ja += W) {
        const int jb = ja + W - 1 < kmax ? ja + W - 1 : kmax;
        const int nw = jb - ja + 1;
        // start the window's columns: z0 = y, z1 = y + hs f0
        for (int it = tid; it < nw * M; it += NT) {
          const int j = ja + it / M, b = it % M;
          double* s = c.base + (size_t)b * c.stride;
          double* col = s + bs_off_col(j);
          const double hs = hj[j] * sc;
          for (int k = 0; k < 6; ++k) {
            col[CZM + k] = s[OY + k];
            col[CZC + k] = s[OY + k] + hs * s[OF0 + k];
          }
        }
        sy.sync();
        for (int t = 1; t <= 2 * jb; ++t) {
          // columns still running at wave step t: 2j >= t
          const int j0 = max(ja, (t + 1) / 2);
          const int ncol = jb - j0 + 1;
          for (int it = tid; it < ncol * M; it += NT) {
            const int j = j0 + it / M, b = it % M;
            bs_deriv(c, bs_off_col(j) + CZC, bs_off_col(j) + CF, b);
          }
          sy.sync();
          tally.derivs += ncol;
          for (int it = tid; it < ncol * M; it += NT) {
            const int j = j0 + it / M, b = it % M;
            double* s = c.base + (size_t)b * c.stride;
            double* col = s + bs_off_col(j);
            const double hs = hj[j] * sc;
            if (t < 2 * j) {
              for (int k = 0; k < 6; ++k) {
                const double zn = col[CZM + k] + 2.0 * hs * col[CF + k];
                col[CZM + k] = col[CZC + k];
                col[CZC + k] = zn;
              }
            } else {  // t == 2j: the column's result T_j1
              double* Tc = s + offT + (j & 1) * kmax * 6;
              for (int k = 0; k < 6; ++k) Tc[k] = 0.5 * (col[CZC + k] + col[CZM + k] + hs * col[CF + k]);
            }
          }
          sy.sync();
          if ((t & 1) || t / 2 < ja) continue;
          const int j = t / 2;  // column j is complete: Neville row j and the test
          bool fail = false;
          for (int b = tid; b < M; b += NT) {
            double* s = c.base + (size_t)b * c.stride;
            double* Tc = s + offT + (j & 1) * kmax * 6;
            double* Tp = s + offT + ((j - 1) & 1) * kmax * 6;
            for (int q = 1; q < j; ++q) {
              const double inv = kNeville.w[j][q];
              for (int k = 0; k < 6; ++k) {
                const double tq = Tc[6 * (q - 1) + k];
                Tc[6 * q + k] = __fma_rn(tq - Tp[6 * (q - 1) + k], inv, tq);
              }
            }
            if (j >= 3 && bs_alive(c, b) &&
                !bs_member_ok(Tc + 6 * (j - 1), Tc + 6 * (j - 2), P.bs_tol, tol_up))
              fail = true;
          }
          if (j < 3) {
            sy.sync();
            continue;
          }
          const bool F = sy.any_to_first(fail);  // valid in tid 0
          if (tid == 0 && !F) {
            s_flags[0] = 1;
            s_flags[1] = j;
          }
          sy.sync();
          if (s_flags[0]) {
            for (int b = tid; b < M; b += NT) {
              double* s = c.base + (size_t)b * c.stride;
              const double* Tc = s + offT + (j & 1) * kmax * 6 + 6 * (j - 1);
              for (int k = 0; k < 6; ++k) s[OY + k] = Tc[k];
            }
            sy.sync();
            break;
          }
        }
      }
    }
    ++attempts;
    int acc = s_flags[0], kacc = s_flags[1];
    double Hacc = H;
    if (!acc) {
      ++tally.halvings;
      if (level >= P.bs_max_halvings) {
        status = NB_E_NOCONV;
        break;
      }
      ++level;
      done *= 2;
      if (sp && attempts > 200000) {
        status = NB_E_TIMEOUT;
        break;
      }
      if (sp) {  // the H/2 attempt ran already: take its outcome
        ++attempts;
        tally.derivs += sderivs;
        if (s_flags[2]) {
          acc = 1;
          kacc = s_flags[3];
          Hacc = 0.5 * H;
          for (int b = tid; b < M; b += NT) {
            const double* Tc = cs.base + (size_t)b * c.stride + offT + (kacc & 1) * kmax * 6 +
                               6 * (kacc - 1);
            double* y = c.base + (size_t)b * c.stride + OY;
            for (int k = 0; k < 6; ++k) y[k] = Tc[k];
          }
          sy.sync();
        } else {
          ++tally.halvings;
          if (level >= P.bs_max_halvings) {
            status = NB_E_NOCONV;
            break;
          }
          ++level;
          done *= 2;
        }
      }
    }
    if (acc) {
      ++done;
      ++tally.substeps;
      if (rec) {
        if (tid == 0) {
          if (rec_n < rec->cap) {
            rec->H[rec_n] = Hacc;
            rec->k[rec_n] = kacc;
          } else {
            rec->counts[2] = 1;
          }
        }
        ++rec_n;
      }
      if (P.merge) {
        if (tid == 0) bs_merge_scan(c, P, El, &merges, rec, rec_n - 1);
        sy.sync();
      }
      if (level > 0 && (done & 1) == 0 && kacc <= kmax - 2) {
        --level;
        done >>= 1;
      }
    }
    if (attempts > 200000) {
      status = NB_E_TIMEOUT;
      break;
    }
    sy.sync();
  }
  tally.merges += merges;
  if (rec && tid == 0) rec->counts[0] = rec_n;
  sy.sync();
  return status;
}

// One CTA as the team: shared scratch s_red (blockDim.x doubles) and two
// shared flag words.
struct BlockTeam {
  double* s_red;
  int* s_flags;
  __device__ int tid() const { return threadIdx.x; }
  __device__ int nthreads() const { return blockDim.x; }
  __device__ int* flags() const { return s_flags; }
  __device__ void sync() const { __syncthreads(); }
  __device__ double max_to_first(double v) const {
    s_red[threadIdx.x] = v;
    __syncthreads();
    double e = 0.0;
    if (threadIdx.x == 0)
      for (int q = 0; q < (int)blockDim.x; ++q) e = fmax(e, s_red[q]);
    return e;
  }  // whether v holds in any thread (here: in all of them)
  __device__ bool any_to_first(bool v) const { return __syncthreads_or(v) != 0; }
};

// One warp as the team (small groups: a CTA integrates one group per warp
// and the barriers are warp barriers). s_flags: this warp's two shared ints.
struct WarpTeam {
  int* s_flags;
  __device__ int tid() const { return threadIdx.x & 31; }
  __device__ int nthreads() const { return 32; }
  __device__ int* flags() const { return s_flags; }
  __device__ void sync() const { __syncwarp(); }
  __device__ double max_to_first(double v) const {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  }  __device__ bool any_to_first(bool v) const { return __any_sync(0xffffffffu, v) != 0; }
};

static __device__ int bs_integrate_group(const BsCtx& c, const Phys& P, double h, double* s_red,
                                         int* s_flags, BsTally& tally, double* El,
                                         BsRec* rec = nullptr) {
  BlockTeam t{s_red, s_flags};
  return bs_integrate(c, P, h, t, tally, El, rec);
}

}  // namespace nb
