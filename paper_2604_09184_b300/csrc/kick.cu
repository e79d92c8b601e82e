// Interaction kick of Eq. Hb with the encounter flags of the changeover.
//
// a_i = G sum_j m_j w_ij (x_j - x_i) / r_ij^3, w = K - r dK/dr (exact gradient
// of H_B), and the pair (i < j) is flagged when r_ij^2 < max(rc_i, rc_j)^2.
//
// B300 design: the FP64 pipe issues ~1/60 of the FP32 rate, so the pair loop
// spends as few FP64 instructions as it can and moves everything else to the
// INT/FP32/MUFU pipes:
//   - the r^-3 refinement and the three accumulations are FP64 (7 FP64
//     instructions per pair in the FP64 mode, 6 in the mixed mode);
//   - dx, dy, dz come from positions held as 128-bit fixed-point integers
//     (fix_of: exact for 2^-36 <= |x| < 2^38 AU): their difference is exact
//     and is rounded to a double by integer ops (fix_diff), which also give
//     the top 64 bits of its square, so r^2 is an aligned integer sum rounded
//     once (sep2_fix, within an ulp of the exact value);
//   - the r^-3 seed is rsqrtf of a float built from r^2's high word with one
//     integer shift-add; its square (exact) and cube (rounded) are built as
//     doubles from integer products of its significand (no F2F conversions,
//     no FP64 multiplies), and the source mass enters the refinement
//     polynomial through m, 1.5 m and 1.875 m staged with the j-tile;
//   - the encounter test first compares the high words of r^2 and
//     max(rc_i^2, rc_j^2) as integers (IEEE order of non-negative doubles),
//     with one unit of slack for the integer r^2; only a near-tie or a close
//     pair takes the exact FP64 branch, which forms dx, dy, dz and r^2 in the
//     FP64 subtractions and fixed rounding that decide the flags, computes the
//     changeover weight and appends the flagged pair with one atomic per warp
//     (ballot + popc).
// j-tiles of 128 bodies (fixed-point positions, m, 1.5 m, 1.875 m) are staged
// through shared memory; each thread owns one target (the integer arithmetic
// takes registers: bounded at 64 for 8 CTAs per SM, 3 % faster than 80 and 6);
// a CTA covers 128 targets x one j-chunk, and the j-chunks' partial sums are
// added in a fixed order by k_finish (deterministic results). The double-single
// kernel has the same shape (one target per thread: 27.7 ms against 30.7 ms
// with two at N = 65538).
#include "nb_internal.cuh"

namespace nb {

constexpr int KNT = 128;  // threads per kick CTA (= j-tile size)
constexpr int KIPT = 1;   // targets per thread (the integer pair arithmetic needs registers:
                          // one target, 64 registers, 8 CTAs per SM)
#ifndef NB_KICK_UNROLL
#define NB_KICK_UNROLL 4
#endif
constexpr int kKickUnroll = NB_KICK_UNROLL;  // j-loop unroll of the FP64/mixed kick (tuning)

struct KickArgs {
  int n, S, jchunk;
  int ib, ie;  // target rows [ib, ie) (all sources 0..n-1 act on them)
  const int* cond;  // if set, the launch does nothing while *cond == 0
  const double *x, *y, *z, *m, *rc, *rc2;
  double* kpart;  // S x 3 x n
  int2* pairs;
  int cap;
  int* counter;
  Ctrl* ctrl;
};

// Append (i, j) for the lanes with f set: one atomicAdd per warp.
__device__ __forceinline__ void emit_pair(bool f, int i, int j, int2* pairs, int cap, int* counter,
                                          Ctrl* ctrl) {
  const unsigned mask = __activemask();
  const unsigned fm = __ballot_sync(mask, f);
  if (fm == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(fm) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(fm));
  base = __shfl_sync(mask, base, leader);
  if (f) {
    const int pos = base + __popc(fm & ((1u << lane) - 1u));
    if (pos < cap)
      pairs[pos] = make_int2(i, j);
    else
      set_status(ctrl, NB_E_OVERFLOW, 1);
  }
}

// The exact branch: coincident bodies, changeover pairs and flag emission.
template <bool FLAGS>
__device__ __forceinline__ double rare_pair(double r2, double sc, double mj, int i, int j,
                                            double rc2i, double rci, const KickArgs& A) {
  double s = sc;
  const double rc2 = fmax(rc2i, __ldg(A.rc2 + j));
  const bool flag = (r2 < rc2) && (i < j);  // coincident distinct bodies are flagged too
  if (r2 == 0.0) {
    s = 0.0;  // no force between coincident bodies (and none on itself)
  } else if (r2 < rc2) {
    const double rcij = fmax(rci, __ldg(A.rc + j));
    const double r = sqrt(r2);
    s = mj * kick_weight(r, rcij) / (r2 * r);
  }
  if (FLAGS) emit_pair(flag, i, j, A.pairs, A.cap, A.counter, A.ctrl);
  return s;
}

template <int PREC>
__global__ void __launch_bounds__(KNT, 8) k_kick(KickArgs A) {
  __shared__ nb_u128 sX[KNT], sY[KNT], sZ[KNT];  // fixed-point positions of the j-tile
  __shared__ double sm[KNT], sm15[KNT], sm1875[KNT];
  __shared__ int sh[KNT];
  __shared__ int s_stop;
  if (threadIdx.x == 0) s_stop = A.ctrl->status || (A.cond && *A.cond == 0);
  __syncthreads();
  if (s_stop) return;
  const int n = A.n;
  const int it = blockIdx.x / A.S;
  const int sidx = blockIdx.x - it * A.S;
  const int i0 = A.ib + it * (KNT * KIPT) + threadIdx.x;

  nb_u128 Xi[KIPT], Yi[KIPT], Zi[KIPT];
  double rc2i[KIPT], rci[KIPT];
  double ax[KIPT], ay[KIPT], az[KIPT];
  double cx[KIPT], cy[KIPT], cz[KIPT];  // compensation (mixed mode)
  int hi[KIPT], ii[KIPT];
#pragma unroll
  for (int k = 0; k < KIPT; ++k) {
    const int i = i0 + k * KNT;
    ii[k] = i;
    if (i < A.ie) {
      Xi[k] = fix_of(A.x[i]);
      Yi[k] = fix_of(A.y[i]);
      Zi[k] = fix_of(A.z[i]);
      rc2i[k] = A.rc2[i];
      rci[k] = A.rc[i];
    } else {  // padding target far from everything, never flagged
      Xi[k] = Yi[k] = Zi[k] = fix_of(1e10);
      rc2i[k] = 0.0;
      rci[k] = 0.0;
    }
    hi[k] = __double2hiint(rc2i[k]);
    ax[k] = ay[k] = az[k] = 0.0;
    cx[k] = cy[k] = cz[k] = 0.0;
  }
  const int j0 = sidx * A.jchunk;
  const int j1 = min(n, j0 + A.jchunk);
  for (int jt = j0; jt < j1; jt += KNT) {
    __syncthreads();
    const int j = jt + threadIdx.x;
    if (j < j1) {
      sX[threadIdx.x] = fix_of(A.x[j]);
      sY[threadIdx.x] = fix_of(A.y[j]);
      sZ[threadIdx.x] = fix_of(A.z[j]);
      const double mj = A.m[j];
      sm[threadIdx.x] = mj;
      sm15[threadIdx.x] = 1.5 * mj;
      sm1875[threadIdx.x] = 1.875 * mj;
      sh[threadIdx.x] = __double2hiint(A.rc2[j]);
    }
    __syncthreads();
    const int cnt = min(KNT, j1 - jt);
    double tx[KIPT], ty[KIPT], tz[KIPT];  // tile sums (mixed mode)
#pragma unroll
    for (int k = 0; k < KIPT; ++k) tx[k] = ty[k] = tz[k] = 0.0;
#pragma unroll kKickUnroll
    for (int q = 0; q < cnt; ++q) {
      const nb_u128 Xj = sX[q], Yj = sY[q], Zj = sZ[q];
      const double mj = sm[q];
      const double mj15 = sm15[q], mj1875 = PREC == NB_PREC_FP64 ? sm1875[q] : 0.0;
      const int hj = sh[q];
#pragma unroll
      for (int k = 0; k < KIPT; ++k) {
        // dx, dy, dz and r^2 on the integer pipe (exact differences of the
        // fixed-point positions, rounded); a pair whose r^2 high word is
        // within one unit of the threshold's takes the exact branch, which
        // decides the flag and the weight from the FP64 subtractions and sep2
        const FixDiff fx = fix_diff(Xj, Xi[k]), fy = fix_diff(Yj, Yi[k]), fz = fix_diff(Zj, Zi[k]);
        const double dx = fx.d, dy = fy.d, dz = fz.d;
        const double r2 = sep2_fix(fx, fy, fz);
        double sc = scale_fast<PREC>(r2, mj, mj15, mj1875);
        if (__double2hiint(r2) <= max(hi[k], hj) + 1) {
          const int i = ii[k] < A.ie ? ii[k] : A.ie - 1, j = jt + q;
          const double ex = __ldg(A.x + j) - __ldg(A.x + i), ey = __ldg(A.y + j) - __ldg(A.y + i),
                       ez = __ldg(A.z + j) - __ldg(A.z + i);
          sc = rare_pair<true>(ii[k] < A.ie ? sep2(ex, ey, ez) : 1e20, sc, mj, ii[k], j, rc2i[k],
                               rci[k], A);
        }
        if (PREC == NB_PREC_FP64) {
          ax[k] = __fma_rn(sc, dx, ax[k]);
          ay[k] = __fma_rn(sc, dy, ay[k]);
          az[k] = __fma_rn(sc, dz, az[k]);
        } else {
          tx[k] = __fma_rn(sc, dx, tx[k]);
          ty[k] = __fma_rn(sc, dy, ty[k]);
          tz[k] = __fma_rn(sc, dz, tz[k]);
        }
      }
    }
    if (PREC != NB_PREC_FP64) {
      // Neumaier-compensated accumulation of the tile sums (TwoSum form).
#pragma unroll
      for (int k = 0; k < KIPT; ++k) {
        double t, b;
        t = ax[k] + tx[k]; b = t - ax[k]; cx[k] += (ax[k] - (t - b)) + (tx[k] - b); ax[k] = t;
        t = ay[k] + ty[k]; b = t - ay[k]; cy[k] += (ay[k] - (t - b)) + (ty[k] - b); ay[k] = t;
        t = az[k] + tz[k]; b = t - az[k]; cz[k] += (az[k] - (t - b)) + (tz[k] - b); az[k] = t;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KIPT; ++k) {
    const int i = ii[k];
    if (i < A.ie) {
      double* p = A.kpart + (size_t)(3 * sidx) * n;
      p[i] = ax[k] + cx[k];
      p[n + i] = ay[k] + cy[k];
      p[2 * n + i] = az[k] + cz[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Unordered-pair kick (FP64, whole system). Each pair {i, j} is evaluated
// once and its term goes to both bodies (Newton's third law): the seeded
// r^-3 (4 FP64 operations), the scales m_j r^-3 and m_i r^-3 and six FMAs,
// 12 FP64 instructions per unordered pair (6 per ordered pair against 7 in
// k_kick), and the integer work (fixed-point differences, r^2, the seed) once
// per pair instead of twice.
// Bodies form NB blocks of kSymBlock. The block pairs (X, Y = X + d mod NB),
// d = 1..NB/2, cover every pair of distinct blocks once (for even NB the
// pairs at d = NB/2 come from the lower block X < NB/2 only); d = 0 is the
// block with itself, one-sided, with the flag taken for i < j. The row-major
// list of NB (NB/2 + 1) tiles is cut into equal ranges, one per CTA; a CTA
// keeps its row's sums in registers (a range spans at most two rows; one
// partial per row and CTA) and writes one partial per tile for block Y.
// In a tile, warp w pairs its 32 bodies of X with the 128 of Y in four
// 32 x 32 sub-tiles: at step s lane l takes body (l + s) mod 32 of the
// sub-tile, and the Y-side sums move one lane down after every step
// (shuffles), so that after 32 steps lane l holds body l's sum; the four
// warps' sums are added in warp order. k_finish adds a body's partials in a
// fixed order (its row's in CTA order, then its column's by d), so the
// results are deterministic. The exact branch (near or inside the changeover
// radius) is that of k_kick with both scales, (m w) / (r^2 r) each.
// ---------------------------------------------------------------------------
struct SymArgs {
  int nb, hrow, tiles, per;
  double* xpart;  // grid x 2 x 3 x kSymBlock
  double* ypart;  // nb x hrow x 3 x kSymBlock
};

static_assert(KNT == kSymBlock, "one thread per body of a block");
// Unroll of the 32-step rotation loop: the loop body holds ~460 instructions
// and the registers are bounded at 64, so unrolling only adds spills (N = 65538:
// 36.7 ms not unrolled, 37.0 and 38.2 ms unrolled 2 and 4 times).
#ifndef NB_SYM_UNROLL
#define NB_SYM_UNROLL 1
#endif
constexpr int kSymUnroll = NB_SYM_UNROLL;

template <bool DIAG>
__device__ __forceinline__ void sym_rare(int i, int j, double mi, double mj, const KickArgs& A,
                                         double& sj, double& si) {
  const bool ok = i < A.n && j < A.n;
  double r2 = 1e20, rc2 = 0.0, rc = 0.0;
  if (ok) {
    r2 = sep2(__ldg(A.x + j) - __ldg(A.x + i), __ldg(A.y + j) - __ldg(A.y + i),
              __ldg(A.z + j) - __ldg(A.z + i));
    rc2 = fmax(__ldg(A.rc2 + i), __ldg(A.rc2 + j));
    rc = fmax(__ldg(A.rc + i), __ldg(A.rc + j));
  }
  // coincident distinct bodies are flagged too
  const bool flag = ok && (r2 < rc2) && (!DIAG || i < j);
  if (ok && r2 == 0.0) {
    sj = 0.0;
    si = 0.0;
  } else if (ok && r2 < rc2) {
    const double r = sqrt(r2);
    const double w = kick_weight(r, rc);
    sj = mj * w / (r2 * r);
    if (!DIAG) si = mi * w / (r2 * r);
  }
  emit_pair(flag, min(i, j), max(i, j), A.pairs, A.cap, A.counter, A.ctrl);
}

__global__ void __launch_bounds__(KNT, kSymCtasPerSm) k_kick_sym(KickArgs A, SymArgs L) {
  __shared__ nb_u128 sX[KNT], sY[KNT], sZ[KNT];  // block Y: fixed-point positions
  __shared__ double sm[KNT];
  __shared__ int sh[KNT];
  __shared__ double sacc[3][4][KNT];  // the warps' Y-side sums of a tile
  __shared__ int s_stop;
  if (threadIdx.x == 0) s_stop = A.ctrl->status || (A.cond && *A.cond == 0);
  __syncthreads();
  if (s_stop) return;
  const int n = A.n;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int H1 = L.hrow + 1;
  const int f0 = blockIdx.x * L.per;
  const int f1 = min(L.tiles, f0 + L.per);
  int X = -1, seg = 0, i = 0, hi = 0;
  nb_u128 Xi = 0, Yi = 0, Zi = 0;
  double mi = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
  for (int f = f0; f < f1; ++f) {
    const int Xf = f / H1, dd = f - Xf * H1;
    if (Xf != X) {
      if (X >= 0) {
        double* p = L.xpart + (size_t)((blockIdx.x * 2 + seg) * 3) * KNT + threadIdx.x;
        p[0] = ax;
        p[KNT] = ay;
        p[2 * KNT] = az;
        seg = 1;
      }
      X = Xf;
      i = X * KNT + threadIdx.x;
      if (i < n) {
        Xi = fix_of(A.x[i]);
        Yi = fix_of(A.y[i]);
        Zi = fix_of(A.z[i]);
        mi = A.m[i];
        hi = __double2hiint(A.rc2[i]);
      } else {  // padding far from everything, massless, never flagged
        Xi = Yi = Zi = fix_of(1e10);
        mi = 0.0;
        hi = 0;
      }
      ax = ay = az = 0.0;
    }
    if (2 * dd == L.nb && X >= L.nb / 2) continue;  // the lower block covers this pair
    int Yb = X + dd;
    if (Yb >= L.nb) Yb -= L.nb;
    const int jb = Yb * KNT;
    __syncthreads();
    {
      const int j = jb + threadIdx.x;
      if (j < n) {
        sX[threadIdx.x] = fix_of(A.x[j]);
        sY[threadIdx.x] = fix_of(A.y[j]);
        sZ[threadIdx.x] = fix_of(A.z[j]);
        sm[threadIdx.x] = A.m[j];
        sh[threadIdx.x] = __double2hiint(A.rc2[j]);
      } else {
        sX[threadIdx.x] = sY[threadIdx.x] = sZ[threadIdx.x] = fix_of(1e10);
        sm[threadIdx.x] = 0.0;
        sh[threadIdx.x] = 0;
      }
    }
    __syncthreads();
    if (dd == 0) {
      // the block with itself: every ordered pair, this body's side only
#pragma unroll 4
      for (int q = 0; q < KNT; ++q) {
        const FixDiff fx = fix_diff(sX[q], Xi), fy = fix_diff(sY[q], Yi), fz = fix_diff(sZ[q], Zi);
        const double r2 = sep2_fix(fx, fy, fz);
        const double mj = sm[q];
        double sj = mj * rinv3_fast(r2), si = 0.0;
        if (__double2hiint(r2) <= max(hi, sh[q]) + 1) sym_rare<true>(i, jb + q, mi, mj, A, sj, si);
        ax = __fma_rn(sj, fx.d, ax);
        ay = __fma_rn(sj, fy.d, ay);
        az = __fma_rn(sj, fz.d, az);
      }
      continue;
    }
#pragma unroll 1
    for (int u = 0; u < 4; ++u) {
      double bx = 0.0, by = 0.0, bz = 0.0;  // Y-side sums, one lane down per step
#pragma unroll kSymUnroll
      for (int s = 0; s < 32; ++s) {
        const int q = 32 * u + ((lane + s) & 31);
        const FixDiff fx = fix_diff(sX[q], Xi), fy = fix_diff(sY[q], Yi), fz = fix_diff(sZ[q], Zi);
        const double r2 = sep2_fix(fx, fy, fz);
        const double mj = sm[q];
        const double r3 = rinv3_fast(r2);
        double sj = mj * r3, si = mi * r3;
        if (__double2hiint(r2) <= max(hi, sh[q]) + 1) sym_rare<false>(i, jb + q, mi, mj, A, sj, si);
        ax = __fma_rn(sj, fx.d, ax);
        ay = __fma_rn(sj, fy.d, ay);
        az = __fma_rn(sj, fz.d, az);
        bx = __fma_rn(-si, fx.d, bx);
        by = __fma_rn(-si, fy.d, by);
        bz = __fma_rn(-si, fz.d, bz);
        const int src = (lane + 1) & 31;
        bx = __shfl_sync(0xffffffffu, bx, src);
        by = __shfl_sync(0xffffffffu, by, src);
        bz = __shfl_sync(0xffffffffu, bz, src);
      }
      sacc[0][wp][32 * u + lane] = bx;
      sacc[1][wp][32 * u + lane] = by;
      sacc[2][wp][32 * u + lane] = bz;
    }
    __syncthreads();
    double* p = L.ypart + ((size_t)Yb * L.hrow + (dd - 1)) * 3 * KNT + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      p[c * KNT] = ((sacc[c][0][threadIdx.x] + sacc[c][1][threadIdx.x]) + sacc[c][2][threadIdx.x]) +
                   sacc[c][3][threadIdx.x];
  }
  if (X >= 0) {
    double* p = L.xpart + (size_t)((blockIdx.x * 2 + seg) * 3) * KNT + threadIdx.x;
    p[0] = ax;
    p[KNT] = ay;
    p[2 * KNT] = az;
  }
}

// A body's sum of the unordered-pair kick's partials, in a fixed order: its
// row's partials in CTA order, then its column's by d.
__device__ __forceinline__ void sym_partials(const Dev& d, int i, double& ax, double& ay,
                                             double& az) {
  const int X = i / kSymBlock, t = i - X * kSymBlock;
  const int H1 = d.sym_hrow + 1;
  const int fa = X * H1, fb = fa + H1 - 1;
  for (int b = fa / d.sym_per; b <= fb / d.sym_per; ++b) {
    const int seg = (b * d.sym_per) / H1 == X ? 0 : 1;
    const double* p = d.sym_xpart + (size_t)((b * 2 + seg) * 3) * kSymBlock + t;
    ax += p[0];
    ay += p[kSymBlock];
    az += p[2 * kSymBlock];
  }
  const double* p = d.sym_ypart + (size_t)X * d.sym_hrow * 3 * kSymBlock + t;
#pragma unroll 4
  for (int dd = 1; dd <= d.sym_hrow; ++dd, p += 3 * kSymBlock) {
    const int Xs = X - dd < 0 ? X - dd + d.sym_nb : X - dd;
    if (2 * dd == d.sym_nb && Xs >= d.sym_nb / 2) continue;
    ax += p[0];
    ay += p[kSymBlock];
    az += p[2 * kSymBlock];
  }
}

// ---------------------------------------------------------------------------
// Double-single kick (NB_PREC_DS). The pair arithmetic runs as double-single
// (unevaluated float pairs, error-free FMA transforms, Dekker/Knuth style) on
// the FP32 pipe, with no FP64 instruction per pair: a lone FP64 instruction
// per pair costs as much pipe time as ~64 FP32 ones on the B300.
//  - Relative coordinates: every coordinate is split on a common grid G = 2^g
//    (k_ds_grid: |c| < 2^23 G for every body not parked beyond 2^19 AU) into
//    a multiple of G and a multiple of G2 = 2^-24 G, each exact as a float,
//    and the float nearest the rest. The multiples subtract exactly in float,
//    so dx carries 2^-48 relative plus 2^-47 G absolute error (2^-66 AU for
//    bodies within 16 AU), in 7 FP32 instructions.
//  - r^2, r^-3, m r^-3 and the products in double-single; each term accurate
//    to a few 2^-48; per-tile sums are float pairs folded into FP64
//    accumulators.
//  - The encounter test compares the float r^2 with a float threshold that
//    over-estimates max(rc_i^2, rc_j^2) by 2^-20; any pair that passes takes
//    the exact FP64 branch of the FP64 kernel (from the FP64 positions), so
//    flags are identical.
// All float arithmetic uses the _rn intrinsics so that no operation is
// contracted or reassociated. The grid depends on all positions only, so a
// row block's kick equals the whole kick's rows bit for bit.
// ---------------------------------------------------------------------------
struct F2 {
  float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F2 ds_mul(F2 a, F2 b) {
  const F2 p = two_prod(a.h, b.h);
  return fast_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}

// The same without the final renormalisation (the low part up to ~3 ulps of
// the high one): for a product that only feeds another product or a sum
// whose two_sum takes the high parts exactly.
__device__ __forceinline__ F2 ds_mul_u(F2 a, F2 b) {
  const F2 p = two_prod(a.h, b.h);
  return F2{p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l))};
}

// d (FP64) -> h + l: h is d truncated to 24 significant bits, l the next 23
// bits; |d| < 2^-74 (irrelevant here) maps to 0.
__device__ __forceinline__ F2 split_d(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  const unsigned sg = hi & 0x80000000u;
  const unsigned hb = ((__funnelshift_l(lo, hi, 3) + 0x40000000u) & 0x7fffffffu) | sg;
  const float km = __fsub_rn(__uint_as_float(0x4b000000u | ((lo >> 6) & 0x7fffffu)), 8388608.0f);
  const float sc = __uint_as_float(((ex - 942u) << 23) | sg);  // +-2^(e - 1069)
  const bool ok = ex >= 949u && ex <= 1150u;
  return {ok ? __uint_as_float(hb) : 0.0f, ok ? __fmul_rn(km, sc) : 0.0f};
}

// Float threshold >= rc^2 (1 + 2^-20) for the encounter pre-test.
__device__ __forceinline__ float rc2_threshold(double rc2) {
  const float f = __double2float_ru(rc2);
  return __uint_as_float(__float_as_uint(f) + 16u);
}

constexpr unsigned kDsParkedExp = 1023 + 19;  // |c| >= 2^19 AU: parked bodies, off the grid
// The finest grid: G >= 2^-64 (G2 >= 2^-88, a normal float), so that a parked
// body (up to 2^38 AU) still has a finite float multiple of G (k <= 2^102)
// however small the live coordinates are.
constexpr unsigned kDsMinExp = 981;

// The largest biased exponent among a body's coordinates (0 when parked).
__device__ __forceinline__ unsigned ds_exp_of(double x, double y, double z) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  const unsigned ey = ((unsigned)__double2hiint(y) >> 20) & 0x7ffu;
  const unsigned ez = ((unsigned)__double2hiint(z) >> 20) & 0x7ffu;
  const unsigned e = max(ex, max(ey, ez));
  return e >= kDsParkedExp ? 0u : e;
}

// The grid exponent of a launch: the largest coordinate exponent of all
// bodies (one CTA; ctrl->ds_exp).
constexpr int DGT = 1024;
__global__ void __launch_bounds__(DGT) k_ds_grid(int n, const double* __restrict__ x,
                                                 const double* __restrict__ y,
                                                 const double* __restrict__ z, Ctrl* ctrl) {
  __shared__ unsigned red[DGT / 32];
  unsigned e = kDsMinExp;
  for (int j = threadIdx.x; j < n; j += DGT) e = max(e, ds_exp_of(x[j], y[j], z[j]));
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x < 32) {
    e = red[threadIdx.x];
    e = __reduce_max_sync(0xffffffffu, e);
    if (threadIdx.x == 0) ctrl->ds_exp = (int)e;
  }
}

// A coordinate on two nested grids: c = h + m + l with h = k G and m = k2 G2
// (G2 = 2^-24 G) exact as floats (|k|, |k2| <= 2^23), and l the float
// nearest to the rest c - k G - k2 G2 (both subtractions exact in FP64,
// |.| <= G2 / 2): absolute error <= 2^-25 G2 = 2^-49 G.
struct DsCoord {
  float h, m, l;
};
__device__ __forceinline__ DsCoord ds_coord(double c, double G, double iG, float Gf) {
  const double k = rint(c * iG);
  const double r = __fma_rn(-k, G, c);
  const double k2 = rint(r * (iG * 16777216.0));
  const double r2 = __fma_rn(-k2, G * 0x1p-24, r);
  return {__fmul_rn(__double2float_rn(k), Gf), __fmul_rn(__double2float_rn(k2), Gf * 0x1p-24f),
          __double2float_rn(r2)};
}

// c_j - c_i as a float pair: the multiples of G and of G2 subtract exactly
// (integers below 2^24 times a power of two); a nonzero difference of the
// first (>= G) dominates the second's (<= G), so fast_two_sum joins them
// exactly, and the rests' difference enters the low part: error below
// 2^-48 |dx| + 2^-47 G (2^-66 AU for bodies within 16 AU).
__device__ __forceinline__ F2 ds_diff(const DsCoord& j, const DsCoord& i) {
  const F2 s = fast_two_sum(__fsub_rn(j.h, i.h), __fsub_rn(j.m, i.m));
  return F2{s.h, __fadd_rn(s.l, __fsub_rn(j.l, i.l))};
}

constexpr int DNT2 = 128;  // threads per DS kick CTA (= j-tile size)
constexpr int DIPT = 1;    // targets per thread
#ifndef NB_DS_MINB
#define NB_DS_MINB 5
#endif
constexpr int kDsMinBlocks = NB_DS_MINB;  // CTAs per SM the registers are bounded for (tuning)

__global__ void __launch_bounds__(DNT2, kDsMinBlocks) k_kick_ds(KickArgs A) {
  // a source's 12 floats as three float4 (three shared loads per pair, broadcast):
  // (x.h, x.m, x.l, y.h), (y.m, y.l, z.h, z.m), (z.l, m.h, m.l, threshold)
  __shared__ float4 sA[DNT2], sB[DNT2], sC[DNT2];
  __shared__ int s_stop, s_exp;
  if (threadIdx.x == 0) {
    s_stop = A.ctrl->status || (A.cond && *A.cond == 0);
    s_exp = A.ctrl->ds_exp;
  }
  __syncthreads();
  if (s_stop) return;
  const unsigned ge = (unsigned)s_exp - 22u;  // biased exponent of G
  const double G = __longlong_as_double((long long)ge << 52);
  const double iG = __longlong_as_double((long long)(2046u - ge) << 52);
  const float Gf = __uint_as_float((ge - 896u) << 23);
  const int n = A.n;
  const int it = blockIdx.x / A.S;
  const int sidx = blockIdx.x - it * A.S;
  const int i0 = A.ib + it * (DNT2 * DIPT) + threadIdx.x;
  DsCoord cx[DIPT], cy[DIPT], cz[DIPT];
  double rc2i[DIPT], rci[DIPT];
  double ax[DIPT], ay[DIPT], az[DIPT];
  float thi[DIPT];
  int ii[DIPT];
#pragma unroll
  for (int k = 0; k < DIPT; ++k) {
    const int i = i0 + k * DNT2;
    ii[k] = i;
    double xi = 1e10, yi = 1e10, zi = 1e10;
    if (i < A.ie) {
      xi = A.x[i]; yi = A.y[i]; zi = A.z[i];
      rc2i[k] = A.rc2[i]; rci[k] = A.rc[i];
    } else {
      rc2i[k] = 0.0; rci[k] = 0.0;
    }
    cx[k] = ds_coord(xi, G, iG, Gf);
    cy[k] = ds_coord(yi, G, iG, Gf);
    cz[k] = ds_coord(zi, G, iG, Gf);
    thi[k] = rc2_threshold(rc2i[k]);
    ax[k] = ay[k] = az[k] = 0.0;
  }
  const int j0 = sidx * A.jchunk;
  const int j1 = min(n, j0 + A.jchunk);
  for (int jt = j0; jt < j1; jt += DNT2) {
    __syncthreads();
    const int j = jt + threadIdx.x;
    if (j < j1) {
      const DsCoord qx = ds_coord(A.x[j], G, iG, Gf), qy = ds_coord(A.y[j], G, iG, Gf),
                    qz = ds_coord(A.z[j], G, iG, Gf);
      const F2 mm = split_d(A.m[j]);
      sA[threadIdx.x] = make_float4(qx.h, qx.m, qx.l, qy.h);
      sB[threadIdx.x] = make_float4(qy.m, qy.l, qz.h, qz.m);
      sC[threadIdx.x] = make_float4(qz.l, mm.h, mm.l, rc2_threshold(A.rc2[j]));
    }
    __syncthreads();
    const int cnt = min(DNT2, j1 - jt);
    F2 tx[DIPT], ty[DIPT], tz[DIPT];
#pragma unroll
    for (int k = 0; k < DIPT; ++k) tx[k] = ty[k] = tz[k] = F2{0.0f, 0.0f};
#pragma unroll 2
    for (int q = 0; q < cnt; ++q) {
      const float4 va = sA[q], vb = sB[q], vc = sC[q];
      const DsCoord qx{va.x, va.y, va.z}, qy{va.w, vb.x, vb.y}, qz{vb.z, vb.w, vc.x};
      const F2 mj{vc.y, vc.z};
      const float thj = vc.w;
#pragma unroll
      for (int k = 0; k < DIPT; ++k) {
        F2 fx = ds_diff(qx, cx[k]), fy = ds_diff(qy, cy[k]), fz = ds_diff(qz, cz[k]);
        // r^2 as a float pair (the 2^-48-relative squares of the low parts dropped)
        F2 px = two_prod(fx.h, fx.h), py = two_prod(fy.h, fy.h), pz = two_prod(fz.h, fz.h);
        px.l = __fmaf_rn(__fmul_rn(2.0f, fx.h), fx.l, px.l);
        py.l = __fmaf_rn(__fmul_rn(2.0f, fy.h), fy.l, py.l);
        pz.l = __fmaf_rn(__fmul_rn(2.0f, fz.h), fz.l, pz.l);
        F2 t = two_sum(px.h, py.h);
        t.l = __fadd_rn(t.l, __fadd_rn(px.l, py.l));
        F2 u = two_sum(t.h, pz.h);
        u.l = __fadd_rn(u.l, __fadd_rn(t.l, pz.l));
        const F2 r2 = fast_two_sum(u.h, u.l);
        // r^-1: float seed y0, residual e = 1 - r^2 y0^2 kept as e_h + e_l,
        // y1 = y0 (1 + e/2 + 3 e^2 / 8)
        const float y0 = rsqrtf(r2.h);
        const F2 q2 = two_prod(y0, y0);
        const F2 s = ds_mul_u(r2, q2);
        const float eh = __fsub_rn(1.0f, s.h);  // exact (Sterbenz)
        // y0 e / 2 = (c.h + c.l - y0 s.l) / 2 with y0 eh = c.h + c.l exactly;
        // the 3 y0 e^2 / 8 term enters the low part as 0.75 y0 eh^2 / 2
        const F2 c = two_prod(y0, eh);
        const float cl =
            __fmaf_rn(__fmul_rn(0.75f, y0), __fmul_rn(eh, eh), __fmaf_rn(y0, -s.l, c.l));
        const F2 yy = fast_two_sum(y0, __fmul_rn(0.5f, c.h));
        const F2 y1{yy.h, __fmaf_rn(0.5f, cl, yy.l)};
        // m_j r^-3 = m_j y1^3
        const F2 y12 = ds_mul_u(y1, y1);
        F2 sc = ds_mul(mj, ds_mul_u(y12, y1));
        if (r2.h <= fmaxf(thi[k], thj)) {
          // possible encounter (or coincident bodies): the exact FP64 branch,
          // from the FP64 positions
          const int i = ii[k] < A.ie ? ii[k] : A.ie - 1, jj = jt + q;
          const double dx = __ldg(A.x + jj) - __ldg(A.x + i), dy = __ldg(A.y + jj) - __ldg(A.y + i),
                       dz = __ldg(A.z + jj) - __ldg(A.z + i);
          const double r2d = ii[k] < A.ie ? sep2(dx, dy, dz) : 1e20;
          const double s64 = rare_pair<true>(r2d, scale_fast<NB_PREC_FP64>(r2d, A.m[jj]),
                                             A.m[jj], ii[k], jj, rc2i[k], rci[k], A);
          sc = split_d(s64);
          fx = split_d(dx);
          fy = split_d(dy);
          fz = split_d(dz);
        }
        const F2 gx = ds_mul_u(sc, fx), gy = ds_mul_u(sc, fy), gz = ds_mul_u(sc, fz);
        F2 w = two_sum(tx[k].h, gx.h);
        tx[k] = F2{w.h, __fadd_rn(w.l, __fadd_rn(tx[k].l, gx.l))};
        w = two_sum(ty[k].h, gy.h);
        ty[k] = F2{w.h, __fadd_rn(w.l, __fadd_rn(ty[k].l, gy.l))};
        w = two_sum(tz[k].h, gz.h);
        tz[k] = F2{w.h, __fadd_rn(w.l, __fadd_rn(tz[k].l, gz.l))};
      }
    }
#pragma unroll
    for (int k = 0; k < DIPT; ++k) {
      ax[k] += (double)tx[k].h + (double)tx[k].l;
      ay[k] += (double)ty[k].h + (double)ty[k].l;
      az[k] += (double)tz[k].h + (double)tz[k].l;
    }
  }
#pragma unroll
  for (int k = 0; k < DIPT; ++k) {
    const int i = ii[k];
    if (i < A.ie) {
      double* p = A.kpart + (size_t)(3 * sidx) * n;
      p[i] = ax[k];
      p[n + i] = ay[k];
      p[2 * n + i] = az[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Double-single unordered-pair kick (NB_PREC_DS, whole system): the tile
// schedule, rotation and partial sums of k_kick_sym with the pair arithmetic
// of k_kick_ds. Per pair {i, j} the float-pair differences, r^2 and r^-3 = y1^3
// once (y1 the refined float-pair r^-1), then m_j r^-3 and m_i r^-3, the
// products with dx, dy, dz and the float-pair sums of both sides. The row
// side's sums are float pairs over a tile (128 pairs) folded into FP64, the
// column side's float pairs over a 32-pair sub-tile, folded into FP64 and
// added over the four warps in warp order. A pair whose float r^2 passes the
// encounter pre-test takes the exact FP64 branch of k_kick_sym (from the FP64
// positions), so flags are identical to the FP64 kicks'.
// ---------------------------------------------------------------------------
#ifndef NB_DS_SYM_MINB
#define NB_DS_SYM_MINB 5
#endif
constexpr int kDsSymMinBlocks = NB_DS_SYM_MINB;  // CTAs per SM the registers are bounded for

// dx, dy, dz, r^2 (high part) and r^-3 of a source staged as three float4
// (x.h, x.m, x.l, y.h), (y.m, y.l, z.h, z.m), (z.l, m.h, m.l, threshold)
// against a target's grid coordinates: the arithmetic of k_kick_ds.
struct DsPairTerm {
  F2 fx, fy, fz, r3;
  float r2h;
};
__device__ __forceinline__ DsPairTerm ds_pair_term(const float4& va, const float4& vb,
                                                   const float4& vc, const DsCoord& cx,
                                                   const DsCoord& cy, const DsCoord& cz) {
  DsPairTerm o;
  const DsCoord qx{va.x, va.y, va.z}, qy{va.w, vb.x, vb.y}, qz{vb.z, vb.w, vc.x};
  o.fx = ds_diff(qx, cx);
  o.fy = ds_diff(qy, cy);
  o.fz = ds_diff(qz, cz);
  F2 px = two_prod(o.fx.h, o.fx.h), py = two_prod(o.fy.h, o.fy.h), pz = two_prod(o.fz.h, o.fz.h);
  px.l = __fmaf_rn(__fmul_rn(2.0f, o.fx.h), o.fx.l, px.l);
  py.l = __fmaf_rn(__fmul_rn(2.0f, o.fy.h), o.fy.l, py.l);
  pz.l = __fmaf_rn(__fmul_rn(2.0f, o.fz.h), o.fz.l, pz.l);
  F2 t = two_sum(px.h, py.h);
  t.l = __fadd_rn(t.l, __fadd_rn(px.l, py.l));
  F2 u = two_sum(t.h, pz.h);
  u.l = __fadd_rn(u.l, __fadd_rn(t.l, pz.l));
  const F2 r2 = fast_two_sum(u.h, u.l);
  const float y0 = rsqrtf(r2.h);
  const F2 q2 = two_prod(y0, y0);
  const F2 s = ds_mul_u(r2, q2);
  const float eh = __fsub_rn(1.0f, s.h);
  const F2 c = two_prod(y0, eh);
  const float cl = __fmaf_rn(__fmul_rn(0.75f, y0), __fmul_rn(eh, eh), __fmaf_rn(y0, -s.l, c.l));
  const F2 yy = fast_two_sum(y0, __fmul_rn(0.5f, c.h));
  const F2 y1{yy.h, __fmaf_rn(0.5f, cl, yy.l)};
  o.r3 = ds_mul(ds_mul_u(y1, y1), y1);
  o.r2h = r2.h;
  return o;
}

// The exact FP64 branch for a pair that passed the float pre-test: r^2 from
// the FP64 positions, the scales of k_kick_sym (seeded r^-3 beyond rc, the
// changeover weight inside, 0 for coincident bodies) and the flag; the
// differences and scales are returned as float pairs.
template <bool DIAG>
__device__ __forceinline__ void ds_sym_rare(int i, int j, const KickArgs& A, DsPairTerm& p,
                                            F2& sj, F2& si) {
  if (i >= A.n || j >= A.n) return;  // padding: massless, far, never flagged
  const double dx = __ldg(A.x + j) - __ldg(A.x + i), dy = __ldg(A.y + j) - __ldg(A.y + i),
               dz = __ldg(A.z + j) - __ldg(A.z + i);
  const double mj = __ldg(A.m + j), mi = __ldg(A.m + i);
  const double r2 = sep2(dx, dy, dz);
  const double r3 = r2 > 0.0 ? rinv3_fast(r2) : 0.0;
  double sj64 = mj * r3, si64 = mi * r3;
  sym_rare<DIAG>(i, j, mi, mj, A, sj64, si64);
  sj = split_d(sj64);
  si = split_d(si64);
  p.fx = split_d(dx);
  p.fy = split_d(dy);
  p.fz = split_d(dz);
}

// s += g as a float pair (the sums' two_sum on the high parts, the low parts added)
__device__ __forceinline__ void ds_acc(F2& s, const F2& g) {
  const F2 w = two_sum(s.h, g.h);
  s = F2{w.h, __fadd_rn(w.l, __fadd_rn(s.l, g.l))};
}

__global__ void __launch_bounds__(KNT, kDsSymMinBlocks) k_kick_ds_sym(KickArgs A, SymArgs L) {
  __shared__ float4 sA[KNT], sB[KNT], sC[KNT];  // block Y, as staged by k_kick_ds
  __shared__ double sacc[3][4][KNT];            // the warps' column sums of a tile
  __shared__ int s_stop, s_exp;
  if (threadIdx.x == 0) {
    s_stop = A.ctrl->status || (A.cond && *A.cond == 0);
    s_exp = A.ctrl->ds_exp;
  }
  __syncthreads();
  if (s_stop) return;
  const unsigned ge = (unsigned)s_exp - 22u;  // biased exponent of G
  const double G = __longlong_as_double((long long)ge << 52);
  const double iG = __longlong_as_double((long long)(2046u - ge) << 52);
  const float Gf = __uint_as_float((ge - 896u) << 23);
  const int n = A.n;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int H1 = L.hrow + 1;
  const int f0 = blockIdx.x * L.per;
  const int f1 = min(L.tiles, f0 + L.per);
  int X = -1, seg = 0, i = 0;
  DsCoord cx{0.0f, 0.0f, 0.0f}, cy = cx, cz = cx;
  F2 mi{0.0f, 0.0f};
  float thi = 0.0f;
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int f = f0; f < f1; ++f) {
    const int Xf = f / H1, dd = f - Xf * H1;
    if (Xf != X) {
      if (X >= 0) {
        double* p = L.xpart + (size_t)((blockIdx.x * 2 + seg) * 3) * KNT + threadIdx.x;
        p[0] = ax;
        p[KNT] = ay;
        p[2 * KNT] = az;
        seg = 1;
      }
      X = Xf;
      i = X * KNT + threadIdx.x;
      const bool live = i < n;
      cx = ds_coord(live ? A.x[i] : 1e10, G, iG, Gf);
      cy = ds_coord(live ? A.y[i] : 1e10, G, iG, Gf);
      cz = ds_coord(live ? A.z[i] : 1e10, G, iG, Gf);
      mi = live ? split_d(A.m[i]) : F2{0.0f, 0.0f};
      thi = rc2_threshold(live ? A.rc2[i] : 0.0);
      ax = ay = az = 0.0;
    }
    if (2 * dd == L.nb && X >= L.nb / 2) continue;  // the lower block covers this pair
    int Yb = X + dd;
    if (Yb >= L.nb) Yb -= L.nb;
    const int jb = Yb * KNT;
    __syncthreads();
    {
      const int j = jb + threadIdx.x;
      const bool live = j < n;
      const DsCoord qx = ds_coord(live ? A.x[j] : 1e10, G, iG, Gf),
                    qy = ds_coord(live ? A.y[j] : 1e10, G, iG, Gf),
                    qz = ds_coord(live ? A.z[j] : 1e10, G, iG, Gf);
      const F2 mm = live ? split_d(A.m[j]) : F2{0.0f, 0.0f};
      sA[threadIdx.x] = make_float4(qx.h, qx.m, qx.l, qy.h);
      sB[threadIdx.x] = make_float4(qy.m, qy.l, qz.h, qz.m);
      sC[threadIdx.x] = make_float4(qz.l, mm.h, mm.l, rc2_threshold(live ? A.rc2[j] : 0.0));
    }
    __syncthreads();
    F2 tx{0.0f, 0.0f}, ty = tx, tz = tx;  // this body's sums over the tile
    if (dd == 0) {
      // the block with itself: every ordered pair, this body's side only
#pragma unroll 1
      for (int q = 0; q < KNT; ++q) {
        const float4 va = sA[q], vb = sB[q], vc = sC[q];
        DsPairTerm p = ds_pair_term(va, vb, vc, cx, cy, cz);
        F2 sj = ds_mul(F2{vc.y, vc.z}, p.r3), si{0.0f, 0.0f};
        if (p.r2h <= fmaxf(thi, vc.w)) ds_sym_rare<true>(i, jb + q, A, p, sj, si);
        ds_acc(tx, ds_mul_u(sj, p.fx));
        ds_acc(ty, ds_mul_u(sj, p.fy));
        ds_acc(tz, ds_mul_u(sj, p.fz));
      }
    } else {
#pragma unroll 1
      for (int u = 0; u < 4; ++u) {
        F2 bx{0.0f, 0.0f}, by = bx, bz = bx;  // column sums, one lane down per step
#pragma unroll 1
        for (int s = 0; s < 32; ++s) {
          const int q = 32 * u + ((lane + s) & 31);
          const float4 va = sA[q], vb = sB[q], vc = sC[q];
          DsPairTerm p = ds_pair_term(va, vb, vc, cx, cy, cz);
          F2 sj = ds_mul(F2{vc.y, vc.z}, p.r3), si = ds_mul(mi, p.r3);
          if (p.r2h <= fmaxf(thi, vc.w)) ds_sym_rare<false>(i, jb + q, A, p, sj, si);
          ds_acc(tx, ds_mul_u(sj, p.fx));
          ds_acc(ty, ds_mul_u(sj, p.fy));
          ds_acc(tz, ds_mul_u(sj, p.fz));
          const F2 gx = ds_mul_u(si, p.fx), gy = ds_mul_u(si, p.fy), gz = ds_mul_u(si, p.fz);
          ds_acc(bx, F2{-gx.h, -gx.l});
          ds_acc(by, F2{-gy.h, -gy.l});
          ds_acc(bz, F2{-gz.h, -gz.l});
          const int src = (lane + 1) & 31;
          bx.h = __shfl_sync(0xffffffffu, bx.h, src);
          bx.l = __shfl_sync(0xffffffffu, bx.l, src);
          by.h = __shfl_sync(0xffffffffu, by.h, src);
          by.l = __shfl_sync(0xffffffffu, by.l, src);
          bz.h = __shfl_sync(0xffffffffu, bz.h, src);
          bz.l = __shfl_sync(0xffffffffu, bz.l, src);
        }
        sacc[0][wp][32 * u + lane] = (double)bx.h + (double)bx.l;
        sacc[1][wp][32 * u + lane] = (double)by.h + (double)by.l;
        sacc[2][wp][32 * u + lane] = (double)bz.h + (double)bz.l;
      }
    }
    ax += (double)tx.h + (double)tx.l;
    ay += (double)ty.h + (double)ty.l;
    az += (double)tz.h + (double)tz.l;
    if (dd == 0) continue;
    __syncthreads();
    double* p = L.ypart + ((size_t)Yb * L.hrow + (dd - 1)) * 3 * KNT + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      p[c * KNT] = ((sacc[c][0][threadIdx.x] + sacc[c][1][threadIdx.x]) + sacc[c][2][threadIdx.x]) +
                   sacc[c][3][threadIdx.x];
  }
  if (X >= 0) {
    double* p = L.xpart + (size_t)((blockIdx.x * 2 + seg) * 3) * KNT + threadIdx.x;
    p[0] = ax;
    p[KNT] = ay;
    p[2 * KNT] = az;
  }
}

// CTAs of a kick launch: target tiles (KNT KIPT targets, DNT2 DIPT for the
// double-single kernel) x S j-chunks
int kick_blocks(int n, int S, int precision) {
  const int t = precision == NB_PREC_DS ? DNT2 * DIPT : KNT * KIPT;
  return ((n + t - 1) / t) * S;
}

static void launch_kick_args(const KickArgs& A, int precision, cudaStream_t st) {
  const int grid = kick_blocks(A.ie - A.ib, A.S, precision);
  if (grid <= 0) return;
  if (precision == NB_PREC_MIXED)
    k_kick<NB_PREC_MIXED><<<grid, KNT, 0, st>>>(A);
  else if (precision == NB_PREC_DS) {
    k_ds_grid<<<1, DGT, 0, st>>>(A.n, A.x, A.y, A.z, A.ctrl);
    k_kick_ds<<<grid, DNT2, 0, st>>>(A);
  }
  else
    k_kick<NB_PREC_FP64><<<grid, KNT, 0, st>>>(A);
}

// Sources per j-chunk. Chunks above 4 tiles take whole tiles (a partial tile
// at every chunk's end cost 0.4 % at N = 65538); shorter ones any length (the
// tile loop stages partial tiles), so that small systems still spread over
// many CTAs (N = 2049: 1088 CTAs instead of 289, 6 % off the step).
static int jchunk_for(int n, int S) {
  int c = (n + S - 1) / S;
  if (c > 4 * KNT) c = ((c + KNT - 1) / KNT) * KNT;
  return c > 0 ? c : KNT;
}

static void launch_kick_sym(const KickArgs& A, const Dev& d, const Phys& P, cudaStream_t st) {
  SymArgs L;
  L.nb = d.sym_nb;
  L.hrow = d.sym_hrow;
  L.tiles = d.sym_nb * (d.sym_hrow + 1);
  L.per = d.sym_per;
  L.xpart = d.sym_xpart;
  L.ypart = d.sym_ypart;
  if (P.precision == NB_PREC_DS) {
    k_ds_grid<<<1, DGT, 0, st>>>(A.n, A.x, A.y, A.z, A.ctrl);
    k_kick_ds_sym<<<d.sym_grid, KNT, 0, st>>>(A, L);
  } else {
    k_kick_sym<<<d.sym_grid, KNT, 0, st>>>(A, L);
  }
}

void launch_kick(const Dev& d, const Phys& P, int /*target_sel*/, cudaStream_t st) {
  KickArgs A;
  A.n = d.n;
  A.S = d.S;
  A.jchunk = jchunk_for(d.n, d.S);
  A.ib = d.row0;  // this rank's rows when sharded, else all
  A.ie = d.row1;
  A.cond = nullptr;
  A.x = d.x; A.y = d.y; A.z = d.z; A.m = d.m; A.rc = d.rc; A.rc2 = d.rc2;
  A.kpart = d.kpart;
  A.pairs = d.ftrial;
  A.cap = d.pair_cap;
  A.counter = &d.ctrl->n_ftrial;
  A.ctrl = d.ctrl;
  if (d.sym)
    launch_kick_sym(A, d, P, st);
  else
    launch_kick_args(A, P.precision, st);
}

void launch_kick_raw(int n, int ib, int ie, const double* x, const double* y, const double* z,
                     const double* m, const double* rc, const double* rc2, int S, int precision,
                     double* kpart, int2* pairs, int cap, Ctrl* ctrl, cudaStream_t st) {
  KickArgs A;
  A.n = n; A.S = S; A.jchunk = jchunk_for(n, S);
  A.ib = ib; A.ie = ie;
  A.cond = nullptr;
  A.x = x; A.y = y; A.z = z; A.m = m; A.rc = rc; A.rc2 = rc2;
  A.kpart = kpart; A.pairs = pairs; A.cap = cap; A.counter = &ctrl->n_ftrial; A.ctrl = ctrl;
  launch_kick_args(A, precision, st);
}

// ---------------------------------------------------------------------------
// k_finish: a_i = G sum_s kpart[s] (fixed order). On a step with
// close-encounter groups, bodies outside the groups also get the change of
// the group bodies' pull: minus their contribution at the trial state, plus
// their contribution at the state the BS integration produced. This equals a
// full re-evaluation of the force at the final positions up to rounding (the
// only pairs whose terms change are those with a group member).
// ---------------------------------------------------------------------------
constexpr int FNT = 256;

// m_j w / r^3 as the kick computes it: the seeded reciprocal root beyond
// rc_ij (m_j with 1.5 m_j and 1.875 m_j in the row kick, m_j times the seeded
// r^-3 in the unordered-pair kick), the exact changeover weight inside, 0 for
// coincident bodies; the range test compares bit patterns.
__device__ __forceinline__ double finish_scale(double dx, double dy, double dz, const double* sj,
                                               int k, double rci, double rc2i, bool sym) {
  const double mj = sj[3 * FNT + k];
  const double r2 = sep2_int(dx, dy, dz);
  // near or inside rc (one high-word unit of slack for the integer r^2), or
  // coincident: the kick's exact branch, decided on the FP64 expression
  if (__double2hiint(r2) <= max(__double2hiint(rc2i), __double2hiint(sj[5 * FNT + k])) + 1) {
    const double r2x = sep2(dx, dy, dz);
    if (nn_less(r2x, rc2i) || nn_less(r2x, sj[5 * FNT + k]) || __double_as_longlong(r2x) == 0ll)
      return pair_scale(r2x, mj, rci, sj[4 * FNT + k]);
  }
  if (sym) return mj * rinv3_fast(r2);
  return scale_fast<NB_PREC_FP64>(r2, mj, sj[6 * FNT + k], sj[7 * FNT + k]);
}

// PH = 0: the whole update in one pass. The step splits it so that the trial
// half can run beside the direct solver: PH = 1 writes the unscaled sum of
// the partials minus the group bodies' trial terms into a; PH = 2 (after the
// direct solver) adds their final terms and applies G and the live mask.
template <int PH>
__global__ void __launch_bounds__(FNT) k_finish_t(Dev d, double G, int with_delta,
                                                 const int* cond) {
  __shared__ int s_stop, s_M;
  // members' trial (so) and final (snw) states: x, y, z, m, rc, rc^2, 1.5 m, 1.875 m
  __shared__ double so[8][FNT], snw[8][FNT];
  if (threadIdx.x == 0) {
    s_stop = d.ctrl->status || (cond && *cond == 0);
    s_M = (with_delta && d.ctrl->n_groups > 0) ? d.ctrl->n_members : 0;
  }
  __syncthreads();
  if (s_stop) return;
  const int n = d.n;
  const int i = blockIdx.x * FNT + threadIdx.x;
  const int M = s_M;
  // this rank's rows (all unless sharded); the closing half leaves the group
  // members' rows to the member re-kick, which recomputes their force in full
  // (and runs beside this kernel)
  const bool row = i >= d.row0 && i < d.row1 && !(PH == 2 && M > 0 && d.member_slot[i] >= 0);
  double ax = 0.0, ay = 0.0, az = 0.0;
  if (row) {
    if (PH == 2) {  // the trial half's result
      ax = d.ax[i]; ay = d.ay[i]; az = d.az[i];
    } else if (d.sym) {
      sym_partials(d, i, ax, ay, az);
    } else {
      for (int s = 0; s < d.S; ++s) {
        const double* p = d.kpart + (size_t)(3 * s) * n;
        ax += p[i];
        ay += p[n + i];
        az += p[2 * n + i];
      }
    }
  }
  const bool delta = row && M > 0 && d.member_slot[i] < 0 && d.alive[i];
  double xi = 0.0, yi = 0.0, zi = 0.0, rci = 0.0, rc2i = 0.0;
  if (delta) {
    xi = d.x[i]; yi = d.y[i]; zi = d.z[i]; rci = d.rc[i]; rc2i = d.rc2[i];
  }
  double cx = 0.0, cy = 0.0, cz = 0.0;
  for (int q0 = 0; q0 < M; q0 += FNT) {
    __syncthreads();
    const int q = q0 + threadIdx.x;
    if (q < M && PH != 2) {
      int b = d.grp_mem[q];
      if (!NB_GUARD(d.ctrl, b >= 0 && b < d.n, 58)) b = 0;
      so[0][threadIdx.x] = d.x[b];
      so[1][threadIdx.x] = d.y[b];
      so[2][threadIdx.x] = d.z[b];
      const double mo = d.m[b];
      so[3][threadIdx.x] = mo;
      so[4][threadIdx.x] = d.rc[b];
      so[5][threadIdx.x] = d.rc2[b];
      so[6][threadIdx.x] = 1.5 * mo;
      so[7][threadIdx.x] = 1.875 * mo;
    }
    if (q < M && PH != 1) {
      const double* g = d.gnew + (size_t)q * 10;
      snw[0][threadIdx.x] = g[0];
      snw[1][threadIdx.x] = g[1];
      snw[2][threadIdx.x] = g[2];
      const double mn = g[9] != 0.0 ? g[6] : 0.0;  // absorbed: no pull
      snw[3][threadIdx.x] = mn;
      snw[4][threadIdx.x] = g[8];
      snw[5][threadIdx.x] = g[8] * g[8];
      snw[6][threadIdx.x] = 1.5 * mn;
      snw[7][threadIdx.x] = 1.875 * mn;
    }
    __syncthreads();
    if (delta) {
      const int cnt = min(FNT, M - q0);
      for (int k = 0; k < cnt; ++k) {
        // the trial kick's term of member k (same arithmetic as the kick:
        // seeded reciprocal root beyond rc, the exact weight inside), then
        // the term at the member's new state
        if (PH != 2) {
          const double dx = so[0][k] - xi, dy = so[1][k] - yi, dz = so[2][k] - zi;
          const double s = finish_scale(dx, dy, dz, &so[0][0], k, rci, rc2i, d.sym);
          cx -= s * dx; cy -= s * dy; cz -= s * dz;
        }
        if (PH != 1) {
          const double dx = snw[0][k] - xi, dy = snw[1][k] - yi, dz = snw[2][k] - zi;
          const double s = finish_scale(dx, dy, dz, &snw[0][0], k, rci, rc2i, d.sym);
          cx += s * dx; cy += s * dy; cz += s * dz;
        }
      }
    }
  }
  if (row) {
    if (PH == 1) {
      d.ax[i] = ax + cx;
      d.ay[i] = ay + cy;
      d.az[i] = az + cz;
    } else {
      const bool live = d.alive[i] != 0;
      d.ax[i] = live ? G * (ax + cx) : 0.0;
      d.ay[i] = live ? G * (ay + cy) : 0.0;
      d.az[i] = live ? G * (az + cz) : 0.0;
    }
  }
}

void launch_finish(const Dev& d, const Phys& P, int with_delta, cudaStream_t st) {
  const int grid = (d.n + FNT - 1) / FNT;
  k_finish_t<0><<<grid, FNT, 0, st>>>(d, P.G, with_delta, nullptr);
}

void launch_finish_part(const Dev& d, const Phys& P, int part, cudaStream_t st) {
  const int grid = (d.n + FNT - 1) / FNT;
  if (part == 1)
    k_finish_t<1><<<grid, FNT, 0, st>>>(d, P.G, 1, nullptr);
  else
    k_finish_t<2><<<grid, FNT, 0, st>>>(d, P.G, 1, nullptr);
}

void launch_force_anew(const Dev& d, const Phys& P, int only_if_ejected, cudaStream_t st) {
  const int* cond = only_if_ejected ? &d.ctrl->n_eject_step : nullptr;
  KickArgs A;
  A.n = d.n;
  A.S = d.S;
  A.jchunk = jchunk_for(d.n, d.S);
  A.ib = 0;
  A.ie = d.n;
  A.cond = cond;
  A.x = d.x; A.y = d.y; A.z = d.z; A.m = d.m; A.rc = d.rc; A.rc2 = d.rc2;
  A.kpart = d.kpart;
  A.pairs = d.ftrial;
  A.cap = d.pair_cap;
  A.counter = &d.ctrl->n_ftrial;
  A.ctrl = d.ctrl;
  if (d.sym)
    launch_kick_sym(A, d, P, st);
  else
    launch_kick_args(A, P.precision, st);
  k_finish_t<0><<<(d.n + FNT - 1) / FNT, FNT, 0, st>>>(d, P.G, 0, cond);
  launch_fsal_init(d, st, cond);
}

// ---------------------------------------------------------------------------
// k_member_kick: full force on every group member at the final positions and
// the new flag set F (pairs with at least one member; all other pairs keep
// their unflagged trial state). One CTA per member, grid-stride.
// ---------------------------------------------------------------------------
constexpr int MNT = 256;

__global__ void __launch_bounds__(MNT) k_member_kick(Dev d, double G) {
  __shared__ int s_stop, s_M;
  __shared__ double red[3 * 32 + 3];
  if (threadIdx.x == 0) {
    s_stop = d.ctrl->status;
    s_M = d.ctrl->n_groups > 0 ? d.ctrl->n_members : 0;
  }
  __syncthreads();
  if (s_stop) return;
  const int M = s_M;
  const int n = d.n;
  KickArgs A;
  A.rc = d.rc;
  A.rc2 = d.rc2;
  A.pairs = d.fprev;
  A.cap = d.pair_cap;
  A.counter = &d.ctrl->n_fprev;
  A.ctrl = d.ctrl;
  for (int q = blockIdx.x; q < M; q += gridDim.x) {
    const int b = d.grp_mem[q];
    if (!NB_GUARD(d.ctrl, b >= 0 && b < d.n, 59)) continue;
    const bool live = d.alive[b] != 0;
    const double xb = d.x[b], yb = d.y[b], zb = d.z[b], rc2b = d.rc2[b], rcb = d.rc[b];
    const int hb = __double2hiint(rc2b);
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (live) {
      for (int j = threadIdx.x; j < n; j += MNT) {
        const double dx = d.x[j] - xb, dy = d.y[j] - yb, dz = d.z[j] - zb;
        const double mj = d.m[j];
        double r2 = sep2_int(dx, dy, dz);
        double sc = scale_fast<NB_PREC_FP64>(r2, mj);
        if (__double2hiint(r2) <= max(hb, __double2hiint(d.rc2[j])) + 1) {
          // flag from the member side: (b, j) when j is not a member or b < j;
          // decided on the FP64 expression of r^2, as in the kick
          r2 = sep2(dx, dy, dz);
          double s = sc;
          const double rc2 = fmax(rc2b, d.rc2[j]);
          const bool close = (r2 < rc2) && d.alive[j] && (j != b);
          const bool flag = close && ((d.member_slot[j] < 0) || (b < j));
          if (r2 == 0.0) {
            s = 0.0;
          } else if (close) {
            const double r = sqrt(r2);
            s = mj * kick_weight(r, fmax(rcb, d.rc[j])) / (r2 * r);
          }
          emit_pair(flag, min(b, j), max(b, j), A.pairs, A.cap, A.counter, A.ctrl);
          sc = s;
        }
        ax = __fma_rn(sc, dx, ax);
        ay = __fma_rn(sc, dy, ay);
        az = __fma_rn(sc, dz, az);
      }
    }
    block_sum3(ax, ay, az, red);
    if (threadIdx.x == 0) {
      d.ax[b] = live ? G * ax : 0.0;
      d.ay[b] = live ? G * ay : 0.0;
      d.az[b] = live ? G * az : 0.0;
    }
  }
}

void launch_member_kick(const Dev& d, const Phys& P, cudaStream_t st) {
  int grid = d.n < 4 * 148 ? d.n : 4 * 148;
  if (grid < 1) grid = 1;
  k_member_kick<<<grid, MNT, 0, st>>>(d, P.G);
}

}  // namespace nb
