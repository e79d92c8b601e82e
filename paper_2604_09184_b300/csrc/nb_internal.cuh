// Internal declarations of libnb: device state layout, control block and the
// device-side physics shared by the kernels of this library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <vector>

#include "nb.h"

namespace nb {

constexpr int kMaxBsK = 12;          // upper bound on bs_kmax
constexpr int kStatN = 14;           // device statistics counters
constexpr int kMlMax = 3;            // deepest multi-level changeover supported
constexpr double kDeadOffset = 1e6;  // absorbed bodies sit at (1e6 (id + 1), 0, 0) AU
// Largest accepted |coordinate| of a live body (the kick's fixed-point
// positions are exact below 2^38 AU).
constexpr double kPosMax = 0x1p37;

// Unordered-pair kick: blocks of kSymBlock bodies, the tile list cut into
// equal ranges, one per CTA, for about NB_SYM_WAVES waves of 8 CTAs per SM on
// 148 SMs (the block scheduler then evens out the SMs: at N = 65538 one wave
// of 112-tile ranges took 40.9 ms, 4, 8 and 16 waves 39.2, 38.4 and 38.0 ms),
// and at least one CTA per block, so that a range spans at most two block
// rows. The grid is fixed by n alone, so the partial sums (and the results)
// do not depend on the device. Automatic selection covers
// kSymMinN <= n <= kSymMaxN (the column partials take 3 x 8 bytes per body
// per block of the other half: 6.4 GB at kSymMaxN).
#ifndef NB_SYM_MINB
#define NB_SYM_MINB 8
#endif
#ifndef NB_SYM_WAVES
#define NB_SYM_WAVES 16
#endif
constexpr int kSymBlock = 128;
constexpr int kSymCtasPerSm = NB_SYM_MINB;  // CTAs per SM the registers are bounded for
constexpr int kSymWave = 148 * kSymCtasPerSm * NB_SYM_WAVES;
constexpr int kSymMinN = 4096;  // kick 0.237 against 0.270 ms at 4096, 0.163 against 0.092 at 2050
constexpr int kSymMaxN = 262144;
struct SymLayout {
  int nb, hrow, tiles, per, grid;
  size_t doubles;  // xpart + ypart
};
inline SymLayout sym_layout(int n) {
  SymLayout L;
  L.nb = (n + kSymBlock - 1) / kSymBlock;
  L.hrow = L.nb / 2;
  L.tiles = L.nb * (L.hrow + 1);
  int g = ((L.nb + kSymWave - 1) / kSymWave) * kSymWave;
  if (g > L.tiles) g = L.tiles;
  L.per = (L.tiles + g - 1) / g;
  L.grid = (L.tiles + L.per - 1) / L.per;
  L.doubles = (size_t)L.grid * 2 * 3 * kSymBlock + (size_t)L.nb * L.hrow * 3 * kSymBlock;
  return L;
}

// Bulirsch-Stoer scratch per group member (doubles): y[6] | f0[6] | per
// extrapolation column j = 1..kmax: zm[6] zc[6] f[6] | T[2][kmax][6] | aux[4].
__host__ __device__ constexpr int bs_off_col(int j) { return 12 + 18 * (j - 1); }
__host__ __device__ constexpr int bs_off_T(int kmax) { return 12 + 18 * kmax; }
__host__ __device__ constexpr int bs_stride_for_kmax(int kmax) { return 16 + 30 * kmax; }

enum StatIdx {
  ST_STEPS = 0,
  ST_FORCE_EVALS,
  ST_ENC_PAIRS,
  ST_GROUPS,
  ST_BS_SUBSTEPS,
  ST_BS_HALVINGS,
  ST_BS_DERIVS,
  ST_MERGES,
  ST_KEPLER_ITERS,
  ST_MOVED,
  ST_LOG_DROPPED,
  ST_EJECTIONS,
  ST_ML_SUBSTEPS,
  ST_ML_GROUPS
};

// Control block in device memory: counters, status and per-step scalars.
struct Ctrl {
  int status;      // first error wins (NB_E_*), 0 while healthy
  int err_where;   // which kernel set it
  int n_ftrial;    // flagged pairs found by the trial kick
  int n_fprev;     // flagged pairs of the cached force (F_prev)
  int n_enc;       // |E| of the current step
  int n_log;       // encounter-log entries written in this nb_step call
  int n_groups;    // close-encounter groups of the current step
  int n_members;   // bodies in those groups
  int n_active;    // bodies not absorbed
  int n_prev_members;
  int pad[2];
  long long step_index;  // global step counter
  double h;              // step size of the current nb_step call
  double E_lost;         // energy removed by mergers
  double dP[3];          // momentum change of group bodies in the current step
  unsigned long long stats[kStatN];
  double m_ejected;  // mass removed beyond eject_r
  int n_eject_step;  // bodies removed at the start of the current step
  int ds_exp;        // the double-single kick's grid: the largest coordinate exponent
};

// Device arrays carved from the caller's workspace (SoA, FP64).
struct Dev {
  int n;          // body slots (fixed; absorbed bodies stay as massless slots)
  int S;          // j-chunks of the kick
  int pair_cap;   // F_trial / F_prev capacity (pairs)
  int log_cap;    // encounter log capacity (entries)
  int member_cap; // group-member capacity (= n)
  int bs_kmax;
  int ppart_n;    // blocks of the O(N) kernels (P partial sums)
  int row0, row1; // target rows of the kick and of the row-wise force finish: [0, n)
                  // unless the system is sharded across ranks (nb_set_shard)
  double *x, *y, *z, *vx, *vy, *vz, *m, *R, *rc, *rc2, *ax, *ay, *az;
  double *xs, *ys, *zs, *vxs, *vys, *vzs;  // saved state after C(h/2)
  int *id, *alive, *member_slot, *uf;
  double* kpart;      // S x 3 x n partial kick sums
  // Unordered-pair kick (each pair evaluated once, FP64, whole system): sym
  // selects it for the step's kicks; sym_nb blocks of kSymBlock bodies,
  // sym_hrow off-diagonal tiles per block row, sym_per tiles per CTA;
  // sym_xpart holds the CTAs' row sums (grid x 2 x 3 x kSymBlock), sym_ypart
  // one partial per tile for its column block (sym_nb x sym_hrow x 3 x
  // kSymBlock). Both live in the kpart allocation.
  int sym, sym_ok, sym_nb, sym_hrow, sym_per, sym_grid;
  double* sym_xpart;
  double* sym_ypart;
  double* ppartA;     // 3 x ppart_n partial momenta (after the opening kick)
  double* ppartB;     // 3 x ppart_n partial momenta (after the drift)
  int2* ftrial;       // pairs of the trial kick
  int2* fprev;        // pairs of the cached force
  unsigned long long* keys;  // sort buffer, 8 x pair_cap
  int* log;           // 3 x log_cap
  int* grp_off;       // member_cap + 1
  int* grp_mem;       // member_cap (body index per member slot)
  double* gscr;       // BS scratch, member_cap x bs_stride doubles
  int bs_stride;
  double* gnew;       // member_cap x 10: x y z vx vy vz m R rc alive(as double)
  double* gEl;        // per-group energy removed by mergers (member_cap)
  double* snap;       // rollback snapshot: 16 x n doubles
  int* snap_i;        // rollback snapshot ints: alive (n) + fprev (2 x pair_cap)
  Ctrl* ctrl;
  Ctrl* snap_ctrl;
  double* eparts;     // energy partial sums
  int eparts_n;
  // multi-level changeover (allocated when ml_levels > 0): a second BS
  // scratch region where the last level's subgroups are gathered, and per
  // level member lists and union-find parents
  double* ml_gscr;    // member_cap x bs_stride
  double* ml_gnew;    // member_cap x 10
  int* ml_list;       // (kMlMax + 1) x member_cap
  int* ml_parent;     // (kMlMax + 1) x member_cap
};

// Parameters as the kernels see them.
struct Phys {
  double G, m0, mu, dt_rcrit, hill_factor, vel_factor, bs_tol;
  int vel_mode, merge, precision, kepler_max_iter, bs_kmax, bs_max_halvings, rcrit_refresh;
  int gas, gas_iter, bs_cluster_min, ml_levels, ml_factor, bs_speculate;
  double gas_rho0, gas_p, gas_eta, gas_cd, eject_r;
};

__device__ __forceinline__ void set_status(Ctrl* c, int code, int where) {
  if (atomicCAS(&c->status, 0, code) == 0) c->err_where = where;
}

// Index checks of the debug build (NB_DEBUG, libnb_debug.so): an index taken
// from device data (a pair list, a member list) that falls outside its array
// sets NB_E_INVALID with the site's code and the access is skipped. In the
// release build the check compiles to `true`.
#ifdef NB_DEBUG
__device__ __forceinline__ bool nb_guard(Ctrl* c, bool ok, int where) {
  if (!ok) set_status(c, NB_E_INVALID, where);
  return ok;
}
#define NB_GUARD(ctrl, cond, where) nb::nb_guard((ctrl), (cond), (where))
#else
#define NB_GUARD(ctrl, cond, where) true
#endif

// ---------------------------------------------------------------------------
// Changeover (the paragraph after Eq. Hc): K goes smoothly from 0 at 0.1 rc to
// 1 at rc. Infinitely differentiable switch in y = (r - 0.1 rc) / (0.9 rc):
// K = f(y) / (f(y) + f(1 - y)) with f(y) = exp(-1/y), so every derivative
// vanishes at both edges and the extrapolation of the close-encounter solver
// stays valid across them. Returns the kick weight w = K - r dK/dr: the pair
// force of Eq. Hb is G m_i m_j w (x_j - x_i) / r^3 and the close part of
// Eq. Ha carries 1 - w.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double kick_weight(double r, double rc) {
  const double y = (r - 0.1 * rc) / (0.9 * rc);
  if (y <= 0.0) return 0.0;
  if (y >= 1.0) return 1.0;
  const double u = 1.0 - y;
  const double f = exp(-1.0 / y), g = exp(-1.0 / u);
  const double s = f + g;
  const double fg = f * g;
  // dK/dy = f g (1/y^2 + 1/(1-y)^2) / (f + g)^2, zero where f g underflows
  const double dKdy = fg > 0.0 ? fg * (1.0 / (y * y) + 1.0 / (u * u)) / (s * s) : 0.0;
  return f / s - r * dKdy / (0.9 * rc);
}

// ---------------------------------------------------------------------------
// FP64 reciprocal roots and reciprocals with few FP64 instructions: a float
// seed from the MUFU unit (float built from the double's high word by one
// integer shift-add, returned to a double by integer ops), refined in FP64.
// ---------------------------------------------------------------------------
// rsqrtf seed of r^2 > 0 rounded toward zero to a float; 2^-126 <= r^2 < 2^128.
// rsqrt_seed_bits returns the float's bit pattern, rsqrt_seed the same value
// as a double.
__device__ __forceinline__ unsigned rsqrt_seed_bits(double r2) {
  const unsigned hr = (unsigned)__double2hiint(r2);
  const float r2f = __uint_as_float((hr << 3) + 0x40000000u);
  return __float_as_uint(rsqrtf(r2f));
}
__device__ __forceinline__ double rsqrt_seed(double r2) {
  const unsigned yb = rsqrt_seed_bits(r2);
  return __hiloint2double((int)((yb >> 3) + 0x38000000u), (int)(yb << 29));
}

// Powers of a positive normal float y0 (bit pattern yb) as doubles, by integer
// arithmetic on its 24-bit significand s: t = y0^2 exactly (s^2 has 48 bits)
// and y3 = y0^3 rounded to 53 bits (s^3 has 72 bits; the lowest 8 are dropped
// before the rounding, so ties may round either way). For y0 in
// [2^-64, 2^64] both are normal doubles. Host-callable so that the bit
// arithmetic can be checked against exact integer products on the CPU.
struct SeedPow {
  double t, y3;
};
__host__ __device__ __forceinline__ int nb_clzll(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}
__host__ __device__ __forceinline__ SeedPow seed_powers(unsigned yb) {
  const unsigned s = (yb & 0x7fffffu) | 0x800000u;
  const unsigned ey = yb >> 23;  // biased float exponent (y0 > 0)
  // s^2 in [2^46, 2^48): shift its leading bit to position 52 and add the
  // exponent field (the leading bit itself carries one unit into it)
  const unsigned long long P = (unsigned long long)s * s;
  const unsigned top = (unsigned)(P >> 47);
  const unsigned long long Qt = P << (6u - top);
  const unsigned long long bt = Qt + ((unsigned long long)(2u * ey + 768u + top) << 52);
  // s^3 / 2^8 in [2^61, 2^64), rounded at bit L - 53 to 53 significant bits
  const unsigned long long A = (unsigned long long)(unsigned)P * s;          // < 2^56
  const unsigned long long B = (unsigned long long)(unsigned)(P >> 32) * s;  // < 2^40
  const unsigned long long R8 = (B << 24) + (A >> 8);
  const int L = 63 - nb_clzll(R8);
  const unsigned long long Q3 = (R8 + (1ull << (L - 53))) >> (L - 52);
  const unsigned long long b3 = Q3 + ((unsigned long long)(L + 3 * (int)ey + 580) << 52);
  SeedPow r;
#ifdef __CUDA_ARCH__
  r.t = __longlong_as_double((long long)bt);
  r.y3 = __longlong_as_double((long long)b3);
#else
  __builtin_memcpy(&r.t, &bt, 8);
  __builtin_memcpy(&r.y3, &b3, 8);
#endif
  return r;
}

// Order of non-negative doubles by their bit patterns (integer compares and
// selects, off the FP64 pipe).
__device__ __forceinline__ bool nn_less(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ double nn_max(double a, double b) { return nn_less(a, b) ? b : a; }
__device__ __forceinline__ double nn_min(double a, double b) { return nn_less(a, b) ? a : b; }

// m / r^3 from the seed y0 ~ r^-1: with e = 1 - r^2 y0^2 (exact residual,
// |e| < 2e-6), r^-3 = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 3e/2 + 15e^2/8 + ...).
// The FP64 mode keeps the e^2 term (truncation ~2^-56 relative), the mixed
// mode ("one Newton step") the linear term only (~1e-11 relative at worst).
// The mass is folded into the polynomial, m15 = 1.5 m and m1875 = 1.875 m
// (per source body, computed once), and y0^2, y0^3 come from seed_powers, so
// the FP64 pipe does 4 operations (3 in the mixed mode).
template <int PREC>
__device__ __forceinline__ double scale_fast(double r2, double m, double m15, double m1875) {
  const SeedPow sp = seed_powers(rsqrt_seed_bits(r2));
  const double e = __fma_rn(-r2, sp.t, 1.0);
  if (PREC == NB_PREC_FP64) return sp.y3 * __fma_rn(__fma_rn(m1875, e, m15), e, m);
  return sp.y3 * __fma_rn(m15, e, m);
}

// 1.5 m and 1.875 m for m >= 0 (zero or normal) by integer ops on m's bits:
// 1.5 m = m + m/2 as a significand sum (truncated, relative error < 2^-52)
// and 1.875 m through the float built from m's high word (relative error
// < 2^-19). Both only multiply e (|e| < 2^-19) and e^2 in the refinement
// polynomial, so their errors enter m r^-3 below 2^-56 relative.
__device__ __forceinline__ void mass_coeffs(double m, double& m15, double& m1875) {
  const unsigned long long B = (unsigned long long)__double_as_longlong(m);
  const unsigned long long M = (B & 0xfffffffffffffull) | 0x10000000000000ull;
  const unsigned long long S = M + (M >> 1);  // [1.5 2^52, 3 2^52)
  const unsigned c = (unsigned)(S >> 53);
  const unsigned long long R = (((B >> 52) + c - 1ull) << 52) + (S >> c);
  const unsigned hm = (unsigned)(B >> 32);
  const unsigned fb = __float_as_uint(__uint_as_float((hm << 3) + 0x40000000u) * 1.875f);
  m15 = B == 0ull ? 0.0 : __longlong_as_double((long long)R);
  m1875 = B == 0ull ? 0.0 : __hiloint2double((int)((fb >> 3) + 0x38000000u), (int)(fb << 29));
}

// The same with the mass as the only per-source input: the coefficients come
// from mass_coeffs, so the FP64 pipe still does 4 operations (3 mixed).
// m in [2^-126, 2^127] or 0.
template <int PREC>
__device__ __forceinline__ double scale_fast(double r2, double m) {
  double m15, m1875;
  mass_coeffs(m, m15, m1875);
  return scale_fast<PREC>(r2, m, m15, m1875);
}

// 1/r from r^2: y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8), error ~1e-17 + rounding.
__device__ __forceinline__ double rinv_fast(double r2) {
  const unsigned yb = rsqrt_seed_bits(r2);
  const double y0 = __hiloint2double((int)((yb >> 3) + 0x38000000u), (int)(yb << 29));
  const double e = __fma_rn(-r2, seed_powers(yb).t, 1.0);
  return __fma_rn(y0 * e, __fma_rn(0.375, e, 0.5), y0);
}

// 1/x for positive normal x with 2^-126 <= x < 2^128: rcp.approx seed r0 of
// the float built from x's high word (relative error < 2^-19), then with the
// exact residual e = 1 - x r0, 1/x = r0 / (1 - e) = r0 (1 + e + e^2) + O(e^3)
// (truncation < 2^-57): 3 FP64 instructions.
__device__ __forceinline__ double rcp_fast(double x) {
  const unsigned hx = (unsigned)__double2hiint(x);
  const float xf = __uint_as_float((hx << 3) + 0x40000000u);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  const unsigned rb = __float_as_uint(rf);
  const double r = __hiloint2double((int)((rb >> 3) + 0x38000000u), (int)(rb << 29));
  const double e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, __fma_rn(e, e, e), r);
}

// ---------------------------------------------------------------------------
// exp(x) for |x| <= 700 with few FP64 instructions, by the table-driven
// method of P. T. P. Tang (ACM TOMS 15, 1989) with 128 table points:
// x = (128 m + j) ln2/128 + r, |r| <= ln2/256 (+ the seed's slack), so
// exp(x) = 2^m 2^(j/128) exp(r). k = 128 m + j is picked in FP32 from a
// float built from x's high word (any nearby integer works: it only sets
// the size of r); r = x - k ln2/128 in two FMAs with ln2/128 split into a
// double and its remainder; exp(r) - 1 by its Taylor polynomial of degree 5
// (truncation < 1e-18 relative); 2^m is added to the exponent field. 8 FP64
// instructions, about 1 ulp. The table holds 2^(j/128) rounded to nearest.
// ---------------------------------------------------------------------------
static __device__ const double kExp2Tab[128] = {
    0x1.0000000000000p+0, 0x1.0163da9fb3335p+0, 0x1.02c9a3e778061p+0, 0x1.04315e86e7f85p+0,
    0x1.059b0d3158574p+0, 0x1.0706b29ddf6dep+0, 0x1.0874518759bc8p+0, 0x1.09e3ecac6f383p+0,
    0x1.0b5586cf9890fp+0, 0x1.0cc922b7247f7p+0, 0x1.0e3ec32d3d1a2p+0, 0x1.0fb66affed31bp+0,
    0x1.11301d0125b51p+0, 0x1.12abdc06c31ccp+0, 0x1.1429aaea92de0p+0, 0x1.15a98c8a58e51p+0,
    0x1.172b83c7d517bp+0, 0x1.18af9388c8deap+0, 0x1.1a35beb6fcb75p+0, 0x1.1bbe084045cd4p+0,
    0x1.1d4873168b9aap+0, 0x1.1ed5022fcd91dp+0, 0x1.2063b88628cd6p+0, 0x1.21f49917ddc96p+0,
    0x1.2387a6e756238p+0, 0x1.251ce4fb2a63fp+0, 0x1.26b4565e27cddp+0, 0x1.284dfe1f56381p+0,
    0x1.29e9df51fdee1p+0, 0x1.2b87fd0dad990p+0, 0x1.2d285a6e4030bp+0, 0x1.2ecafa93e2f56p+0,
    0x1.306fe0a31b715p+0, 0x1.32170fc4cd831p+0, 0x1.33c08b26416ffp+0, 0x1.356c55f929ff1p+0,
    0x1.371a7373aa9cbp+0, 0x1.38cae6d05d866p+0, 0x1.3a7db34e59ff7p+0, 0x1.3c32dc313a8e5p+0,
    0x1.3dea64c123422p+0, 0x1.3fa4504ac801cp+0, 0x1.4160a21f72e2ap+0, 0x1.431f5d950a897p+0,
    0x1.44e086061892dp+0, 0x1.46a41ed1d0057p+0, 0x1.486a2b5c13cd0p+0, 0x1.4a32af0d7d3dep+0,
    0x1.4bfdad5362a27p+0, 0x1.4dcb299fddd0dp+0, 0x1.4f9b2769d2ca7p+0, 0x1.516daa2cf6642p+0,
    0x1.5342b569d4f82p+0, 0x1.551a4ca5d920fp+0, 0x1.56f4736b527dap+0, 0x1.58d12d497c7fdp+0,
    0x1.5ab07dd485429p+0, 0x1.5c9268a5946b7p+0, 0x1.5e76f15ad2148p+0, 0x1.605e1b976dc09p+0,
    0x1.6247eb03a5585p+0, 0x1.6434634ccc320p+0, 0x1.6623882552225p+0, 0x1.68155d44ca973p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6c012750bdabfp+0, 0x1.6dfb23c651a2fp+0, 0x1.6ff7df9519484p+0,
    0x1.71f75e8ec5f74p+0, 0x1.73f9a48a58174p+0, 0x1.75feb564267c9p+0, 0x1.780694fde5d3fp+0,
    0x1.7a11473eb0187p+0, 0x1.7c1ed0130c132p+0, 0x1.7e2f336cf4e62p+0, 0x1.80427543e1a12p+0,
    0x1.82589994cce13p+0, 0x1.8471a4623c7adp+0, 0x1.868d99b4492edp+0, 0x1.88ac7d98a6699p+0,
    0x1.8ace5422aa0dbp+0, 0x1.8cf3216b5448cp+0, 0x1.8f1ae99157736p+0, 0x1.9145b0b91ffc6p+0,
    0x1.93737b0cdc5e5p+0, 0x1.95a44cbc8520fp+0, 0x1.97d829fde4e50p+0, 0x1.9a0f170ca07bap+0,
    0x1.9c49182a3f090p+0, 0x1.9e86319e32323p+0, 0x1.a0c667b5de565p+0, 0x1.a309bec4a2d33p+0,
    0x1.a5503b23e255dp+0, 0x1.a799e1330b358p+0, 0x1.a9e6b5579fdbfp+0, 0x1.ac36bbfd3f37ap+0,
    0x1.ae89f995ad3adp+0, 0x1.b0e07298db666p+0, 0x1.b33a2b84f15fbp+0, 0x1.b59728de5593ap+0,
    0x1.b7f76f2fb5e47p+0, 0x1.ba5b030a1064ap+0, 0x1.bcc1e904bc1d2p+0, 0x1.bf2c25bd71e09p+0,
    0x1.c199bdd85529cp+0, 0x1.c40ab5fffd07ap+0, 0x1.c67f12e57d14bp+0, 0x1.c8f6d9406e7b5p+0,
    0x1.cb720dcef9069p+0, 0x1.cdf0b555dc3fap+0, 0x1.d072d4a07897cp+0, 0x1.d2f87080d89f2p+0,
    0x1.d5818dcfba487p+0, 0x1.d80e316c98398p+0, 0x1.da9e603db3285p+0, 0x1.dd321f301b460p+0,
    0x1.dfc97337b9b5fp+0, 0x1.e264614f5a129p+0, 0x1.e502ee78b3ff6p+0, 0x1.e7a51fbc74c83p+0,
    0x1.ea4afa2a490dap+0, 0x1.ecf482d8e67f1p+0, 0x1.efa1bee615a27p+0, 0x1.f252b376bba97p+0,
    0x1.f50765b6e4540p+0, 0x1.f7bfdad9cbe14p+0, 0x1.fa7c1819e90d8p+0, 0x1.fd3c22b8f71f1p+0,
};

__device__ __forceinline__ double exp_fast(double x) {
  const unsigned hx = (unsigned)__double2hiint(x);
  const unsigned ex = (hx >> 20) & 0x7ffu;
  // float of x from its sign, exponent and top 20 fraction bits; |x| < 2^-9
  // takes k = 0 (r = x is already small enough)
  const float xf = __uint_as_float((hx & 0x80000000u) | ((ex - 896u) << 23) | ((hx & 0xfffffu) << 3));
  const int k = ex < 1014u ? 0 : __float2int_rn(xf * 184.6649652337873f);  // 128 / ln2
  // k as a double by integer ops (|k| < 2^24 is exact in a float)
  const unsigned kb = __float_as_uint((float)k);
  const double kd = k == 0 ? 0.0
                           : __hiloint2double((int)((kb & 0x80000000u) | (((kb & 0x7fffffffu) >> 3) + 0x38000000u)),
                                              (int)(kb << 29));
  double r = __fma_rn(-kd, 0x1.62e42fefa39efp-8, x);  // ln2/128, rounded
  r = __fma_rn(-kd, 0x1.abc9e3b39803fp-63, r);        // its remainder
  double p = __fma_rn(r, 1.0 / 120.0, 1.0 / 24.0);
  p = __fma_rn(p, r, 1.0 / 6.0);
  p = __fma_rn(p, r, 0.5);
  p = __fma_rn(p, r, 1.0);
  const double T = __ldg(&kExp2Tab[k & 127]);
  const double e = __fma_rn(T, p * r, T);
  return __hiloint2double(__double2hiint(e) + (k >> 7) * (1 << 20), __double2loint(e));
}


// Squared separation in the fixed rounding that decides encounter flags:
// fma(dz, dz, fma(dy, dy, dx*dx)), every operation correctly rounded.
__device__ __forceinline__ double sep2(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// r^2 = dx^2 + dy^2 + dz^2 by integer arithmetic, rounded to nearest from a
// sum exact to ~2^-60 relative (at most one ulp from the exact value; sep2
// may differ from it by an ulp): each significand, normalised to 64 bits, is
// squared to its top 64 bits (a 64 x 64 -> 128-bit high product), the three
// are aligned to the largest and added, and the sum is rounded to 53 bits.
// No FP64 instruction; zero and subnormal components count as zero; 0 for
// coincident bodies; components below 2^500 in size. Host-callable so that it
// can be checked on the CPU.
__host__ __device__ __forceinline__ unsigned long long nb_umulhi64(unsigned long long a,
                                                                  unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}
__host__ __device__ __forceinline__ unsigned long long nb_dbits(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  __builtin_memcpy(&b, &v, 8);
  return b;
#endif
}
// top 64 bits of the square of |v|'s significand and 2 x v's exponent field
__host__ __device__ __forceinline__ unsigned long long sq_top(double v, int& key) {
  const unsigned long long b = nb_dbits(v);
  const int ex = (int)((b >> 52) & 0x7ffu);
  const unsigned long long mn = ((b << 11) | 0x8000000000000000ull);
  key = ex == 0 ? -4096 : 2 * ex;
  return ex == 0 ? 0ull : nb_umulhi64(mn, mn);  // [2^62, 2^64)
}
__host__ __device__ __forceinline__ double sep2_int(double dx, double dy, double dz) {
  int kx, ky, kz;
  const unsigned long long qx = sq_top(dx, kx), qy = sq_top(dy, ky), qz = sq_top(dz, kz);
  const int K = kx > ky ? (kx > kz ? kx : kz) : (ky > kz ? ky : kz);
  // value of q with key k: q 2^(k - 2108); aligned to K with 2 bits of headroom
  const int sx = K - kx + 2, sy = K - ky + 2, sz = K - kz + 2;
  const unsigned long long S = (sx < 64 ? qx >> sx : 0ull) + (sy < 64 ? qy >> sy : 0ull) +
                               (sz < 64 ? qz >> sz : 0ull);  // r^2 = S 2^(K - 2106)
  if (S == 0ull) return 0.0;
  const int L = 63 - nb_clzll(S);  // >= 60 (the largest term is >= 2^60)
  const unsigned long long Q = (S + (1ull << (L - 53))) >> (L - 52);
  const unsigned long long bits = Q + ((unsigned long long)(L + K - 1084) << 52);
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double r;
  __builtin_memcpy(&r, &bits, 8);
  return r;
#endif
}

// Positions as signed 128-bit fixed-point numbers X = x 2^88 (two's
// complement in an unsigned __int128): exact for 2^-36 <= |x| < 2^38 AU,
// truncated below (error < 2^-88 AU), saturated at 2^38 AU beyond (only
// absorbed bodies, which have no mass and no changeover radius, can sit
// there: at 1e6 (id + 1) AU, beyond 2^38 AU from id ~ 275 000).
// The difference of two of them is exact, so the kick forms dx, dy, dz on the
// integer pipe: fix_diff rounds X_j - X_i to a double (to nearest, ties
// upward; a negative difference is taken one unit of 2^-88 AU small, which
// matters only below ~2^-35 AU) and returns the top 64 bits of its square for
// sep2_fix.
typedef unsigned __int128 nb_u128;
__host__ __device__ __forceinline__ nb_u128 fix_of(double x) {
  const unsigned long long b = nb_dbits(x);
  const int ex = (int)((b >> 52) & 0x7ffu);
  const nb_u128 m = (nb_u128)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = ex - 987;  // x = m 2^(ex - 1075) = m 2^(sh - 88)
  nb_u128 mag = ex == 0 ? (nb_u128)0
                        : (sh >= 0 ? (sh <= 73 ? m << sh : ((nb_u128)1 << 126))
                                   : (sh > -53 ? m >> (-sh) : (nb_u128)0));
  return (b >> 63) ? (nb_u128)0 - mag : mag;
}
struct FixDiff {
  double d;               // X_j - X_i as a double
  unsigned long long sq;  // top 64 bits of the square of the normalised magnitude
  int key;                // 2 L, L the leading bit of the magnitude (-4096 for zero)
};
__host__ __device__ __forceinline__ FixDiff fix_diff(nb_u128 xj, nb_u128 xi) {
  const nb_u128 dv = xj - xi;
  const unsigned long long hw = (unsigned long long)(dv >> 64);
  const unsigned long long sgn = (unsigned long long)((long long)hw >> 63);  // ~0 if negative
  // one's-complement magnitude: |dv| for dv >= 0, |dv| - 1 (one unit, 2^-88 AU)
  // below it for dv < 0, which changes the result only for |dx| < ~2^-35 AU
  const unsigned long long h = hw ^ sgn, l = (unsigned long long)dv ^ sgn;
  FixDiff r;
  if ((h | l) == 0ull) {
    r.d = 0.0;
    r.sq = 0ull;
    r.key = -4096;
    return r;
  }
  int L;
  unsigned long long N;  // the magnitude's top 64 bits, bit 63 set
  if (h) {
    const int s = nb_clzll(h);
    N = s ? (h << s) | (l >> (64 - s)) : h;
    L = 127 - s;
  } else {  // |dx| < 2^-24 AU
    const int s = nb_clzll(l);
    N = l << s;
    L = 63 - s;
  }
  // round at bit 10 (without forming N + 2^10, which can overflow 64 bits):
  // 53 bits, 2^53 on a carry (which the exponent add absorbs)
  const unsigned long long Q = (N >> 11) + ((N >> 10) & 1ull);
  const unsigned long long bits = (sgn << 63) + Q + ((unsigned long long)(L + 934) << 52);
#ifdef __CUDA_ARCH__
  r.d = __longlong_as_double((long long)bits);
#else
  __builtin_memcpy(&r.d, &bits, 8);
#endif
  r.sq = nb_umulhi64(N, N);  // [2^62, 2^64): d^2 = sq 2^(2L - 238)
  r.key = 2 * L;
  return r;
}
// r^2 from the three fix_diff squares (aligned sum rounded to 53 bits, as
// in sep2_int): within half an ulp plus ~2^-58 of the exact value.
__host__ __device__ __forceinline__ double sep2_fix(const FixDiff& a, const FixDiff& b,
                                                   const FixDiff& c) {
  const int K = a.key > b.key ? (a.key > c.key ? a.key : c.key) : (b.key > c.key ? b.key : c.key);
  const int sa = K - a.key + 2, sb = K - b.key + 2, sc = K - c.key + 2;
  const unsigned long long S = (sa < 64 ? a.sq >> sa : 0ull) + (sb < 64 ? b.sq >> sb : 0ull) +
                               (sc < 64 ? c.sq >> sc : 0ull);  // r^2 = S 2^(K - 236)
  if (S == 0ull) return 0.0;
  const int L = 63 - nb_clzll(S);
  const unsigned long long Q = (S + (1ull << (L - 53))) >> (L - 52);
  const unsigned long long bits = Q + ((unsigned long long)(L + K + 786) << 52);
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double r;
  __builtin_memcpy(&r, &bits, 8);
  return r;
#endif
}

// r^-3 alone for the unordered-pair kick (which scales it by each body's
// mass), with one FP64 instruction: r^-3 = y0^3 p, p = (1 - e)^(-3/2) =
// 1 + 3e/2 + 15e^2/8 + O(e^3), e = 1 - r^2 y0^2, and p formed on the integer
// pipe. r^2 = R 2^(er - 1075) (R its 53-bit significand) and y0^2 = s^2
// 2^(2 ey - 300) (s the seed's 24-bit significand), so r^2 y0^2 = R s^2 2^-K
// with K = 1375 - er - 2 ey: the 101-bit product R s^2 is exact, and
// D = (2^K - R s^2) 2^(63 - K), rounded toward minus infinity, is e in units
// of 2^-63 (|D| < 2^45 for |e| < 2^-18). p - 1 = 1.5 e + 1.875 e^2 is then an
// integer in the same units (e^2 from the square of D / 2^14, error below
// 2^-60 in all), and p's bits follow by rounding that integer to p's ulp
// (2^-52 above 1, 2^-53 below). With y3 = y0^3 rounded (seed_powers) and the
// one rounded product, r^-3 is within ~1.6 ulp (the e^3 term, < 2^-55.7 for
// |e| < 2e-6, as in scale_fast). The product y3 p stays on the FP64 pipe:
// forming it from the 117-bit integer product too (1.0 ulp) made the kick
// 9 % slower at N = 65538 (40.1 against 36.7 ms), the integer pipe being the
// busier one by then. Valid for seeds with |e| < 2^-18 and
// 2^-126 <= r^2 < 2^128 (the seed's range). Host-callable with the seed's
// bits as an input, so that it can be checked on the CPU.
__host__ __device__ __forceinline__ double rinv3_from_seed(double r2, unsigned yb) {
  const unsigned long long B = nb_dbits(r2);
  const int er = (int)(B >> 52);
  const unsigned long long R = (B & 0xfffffffffffffull) | 0x10000000000000ull;
  const unsigned s = (yb & 0x7fffffu) | 0x800000u;
  const int ey = (int)(yb >> 23);
  const unsigned long long S2 = (unsigned long long)s * s;  // < 2^48
  const nb_u128 P = (nb_u128)R * S2;                        // < 2^101
  const int K = 1375 - er - 2 * ey;                         // r^2 y0^2 = P 2^-K, K in 98..101
  const long long D = (long long)((__int128)(((nb_u128)1 << K) - P) >> (K - 63));
  const unsigned long long a = (unsigned long long)(D < 0 ? -D : D) >> 14;
  const long long q = (long long)((a * a) >> 35);        // e^2 in units of 2^-63
  const long long dp = D + (D >> 1) + ((q << 1) - (q >> 3));  // p - 1 = 1.5 e + 1.875 e^2
  const unsigned long long pb =
      dp >= 0 ? 0x3ff0000000000000ull + (((unsigned long long)dp + 1024ull) >> 11)
              : 0x3ff0000000000000ull - (((unsigned long long)(-dp) + 512ull) >> 10);
  double p;
#ifdef __CUDA_ARCH__
  p = __longlong_as_double((long long)pb);
  return __dmul_rn(seed_powers(yb).y3, p);
#else
  __builtin_memcpy(&p, &pb, 8);
  return seed_powers(yb).y3 * p;
#endif
}
__device__ __forceinline__ double rinv3_fast(double r2) {
  return rinv3_from_seed(r2, rsqrt_seed_bits(r2));
}

// m_j w / r^3 for one pair with full-precision r (used off the hot loop).
// w = 1 when r^2 >= rc^2 with rc = max(rc_i, rc_j); 0 for coincident bodies.
__device__ __forceinline__ double pair_scale(double r2, double mj, double rci, double rcj) {
  if (r2 == 0.0 || mj == 0.0) return 0.0;
  const double rc = fmax(rci, rcj);
  const double r = sqrt(r2);
  const double w = (r2 < rc * rc) ? kick_weight(r, rc) : 1.0;
  return mj * w / (r2 * r);
}

// Critical radius of Eq. rcrit. R_Hill = |x| (m / 3 m0)^(1/3); the velocity
// term uses |v - v_circ(x)| (vel_mode 0: speed relative to the local circular
// prograde orbit) or |v| (vel_mode 1).
__device__ __forceinline__ double rcrit(const Phys& P, double x, double y, double z, double vx,
                                        double vy, double vz, double m) {
  const double r = sqrt(x * x + y * y + z * z);
  const double rh = r * cbrt(m / (3.0 * P.m0));
  double vr;
  if (P.vel_mode == 0) {
    const double rxy = sqrt(x * x + y * y);
    double cx = 0.0, cy = 0.0;
    if (rxy > 0.0 && r > 0.0) {
      const double vk = sqrt(P.G * P.m0 / r);
      cx = -vk * y / rxy;
      cy = vk * x / rxy;
    }
    const double dx = vx - cx, dy = vy - cy;
    vr = sqrt(dx * dx + dy * dy + vz * vz);
  } else {
    vr = sqrt(vx * vx + vy * vy + vz * vz);
  }
  return fmax(P.hill_factor * rh, P.vel_factor * fabs(P.dt_rcrit) * vr);
}

// Deterministic block reduction of three doubles (fixed shuffle tree, fixed
// warp order). Valid in thread 0 on return. smem: >= 3 * 32 doubles.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* smem) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) {
    smem[3 * w] = a;
    smem[3 * w + 1] = b;
    smem[3 * w + 2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int k = 0; k < nw; ++k) {
      a += smem[3 * k];
      b += smem[3 * k + 1];
      c += smem[3 * k + 2];
    }
  }
  __syncthreads();
}

// Sum of the 3 x nparts partial momenta in a fixed order; every block that
// calls it obtains the same bits. Result valid in all threads.
__device__ __forceinline__ void reduce_parts3(const double* parts, int nparts, double* smem,
                                              double out[3]) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
    a += parts[3 * k];
    b += parts[3 * k + 1];
    c += parts[3 * k + 2];
  }
  block_sum3(a, b, c, smem);
  if (threadIdx.x == 0) {
    smem[96] = a;
    smem[97] = b;
    smem[98] = c;
  }
  __syncthreads();
  out[0] = smem[96];
  out[1] = smem[97];
  out[2] = smem[98];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Host-side launchers (one per kernel family), defined in the .cu files.
// ---------------------------------------------------------------------------
int kick_blocks(int n, int S, int precision);
int ppart_blocks(int n);
void launch_kick(const Dev& d, const Phys& P, int target_sel, cudaStream_t st);
void launch_kick_raw(int n, int ib, int ie, const double* x, const double* y, const double* z,
                     const double* m, const double* rc, const double* rc2, int S, int precision,
                     double* kpart, int2* pairs, int cap, Ctrl* ctrl, cudaStream_t st);
void launch_finish(const Dev& d, const Phys& P, int with_delta, cudaStream_t st);
// part 1: partial sums minus the group bodies' trial terms (unscaled); part 2:
// plus their final terms, times G (the step runs part 1 beside the direct solver)
void launch_finish_part(const Dev& d, const Phys& P, int part, cudaStream_t st);
void launch_member_kick(const Dev& d, const Phys& P, cudaStream_t st);
void launch_open_h(const Dev& d, double h, cudaStream_t st);
void launch_drift_h(const Dev& d, const Phys& P, double h, cudaStream_t st);
void launch_close_h(const Dev& d, const Phys& P, double h, int last, cudaStream_t st);
void launch_encounter(const Dev& d, const Phys& P, cudaStream_t st);
void launch_bs(const Dev& d, const Phys& P, double h, cudaStream_t st,
               cudaStream_t side = nullptr);
int bs_launches(const Dev& d, const Phys& P);  // kernels launch_bs launches
void launch_scatter(const Dev& d, const Phys& P, cudaStream_t st);
void launch_init_in(const Dev& d, const Phys& P, const double* x3, const double* v3,
                    const double* m, const double* R, const double* rc, const int* ids,
                    cudaStream_t st);
void launch_fsal_init(const Dev& d, cudaStream_t st, const int* cond = nullptr);
void launch_refresh_rcrit(const Dev& d, const Phys& P, cudaStream_t st);
void launch_gas(const Dev& d, const Phys& P, double tau, cudaStream_t st);
void launch_eject(const Dev& d, const Phys& P, cudaStream_t st);
// force and flags at the current positions (the start-of-step evaluation);
// with only_if_ejected, nothing happens unless bodies were removed this step
void launch_force_anew(const Dev& d, const Phys& P, int only_if_ejected, cudaStream_t st);
void launch_energy(const Dev& d, const Phys& P, double* out8, cudaStream_t st);
void launch_kepler_raw(int n, double mu, double* x3, double* v3, double dt, int max_iter,
                       int* status, cudaStream_t st);
int energy_blocks(int n);
void launch_gather(const Dev& d, double* x3, double* v3, double* m, double* R, double* rc,
                   int* ids, int* count, cudaStream_t st);
void launch_a_convert(const Dev& d, double* a3, int to_soa, cudaStream_t st);
void launch_raw_prep(int n, const double* x3, const double* rc, double* x, double* y, double* z,
                     double* rc2, Ctrl* ctrl, cudaStream_t st);
void launch_raw_finish(int n, int ib, int ie, int S, const double* kpart, double G, double* a3,
                       cudaStream_t st);
int peak_blocks();
int measure_peaks(double* fp64, double* fp32, void* scratch, cudaStream_t st);

// NVTX range around a host-side phase (what a profiler shows as the phase
// that enqueued the kernels); free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace nb

// Host handle of one system (C ABI type nb_system).
struct nb_system {
  nb::Dev d;
  nb::Phys P;
  nb_params prm;
  cudaStream_t st;
  double* out8;  // device: energy results
  int* cnt;      // device: gather count
  char err[256];
  // a second stream for the trial half of the force update, which runs beside
  // the direct solver, and the fork/join events
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // kick timing (CUDA events on the launching stream) and launch counting
  int timing;
  std::vector<cudaEvent_t>* events;
  double kick_ms;
  long long kick_launches;
  long long launches;
  // row sharding across ranks (nb_set_shard): this rank's block of target
  // rows, the caller's all-gather and the exchange buffers (caller memory)
  int shard_rank, shard_world, shard_chunk;
  nb_allgather_fn shard_fn;
  void* shard_user;
  char* shard_buf;
  // CUDA graphs of the plain step (no split phases, unsharded, untimed) for
  // one dt: a middle step (its closing kick fused with the next opening one)
  // and a last step, captured on a private stream and launched on st
  cudaStream_t cap;
  cudaGraphExec_t gx_mid, gx_last;
  double g_dt;
  int g_fail;  // capture unavailable: direct launches
};

namespace nb {
// The all-gather of a sharded step: 1 = the trial kick's flagged pairs of
// every rank, 2 = every rank's rows of the force (nothing when unsharded).
int shard_exchange(nb_system* s, int which);
// Drop the plain step's CUDA graphs (after a change of the Dev or Phys they captured).
void drop_step_graphs(nb_system* s);
}  // namespace nb
