// Close encounters: the encounter set, independent groups, and the direct
// solver for H_A restricted to each group (section "The hybrid symplectic
// integrator"; groups per section "Increasing N"; perfect mergers per
// "Detailing the outcomes of collisions").
//
// k_encounter (one CTA): E = F_prev U F_trial as sorted unique (i, j) keys,
//   appended to the encounter log; connected components of E (each body
//   labelled with its component's smallest body); member slots ordered by
//   (smallest member, body). Sorts, compactions and labels run over the
//   whole CTA, in shared memory when E is small.
// k_bs (one CTA per group, grid-stride): Gragg modified midpoint with
//   n_k = 2k substeps and Neville extrapolation in the substep squared,
//   restarting from the state saved after C(h/2). Substep halving on
//   failure, doubling back after an early success on an aligned boundary,
//   merging scan after every accepted substep.
// k_bs_cluster (one thread-block cluster of 16 CTAs, else 8, per large group, groups
//   of at least bs_cluster_min bodies): the same solver with the group's
//   (column, member) work items spread over the cluster's threads and the
//   hardware cluster barrier between phases; results are bit-identical to
//   the single-CTA solver (same arithmetic per item, max-reductions only).
// k_scatter (one CTA): momentum change of the group bodies, energy removed
//   by mergers, and the write-back of the group results.
#include <cooperative_groups.h>

#include "bs.cuh"
#include "kepler.cuh"
#include "nb_internal.cuh"

namespace cg = cooperative_groups;

namespace nb {

constexpr int ENT = 1024;  // threads of k_encounter
constexpr int BNT = 64;    // threads of a BS CTA
constexpr int kWarpGroupMax = 8;  // groups of up to 8 bodies run on one warp
// the warp teams' scratch of a CTA fits the 48 KB of dynamic shared memory
// that needs no opt-in, with room for the kernel's static shared memory
static_assert((size_t)(BNT / 32) * kWarpGroupMax * bs_stride_for_kmax(kMaxBsK) * sizeof(double) <=
                  48 * 1024 - 1024, "warp-team scratch exceeds 47 KB");

// Which solver takes a group of M bodies: 2 = a cluster (bs_cluster_min > 0
// and M >= it), 1 = one warp (M <= kWarpGroupMax), 0 = one CTA. The
// multi-level path runs every group on one CTA.
__host__ __device__ inline int group_route(const Phys& P, int M) {
  if (P.ml_levels > 0) return 0;
  if (P.bs_cluster_min > 0 && M >= P.bs_cluster_min) return 2;
  return M <= kWarpGroupMax ? 1 : 0;
}
constexpr int CCL_MAX = 16;  // CTAs per cluster of the large-group solver (16: opt-in size)
constexpr int CNT = 128;     // threads per CTA of the large-group solver

__device__ void bitonic_sort(unsigned long long* a, int P2) {
  for (int k = 2; k <= P2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long ai = a[i], aj = a[ixj];
          if ((ai > aj) == up) {
            a[i] = aj;
            a[ixj] = ai;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Exclusive prefix sum of one count per thread over the CTA (ENT threads);
// *total receives the sum. ws: ENT/32 ints of shared scratch. Every thread
// must call it (it holds barriers).
static_assert(ENT == 1024, "the scan below takes 32 warps");
__device__ __forceinline__ int block_excl_scan(int v, int* ws, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int excl = x - v + (w > 0 ? ws[w - 1] : 0);
  *total = ws[31];
  __syncthreads();  // ws free for the next call
  return excl;
}

// In-place unique of the sorted a[0, n) by the whole CTA, in chunks of ENT:
// returns the count. A chunk reads its elements and predecessors before its
// scan's barriers and writes after them, to positions below its own start
// or within it; the last original value of a chunk is carried in *carry.
__device__ int block_unique_sorted(unsigned long long* a, int n, int* ws,
                                   unsigned long long* carry) {
  int out = 0;
  for (int base = 0; base < n; base += ENT) {
    const int k = base + threadIdx.x;
    unsigned long long v = 0ull, prev = 0ull;
    if (k < n) {
      v = a[k];
      prev = threadIdx.x > 0 ? a[k - 1] : (base > 0 ? *carry : 0ull);
    }
    const int f = (k < n && (k == 0 || v != prev)) ? 1 : 0;
    int tot;
    const int pos = block_excl_scan(f, ws, &tot);
    if (threadIdx.x == ENT - 1) *carry = v;
    if (f) a[out + pos] = v;
    out += tot;
    __syncthreads();
  }
  return out;
}

// Connected components of the nb bodies joined by the nE edges (local
// indices packed as a << 32 | b): label[k] becomes the smallest index of
// k's component, the root the serial union-find by smaller index reaches.
// Labels only decrease and stay indices of the same component, so passes of
// min-propagation over the edges and pointer jumping reach that fixed point
// whatever order the atomics take; a pass with a change lowers the sum of
// the labels, which bounds the passes. s_flag: one shared int.
__device__ void block_components(int* label, int nb, const unsigned long long* edges, int nE,
                                 int* s_flag, Ctrl* C) {
  for (int k = threadIdx.x; k < nb; k += ENT) label[k] = k;
  const long long cap = (long long)nb * nb / 2 + 2;
  for (long long pass = 0;; ++pass) {
    __syncthreads();  // the previous pass's reads of *s_flag are done
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < nE; e += ENT) {
      const int a = (int)(edges[e] >> 32), b = (int)(edges[e] & 0xffffffffu);
      const int la = label[a], lb = label[b];
      if (la != lb) {
        const int m = min(la, lb);
        atomicMin(&label[a], m);
        atomicMin(&label[b], m);
        *s_flag = 1;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += ENT) {
      const int l = label[k], ll = label[l];
      if (ll < l) atomicMin(&label[k], ll);
    }
    __syncthreads();
    if (*s_flag == 0) break;
    if (pass > cap) {  // cannot happen (see above); reported rather than looped on
      if (threadIdx.x == 0) set_status(C, NB_E_INVALID, 60);
      break;
    }
  }
}

__device__ __forceinline__ int lower_bound_u64(const unsigned long long* a, int n,
                                               unsigned long long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Encounter sets of at most kEncSmall keys (F_prev plus F_trial, the common
// case) keep every array in shared memory: pair keys and group keys
// (next_pow2(nb) <= 2 kEncSmall), body keys (next_pow2(2 nE) <= 2 kEncSmall),
// labels and edges; larger sets use the workspace's key regions.
constexpr int kEncSmall = 512;

__global__ void __launch_bounds__(ENT) k_encounter(Dev d) {
  __shared__ int s_stop, s_nT, s_nP, s_step, s_flag;
  __shared__ int ws[ENT / 32];
  __shared__ unsigned long long s_carry;
  __shared__ unsigned long long sKA[2 * kEncSmall], sKB[2 * kEncSmall], sEdge[kEncSmall];
  __shared__ int sLab[2 * kEncSmall];
  Ctrl* C = d.ctrl;
  if (threadIdx.x == 0) {
    s_stop = C->status;
    s_nT = min(C->n_ftrial, d.pair_cap);
    s_nP = min(C->n_fprev, d.pair_cap);
    s_step = (int)C->step_index;
  }
  __syncthreads();
  if (s_stop) return;
  // previous members are no longer members
  const int nprev = C->n_prev_members;
  for (int q = threadIdx.x; q < nprev; q += ENT) {
    const int b = d.grp_mem[q];
    if (NB_GUARD(C, q < d.member_cap && b >= 0 && b < d.n, 50)) d.member_slot[b] = -1;
  }
  const int nT = s_nT, nP = s_nP, nK = nT + nP;
  const bool small = nK <= kEncSmall;
  // global regions: A holds <= next_pow2(2 pair_cap) pair keys, then the
  // edges at 2 pair_cap, later <= 4 pair_cap group keys; B holds <= 4
  // pair_cap body keys (pair_cap is a power of 2)
  unsigned long long* kA = small ? sKA : d.keys;
  unsigned long long* kB = small ? sKB : d.keys + 4 * (size_t)d.pair_cap;
  unsigned long long* edges = small ? sEdge : d.keys + 2 * (size_t)d.pair_cap;
  int* label = small ? sLab : d.uf;
  const int P2 = next_pow2(nK > 0 ? nK : 1);
  for (int k = threadIdx.x; k < P2; k += ENT) {
    unsigned long long key = ~0ull;
    if (k < nP) {
      const int2 p = d.fprev[k];
      if (NB_GUARD(C, p.x >= 0 && p.x < p.y && p.y < d.n, 51))
        key = ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.y;
    } else if (k < nK) {
      const int2 p = d.ftrial[k - nP];
      if (NB_GUARD(C, p.x >= 0 && p.x < p.y && p.y < d.n, 52))
        key = ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.y;
    }
    kA[k] = key;
  }
  __syncthreads();
  bitonic_sort(kA, P2);
  // unique pairs; a pair refused by a guard sorts last as ~0 and is cut
  int nE = block_unique_sorted(kA, nK, ws, &s_carry);
  if (nE > 0 && kA[nE - 1] == ~0ull) --nE;
  // encounter log: (step, id_i, id_j)
  const int base = C->n_log;
  for (int k = threadIdx.x; k < nE; k += ENT) {
    const int pos = base + k;
    if (pos < d.log_cap) {
      const int i = (int)(kA[k] >> 32), j = (int)(kA[k] & 0xffffffffu);
      if (!NB_GUARD(C, i >= 0 && i < d.n && j >= 0 && j < d.n, 53)) continue;
      d.log[3 * pos] = s_step;
      d.log[3 * pos + 1] = d.id[i];
      d.log[3 * pos + 2] = d.id[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int fit = max(0, min(nE, d.log_cap - base));
    C->stats[ST_LOG_DROPPED] += (unsigned long long)(nE - fit);
    C->n_log = base + nE;  // entries beyond log_cap are counted, not stored
    C->n_enc = nE;
    C->stats[ST_ENC_PAIRS] += (unsigned long long)nE;
    C->stats[ST_FORCE_EVALS] += 1ull;
  }
  if (nE == 0) {
    if (threadIdx.x == 0) {
      C->n_groups = 0;
      C->n_members = 0;
      C->n_prev_members = 0;
      C->n_fprev = nT;
    }
    for (int k = threadIdx.x; k < nT; k += ENT) d.fprev[k] = d.ftrial[k];
    return;
  }
  // bodies appearing in E, sorted and unique
  const int P2b = next_pow2(2 * nE);
  for (int k = threadIdx.x; k < P2b; k += ENT) {
    unsigned long long v = ~0ull;
    if (k < 2 * nE) v = (k & 1) ? (kA[k >> 1] & 0xffffffffu) : (kA[k >> 1] >> 32);
    kB[k] = v;
  }
  __syncthreads();
  bitonic_sort(kB, P2b);
  const int nb = block_unique_sorted(kB, 2 * nE, ws, &s_carry);
  // the pairs as edges between local body indices, then the components
  for (int k = threadIdx.x; k < nE; k += ENT) {
    const int a = lower_bound_u64(kB, nb, kA[k] >> 32);
    const int b = lower_bound_u64(kB, nb, kA[k] & 0xffffffffu);
    edges[k] = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
  }
  block_components(label, nb, edges, nE, &s_flag, C);
  // group keys (root body, body) reuse region A
  const int P2g = next_pow2(nb);
  for (int k = threadIdx.x; k < P2g; k += ENT) {
    unsigned long long v = ~0ull;
    if (k < nb) v = (kB[label[k]] << 32) | kB[k];
    kA[k] = v;
  }
  __syncthreads();
  bitonic_sort(kA, P2g);
  for (int k = threadIdx.x; k < nb; k += ENT) {
    const int body = (int)(kA[k] & 0xffffffffu);
    if (!NB_GUARD(C, k < d.member_cap && body >= 0 && body < d.n, 54)) continue;
    d.grp_mem[k] = body;
    d.member_slot[body] = k;
  }
  // group offsets: where the root changes
  int g = 0;
  for (int b0 = 0; b0 < nb; b0 += ENT) {
    const int k = b0 + threadIdx.x;
    const int f = (k < nb && (k == 0 || (kA[k] >> 32) != (kA[k - 1] >> 32))) ? 1 : 0;
    int tot;
    const int pos = block_excl_scan(f, ws, &tot);
    if (f) d.grp_off[g + pos] = k;
    g += tot;
  }
  if (threadIdx.x == 0) {
    d.grp_off[g] = nb;
    C->n_groups = g;
    C->n_members = nb;
    C->n_prev_members = nb;
    C->stats[ST_GROUPS] += (unsigned long long)g;
    C->stats[ST_MOVED] += (unsigned long long)nb;
  }
}

void launch_encounter(const Dev& d, const Phys& P, cudaStream_t st) {
  (void)P;
  k_encounter<<<1, ENT, 0, st>>>(d);
}

// ---------------------------------------------------------------------------
// Multi-level changeover (section "Increasing N"), one CTA per level-0 group.
// Level l has radii r_crit f^-l and substeps tau / f. ml_level<LV>(S, tau)
// moves the members S over tau under their Kepler motion and the close part
// of their interaction with weight 1 - w_LV: at LV = ml_levels by the direct
// solver (the members gathered into the second scratch region, radii scaled
// by f^-LV), below it by f substeps K A K with the kick weight
// w_(LV+1) - w_LV and the level-(LV+1) groups (pairs within the next radii at
// the substep's start or after the trial Kepler drift, restarted from the
// substep's start) integrated by ml_level<LV+1>. The recursion is unrolled at
// compile time (kMlMax levels), so no device stack is used. Members are the
// group's slots 0..M-1; their state lives in the y fields of the group's
// scratch; the column fields hold the per-level saved states and the kick
// accelerations (the direct solver works in the second region).
// ---------------------------------------------------------------------------
struct MlCtx {
  BsCtx a;       // the group's scratch (region A)
  double* bbase; // the group's slots in the second region
  double* bg;
  int* list;     // (kMlMax + 1) x M
  int* parent;   // (kMlMax + 1) x M
  int L, f, Mg;
  Phys P;
  double* s_red;
  int* s_flags;
  int* s_int;    // 2 shared ints: a count and an error flag
  BsTally* tally;
  double El;     // energy removed by mergers (thread 0)
};

// f^-level by repeated division (the oracle computes it the same way)
__device__ __forceinline__ double ml_scale(int f, int level) {
  double s = 1.0;
  for (int l = 0; l < level; ++l) s /= (double)f;
  return s;
}

__device__ __forceinline__ double* ml_y(const MlCtx& m, int i) {
  return m.a.base + (size_t)i * m.a.stride + OY;
}

__device__ __forceinline__ double ml_pw(double q2, double q, double rcl) {
  return (q2 < rcl * rcl) ? kick_weight(q, rcl) : 1.0;
}

// K_level(tau) over the live members of S: v += tau sum G m_j (w_level -
// w_(level-1)) d / r^3, accelerations first (all of them), then applied.
__device__ void ml_kick(MlCtx& m, const int* S, int ns, int level, double tau) {
  const double sl = ml_scale(m.f, level), sp = ml_scale(m.f, level - 1);
  const double* g = m.a.g;
  for (int a = threadIdx.x; a < ns; a += blockDim.x) {
    const int i = S[a];
    double* acc = m.a.base + (size_t)i * m.a.stride + bs_off_col(1) + CZC;
    acc[0] = acc[1] = acc[2] = 0.0;
    if (g[10 * i + 9] == 0.0) continue;
    const double* yi = ml_y(m, i);
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int b = 0; b < ns; ++b) {
      const int j = S[b];
      if (j == i || g[10 * j + 9] == 0.0) continue;
      const double* yj = ml_y(m, j);
      const double dx = yj[0] - yi[0], dy = yj[1] - yi[1], dz = yj[2] - yi[2];
      const double q2 = sep2(dx, dy, dz);
      if (q2 == 0.0) continue;
      const double q = sqrt(q2);
      const double rcp = fmax(g[10 * i + 8], g[10 * j + 8]);
      const double dw = ml_pw(q2, q, rcp * sl) - ml_pw(q2, q, rcp * sp);
      if (dw == 0.0) continue;
      const double fr = m.P.G * g[10 * j + 6] * dw / (q2 * q);
      ax += fr * dx;
      ay += fr * dy;
      az += fr * dz;
    }
    acc[0] = ax; acc[1] = ay; acc[2] = az;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < ns; a += blockDim.x) {
    const int i = S[a];
    if (g[10 * i + 9] == 0.0) continue;
    double* y = ml_y(m, i);
    const double* acc = m.a.base + (size_t)i * m.a.stride + bs_off_col(1) + CZC;
    y[3] += tau * acc[0];
    y[4] += tau * acc[1];
    y[5] += tau * acc[2];
  }
  __syncthreads();
}

// pairs (a < b) of S within the radii r_crit * sl join in parent[] (thread 0)
__device__ void ml_flag(const MlCtx& m, const int* S, int ns, double sl, int* parent) {
  const double* g = m.a.g;
  for (int a = 0; a < ns; ++a) {
    const int i = S[a];
    if (g[10 * i + 9] == 0.0) continue;
    const double* yi = ml_y(m, i);
    for (int b = a + 1; b < ns; ++b) {
      const int j = S[b];
      if (g[10 * j + 9] == 0.0) continue;
      const double* yj = ml_y(m, j);
      const double q2 = sep2(yj[0] - yi[0], yj[1] - yi[1], yj[2] - yi[2]);
      const double rcl = fmax(g[10 * i + 8], g[10 * j + 8]) * sl;
      if (!(q2 < rcl * rcl)) continue;
      int ra = a, rb = b;
      while (parent[ra] != ra) ra = parent[ra];
      while (parent[rb] != rb) rb = parent[rb];
      if (ra < rb)
        parent[rb] = ra;
      else if (rb < ra)
        parent[ra] = rb;
    }
  }
}

// The direct solver on S with the radii of level LV, in the second region.
__device__ int ml_direct(MlCtx& m, const int* S, int ns, double tau, int level) {
  const double scale = ml_scale(m.f, level);
  BsCtx c = m.a;
  c.base = m.bbase;
  c.g = m.bg;
  c.M = ns;
  c.rc_scale = scale;
  for (int a = threadIdx.x; a < ns; a += blockDim.x) {
    const int i = S[a];
    const double* ya = ml_y(m, i);
    double* yb = c.base + (size_t)a * c.stride + OY;
    for (int k = 0; k < 6; ++k) yb[k] = ya[k];
    const double* ga = m.a.g + 10 * i;
    double* gb = c.g + 10 * a;
    for (int k = 6; k < 10; ++k) gb[k] = ga[k];
    bs_set_aux(c, a, m.P.G, gb[6], gb[8] * scale);
  }
  __syncthreads();
  double El = 0.0;
  const int st = bs_integrate_group(c, m.P, tau, m.s_red, m.s_flags, *m.tally, &El);
  if (threadIdx.x == 0) m.El += El;
  for (int a = threadIdx.x; a < ns; a += blockDim.x) {
    const int i = S[a];
    double* ya = ml_y(m, i);
    const double* yb = c.base + (size_t)a * c.stride + OY;
    for (int k = 0; k < 6; ++k) ya[k] = yb[k];
    double* ga = m.a.g + 10 * i;
    const double* gb = c.g + 10 * a;
    for (int k = 6; k < 10; ++k) ga[k] = gb[k];
  }
  __syncthreads();
  return st;
}

template <int LV>
__device__ int ml_level(MlCtx& m, const int* S, int ns, double tau) {
  if (LV >= m.L) return ml_direct(m, S, ns, tau, LV);
  if constexpr (LV >= kMlMax) {
    return NB_E_INVALID;  // unreachable: ml_levels <= kMlMax
  } else {
    const int tid = threadIdx.x, NT = blockDim.x;
    const double t1 = tau / (double)m.f;
    const double sn = ml_scale(m.f, LV + 1);
    int* parent = m.parent + (size_t)(LV + 1) * m.Mg;
    int* sub = m.list + (size_t)(LV + 1) * m.Mg;
    const int save = bs_off_col(LV + 1) + CZM;  // this level's substep-start state
    const double mu = m.P.mu;
    int status = 0;
    for (int k = 0; k < m.f && !status; ++k) {
      ml_kick(m, S, ns, LV + 1, 0.5 * t1);
      if (tid == 0) {
        for (int a = 0; a < ns; ++a) parent[a] = a;
        ml_flag(m, S, ns, sn, parent);
        m.s_int[1] = 0;
      }
      for (int a = tid; a < ns; a += NT) {
        double* y = ml_y(m, S[a]);
        double* sv = m.a.base + (size_t)S[a] * m.a.stride + save;
        for (int q = 0; q < 6; ++q) sv[q] = y[q];
      }
      __syncthreads();
      for (int a = tid; a < ns; a += NT) {
        const int i = S[a];
        if (m.a.g[10 * i + 9] == 0.0) continue;
        double* y = ml_y(m, i);
        int it;
        if (kepler_drift(mu, y[0], y[1], y[2], y[3], y[4], y[5], t1, m.P.kepler_max_iter, &it))
          m.s_int[1] = 1;
      }
      __syncthreads();
      if (tid == 0) {
        ml_flag(m, S, ns, sn, parent);
        for (int a = 0; a < ns; ++a) {
          int r = a;
          while (parent[r] != r) r = parent[r];
          parent[a] = r;
        }
      }
      __syncthreads();
      if (m.s_int[1]) status = NB_E_NOCONV;
      for (int a = 0; a < ns && !status; ++a) {
        if (parent[a] != a) continue;
        if (tid == 0) {
          int nsub = 0;
          for (int b = a; b < ns; ++b)
            if (parent[b] == a) sub[nsub++] = S[b];
          m.s_int[0] = nsub;
        }
        __syncthreads();
        const int nsub = m.s_int[0];
        if (nsub < 2) continue;
        for (int b = a + tid; b < ns; b += NT) {
          if (parent[b] != a) continue;
          double* y = ml_y(m, S[b]);
          const double* sv = m.a.base + (size_t)S[b] * m.a.stride + save;
          for (int q = 0; q < 6; ++q) y[q] = sv[q];
        }
        __syncthreads();
        if (tid == 0) m.tally->ml_groups += 1;
        status = ml_level<LV + 1>(m, sub, nsub, t1);
      }
      if (status) break;
      ml_kick(m, S, ns, LV + 1, 0.5 * t1);
      if (tid == 0) m.tally->ml_substeps += 1;
    }
    return status;
  }
}

// One CTA per group: the direct solver (ML = false) or the multi-level
// changeover (ML = true, its own kernel so that the direct solver's kernel
// keeps its registers).
template <bool ML>
__global__ void __maxnreg__(128) k_bs_t(Dev d, Phys P, double h) {
  __shared__ int s_stop, s_ng;
  __shared__ double s_red[BNT];
  __shared__ int s_flags[4];
  __shared__ int s_int[2];
  if (threadIdx.x == 0) {
    s_stop = d.ctrl->status;
    s_ng = d.ctrl->n_groups;
  }
  __syncthreads();
  if (s_stop) return;
  BsTally tally{0, 0, 0, 0};
  if constexpr (!ML) {
    // small groups: one per warp, with warp barriers only; the group's scratch
    // (kWarpGroupMax slots of bs_stride doubles per warp) in dynamic shared
    // memory (the CTA's other groups keep theirs in gscr)
    __shared__ int s_wflags[BNT / 32][4];
    extern __shared__ double s_bscr[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTeam wt{s_wflags[warp]};
    for (int grp = blockIdx.x * (BNT / 32) + warp; grp < s_ng; grp += gridDim.x * (BNT / 32)) {
      const int off = d.grp_off[grp];
      const int M = d.grp_off[grp + 1] - off;
      if (group_route(P, M) != 1) continue;
      BsCtx c;
      c.M = M;
      c.stride = d.bs_stride;
      c.base = s_bscr + (size_t)warp * kWarpGroupMax * d.bs_stride;  // the warp's scratch
      c.g = d.gnew + (size_t)off * 10;
      c.kmax = P.bs_kmax;
      c.G = P.G;
      c.mu = P.mu;
      c.mu15 = 1.5 * P.mu;
      c.mu1875 = 1.875 * P.mu;
      for (int b = lane; b < M; b += 32) {
        const int body = d.grp_mem[off + b];
        if (!NB_GUARD(d.ctrl, body >= 0 && body < d.n && off + b < d.member_cap, 57)) continue;
        double* y = c.base + (size_t)b * c.stride + OY;
        y[0] = d.xs[body]; y[1] = d.ys[body]; y[2] = d.zs[body];
        y[3] = d.vxs[body]; y[4] = d.vys[body]; y[5] = d.vzs[body];
        double* g = c.g + 10 * b;
        g[6] = d.m[body];
        g[7] = d.R[body];
        g[8] = d.rc[body];
        g[9] = 1.0;
        bs_set_aux(c, b, P.G, g[6], g[8]);
      }
      __syncwarp();
      double El = 0.0;
      // groups of up to 4 bodies speculate on the half-size attempt in the
      // warp's spare slots and lanes
      double* spec =
          P.bs_speculate && 2 * M <= kWarpGroupMax ? c.base + (size_t)M * c.stride : nullptr;
      const int status = bs_integrate(c, P, h, wt, tally, &El, (BsRec*)nullptr, spec);
      if (status && lane == 0) set_status(d.ctrl, status, 30);
      for (int b = lane; b < M; b += 32) {
        const double* y = c.base + (size_t)b * c.stride + OY;
        double* g = c.g + 10 * b;
        for (int k = 0; k < 6; ++k) g[k] = y[k];
      }
      if (lane == 0) d.gEl[grp] = El;
      __syncwarp();
    }
    // the warps' counters go through warp 0 of each CTA below; fold them
    // into thread 0's tally (each warp's lane 0 holds its own)
    __shared__ long long s_tal[BNT / 32][4];
    if (lane == 0) {
      s_tal[warp][0] = tally.derivs;
      s_tal[warp][1] = tally.substeps;
      s_tal[warp][2] = tally.halvings;
      s_tal[warp][3] = tally.merges;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tally.derivs = tally.substeps = tally.halvings = tally.merges = 0;
      for (int w = 0; w < BNT / 32; ++w) {
        tally.derivs += s_tal[w][0];
        tally.substeps += s_tal[w][1];
        tally.halvings += s_tal[w][2];
        tally.merges += s_tal[w][3];
      }
    }
  }
  for (int grp = blockIdx.x; grp < s_ng; grp += gridDim.x) {
    const int off = d.grp_off[grp];
    if (!ML && group_route(P, d.grp_off[grp + 1] - off) != 0) continue;  // a warp or a cluster
    BsCtx c;
    c.M = d.grp_off[grp + 1] - off;
    c.stride = d.bs_stride;
    c.base = d.gscr + (size_t)off * d.bs_stride;
    c.g = d.gnew + (size_t)off * 10;
    c.kmax = P.bs_kmax;
    c.G = P.G;
    c.mu = P.mu;
    c.mu15 = 1.5 * P.mu;
    c.mu1875 = 1.875 * P.mu;
    for (int b = threadIdx.x; b < c.M; b += blockDim.x) {
      const int body = d.grp_mem[off + b];
      if (!NB_GUARD(d.ctrl, body >= 0 && body < d.n && off + b < d.member_cap, 57)) continue;
      double* y = c.base + (size_t)b * c.stride + OY;
      y[0] = d.xs[body]; y[1] = d.ys[body]; y[2] = d.zs[body];
      y[3] = d.vxs[body]; y[4] = d.vys[body]; y[5] = d.vzs[body];
      double* g = c.g + 10 * b;
      g[6] = d.m[body];
      g[7] = d.R[body];
      g[8] = d.rc[body];
      g[9] = 1.0;
      bs_set_aux(c, b, P.G, g[6], g[8]);
    }
    __syncthreads();
    double El = 0.0;
    int status;
    if constexpr (ML) {
      MlCtx m;
      m.a = c;
      m.bbase = d.ml_gscr + (size_t)off * d.bs_stride;
      m.bg = d.ml_gnew + (size_t)off * 10;
      m.list = d.ml_list + (size_t)(kMlMax + 1) * off;
      m.parent = d.ml_parent + (size_t)(kMlMax + 1) * off;
      m.L = P.ml_levels;
      m.f = P.ml_factor;
      m.Mg = c.M;
      m.P = P;
      m.s_red = s_red;
      m.s_flags = s_flags;
      m.s_int = s_int;
      m.tally = &tally;
      m.El = 0.0;
      for (int b = threadIdx.x; b < c.M; b += blockDim.x) m.list[b] = b;
      __syncthreads();
      status = ml_level<0>(m, m.list, c.M, h);
      El = m.El;
    } else {
      status = bs_integrate_group(c, P, h, s_red, s_flags, tally, &El);
    }
    if (status && threadIdx.x == 0) set_status(d.ctrl, status, 30);
    for (int b = threadIdx.x; b < c.M; b += blockDim.x) {
      const double* y = c.base + (size_t)b * c.stride + OY;
      double* g = c.g + 10 * b;
      for (int k = 0; k < 6; ++k) g[k] = y[k];
    }
    if (threadIdx.x == 0) d.gEl[grp] = El;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&d.ctrl->stats[ST_BS_DERIVS], (unsigned long long)tally.derivs);
    atomicAdd(&d.ctrl->stats[ST_BS_SUBSTEPS], (unsigned long long)tally.substeps);
    atomicAdd(&d.ctrl->stats[ST_BS_HALVINGS], (unsigned long long)tally.halvings);
    atomicAdd(&d.ctrl->stats[ST_MERGES], (unsigned long long)tally.merges);
    atomicAdd(&d.ctrl->stats[ST_ML_SUBSTEPS], (unsigned long long)tally.ml_substeps);
    atomicAdd(&d.ctrl->stats[ST_ML_GROUPS], (unsigned long long)tally.ml_groups);
  }
}

// A thread-block cluster as the Bulirsch-Stoer team: flags and the per-CTA
// maxima live in the shared memory of the cluster's first CTA (read by the
// others through distributed shared memory); the barrier is the cluster's.
struct ClusterTeam {
  int* s_flags;    // CTA 0's flags (mapped)
  double* s_slot;  // CTA 0's per-CTA maxima (mapped), one per CTA of the cluster
  double* s_red;   // this CTA's reduction scratch, CNT entries
  int ncta;        // CTAs in the cluster
  __device__ int tid() const { return (int)cg::this_cluster().block_rank() * CNT + threadIdx.x; }
  __device__ int nthreads() const { return ncta * CNT; }
  __device__ int* flags() const { return s_flags; }
  __device__ void sync() const { cg::this_cluster().sync(); }
  __device__ double max_to_first(double v) const {
    s_red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double e = 0.0;
      for (int q = 0; q < CNT; ++q) e = fmax(e, s_red[q]);
      s_slot[cg::this_cluster().block_rank()] = e;
    }
    cg::this_cluster().sync();
    double e = 0.0;
    if (tid() == 0)
      for (int q = 0; q < ncta; ++q) e = fmax(e, s_slot[q]);
    return e;
  }  // whether v holds in any thread (valid in the first thread)
  __device__ bool any_to_first(bool v) const { return max_to_first(v ? 1.0 : 0.0) > 0.0; }
};

__global__ void __launch_bounds__(CNT) k_bs_cluster(Dev d, Phys P, double h, int min_m) {
  __shared__ double s_red[CNT];
  __shared__ double s_slot_own[CCL_MAX];
  __shared__ int s_flags_own[4];
  __shared__ int s_ctl[2];
  cg::cluster_group cl = cg::this_cluster();
  // the cluster's first CTA reads the control block once; every CTA takes
  // its values from there, so all CTAs of the cluster decide alike
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    s_ctl[0] = d.ctrl->status;
    s_ctl[1] = d.ctrl->n_groups;
  }
  cl.sync();
  const int* ctl0 = cl.map_shared_rank(s_ctl, 0);
  const int stop = ctl0[0], ng = ctl0[1];
  if (stop) {
    cl.sync();  // CTA 0's shared memory stays until every CTA has read it
    return;
  }
  const int ncta = (int)cl.num_blocks();
  ClusterTeam team{cl.map_shared_rank(s_flags_own, 0), cl.map_shared_rank(s_slot_own, 0), s_red,
                   ncta};
  const int cid = blockIdx.x / ncta, ncl = gridDim.x / ncta;
  const int tid = team.tid(), NT = team.nthreads();
  BsTally tally{0, 0, 0, 0};
  for (int grp = cid; grp < ng; grp += ncl) {
    const int off = d.grp_off[grp];
    const int M = d.grp_off[grp + 1] - off;
    if (group_route(P, M) != 2) continue;
    BsCtx c;
    c.M = M;
    c.stride = d.bs_stride;
    c.base = d.gscr + (size_t)off * d.bs_stride;
    c.g = d.gnew + (size_t)off * 10;
    c.kmax = P.bs_kmax;
    c.G = P.G;
    c.mu = P.mu;
    c.mu15 = 1.5 * P.mu;
    c.mu1875 = 1.875 * P.mu;
    for (int b = tid; b < M; b += NT) {
      const int body = d.grp_mem[off + b];
      if (!NB_GUARD(d.ctrl, body >= 0 && body < d.n && off + b < d.member_cap, 57)) continue;
      double* y = c.base + (size_t)b * c.stride + OY;
      y[0] = d.xs[body]; y[1] = d.ys[body]; y[2] = d.zs[body];
      y[3] = d.vxs[body]; y[4] = d.vys[body]; y[5] = d.vzs[body];
      double* g = c.g + 10 * b;
      g[6] = d.m[body];
      g[7] = d.R[body];
      g[8] = d.rc[body];
      g[9] = 1.0;
      bs_set_aux(c, b, P.G, g[6], g[8]);
    }
    cl.sync();
    double El = 0.0;
    const int status = bs_integrate(c, P, h, team, tally, &El, (BsRec*)nullptr);
    if (status && tid == 0) set_status(d.ctrl, status, 31);
    for (int b = tid; b < M; b += NT) {
      const double* y = c.base + (size_t)b * c.stride + OY;
      double* g = c.g + 10 * b;
      for (int k = 0; k < 6; ++k) g[k] = y[k];
    }
    if (tid == 0) d.gEl[grp] = El;
    cl.sync();
  }
  if (tid == 0) {
    atomicAdd(&d.ctrl->stats[ST_BS_DERIVS], (unsigned long long)tally.derivs);
    atomicAdd(&d.ctrl->stats[ST_BS_SUBSTEPS], (unsigned long long)tally.substeps);
    atomicAdd(&d.ctrl->stats[ST_BS_HALVINGS], (unsigned long long)tally.halvings);
    atomicAdd(&d.ctrl->stats[ST_MERGES], (unsigned long long)tally.merges);
  }
  // no CTA may exit while another still reads its shared memory
  cl.sync();
}

// Cluster size for the large-group solver: 16 CTAs (opt-in size) where the
// device can schedule such clusters, else the portable 8; as many clusters
// as fit on the device at once.
static int cluster_shape(int* ncl) {
  static int size = 0, count = 0;
  if (!size) {
    cudaFuncSetAttribute(k_bs_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c = CCL_MAX; c >= 8 && !size; c /= 2) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(CNT, 1, 1);
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int active = 0;
      if (cudaOccupancyMaxActiveClusters(&active, k_bs_cluster, &cfg) == cudaSuccess && active > 0) {
        size = c;
        count = active;
      }
    }
    cudaGetLastError();  // a refused size leaves an error behind
    if (!size) {
      size = 8;
      count = 1;
    }
  }
  *ncl = count;
  return size;
}

void launch_bs_cluster(const Dev& d, const Phys& P, double h, cudaStream_t st) {
  int ncl = 1;
  const int c = cluster_shape(&ncl);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = c;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(c * ncl, 1, 1);
  cfg.blockDim = dim3(CNT, 1, 1);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_bs_cluster, d, P, h, P.bs_cluster_min);
}

int bs_launches(const Dev& d, const Phys& P) {
  return (P.ml_levels == 0 && P.bs_cluster_min > 0 && d.n >= P.bs_cluster_min) ? 2 : 1;
}

void launch_bs(const Dev& d, const Phys& P, double h, cudaStream_t st, cudaStream_t side) {
  int grid = d.n < 2 * 148 ? d.n : 2 * 148;
  if (grid < 1) grid = 1;
  if (P.ml_levels > 0) {
    k_bs_t<true><<<grid, BNT, 0, st>>>(d, P, h);
    return;
  }
  // <= 48 KB for bs_kmax <= 12 (2 warps x 8 slots x 376 doubles)
  const size_t wsm = (size_t)(BNT / 32) * kWarpGroupMax * d.bs_stride * sizeof(double);
  k_bs_t<false><<<grid, BNT, wsm, st>>>(d, P, h);
  // the cluster solver takes the other groups (disjoint rows of gnew): on the
  // side stream, when there is one, it runs beside the warp and CTA solver
  if (bs_launches(d, P) == 2) launch_bs_cluster(d, P, h, side ? side : st);
}

// ---------------------------------------------------------------------------
constexpr int SNT = 256;

__global__ void __launch_bounds__(SNT) k_scatter(Dev d) {
  __shared__ int s_stop, s_ng, s_M;
  __shared__ double red[3 * 32 + 3];
  Ctrl* C = d.ctrl;
  if (threadIdx.x == 0) {
    s_stop = C->status;
    s_ng = C->n_groups;
    s_M = C->n_members;
  }
  __syncthreads();
  if (s_stop || s_ng == 0) return;
  const int M = s_M;
  double px = 0.0, py = 0.0, pz = 0.0;
  int dead = 0;
  for (int q = threadIdx.x; q < M; q += SNT) {
    const int b = d.grp_mem[q];
    if (!NB_GUARD(C, b >= 0 && b < d.n, 55)) continue;
    const double* g = d.gnew + (size_t)q * 10;
    const double mn = g[9] != 0.0 ? g[6] : 0.0;
    px += mn * g[3] - d.m[b] * d.vx[b];
    py += mn * g[4] - d.m[b] * d.vy[b];
    pz += mn * g[5] - d.m[b] * d.vz[b];
    dead += g[9] != 0.0 ? 0 : 1;
  }
  block_sum3(px, py, pz, red);
  __shared__ int s_dead;
  if (threadIdx.x == 0) s_dead = 0;
  __syncthreads();
  atomicAdd(&s_dead, dead);
  __syncthreads();
  if (threadIdx.x == 0) {
    C->dP[0] = px;
    C->dP[1] = py;
    C->dP[2] = pz;
    double El = 0.0;
    for (int g = 0; g < s_ng; ++g) El += d.gEl[g];
    C->E_lost += El;
    C->n_active -= s_dead;
    C->n_fprev = 0;  // rebuilt by k_member_kick
  }
  __syncthreads();
  for (int q = threadIdx.x; q < M; q += SNT) {
    const int b = d.grp_mem[q];
    if (!NB_GUARD(C, b >= 0 && b < d.n, 56)) continue;
    const double* g = d.gnew + (size_t)q * 10;
    if (g[9] != 0.0) {
      d.x[b] = g[0]; d.y[b] = g[1]; d.z[b] = g[2];
      d.vx[b] = g[3]; d.vy[b] = g[4]; d.vz[b] = g[5];
      d.m[b] = g[6]; d.R[b] = g[7]; d.rc[b] = g[8]; d.rc2[b] = g[8] * g[8];
    } else {  // absorbed: a massless slot far from every body, never flagged
      d.alive[b] = 0;
      d.x[b] = kDeadOffset * (double)(d.id[b] + 1);
      d.y[b] = 0.0; d.z[b] = 0.0;
      d.vx[b] = 0.0; d.vy[b] = 0.0; d.vz[b] = 0.0;
      d.m[b] = 0.0; d.R[b] = 0.0; d.rc[b] = 0.0; d.rc2[b] = 0.0;
    }
  }
}

void launch_scatter(const Dev& d, const Phys& P, cudaStream_t st) {
  (void)P;
  k_scatter<<<1, SNT, 0, st>>>(d);
}

}  // namespace nb
