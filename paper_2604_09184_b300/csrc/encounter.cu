// Close encounters: the encounter set, independent groups, and the direct
// solver for H_A restricted to each group (section "The hybrid symplectic
// integrator"; groups per section "Increasing N"; perfect mergers per
// "Detailing the outcomes of collisions").
//
// k_encounter (one CTA): E = F_prev U F_trial as sorted unique (i, j) keys,
//   appended to the encounter log; connected components of E by union-find;
//   member slots ordered by (smallest member, body).
// k_bs (one CTA per group, grid-stride): Gragg modified midpoint with
//   n_k = 2k substeps and Neville extrapolation in the substep squared,
//   restarting from the state saved after C(h/2). Substep halving on
//   failure, doubling back after an early success on an aligned boundary,
//   merging scan after every accepted substep.
// k_scatter (one CTA): momentum change of the group bodies, energy removed
//   by mergers, and the write-back of the group results.
#include "nb_internal.cuh"

namespace nb {

constexpr int ENT = 1024;  // threads of k_encounter
constexpr int BNT = 64;    // threads of a BS CTA

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

__device__ __forceinline__ int uf_find(int* uf, int k) {
  while (uf[k] != k) {
    uf[k] = uf[uf[k]];
    k = uf[k];
  }
  return k;
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

__global__ void __launch_bounds__(ENT) k_encounter(Dev d) {
  __shared__ int s_stop, s_nT, s_nP, s_nE, s_nb, s_step;
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
  for (int q = threadIdx.x; q < nprev; q += ENT) d.member_slot[d.grp_mem[q]] = -1;
  const int nT = s_nT, nP = s_nP, nK = nT + nP;
  // region A holds <= next_pow2(2 pair_cap) pair keys and later <= 4 pair_cap
  // group keys; region B holds <= 4 pair_cap body keys (pair_cap is a power of 2)
  unsigned long long* kA = d.keys;
  unsigned long long* kB = d.keys + 4 * (size_t)d.pair_cap;
  const int P2 = next_pow2(nK > 0 ? nK : 1);
  for (int k = threadIdx.x; k < P2; k += ENT) {
    unsigned long long key = ~0ull;
    if (k < nP) {
      const int2 p = d.fprev[k];
      key = ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.y;
    } else if (k < nK) {
      const int2 p = d.ftrial[k - nP];
      key = ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.y;
    }
    kA[k] = key;
  }
  __syncthreads();
  bitonic_sort(kA, P2);
  if (threadIdx.x == 0) {
    int ne = 0;
    for (int k = 0; k < nK; ++k) {
      if (ne > 0 && kA[k] == kA[ne - 1]) continue;
      kA[ne++] = kA[k];
    }
    s_nE = ne;
  }
  __syncthreads();
  const int nE = s_nE;
  // encounter log: (step, id_i, id_j)
  const int base = C->n_log;
  for (int k = threadIdx.x; k < nE; k += ENT) {
    const int pos = base + k;
    if (pos < d.log_cap) {
      const int i = (int)(kA[k] >> 32), j = (int)(kA[k] & 0xffffffffu);
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
  if (threadIdx.x == 0) {
    int nb = 0;
    for (int k = 0; k < 2 * nE; ++k) {
      if (nb > 0 && kB[k] == kB[nb - 1]) continue;
      kB[nb++] = kB[k];
    }
    s_nb = nb;
    for (int k = 0; k < nb; ++k) d.uf[k] = k;
    // union by the smaller local index (= smaller body index)
    for (int k = 0; k < nE; ++k) {
      const int a = lower_bound_u64(kB, nb, kA[k] >> 32);
      const int b = lower_bound_u64(kB, nb, kA[k] & 0xffffffffu);
      const int ra = uf_find(d.uf, a), rb = uf_find(d.uf, b);
      if (ra < rb)
        d.uf[rb] = ra;
      else if (rb < ra)
        d.uf[ra] = rb;
    }
    for (int k = 0; k < nb; ++k) d.uf[k] = uf_find(d.uf, k);  // flatten
  }
  __syncthreads();
  const int nb = s_nb;
  // group keys (root body, body) reuse region A
  const int P2g = next_pow2(nb);
  for (int k = threadIdx.x; k < P2g; k += ENT) {
    unsigned long long v = ~0ull;
    if (k < nb) v = (kB[d.uf[k]] << 32) | kB[k];
    kA[k] = v;
  }
  __syncthreads();
  bitonic_sort(kA, P2g);
  for (int k = threadIdx.x; k < nb; k += ENT) {
    const int body = (int)(kA[k] & 0xffffffffu);
    d.grp_mem[k] = body;
    d.member_slot[body] = k;
  }
  if (threadIdx.x == 0) {
    int g = 0;
    for (int k = 0; k < nb; ++k)
      if (k == 0 || (kA[k] >> 32) != (kA[k - 1] >> 32)) d.grp_off[g++] = k;
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
// Bulirsch-Stoer for one group per CTA.
// Scratch per member slot (stride doubles): y[6] | zm[6] | zc[6] | f[6] |
// T[2][kmax][6]. Working copies of m, R, rc, alive live in gnew[slot*10+6..9].
// ---------------------------------------------------------------------------
constexpr int OY = 0, OZM = 6, OZC = 12, OF = 18, OT = 24;

struct BsCtx {
  double* base;  // scratch of the group's first slot
  double* g;     // gnew of the group's first slot
  int stride, M, kmax;
  double G, mu;
};

__device__ __forceinline__ bool bs_alive(const BsCtx& c, int b) { return c.g[10 * b + 9] != 0.0; }

// f = d/dt of field fo for member b (Eq. Ha restricted to the group).
__device__ void bs_deriv(const BsCtx& c, int fo, int b) {
  const double* yb = c.base + (size_t)b * c.stride + fo;
  double* fb = c.base + (size_t)b * c.stride + OF;
  if (!bs_alive(c, b)) {
    for (int k = 0; k < 6; ++k) fb[k] = 0.0;
    return;
  }
  fb[0] = yb[3];
  fb[1] = yb[4];
  fb[2] = yb[5];
  const double r2 = yb[0] * yb[0] + yb[1] * yb[1] + yb[2] * yb[2];
  const double r = sqrt(r2);
  const double ks = -c.mu / (r2 * r);
  double ax = ks * yb[0], ay = ks * yb[1], az = ks * yb[2];
  const double rcb = c.g[10 * b + 8];
  for (int q = 0; q < c.M; ++q) {
    if (q == b || !bs_alive(c, q)) continue;
    const double* yq = c.base + (size_t)q * c.stride + fo;
    const double dx = yq[0] - yb[0], dy = yq[1] - yb[1], dz = yq[2] - yb[2];
    const double q2 = sep2(dx, dy, dz);
    if (q2 == 0.0) continue;
    const double rc = fmax(rcb, c.g[10 * q + 8]);
    if (!(q2 < rc * rc)) continue;  // 1 - w = 0 beyond rc
    const double qq = sqrt(q2);
    const double w = kick_weight(qq, rc);
    const double f = c.G * c.g[10 * q + 6] * (1.0 - w) / (q2 * qq);
    ax += f * dx;
    ay += f * dy;
    az += f * dz;
  }
  fb[3] = ax;
  fb[4] = ay;
  fb[5] = az;
}

__device__ double pair_energy(const Phys& P, const double* a, double ma, const double* b,
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

// Perfect merging on contact, scanned in ascending slot (= body) order.
__device__ void bs_merge_scan(const BsCtx& c, const Phys& P, double* El, int* merges) {
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
      *merges += 1;
    }
  }
}

__global__ void __launch_bounds__(BNT) k_bs(Dev d, Phys P, double h) {
  __shared__ int s_stop, s_ng;
  __shared__ double s_err[BNT];
  __shared__ int s_acc, s_kacc;
  if (threadIdx.x == 0) {
    s_stop = d.ctrl->status;
    s_ng = d.ctrl->n_groups;
  }
  __syncthreads();
  if (s_stop) return;
  const int kmax = P.bs_kmax;
  long long derivs = 0, substeps = 0, halvings = 0;
  int merges = 0;
  for (int grp = blockIdx.x; grp < s_ng; grp += gridDim.x) {
    const int off = d.grp_off[grp];
    BsCtx c;
    c.M = d.grp_off[grp + 1] - off;
    c.stride = d.bs_stride;
    c.base = d.gscr + (size_t)off * d.bs_stride;
    c.g = d.gnew + (size_t)off * 10;
    c.kmax = kmax;
    c.G = P.G;
    c.mu = P.mu;
    for (int b = threadIdx.x; b < c.M; b += BNT) {
      const int body = d.grp_mem[off + b];
      double* y = c.base + (size_t)b * c.stride + OY;
      y[0] = d.xs[body]; y[1] = d.ys[body]; y[2] = d.zs[body];
      y[3] = d.vxs[body]; y[4] = d.vys[body]; y[5] = d.vzs[body];
      double* g = c.g + 10 * b;
      g[6] = d.m[body];
      g[7] = d.R[body];
      g[8] = d.rc[body];
      g[9] = 1.0;
    }
    __syncthreads();
    double El = 0.0;
    int level = 0;
    long long done = 0;
    int status = 0;
    long long attempts = 0;
    while (done < (1ll << level)) {
      const double H = ldexp(h, -level);
      if (threadIdx.x == 0) {
        s_acc = 0;
        s_kacc = 0;
      }
      for (int j = 1; j <= kmax; ++j) {
        const int nsub = 2 * j;
        const double hs = H / nsub;
        for (int b = threadIdx.x; b < c.M; b += BNT) bs_deriv(c, OY, b);
        __syncthreads();
        for (int b = threadIdx.x; b < c.M; b += BNT) {
          double* s = c.base + (size_t)b * c.stride;
          for (int k = 0; k < 6; ++k) {
            s[OZM + k] = s[OY + k];
            s[OZC + k] = s[OY + k] + hs * s[OF + k];
          }
        }
        __syncthreads();
        for (int m = 1; m < nsub; ++m) {
          for (int b = threadIdx.x; b < c.M; b += BNT) bs_deriv(c, OZC, b);
          __syncthreads();
          for (int b = threadIdx.x; b < c.M; b += BNT) {
            double* s = c.base + (size_t)b * c.stride;
            for (int k = 0; k < 6; ++k) {
              const double zn = s[OZM + k] + 2.0 * hs * s[OF + k];
              s[OZM + k] = s[OZC + k];
              s[OZC + k] = zn;
            }
          }
          __syncthreads();
        }
        for (int b = threadIdx.x; b < c.M; b += BNT) bs_deriv(c, OZC, b);
        __syncthreads();
        derivs += nsub + 1;
        double emax = 0.0;
        for (int b = threadIdx.x; b < c.M; b += BNT) {
          double* s = c.base + (size_t)b * c.stride;
          double* Tc = s + OT + (j & 1) * kmax * 6;
          double* Tp = s + OT + ((j - 1) & 1) * kmax * 6;
          for (int k = 0; k < 6; ++k) Tc[k] = 0.5 * (s[OZC + k] + s[OZM + k] + hs * s[OF + k]);
          for (int q = 1; q < j; ++q) {
            const double ratio = (double)(2 * j) / (double)(2 * (j - q));
            const double den = ratio * ratio - 1.0;
            for (int k = 0; k < 6; ++k) {
              const double t = Tc[6 * (q - 1) + k];
              Tc[6 * q + k] = t + (t - Tp[6 * (q - 1) + k]) / den;
            }
          }
          if (j >= 3 && bs_alive(c, b)) {
            const double* A = Tc + 6 * (j - 1);
            const double* B = Tc + 6 * (j - 2);
            for (int part = 0; part < 2; ++part) {
              double dm = 0.0, ym = 0.0;
              for (int k = 3 * part; k < 3 * part + 3; ++k) {
                dm = fmax(dm, fabs(A[k] - B[k]));
                ym = fmax(ym, fabs(A[k]));
              }
              emax = fmax(emax, dm / (ym + 1e-300));
            }
          }
        }
        s_err[threadIdx.x] = emax;
        __syncthreads();
        if (threadIdx.x == 0) {
          double e = 0.0;
          for (int t = 0; t < BNT; ++t) e = fmax(e, s_err[t]);
          if (j >= 3 && e <= P.bs_tol) {
            s_acc = 1;
            s_kacc = j;
          }
        }
        __syncthreads();
        if (s_acc) {
          for (int b = threadIdx.x; b < c.M; b += BNT) {
            double* s = c.base + (size_t)b * c.stride;
            const double* Tc = s + OT + (j & 1) * kmax * 6 + 6 * (j - 1);
            for (int k = 0; k < 6; ++k) s[OY + k] = Tc[k];
          }
          __syncthreads();
          break;
        }
      }
      ++attempts;
      if (s_acc) {
        ++done;
        ++substeps;
        if (P.merge) {
          if (threadIdx.x == 0) bs_merge_scan(c, P, &El, &merges);
          __syncthreads();
        }
        if (level > 0 && (done & 1) == 0 && s_kacc <= kmax - 2) {
          --level;
          done >>= 1;
        }
      } else {
        ++halvings;
        if (level >= P.bs_max_halvings) {
          status = NB_E_NOCONV;
          break;
        }
        ++level;
        done *= 2;
      }
      if (attempts > 200000) {
        status = NB_E_TIMEOUT;
        break;
      }
      __syncthreads();
    }
    if (status && threadIdx.x == 0) set_status(d.ctrl, status, 30);
    for (int b = threadIdx.x; b < c.M; b += BNT) {
      const double* y = c.base + (size_t)b * c.stride + OY;
      double* g = c.g + 10 * b;
      for (int k = 0; k < 6; ++k) g[k] = y[k];
    }
    if (threadIdx.x == 0) d.gEl[grp] = El;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&d.ctrl->stats[ST_BS_DERIVS], (unsigned long long)derivs);
    atomicAdd(&d.ctrl->stats[ST_BS_SUBSTEPS], (unsigned long long)substeps);
    atomicAdd(&d.ctrl->stats[ST_BS_HALVINGS], (unsigned long long)halvings);
    atomicAdd(&d.ctrl->stats[ST_MERGES], (unsigned long long)merges);
  }
}

void launch_bs(const Dev& d, const Phys& P, double h, cudaStream_t st) {
  int grid = d.n < 2 * 148 ? d.n : 2 * 148;
  if (grid < 1) grid = 1;
  k_bs<<<grid, BNT, 0, st>>>(d, P, h);
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
