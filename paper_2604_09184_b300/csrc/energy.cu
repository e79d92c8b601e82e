// Energy and momentum diagnostics: E = H_A + H_B + H_C (Eqs. Ha, Hb, Hc; the
// changeover K cancels between the close part of H_A and H_B, leaving the
// Newtonian pair sum), L = sum m x cross v, P = sum m v.
//
// The O(N^2) pair potential uses 1/r from the same float seed as the kick,
// refined to FP64 (second order in the residual). Per-thread and per-block
// sums are Neumaier-compensated; the final reduction runs in a fixed order.
#include <cmath>

#include "nb_internal.cuh"

namespace nb {

constexpr int ENT2 = 256;
constexpr int ECOMP = 8;  // KE + star potential, pair potential, L(3), P(3)

struct Neu {
  double s, c;
  __device__ void add(double x) {
    const double t = s + x;
    const double b = t - s;
    c += (s - (t - b)) + (x - b);
    s = t;
  }
};

__device__ __forceinline__ double inv_r(double r2) {
  const unsigned hr = (unsigned)__double2hiint(r2);
  const float r2f = __uint_as_float((hr << 3) + 0x40000000u);
  const unsigned yb = __float_as_uint(rsqrtf(r2f));
  const double y0 = __hiloint2double((int)((yb >> 3) + 0x38000000u), (int)(yb << 29));
  const double e = __fma_rn(-r2, y0 * y0, 1.0);  // y0 (1 - e)^(-1/2)
  return __fma_rn(y0, e * __fma_rn(0.375, e, 0.5), y0);
}

__global__ void __launch_bounds__(ENT2) k_energy_parts(Dev d, Phys P) {
  __shared__ double sx[ENT2], sy[ENT2], sz[ENT2], sm[ENT2];
  __shared__ double red[2 * ECOMP * ENT2];
  const int n = d.n;
  const int i = blockIdx.x * ENT2 + threadIdx.x;
  const bool live = i < n && d.alive[i];
  const double xi = live ? d.x[i] : 0.0, yi = live ? d.y[i] : 0.0, zi = live ? d.z[i] : 0.0;
  const double mi = live ? d.m[i] : 0.0;
  Neu pot{0.0, 0.0};
  for (int jt = 0; jt < n; jt += ENT2) {
    __syncthreads();
    const int j = jt + threadIdx.x;
    if (j < n) {
      sx[threadIdx.x] = d.x[j];
      sy[threadIdx.x] = d.y[j];
      sz[threadIdx.x] = d.z[j];
      sm[threadIdx.x] = d.m[j];
    }
    __syncthreads();
    const int cnt = min(ENT2, n - jt);
    if (live) {
      double t = 0.0;
      for (int q = 0; q < cnt; ++q) {
        const double dx = sx[q] - xi, dy = sy[q] - yi, dz = sz[q] - zi;
        const double r2 = sep2(dx, dy, dz);
        if (r2 == 0.0) continue;
        t += sm[q] * inv_r(r2);
      }
      pot.add(t);
    }
  }
  double v[ECOMP] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (live) {
    const double vx = d.vx[i], vy = d.vy[i], vz = d.vz[i];
    const double r = sqrt(xi * xi + yi * yi + zi * zi);
    v[0] = 0.5 * mi * (vx * vx + vy * vy + vz * vz) - P.G * P.m0 * mi / r;
    v[1] = -0.5 * P.G * mi * (pot.s + pot.c);  // each pair is counted twice
    v[2] = mi * (yi * vz - zi * vy);
    v[3] = mi * (zi * vx - xi * vz);
    v[4] = mi * (xi * vy - yi * vx);
    v[5] = mi * vx;
    v[6] = mi * vy;
    v[7] = mi * vz;
  }
  for (int k = 0; k < ECOMP; ++k) red[k * ENT2 + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < ECOMP) {
    Neu a{0.0, 0.0};
    for (int t = 0; t < ENT2; ++t) a.add(red[threadIdx.x * ENT2 + t]);
    d.eparts[2 * (ECOMP * blockIdx.x + threadIdx.x)] = a.s;
    d.eparts[2 * (ECOMP * blockIdx.x + threadIdx.x) + 1] = a.c;
  }
}

__global__ void k_energy_final(Dev d, Phys P, int nblocks, double* out8) {
  __shared__ double acc[ECOMP];
  if (threadIdx.x < ECOMP) {
    Neu a{0.0, 0.0};
    for (int b = 0; b < nblocks; ++b) {
      a.add(d.eparts[2 * (ECOMP * b + threadIdx.x)]);
      a.add(d.eparts[2 * (ECOMP * b + threadIdx.x) + 1]);
    }
    acc[threadIdx.x] = a.s + a.c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double Px = acc[5], Py = acc[6], Pz = acc[7];
    Neu e{0.0, 0.0};
    e.add(acc[0]);
    e.add(acc[1]);
    e.add((Px * Px + Py * Py + Pz * Pz) / (2.0 * P.m0));
    out8[0] = e.s + e.c;
    out8[1] = acc[2];
    out8[2] = acc[3];
    out8[3] = acc[4];
    out8[4] = Px;
    out8[5] = Py;
    out8[6] = Pz;
    out8[7] = d.ctrl->E_lost;
  }
}

int energy_blocks(int n) { return (n + ENT2 - 1) / ENT2; }

// ---------------------------------------------------------------------------
// Gradient of E = H_A + H_B + H_C with respect to the state (x, v, m) of the
// live bodies, for losses that contain the total energy:
//   dE/dx_i = G m_i (m0 x_i / |x_i|^3 + sum_j m_j (x_i - x_j) / r_ij^3)
//   dE/dv_i = m_i (v_i + P / m0)                      (P = sum_j m_j v_j)
//   dE/dm_i = |v_i|^2 / 2 - G m0 / |x_i| - G sum_j m_j / r_ij + P . v_i / m0
// Arrays interleaved [n][3] as at the boundary. P is reduced in a fixed order
// (per-block Neumaier sums, then the blocks in order), so results do not
// depend on the launch.
constexpr int EGT = 256;

__global__ void __launch_bounds__(EGT) k_egrad_momentum(int n, const double* __restrict__ v,
                                                        const double* __restrict__ m,
                                                        const int* __restrict__ alive,
                                                        double* __restrict__ parts) {
  __shared__ double red[3 * EGT];
  const int i = blockIdx.x * EGT + threadIdx.x;
  const bool live = i < n && (!alive || alive[i]);
  for (int k = 0; k < 3; ++k) red[k * EGT + threadIdx.x] = live ? m[i] * v[3 * i + k] : 0.0;
  __syncthreads();
  if (threadIdx.x < 3) {
    Neu a{0.0, 0.0};
    for (int t = 0; t < EGT; ++t) a.add(red[threadIdx.x * EGT + t]);
    parts[2 * (3 * blockIdx.x + threadIdx.x)] = a.s;
    parts[2 * (3 * blockIdx.x + threadIdx.x) + 1] = a.c;
  }
}

// Source chunks of the pair sums: about 8 CTAs per SM over target tiles x
// chunks, chunks of at least 64 sources, at most 64 chunks. Depends on n only.
constexpr int EPT = 128;  // targets (threads) per CTA of the pair sums
inline int egrad_split(int n) {
  const int tiles = (n + EPT - 1) / EPT;
  int S = (8 * 148 + tiles - 1) / tiles;
  if (S > n / 64) S = n / 64;
  if (S > 64) S = 64;
  return S < 1 ? 1 : S;
}

// Partial pair sums of the j-chunk blockIdx.y for the targets of the tile
// blockIdx.x: sum_j m_j (x_i - x_j) / r^3 and sum_j m_j / r into part
// [S][4][n]. r^2 on the integer pipe and 1/r from the seeded reciprocal root.
__global__ void __launch_bounds__(EPT) k_egrad_pairs(int n, int chunk, const double* __restrict__ x,
                                                    const double* __restrict__ m,
                                                    const int* __restrict__ alive,
                                                    double* __restrict__ part) {
  __shared__ double sx[EPT], sy[EPT], sz[EPT], sm[EPT];
  const int i = blockIdx.x * EPT + threadIdx.x;
  const bool live = i < n && (!alive || alive[i]);
  const double xi = live ? x[3 * i] : 0.0, yi = live ? x[3 * i + 1] : 0.0,
               zi = live ? x[3 * i + 2] : 0.0;
  const int j0 = blockIdx.y * chunk, j1 = min(n, j0 + chunk);
  double fx = 0.0, fy = 0.0, fz = 0.0, pot = 0.0;
  for (int jt = j0; jt < j1; jt += EPT) {
    __syncthreads();
    const int j = jt + threadIdx.x;
    if (j < j1) {
      sx[threadIdx.x] = x[3 * j];
      sy[threadIdx.x] = x[3 * j + 1];
      sz[threadIdx.x] = x[3 * j + 2];
      sm[threadIdx.x] = (!alive || alive[j]) ? m[j] : 0.0;
    }
    __syncthreads();
    const int cnt = min(EPT, j1 - jt);
    if (live) {
      for (int q = 0; q < cnt; ++q) {
        const double dx = xi - sx[q], dy = yi - sy[q], dz = zi - sz[q];
        const double r2 = sep2_int(dx, dy, dz);
        if (__double_as_longlong(r2) == 0ll) continue;  // the body itself
        const double ir = rinv_fast(r2);
        const double mir = sm[q] * ir;
        const double mir3 = mir * (ir * ir);
        fx = __fma_rn(mir3, dx, fx);
        fy = __fma_rn(mir3, dy, fy);
        fz = __fma_rn(mir3, dz, fz);
        pot += mir;
      }
    }
  }
  if (i < n) {
    double* o = part + (size_t)blockIdx.y * 4 * n;
    o[i] = fx;
    o[n + i] = fy;
    o[2 * n + i] = fz;
    o[3 * n + i] = pot;
  }
}

// The chunks' partial sums in chunk order, the momentum from the per-block
// sums in block order, and the gradient of every body.
__global__ void __launch_bounds__(EGT) k_egrad(int n, int S, const double* __restrict__ part,
                                               const double* __restrict__ x,
                                               const double* __restrict__ v,
                                               const double* __restrict__ m,
                                               const int* __restrict__ alive, double G, double m0,
                                               int nparts, const double* __restrict__ parts,
                                               double* __restrict__ gx, double* __restrict__ gv,
                                               double* __restrict__ gm) {
  __shared__ double Psh[3];
  if (threadIdx.x < 3) {
    Neu a{0.0, 0.0};
    for (int b = 0; b < nparts; ++b) {
      a.add(parts[2 * (3 * b + threadIdx.x)]);
      a.add(parts[2 * (3 * b + threadIdx.x) + 1]);
    }
    Psh[threadIdx.x] = a.s + a.c;
  }
  __syncthreads();
  const int i = blockIdx.x * EGT + threadIdx.x;
  if (i >= n) return;
  const bool live = !alive || alive[i];
  if (!live) {
    for (int k = 0; k < 3; ++k) {
      gx[3 * i + k] = 0.0;
      gv[3 * i + k] = 0.0;
    }
    gm[i] = 0.0;
    return;
  }
  double fx = 0.0, fy = 0.0, fz = 0.0, pot = 0.0;
  for (int c = 0; c < S; ++c) {
    const double* o = part + (size_t)c * 4 * n;
    fx += o[i];
    fy += o[n + i];
    fz += o[2 * n + i];
    pot += o[3 * n + i];
  }
  const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
  const double mi = m[i];
  const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
  const double r = sqrt(xi * xi + yi * yi + zi * zi);
  const double c0 = m0 / (r * r * r);
  gx[3 * i] = G * mi * __fma_rn(c0, xi, fx);
  gx[3 * i + 1] = G * mi * __fma_rn(c0, yi, fy);
  gx[3 * i + 2] = G * mi * __fma_rn(c0, zi, fz);
  const double Px = Psh[0], Py = Psh[1], Pz = Psh[2];
  gv[3 * i] = mi * (vx + Px / m0);
  gv[3 * i + 1] = mi * (vy + Py / m0);
  gv[3 * i + 2] = mi * (vz + Pz / m0);
  gm[i] = 0.5 * (vx * vx + vy * vy + vz * vz) - G * m0 / r - G * pot +
          (Px * vx + Py * vy + Pz * vz) / m0;
}

void launch_energy(const Dev& d, const Phys& P, double* out8, cudaStream_t st) {
  const int nb = energy_blocks(d.n);
  k_energy_parts<<<nb, ENT2, 0, st>>>(d, P);
  k_energy_final<<<1, 32, 0, st>>>(d, P, nb, out8);
}

}  // namespace nb

extern "C" size_t nb_energy_grad_scratch_bytes(int n) {
  if (n < 1) return 0;
  // the momentum's per-block sums, then the pair sums' partials (256-byte aligned)
  const size_t mom = (sizeof(double) * 6 * (size_t)((n + nb::EGT - 1) / nb::EGT) + 255) & ~(size_t)255;
  return mom + sizeof(double) * 4 * (size_t)n * (size_t)nb::egrad_split(n);
}

extern "C" int nb_energy_grad(int n, const double* x, const double* v, const double* m,
                              const int* alive, double G, double m0, double* gx, double* gv,
                              double* gm, void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 1 || !x || !v || !m || !gx || !gv || !gm) return NB_E_INVALID;
  if (!std::isfinite(G) || !std::isfinite(m0) || !(m0 > 0.0)) return NB_E_INVALID;
  if (!scratch || scratch_bytes < nb_energy_grad_scratch_bytes(n) || ((uintptr_t)scratch & 7))
    return NB_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (n + nb::EGT - 1) / nb::EGT;
  const int S = nb::egrad_split(n);
  double* parts = (double*)scratch;
  double* part = (double*)((char*)scratch +
                           ((sizeof(double) * 6 * (size_t)nb + 255) & ~(size_t)255));
  nb::k_egrad_momentum<<<nb, nb::EGT, 0, st>>>(n, v, m, alive, parts);
  nb::k_egrad_pairs<<<dim3((n + nb::EPT - 1) / nb::EPT, S), nb::EPT, 0, st>>>(
      n, (n + S - 1) / S, x, m, alive, part);
  nb::k_egrad<<<nb, nb::EGT, 0, st>>>(n, S, part, x, v, m, alive, G, m0, nb, parts, gx, gv, gm);
  if (cudaGetLastError() != cudaSuccess) return NB_E_CUDA;
  return NB_OK;
}
