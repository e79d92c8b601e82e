// O(N) parts of the step: the kick flow of H_B with the cached force (Eq. Hb),
// the momentum drift of H_C (Eq. Hc) and the Kepler drift of H_A's first sum
// (Eq. Ha), plus system initialisation.
//
// One step is B(h/2) C(h/2) A(h) C(h/2) B(h/2). k_open applies the first
// B(h/2); k_drift applies C(h/2), saves the state for the close-encounter
// solver and Kepler-drifts every body; k_close applies C(h/2) and B(h/2) and,
// between two steps of one call, the next step's opening B(h/2) as a second,
// separate addition. Partial momenta are summed per block in a fixed order
// and re-reduced in a fixed order by the consumer, so results are
// deterministic.
#include "kepler.cuh"
#include "nb_internal.cuh"

namespace nb {

constexpr int DNT = 256;  // threads per block of the O(N) kernels

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DNT) k_open(Dev d, double hh) {
  __shared__ int s_stop;
  __shared__ double red[3 * 32 + 3];
  if (threadIdx.x == 0) s_stop = d.ctrl->status;
  __syncthreads();
  if (s_stop) return;
  const int i = blockIdx.x * DNT + threadIdx.x;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (i < d.n && d.alive[i]) {
    // explicit FMAs: the same rounding as the fused opening kick of k_close
    const double vx = __fma_rn(hh, d.ax[i], d.vx[i]);
    const double vy = __fma_rn(hh, d.ay[i], d.vy[i]);
    const double vz = __fma_rn(hh, d.az[i], d.vz[i]);
    d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
    const double m = d.m[i];
    px = m * vx; py = m * vy; pz = m * vz;
  }
  block_sum3(px, py, pz, red);
  if (threadIdx.x == 0) {
    d.ppartA[3 * blockIdx.x] = px;
    d.ppartA[3 * blockIdx.x + 1] = py;
    d.ppartA[3 * blockIdx.x + 2] = pz;
  }
}

__global__ void __launch_bounds__(DNT) k_drift(Dev d, Phys P, double h) {
  __shared__ int s_stop;
  __shared__ double red[3 * 32 + 3];
  __shared__ unsigned long long s_it;
  if (threadIdx.x == 0) {
    s_stop = d.ctrl->status;
    s_it = 0ull;
  }
  __syncthreads();
  if (s_stop) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.ctrl->n_ftrial = 0;  // consumed by the next kick
  double Pt[3];
  reduce_parts3(d.ppartA, d.ppart_n, red, Pt);
  const double hh = 0.5 * h;
  const int i = blockIdx.x * DNT + threadIdx.x;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (i < d.n && d.alive[i]) {
    double x = d.x[i] + hh * Pt[0] / P.m0;
    double y = d.y[i] + hh * Pt[1] / P.m0;
    double z = d.z[i] + hh * Pt[2] / P.m0;
    double vx = d.vx[i], vy = d.vy[i], vz = d.vz[i];
    d.xs[i] = x; d.ys[i] = y; d.zs[i] = z;
    d.vxs[i] = vx; d.vys[i] = vy; d.vzs[i] = vz;
    int it = 0;
    const int st = kepler_drift(P.mu, x, y, z, vx, vy, vz, h, P.kepler_max_iter, &it);
    if (st) set_status(d.ctrl, st, 10);
    atomicAdd(&s_it, (unsigned long long)it);
    d.x[i] = x; d.y[i] = y; d.z[i] = z;
    d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
    const double m = d.m[i];
    px = m * vx; py = m * vy; pz = m * vz;
  }
  block_sum3(px, py, pz, red);
  if (threadIdx.x == 0) {
    d.ppartB[3 * blockIdx.x] = px;
    d.ppartB[3 * blockIdx.x + 1] = py;
    d.ppartB[3 * blockIdx.x + 2] = pz;
    atomicAdd(&d.ctrl->stats[ST_KEPLER_ITERS], s_it);
  }
}

__global__ void __launch_bounds__(DNT) k_close(Dev d, Phys P, double h, int last) {
  __shared__ int s_stop;
  __shared__ double red[3 * 32 + 3];
  if (threadIdx.x == 0) s_stop = d.ctrl->status;
  __syncthreads();
  if (s_stop) return;
  double Pt[3];
  reduce_parts3(d.ppartB, d.ppart_n, red, Pt);
  if (d.ctrl->n_groups > 0) {
    Pt[0] += d.ctrl->dP[0];
    Pt[1] += d.ctrl->dP[1];
    Pt[2] += d.ctrl->dP[2];
  }
  const double hh = 0.5 * h;
  const int i = blockIdx.x * DNT + threadIdx.x;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (i < d.n && d.alive[i]) {
    d.x[i] += hh * Pt[0] / P.m0;
    d.y[i] += hh * Pt[1] / P.m0;
    d.z[i] += hh * Pt[2] / P.m0;
    const double ax = d.ax[i], ay = d.ay[i], az = d.az[i];
    double vx = __fma_rn(hh, ax, d.vx[i]), vy = __fma_rn(hh, ay, d.vy[i]),
           vz = __fma_rn(hh, az, d.vz[i]);
    if (!last) {  // the next step's opening B(h/2), rounded as k_open rounds it
      vx = __fma_rn(hh, ax, vx);
      vy = __fma_rn(hh, ay, vy);
      vz = __fma_rn(hh, az, vz);
      const double m = d.m[i];
      px = m * vx; py = m * vy; pz = m * vz;
    }
    d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
  }
  if (!last) {
    block_sum3(px, py, pz, red);
    if (threadIdx.x == 0) {
      d.ppartA[3 * blockIdx.x] = px;
      d.ppartA[3 * blockIdx.x + 1] = py;
      d.ppartA[3 * blockIdx.x + 2] = pz;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctrl->step_index += 1;
    d.ctrl->stats[ST_STEPS] += 1ull;
  }
}

int ppart_blocks(int n) { return (n + DNT - 1) / DNT; }

void launch_open_h(const Dev& d, double h, cudaStream_t st) {
  k_open<<<d.ppart_n, DNT, 0, st>>>(d, 0.5 * h);
}

void launch_drift_h(const Dev& d, const Phys& P, double h, cudaStream_t st) {
  k_drift<<<d.ppart_n, DNT, 0, st>>>(d, P, h);
}

void launch_close_h(const Dev& d, const Phys& P, double h, int last, cudaStream_t st) {
  k_close<<<d.ppart_n, DNT, 0, st>>>(d, P, h, last);
}

// ---------------------------------------------------------------------------
// Initialisation from staged inputs: interleaved x, v [n][3], m, R, optional
// rc and ids. Validates and writes the SoA state.
// ---------------------------------------------------------------------------
struct InitIn {
  const double *x3, *v3, *m, *R, *rc;
  const int* ids;
};

__global__ void __launch_bounds__(DNT) k_init(Dev d, Phys P, InitIn in) {
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= d.n) return;
  const double x = in.x3[3 * i], y = in.x3[3 * i + 1], z = in.x3[3 * i + 2];
  const double vx = in.v3[3 * i], vy = in.v3[3 * i + 1], vz = in.v3[3 * i + 2];
  const double m = in.m[i], R = in.R[i];
  bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) &&
            isfinite(vz) && isfinite(m) && m > 0.0 && isfinite(R) && R >= 0.0;
  // the kick's fixed-point positions cover |x| < 2^38 AU
  ok = ok && fabs(x) < kPosMax && fabs(y) < kPosMax && fabs(z) < kPosMax;
  ok = ok && (x != 0.0 || y != 0.0 || z != 0.0);
  double rc = 0.0;
  if (in.rc) {
    rc = in.rc[i];
    ok = ok && isfinite(rc) && rc > 0.0;
  } else if (ok) {
    rc = rcrit(P, x, y, z, vx, vy, vz, m);
    ok = ok && isfinite(rc) && rc > 0.0;
  }
  int id = i;
  if (in.ids) {
    id = in.ids[i];
    if (i > 0 && in.ids[i - 1] >= id) ok = false;
  }
  if (!ok) set_status(d.ctrl, NB_E_INVALID, 20);
  d.x[i] = x; d.y[i] = y; d.z[i] = z;
  d.vx[i] = vx; d.vy[i] = vy; d.vz[i] = vz;
  d.m[i] = m; d.R[i] = R; d.rc[i] = rc; d.rc2[i] = rc * rc;
  d.ax[i] = d.ay[i] = d.az[i] = 0.0;
  d.id[i] = id;
  d.alive[i] = 1;
  d.member_slot[i] = -1;
}

void launch_init_in(const Dev& d, const Phys& P, const double* x3, const double* v3,
                    const double* m, const double* R, const double* rc, const int* ids,
                    cudaStream_t st) {
  InitIn in{x3, v3, m, R, rc, ids};
  k_init<<<d.ppart_n, DNT, 0, st>>>(d, P, in);
}

__global__ void k_fsal_init(Dev d, const int* cond) {
  __shared__ int s_n;
  if (cond && *cond == 0) return;
  if (threadIdx.x == 0) {
    int nt = d.ctrl->n_ftrial;
    if (nt > d.pair_cap) {
      set_status(d.ctrl, NB_E_OVERFLOW, 21);
      nt = d.pair_cap;
    }
    s_n = nt;
    d.ctrl->n_fprev = nt;
    d.ctrl->stats[ST_FORCE_EVALS] += 1ull;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < s_n; k += blockDim.x) d.fprev[k] = d.ftrial[k];
}

void launch_fsal_init(const Dev& d, cudaStream_t st, const int* cond) {
  k_fsal_init<<<1, 1024, 0, st>>>(d, cond);
}

// Eq. rcrit for every live body from its current state (rcrit_refresh = 1,
// at the start of a step); clears the trial-flag count for the force
// evaluation that follows.
__global__ void __launch_bounds__(DNT) k_refresh_rcrit(Dev d, Phys P) {
  if (d.ctrl->status) return;
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i == 0) d.ctrl->n_ftrial = 0;
  if (i >= d.n || !d.alive[i]) return;
  const double rc = rcrit(P, d.x[i], d.y[i], d.z[i], d.vx[i], d.vy[i], d.vz[i], d.m[i]);
  d.rc[i] = rc;
  d.rc2[i] = rc * rc;
}

void launch_refresh_rcrit(const Dev& d, const Phys& P, cudaStream_t st) {
  k_refresh_rcrit<<<d.ppart_n, DNT, 0, st>>>(d, P);
}

// ---------------------------------------------------------------------------
// Gas drag G(tau) by the implicit midpoint method (Eq. implicit):
// v' = v + tau a_f(x, (v + v') / 2), fixed-point iteration to 1e-15 of |v'|.
// a_f = -(C_D pi R^2 rho / (2 m)) |u| u, u = v + P / m0 - v_gas, the gas
// circling the star at (1 - eta) sqrt(G m0 / s), rho = rho0 s^-p (s the
// cylindrical radius). P (the momentum at the operator's start) is summed
// per block by k_gas_parts and re-reduced in a fixed order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DNT) k_gas_parts(Dev d) {
  __shared__ double red[3 * 32 + 3];
  if (d.ctrl->status) return;
  const int i = blockIdx.x * DNT + threadIdx.x;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (i < d.n && d.alive[i]) {
    const double m = d.m[i];
    px = m * d.vx[i]; py = m * d.vy[i]; pz = m * d.vz[i];
  }
  block_sum3(px, py, pz, red);
  if (threadIdx.x == 0) {
    d.ppartB[3 * blockIdx.x] = px;
    d.ppartB[3 * blockIdx.x + 1] = py;
    d.ppartB[3 * blockIdx.x + 2] = pz;
  }
}

__device__ __forceinline__ void drag_acc(const Phys& P, double x, double y, const double u0[3],
                                         double kcoef, double a[3]) {
  const double s = sqrt(x * x + y * y);
  double gx = 0.0, gy = 0.0;
  if (s > 0.0) {
    const double vk = (1.0 - P.gas_eta) * sqrt(P.G * P.m0 / s);
    gx = -vk * y / s;
    gy = vk * x / s;
  }
  const double ux = u0[0] - gx, uy = u0[1] - gy, uz = u0[2];
  const double un = sqrt(ux * ux + uy * uy + uz * uz);
  const double kd = kcoef * pow(s, -P.gas_p);
  a[0] = -kd * un * ux;
  a[1] = -kd * un * uy;
  a[2] = -kd * un * uz;
}

__global__ void __launch_bounds__(DNT) k_gas(Dev d, Phys P, double tau) {
  __shared__ int s_stop;
  __shared__ double red[3 * 32 + 3];
  if (threadIdx.x == 0) s_stop = d.ctrl->status;
  __syncthreads();
  if (s_stop) return;
  double Pt[3];
  reduce_parts3(d.ppartB, d.ppart_n, red, Pt);
  const double cx = Pt[0] / P.m0, cy = Pt[1] / P.m0, cz = Pt[2] / P.m0;
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= d.n || !d.alive[i] || !(d.R[i] > 0.0)) return;
  const double x = d.x[i], y = d.y[i];
  const double R = d.R[i];
  const double kcoef = P.gas_cd * 3.14159265358979323846 * R * R * P.gas_rho0 / (2.0 * d.m[i]);
  const double v0[3] = {d.vx[i], d.vy[i], d.vz[i]};
  double w[3] = {v0[0], v0[1], v0[2]};
  bool ok = false;
  for (int it = 0; it < P.gas_iter; ++it) {
    const double u[3] = {0.5 * (v0[0] + w[0]) + cx, 0.5 * (v0[1] + w[1]) + cy,
                         0.5 * (v0[2] + w[2]) + cz};
    double a[3];
    drag_acc(P, x, y, u, kcoef, a);
    double dmax = 0.0, wmax = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double wn = v0[k] + tau * a[k];
      dmax = fmax(dmax, fabs(wn - w[k]));
      wmax = fmax(wmax, fabs(wn));
      w[k] = wn;
    }
    if (dmax <= 1e-15 * wmax) {
      ok = true;
      break;
    }
  }
  if (!ok) set_status(d.ctrl, NB_E_NOCONV, 26);
  d.vx[i] = w[0];
  d.vy[i] = w[1];
  d.vz[i] = w[2];
}

void launch_gas(const Dev& d, const Phys& P, double tau, cudaStream_t st) {
  k_gas_parts<<<d.ppart_n, DNT, 0, st>>>(d);
  k_gas<<<d.ppart_n, DNT, 0, st>>>(d, P, tau);
}

// ---------------------------------------------------------------------------
// Ejection at the start of a step: bodies beyond eject_r leave, in ascending
// index order; each takes away its kinetic and star-potential energy, its
// mutual potential with the bodies still present and the change of the
// |P|^2 / (2 m0) term of Eq. Hc (booked in E_lost). One CTA; the scan is
// O(N) per step and each removal O(N) (removals are rare).
// ---------------------------------------------------------------------------
constexpr int ENT2 = 1024;

__global__ void __launch_bounds__(ENT2) k_eject(Dev d, Phys P) {
  __shared__ double red[3 * 32 + 3];
  __shared__ int s_next, s_count;
  if (d.ctrl->status) return;
  if (threadIdx.x == 0) s_count = 0;
  const double r2max = P.eject_r * P.eject_r;
  int start = 0;
  for (;;) {
    if (threadIdx.x == 0) s_next = d.n;
    __syncthreads();
    // the lowest index at or after `start` beyond eject_r
    for (int i = start + threadIdx.x; i < d.n; i += ENT2) {
      if (!d.alive[i]) continue;
      const double x = d.x[i], y = d.y[i], z = d.z[i];
      if (x * x + y * y + z * z > r2max) {
        atomicMin(&s_next, i);
        break;
      }
    }
    __syncthreads();
    const int e = s_next;
    if (e >= d.n) break;
    const double xe = d.x[e], ye = d.y[e], ze = d.z[e], me = d.m[e];
    const double vxe = d.vx[e], vye = d.vy[e], vze = d.vz[e];
    double px = 0.0, py = 0.0, pot = 0.0;
    double pz = 0.0;
    for (int j = threadIdx.x; j < d.n; j += ENT2) {
      if (!d.alive[j]) continue;
      const double mj = d.m[j];
      px += mj * d.vx[j]; py += mj * d.vy[j]; pz += mj * d.vz[j];
      if (j == e) continue;
      const double dx = d.x[j] - xe, dy = d.y[j] - ye, dz = d.z[j] - ze;
      pot -= P.G * me * mj / sqrt(dx * dx + dy * dy + dz * dz);
    }
    block_sum3(px, py, pz, red);
    double dum1 = 0.0, dum2 = 0.0;
    block_sum3(pot, dum1, dum2, red);
    if (threadIdx.x == 0) {
      const double P2 = px * px + py * py + pz * pz;
      const double qx = px - me * vxe, qy = py - me * vye, qz = pz - me * vze;
      const double Pn2 = qx * qx + qy * qy + qz * qz;
      const double v2 = vxe * vxe + vye * vye + vze * vze;
      const double r = sqrt(xe * xe + ye * ye + ze * ze);
      const double eb = 0.5 * me * v2 - P.G * P.m0 * me / r;
      Ctrl* C = d.ctrl;
      C->E_lost += eb + pot + (P2 - Pn2) / (2.0 * P.m0);
      C->m_ejected += me;
      C->stats[ST_EJECTIONS] += 1ull;
      C->n_active -= 1;
      s_count += 1;
      d.alive[e] = 0;
      d.x[e] = kDeadOffset * (double)(d.id[e] + 1);
      d.y[e] = 0.0; d.z[e] = 0.0;
      d.vx[e] = 0.0; d.vy[e] = 0.0; d.vz[e] = 0.0;
      d.m[e] = 0.0; d.R[e] = 0.0; d.rc[e] = 0.0; d.rc2[e] = 0.0;
    }
    __syncthreads();
    start = e + 1;
  }
  if (threadIdx.x == 0) {
    d.ctrl->n_eject_step = s_count;
    if (s_count) d.ctrl->n_ftrial = 0;  // for the force evaluation that follows
  }
}

void launch_eject(const Dev& d, const Phys& P, cudaStream_t st) { k_eject<<<1, ENT2, 0, st>>>(d, P); }

// ---------------------------------------------------------------------------
// Standalone Kepler drift of interleaved device arrays.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DNT) k_kepler_raw(int n, double mu, double* x3, double* v3,
                                                    double h, int max_iter, int* status) {
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= n) return;
  double x = x3[3 * i], y = x3[3 * i + 1], z = x3[3 * i + 2];
  double vx = v3[3 * i], vy = v3[3 * i + 1], vz = v3[3 * i + 2];
  int it;
  const int st = kepler_drift(mu, x, y, z, vx, vy, vz, h, max_iter, &it);
  if (st) atomicCAS(status, 0, st);
  x3[3 * i] = x; x3[3 * i + 1] = y; x3[3 * i + 2] = z;
  v3[3 * i] = vx; v3[3 * i + 1] = vy; v3[3 * i + 2] = vz;
}

void launch_kepler_raw(int n, double mu, double* x3, double* v3, double dt, int max_iter,
                       int* status, cudaStream_t st) {
  if (n <= 0) return;
  k_kepler_raw<<<(n + DNT - 1) / DNT, DNT, 0, st>>>(n, mu, x3, v3, dt, max_iter, status);
}

}  // namespace nb

namespace nb {

// ---------------------------------------------------------------------------
// Gather the active bodies (ascending slot = ascending id) into interleaved
// outputs. One CTA scans the alive flags chunk by chunk.
// ---------------------------------------------------------------------------
struct GatherOut {
  double *x3, *v3, *m, *R, *rc;
  int* ids;
  int* count;
};

// The live bodies in slot order (ascending id), compacted: blocks of GNT
// slots count their live bodies (k_gather_count), then each block writes its
// own at the sum of the counts before it (k_gather), so the order is that of
// a sequential scan whatever the grid.
constexpr int GNT = 1024;
__global__ void __launch_bounds__(GNT) k_gather_count(Dev d, int* bcnt) {
  __shared__ int warp_tot[GNT / 32];
  const int i = blockIdx.x * GNT + threadIdx.x;
  const int f = (i < d.n && d.alive[i]) ? 1 : 0;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int t = __reduce_add_sync(0xffffffffu, warp_tot[threadIdx.x]);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(GNT) k_gather(Dev d, GatherOut o, const int* bcnt) {
  __shared__ int warp_tot[GNT / 32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
    int b = 0;
    for (int k = lane; k < (int)blockIdx.x; k += 32) b += bcnt[k];
    b = __reduce_add_sync(0xffffffffu, b);
    if (lane == 0) {
      s_base = b;
      if (blockIdx.x == gridDim.x - 1 && o.count) *o.count = b + bcnt[blockIdx.x];
    }
  }
  const int i = blockIdx.x * GNT + threadIdx.x;
  const int f = (i < d.n && d.alive[i]) ? 1 : 0;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  const int wpre = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[wid] = __popc(bal);
  __syncthreads();
  int off = 0;
  for (int w = 0; w < wid; ++w) off += warp_tot[w];
  const int pos = s_base + off + wpre;
  if (f) {
    if (o.x3) { o.x3[3 * pos] = d.x[i]; o.x3[3 * pos + 1] = d.y[i]; o.x3[3 * pos + 2] = d.z[i]; }
    if (o.v3) { o.v3[3 * pos] = d.vx[i]; o.v3[3 * pos + 1] = d.vy[i]; o.v3[3 * pos + 2] = d.vz[i]; }
    if (o.m) o.m[pos] = d.m[i];
    if (o.R) o.R[pos] = d.R[i];
    if (o.rc) o.rc[pos] = d.rc[i];
    if (o.ids) o.ids[pos] = d.id[i];
  }
}

// bcnt: one int per block of GNT slots (the workspace's union-find labels,
// free outside the encounter kernel)
void launch_gather(const Dev& d, double* x3, double* v3, double* m, double* R, double* rc,
                   int* ids, int* count, cudaStream_t st) {
  GatherOut o{x3, v3, m, R, rc, ids, count};
  const int nb = (d.n + GNT - 1) / GNT;
  k_gather_count<<<nb, GNT, 0, st>>>(d, d.uf);
  k_gather<<<nb, GNT, 0, st>>>(d, o, d.uf);
}

// Interleaved <-> SoA helpers for the cached force.
__global__ void __launch_bounds__(DNT) k_a_to_soa(Dev d, const double* a3) {
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= d.n) return;
  d.ax[i] = a3[3 * i];
  d.ay[i] = a3[3 * i + 1];
  d.az[i] = a3[3 * i + 2];
}

__global__ void __launch_bounds__(DNT) k_a_to_aos(Dev d, double* a3) {
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= d.n) return;
  a3[3 * i] = d.ax[i];
  a3[3 * i + 1] = d.ay[i];
  a3[3 * i + 2] = d.az[i];
}

void launch_a_convert(const Dev& d, double* a3, int to_soa, cudaStream_t st) {
  if (to_soa)
    k_a_to_soa<<<d.ppart_n, DNT, 0, st>>>(d, a3);
  else
    k_a_to_aos<<<d.ppart_n, DNT, 0, st>>>(d, a3);
}

// Standalone kick helpers: interleaved positions to SoA (+ rc^2), and the
// fixed-order sum of the j-chunk partials times G into interleaved a.
__global__ void __launch_bounds__(DNT) k_raw_prep(int n, const double* x3, const double* rc,
                                                  double* x, double* y, double* z, double* rc2,
                                                  Ctrl* ctrl) {
  const int i = blockIdx.x * DNT + threadIdx.x;
  if (i >= n) return;
  x[i] = x3[3 * i];
  y[i] = x3[3 * i + 1];
  z[i] = x3[3 * i + 2];
  rc2[i] = rc[i] * rc[i];
  // the kick's fixed-point positions cover |x| < 2^38 AU (NaN fails too)
  if (!(fabs(x[i]) < kPosMax && fabs(y[i]) < kPosMax && fabs(z[i]) < kPosMax))
    set_status(ctrl, NB_E_INVALID, 22);
}

// a3 holds rows [ib, ie): row i goes to a3[3 (i - ib)].
__global__ void __launch_bounds__(DNT) k_raw_finish(int n, int ib, int ie, int S,
                                                    const double* kpart, double G, double* a3) {
  const int i = ib + blockIdx.x * DNT + threadIdx.x;
  if (i >= ie) return;
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int s = 0; s < S; ++s) {
    const double* p = kpart + (size_t)(3 * s) * n;
    ax += p[i];
    ay += p[n + i];
    az += p[2 * n + i];
  }
  double* o = a3 + 3 * (size_t)(i - ib);
  o[0] = G * ax;
  o[1] = G * ay;
  o[2] = G * az;
}

void launch_raw_prep(int n, const double* x3, const double* rc, double* x, double* y, double* z,
                     double* rc2, Ctrl* ctrl, cudaStream_t st) {
  k_raw_prep<<<(n + DNT - 1) / DNT, DNT, 0, st>>>(n, x3, rc, x, y, z, rc2, ctrl);
}

void launch_raw_finish(int n, int ib, int ie, int S, const double* kpart, double G, double* a3,
                       cudaStream_t st) {
  if (ie <= ib) return;
  k_raw_finish<<<(ie - ib + DNT - 1) / DNT, DNT, 0, st>>>(n, ib, ie, S, kpart, G, a3);
}

}  // namespace nb
