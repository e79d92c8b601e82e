// C ABI of libnb (declared in include/nb.h): workspace layout, system
// lifetime, the step driver and the single-kernel entry points.
//
// Every step of the integrator runs in device kernels on the caller's
// stream; the host only orders launches, snapshots the state for rollback
// and reads the control block once per nb_step() call.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nb_internal.cuh"

using namespace nb;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int round_pow2(int v) {
  int p = 1;
  while (p < v && p < (1 << 30)) p <<= 1;
  return p;
}

int auto_split(int n) {
  // About 48 kick CTAs per SM over the launch per 256 targets (~97 for the
  // kernels' 128-target tiles), so the last partial wave is a small fraction
  // of the kernel: at N = 65538 the FP64 kick took 61.0, 60.0, 59.6, 58.9 and
  // 58.6 ms with S = 8, 14, 20, 28 and 64. Beyond S ~ 28 the partial sums
  // (S x 3 x N doubles) outgrow L2: at S = 56 the kick wrote 36.5 MB to DRAM
  // per launch (1.1 MB at S = 28) for a 0.4 ms gain, so S stays near 28.
  // At most 64 chunks of at least 32 sources (chunks of any length: at
  // N = 2049 whole 128-body chunks left 289 CTAs, two per SM).
  const int itiles = (n + 255) / 256;
  int S = (148 * 48 + itiles - 1) / itiles;
  const int maxS = (n + 31) / 32;
  if (S > 64) S = 64;
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  return S;
}

struct Carver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = align256(off);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Lay out the workspace; with base == nullptr only the size is computed.
size_t layout(const nb_params& p, int n, char* base, Dev* out) {
  Dev d;
  memset(&d, 0, sizeof(d));
  d.n = n;
  d.row0 = 0;
  d.row1 = n;
  d.S = p.kick_split > 0 ? p.kick_split : auto_split(n);
  const int cap = p.pair_capacity > 0 ? p.pair_capacity : (4 * n > 4096 ? 4 * n : 4096);
  d.pair_cap = round_pow2(cap);
  d.log_cap = p.log_capacity > 0 ? p.log_capacity : (1 << 20);
  d.member_cap = n;
  d.bs_kmax = p.bs_kmax < 3 ? 3 : (p.bs_kmax > kMaxBsK ? kMaxBsK : p.bs_kmax);
  d.bs_stride = bs_stride_for_kmax(d.bs_kmax);
  d.ppart_n = ppart_blocks(n);
  d.eparts_n = energy_blocks(n);
  Carver c{base, 0};
  double** arr[] = {&d.x, &d.y, &d.z, &d.vx, &d.vy, &d.vz, &d.m, &d.R, &d.rc, &d.rc2,
                    &d.ax, &d.ay, &d.az, &d.xs, &d.ys, &d.zs, &d.vxs, &d.vys, &d.vzs};
  for (double** a : arr) *a = c.take<double>(n);
  d.id = c.take<int>(n);
  d.alive = c.take<int>(n);
  d.member_slot = c.take<int>(n);
  d.uf = c.take<int>(n > 64 ? n : 64);
  // the unordered-pair kick's partials share the kpart allocation
  const bool sym = (p.precision == NB_PREC_FP64 || p.precision == NB_PREC_DS) &&
                   (p.kick_symmetric == 1 ? n <= kSymMaxN
                                          : p.kick_symmetric == 0 && n >= kSymMinN && n <= kSymMaxN);
  size_t kpart_n = (size_t)3 * d.S * n;
  if (sym) {
    const SymLayout L = sym_layout(n);
    d.sym = d.sym_ok = 1;
    d.sym_nb = L.nb;
    d.sym_hrow = L.hrow;
    d.sym_per = L.per;
    d.sym_grid = L.grid;
    if (L.doubles > kpart_n) kpart_n = L.doubles;
  }
  d.kpart = c.take<double>(kpart_n);
  if (sym) {
    d.sym_xpart = d.kpart;
    d.sym_ypart = d.kpart + (size_t)d.sym_grid * 2 * 3 * kSymBlock;
  }
  d.ppartA = c.take<double>((size_t)3 * d.ppart_n);
  d.ppartB = c.take<double>((size_t)3 * d.ppart_n);
  d.ftrial = c.take<int2>(d.pair_cap);
  d.fprev = c.take<int2>(d.pair_cap);
  d.keys = c.take<unsigned long long>((size_t)8 * d.pair_cap);
  d.log = c.take<int>((size_t)3 * d.log_cap);
  d.grp_off = c.take<int>((size_t)n + 1);
  d.grp_mem = c.take<int>(n);
  d.gscr = c.take<double>((size_t)n * d.bs_stride);
  d.gnew = c.take<double>((size_t)n * 10);
  d.gEl = c.take<double>(n);
  if (p.ml_levels > 0) {
    d.ml_gscr = c.take<double>((size_t)n * d.bs_stride);
    d.ml_gnew = c.take<double>((size_t)n * 10);
    d.ml_list = c.take<int>((size_t)(kMlMax + 1) * n);
    d.ml_parent = c.take<int>((size_t)(kMlMax + 1) * n);
  }
  d.snap = c.take<double>((size_t)16 * n);
  d.snap_i = c.take<int>((size_t)n + 2 * (size_t)d.pair_cap);
  d.ctrl = c.take<Ctrl>(1);
  d.snap_ctrl = c.take<Ctrl>(1);
  d.eparts = c.take<double>((size_t)2 * 8 * d.eparts_n);
  if (out) *out = d;
  return align256(c.off) + 256 * 2;  // + out8 and gather count
}

Phys make_phys(const nb_params& p) {
  Phys P{};
  P.G = p.G;
  P.m0 = p.m0;
  P.mu = p.G * p.m0;
  P.dt_rcrit = p.dt_rcrit;
  P.hill_factor = p.hill_factor;
  P.vel_factor = p.vel_factor;
  P.bs_tol = p.bs_tol;
  P.vel_mode = p.vel_mode;
  P.merge = p.merge;
  P.precision = p.precision;
  P.kepler_max_iter = p.kepler_max_iter;
  P.bs_kmax = p.bs_kmax < 3 ? 3 : (p.bs_kmax > kMaxBsK ? kMaxBsK : p.bs_kmax);
  P.bs_max_halvings = p.bs_max_halvings > 40 ? 40 : p.bs_max_halvings;
  P.rcrit_refresh = p.rcrit_refresh;
  P.gas = p.gas;
  P.gas_iter = p.gas_iter;
  P.gas_rho0 = p.gas_rho0;
  P.gas_p = p.gas_p;
  P.gas_eta = p.gas_eta;
  P.gas_cd = p.gas_cd;
  P.eject_r = p.eject_r;
  P.bs_cluster_min = p.bs_cluster_min;
  P.ml_levels = p.ml_levels;
  P.ml_factor = p.ml_factor;
  P.bs_speculate = p.bs_speculate;
  return P;
}

bool params_ok(const nb_params* p) {
  if (!p) return false;
  if (!(p->G > 0.0) || !(p->m0 > 0.0) || !std::isfinite(p->dt_rcrit)) return false;
  if (!(p->hill_factor >= 0.0) || !(p->vel_factor >= 0.0)) return false;
  if (p->precision < NB_PREC_FP64 || p->precision > NB_PREC_DS) return false;
  if (p->kepler_max_iter < 1 || p->bs_max_halvings < 0 || !(p->bs_tol > 0.0)) return false;
  if (p->pair_capacity < 0 || p->log_capacity < 0 || p->kick_split < 0) return false;
  if (p->rcrit_refresh != 0 && p->rcrit_refresh != 1) return false;
  if (p->gas != 0 && p->gas != 1) return false;
  if (p->gas && (!(p->gas_rho0 >= 0.0) || !std::isfinite(p->gas_p) || !(p->gas_eta <= 1.0) ||
                 !(p->gas_cd >= 0.0) || p->gas_iter < 1))
    return false;
  if (!(p->eject_r >= 0.0) || !std::isfinite(p->eject_r) || p->eject_r >= 0.5 * kDeadOffset)
    return false;
  if (p->bs_cluster_min < 0) return false;
  if (p->ml_levels < 0 || p->ml_levels > kMlMax || p->ml_factor < 2 || p->ml_factor > 64)
    return false;
  if (p->bs_speculate != 0 && p->bs_speculate != 1) return false;
  if (p->kick_symmetric < -1 || p->kick_symmetric > 1) return false;
  return true;
}

int cuda_fail(nb_system* s, cudaError_t e, const char* what) {
  if (s) snprintf(s->err, sizeof(s->err), "%s: %s", what, cudaGetErrorString(e));
  return NB_E_CUDA;
}

#define NB_CU(call)                                         \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

int read_ctrl(nb_system* s, Ctrl* h) {
  NB_CU(cudaMemcpyAsync(h, s->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->st));
  NB_CU(cudaStreamSynchronize(s->st));
  return NB_OK;
}

// Copy the mutable state into (dir = 0) or back from (dir = 1) the snapshot.
int snapshot(nb_system* s, int dir) {
  const Dev& d = s->d;
  const size_t nb = sizeof(double) * d.n;
  double* arr[] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.m, d.R, d.rc, d.rc2, d.ax, d.ay, d.az};
  for (int k = 0; k < 13; ++k) {
    double* sp = d.snap + (size_t)k * d.n;
    if (dir == 0)
      NB_CU(cudaMemcpyAsync(sp, arr[k], nb, cudaMemcpyDeviceToDevice, s->st));
    else
      NB_CU(cudaMemcpyAsync(arr[k], sp, nb, cudaMemcpyDeviceToDevice, s->st));
  }
  const size_t ni = sizeof(int) * d.n, np = sizeof(int2) * d.pair_cap;
  if (dir == 0) {
    NB_CU(cudaMemcpyAsync(d.snap_i, d.alive, ni, cudaMemcpyDeviceToDevice, s->st));
    NB_CU(cudaMemcpyAsync(d.snap_i + d.n, d.fprev, np, cudaMemcpyDeviceToDevice, s->st));
    NB_CU(cudaMemcpyAsync(d.snap_ctrl, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, s->st));
  } else {
    NB_CU(cudaMemcpyAsync(d.alive, d.snap_i, ni, cudaMemcpyDeviceToDevice, s->st));
    NB_CU(cudaMemcpyAsync(d.fprev, d.snap_i + d.n, np, cudaMemcpyDeviceToDevice, s->st));
    NB_CU(cudaMemsetAsync(d.member_slot, 0xff, ni, s->st));
    Ctrl h;
    NB_CU(cudaMemcpyAsync(&h, d.snap_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
    h.n_prev_members = 0;
    h.n_groups = 0;
    h.n_log = 0;
    h.status = 0;
    NB_CU(cudaMemcpyAsync(d.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
  }
  return NB_OK;
}

const char* where_name(int w) {
  switch (w) {
    case 1: return "kick (flagged-pair buffer)";
    case 10: return "Kepler drift";
    case 20: return "input validation";
    case 21: return "initial flag set";
    case 22: return "coordinate range of the standalone kick";
    case 30: return "Bulirsch-Stoer";
    case 70: return "another rank's kick (sharded step)";
    case 71: return "flagged-pair buffer (sharded step, all ranks together)";
    default: return "device";
  }
}

// A failed exchange of a sharded step: wait for the enqueued work, restore
// the state of the call's start and report.
int shard_fail(nb_system* s, int rc) {
  cudaStreamSynchronize(s->st);
  snprintf(s->err, sizeof(s->err), "the all-gather of a sharded step failed (state rolled back)");
  const int r2 = snapshot(s, 1);
  return r2 ? r2 : rc;
}

}  // namespace

namespace nb {
// Drop the plain step's graphs (their kernels hold the Dev and Phys of the
// capture by value: recaptured at the next step).
void drop_step_graphs(nb_system* s) {
  if (s->gx_mid) cudaGraphExecDestroy(s->gx_mid);
  if (s->gx_last) cudaGraphExecDestroy(s->gx_last);
  s->gx_mid = nullptr;
  s->gx_last = nullptr;
}
}  // namespace nb

extern "C" {

void nb_default_params(nb_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->G = 2.959122082855911e-4;
  p->m0 = 1.0;
  p->dt_rcrit = 6.0;
  p->hill_factor = 3.0;
  p->vel_factor = 0.4;
  p->vel_mode = 0;
  p->merge = 1;
  p->precision = NB_PREC_FP64;
  p->kepler_max_iter = 30;
  p->bs_tol = 1e-14;
  p->bs_kmax = 8;
  p->bs_max_halvings = 20;
  p->pair_capacity = 0;
  p->log_capacity = 0;
  p->kick_split = 0;
  p->rcrit_refresh = 0;
  p->gas = 0;
  p->gas_rho0 = 2.36e-3;
  p->gas_p = 2.75;
  p->gas_eta = 2e-3;
  p->gas_cd = 1.0;
  p->gas_iter = 30;
  p->eject_r = 0.0;
  p->bs_cluster_min = 64;
  p->ml_levels = 0;
  p->ml_factor = 3;
  p->bs_speculate = 1;
  p->kick_symmetric = 0;
}

size_t nb_workspace_bytes(const nb_params* p, int n) {
  if (!params_ok(p) || n < 1) return 0;
  return layout(*p, n, nullptr, nullptr);
}

const char* nb_status_string(int status) {
  switch (status) {
    case NB_OK: return "ok";
    case NB_E_INVALID: return "invalid argument";
    case NB_E_CUDA: return "CUDA error";
    case NB_E_OVERFLOW: return "buffer overflow";
    case NB_E_NOCONV: return "iteration cap reached";
    case NB_E_TIMEOUT: return "bounded loop gave up";
    case NB_E_WORKSPACE: return "workspace too small or misaligned";
    default: return "unknown status";
  }
}

const char* nb_last_error(const nb_system* s) { return s ? s->err : "no system"; }

int nb_init_system(nb_system** out, const nb_params* p, int n, const double* x, const double* v,
                   const double* m, const double* R, const double* rc_override, const int* ids,
                   void* workspace, size_t ws_bytes, void* stream, int inputs_on_device) {
  if (!out) return NB_E_INVALID;
  *out = nullptr;
  if (!params_ok(p) || n < 1 || !x || !v || !m || !R) return NB_E_INVALID;
  if (p->kick_symmetric == 1 && p->precision != NB_PREC_MIXED && n > kSymMaxN) return NB_E_INVALID;
  const size_t need = layout(*p, n, nullptr, nullptr);
  if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return NB_E_WORKSPACE;
  nb_system* s = (nb_system*)calloc(1, sizeof(nb_system));
  if (!s) return NB_E_INVALID;
  s->events = new std::vector<cudaEvent_t>();
  s->prm = *p;
  s->st = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    nb_destroy(s);
    return NB_E_CUDA;
  }
  s->P = make_phys(*p);
  layout(*p, n, (char*)workspace, &s->d);
  const size_t tail = align256(need - 512);
  s->out8 = (double*)((char*)workspace + tail);
  s->cnt = (int*)((char*)workspace + tail + 256);
  Dev& d = s->d;
  int rc = NB_OK;
  do {
    Ctrl h;
    memset(&h, 0, sizeof(h));
    h.n_active = n;
    if (cudaMemcpyAsync(d.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, s->st) != cudaSuccess) {
      rc = NB_E_CUDA;
      break;
    }
    const double *ix = x, *iv = v, *im = m, *iR = R, *irc = rc_override;
    const int* iid = ids;
    if (!inputs_on_device) {  // stage host inputs in the snapshot area
      double* st = d.snap;
      const size_t b3 = sizeof(double) * 3 * n, b1 = sizeof(double) * n;
      cudaMemcpyAsync(st, x, b3, cudaMemcpyHostToDevice, s->st);
      cudaMemcpyAsync(st + 3 * n, v, b3, cudaMemcpyHostToDevice, s->st);
      cudaMemcpyAsync(st + 6 * n, m, b1, cudaMemcpyHostToDevice, s->st);
      cudaMemcpyAsync(st + 7 * n, R, b1, cudaMemcpyHostToDevice, s->st);
      ix = st; iv = st + 3 * n; im = st + 6 * n; iR = st + 7 * n;
      if (rc_override) {
        cudaMemcpyAsync(st + 8 * n, rc_override, b1, cudaMemcpyHostToDevice, s->st);
        irc = st + 8 * n;
      }
      if (ids) {
        cudaMemcpyAsync(d.snap_i, ids, sizeof(int) * n, cudaMemcpyHostToDevice, s->st);
        iid = d.snap_i;
      }
    }
    cudaMemsetAsync(d.member_slot, 0xff, sizeof(int) * n, s->st);
    launch_init_in(d, s->P, ix, iv, im, iR, irc, iid, s->st);
    launch_kick(d, s->P, 0, s->st);
    launch_finish(d, s->P, 0, s->st);
    launch_fsal_init(d, s->st);
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      cuda_fail(s, e, "nb_init_system");
      rc = NB_E_CUDA;
      break;
    }
    Ctrl c;
    if (read_ctrl(s, &c) != NB_OK) {
      rc = NB_E_CUDA;
      break;
    }
    if (c.status) {
      snprintf(s->err, sizeof(s->err), "%s during %s", nb_status_string(c.status),
               where_name(c.err_where));
      rc = c.status;
    }
  } while (0);
  s->launches += 4;
  if (rc != NB_OK) {
    nb_destroy(s);
    return rc;
  }
  *out = s;
  return NB_OK;
}

int nb_set_fsal(nb_system* s, const double* a, const int* pairs_ij, int npairs, int on_device) {
  if (!s || !a || npairs < 0 || (npairs > 0 && !pairs_ij)) return NB_E_INVALID;
  if (npairs > s->d.pair_cap) return NB_E_OVERFLOW;
  const Dev& d = s->d;
  double* tmp = d.snap;  // staging
  NB_CU(cudaMemcpyAsync(tmp, a, sizeof(double) * 3 * d.n,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  launch_a_convert(d, tmp, 1, s->st);
  if (npairs)
    NB_CU(cudaMemcpyAsync(d.fprev, pairs_ij, sizeof(int2) * npairs,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  NB_CU(cudaMemcpyAsync(&d.ctrl->n_fprev, &npairs, sizeof(int), cudaMemcpyHostToDevice, s->st));
  NB_CU(cudaStreamSynchronize(s->st));
  return NB_OK;
}

// One plain step (no split phases, unsharded, untimed) on stream st, with
// the closing kick fused with the next opening one unless last: the same
// launches, in the same order, as the general loop of nb_step.
static int enqueue_plain_step(nb_system* s, cudaStream_t st, double dt, bool last) {
  const Dev& d = s->d;
  launch_drift_h(d, s->P, dt, st);
  launch_kick(d, s->P, 0, st);
  launch_encounter(d, s->P, st);
  NB_CU(cudaEventRecord(s->ev_fork, st));
  NB_CU(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
  launch_finish_part(d, s->P, 1, s->side);
  launch_bs(d, s->P, dt, st, s->side);
  NB_CU(cudaEventRecord(s->ev_join, s->side));
  NB_CU(cudaStreamWaitEvent(st, s->ev_join, 0));
  // the closing half of the force update (rows outside the groups) beside
  // the scatter and the members' re-kick (the members' rows)
  NB_CU(cudaEventRecord(s->ev_fork, st));
  NB_CU(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
  launch_finish_part(d, s->P, 2, s->side);
  NB_CU(cudaEventRecord(s->ev_join, s->side));
  launch_scatter(d, s->P, st);
  launch_member_kick(d, s->P, st);
  NB_CU(cudaStreamWaitEvent(st, s->ev_join, 0));
  launch_close_h(d, s->P, dt, last, st);
  return NB_OK;
}

static int capture_plain_step(nb_system* s, double dt, bool last, cudaGraphExec_t* out) {
  *out = nullptr;
  if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return NB_E_CUDA;
  }
  const int rc = enqueue_plain_step(s, s->cap, dt, last);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->cap, &g);
  if (rc != NB_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return NB_E_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return NB_E_CUDA;
  }
  return NB_OK;
}

// The plain step's graphs for dt, captured at the first call with that dt.
// NB_E_CUDA when capture is unavailable (nb_step then launches directly).
static int step_graphs(nb_system* s, double dt) {
  if (s->g_fail) return NB_E_CUDA;
  if (s->gx_mid && s->gx_last && s->g_dt == dt) return NB_OK;
  drop_step_graphs(s);
  if (!s->cap && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->cap = nullptr;
    s->g_fail = 1;
    return NB_E_CUDA;
  }
  if (capture_plain_step(s, dt, false, &s->gx_mid) != NB_OK ||
      capture_plain_step(s, dt, true, &s->gx_last) != NB_OK) {
    drop_step_graphs(s);
    s->g_fail = 1;
    return NB_E_CUDA;
  }
  s->g_dt = dt;
  return NB_OK;
}

int nb_step(nb_system* s, int nsteps, double dt) {
  if (!s || nsteps < 0 || !std::isfinite(dt)) return NB_E_INVALID;
  if (nsteps == 0) return NB_OK;
  const Dev& d = s->d;
  int rc = snapshot(s, 0);
  if (rc) return rc;
  NB_CU(cudaMemsetAsync(&d.ctrl->n_log, 0, sizeof(int), s->st));
  if (s->timing) {
    while ((int)s->events->size() < 2 * nsteps) {
      cudaEvent_t e;
      NB_CU(cudaEventCreate(&e));
      s->events->push_back(e);
    }
  }
  NvtxRange whole("nb_step");
  const int refresh = s->P.rcrit_refresh;
  const int eject = s->P.eject_r > 0.0;
  const int gas = s->P.gas;
  const int split = refresh || eject || gas;  // no fusion of closing and opening kicks
  if (!split) launch_open_h(d, dt, s->st);
  // the plain step as CUDA graphs: the same launches without the gaps
  // between dependent launches (which matter where the step is short)
  const bool graphs = !split && !s->timing && s->shard_world <= 1 && step_graphs(s, dt) == NB_OK;
  if (graphs) {
    for (int k = 0; k + 1 < nsteps; ++k) NB_CU(cudaGraphLaunch(s->gx_mid, s->st));
    NB_CU(cudaGraphLaunch(s->gx_last, s->st));
  }
  for (int k = 0; k < (graphs ? 0 : nsteps); ++k) {
    if (split) {
      // step start: ejection, Eq. rcrit anew, the cached force and flags
      // anew where either changed, then G(h/2) and the opening B(h/2)
      NvtxRange r("step start: eject / rcrit / force / gas / B(h/2)");
      if (eject) launch_eject(d, s->P, s->st);
      if (refresh) launch_refresh_rcrit(d, s->P, s->st);
      if (refresh || eject) launch_force_anew(d, s->P, !refresh, s->st);
      if (gas) launch_gas(d, s->P, 0.5 * dt, s->st);
      launch_open_h(d, dt, s->st);
    }
    {
      NvtxRange r("C(h/2) + Kepler drift A(h)");
      launch_drift_h(d, s->P, dt, s->st);
    }
    {
      NvtxRange r("kick + flags at the trial positions");
      if (s->timing) NB_CU(cudaEventRecord((*s->events)[2 * k], s->st));
      launch_kick(d, s->P, 0, s->st);
      if (s->timing) NB_CU(cudaEventRecord((*s->events)[2 * k + 1], s->st));
      // sharded: every rank's flagged pairs (nothing when not sharded)
      rc = shard_exchange(s, 1);
      if (rc) return shard_fail(s, rc);
    }
    {
      NvtxRange r("encounter set, groups, direct solver (trial half of the force beside it)");
      launch_encounter(d, s->P, s->st);
      // the trial half of the incremental force update needs only the groups
      // and the trial state, so it runs on the side stream while the direct
      // solver (a few latency-bound CTAs) runs on the launching stream
      NB_CU(cudaEventRecord(s->ev_fork, s->st));
      NB_CU(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
      launch_finish_part(d, s->P, 1, s->side);
      launch_bs(d, s->P, dt, s->st, s->side);  // the cluster solver's launch on the side stream
      NB_CU(cudaEventRecord(s->ev_join, s->side));
      NB_CU(cudaStreamWaitEvent(s->st, s->ev_join, 0));
    }
    {
      NvtxRange r("final force (incremental) and scatter");
      // the closing half of the force update (rows outside the groups) on
      // the side stream beside the scatter and the members' re-kick
      NB_CU(cudaEventRecord(s->ev_fork, s->st));
      NB_CU(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
      launch_finish_part(d, s->P, 2, s->side);
      NB_CU(cudaEventRecord(s->ev_join, s->side));
      launch_scatter(d, s->P, s->st);
      launch_member_kick(d, s->P, s->st);
      NB_CU(cudaStreamWaitEvent(s->st, s->ev_join, 0));
      // sharded: every rank's rows of the force (nothing when not sharded)
      rc = shard_exchange(s, 2);
      if (rc) return shard_fail(s, rc);
    }
    {
      NvtxRange r("C(h/2) + B(h/2)");
      launch_close_h(d, s->P, dt, split || k == nsteps - 1, s->st);
      if (gas) launch_gas(d, s->P, 0.5 * dt, s->st);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(s, e, "nb_step launch");
  Ctrl c;
  rc = read_ctrl(s, &c);
  if (rc) return rc;
  // kernels per step: open (split) or once per call, drift, kick, encounter,
  // the direct solver (1 or 2), finish (2 halves), scatter, member re-kick,
  // close; and eject 1, r_crit 1, the force anew 3, gas 2 + 2
  const long long per_step = 8 + bs_launches(d, s->P) + (split ? 1 : 0) + (eject ? 1 : 0) +
                             (refresh ? 1 : 0) + ((refresh || eject) ? 3 : 0) + (gas ? 4 : 0) +
                             (s->shard_world > 1 ? 4 : 0) +
                             // the double-single kick's grid, before each kick
                             (s->P.precision == NB_PREC_DS ? 1 + ((refresh || eject) ? 1 : 0) : 0);
  s->launches += (split ? 0 : 1) + per_step * nsteps;
  if (s->timing) {
    for (int k = 0; k < nsteps; ++k) {
      float ms = 0.f;
      NB_CU(cudaEventElapsedTime(&ms, (*s->events)[2 * k], (*s->events)[2 * k + 1]));
      s->kick_ms += ms;
    }
    s->kick_launches += nsteps;
  }
  if (c.status) {
    snprintf(s->err, sizeof(s->err), "%s during %s (state rolled back)",
             nb_status_string(c.status), where_name(c.err_where));
    const int st = c.status;
    rc = snapshot(s, 1);
    return rc ? rc : st;
  }
  return NB_OK;
}

int nb_energy_momentum(nb_system* s, double* E, double L[3], double P[3], double* E_lost) {
  if (!s) return NB_E_INVALID;
  launch_energy(s->d, s->P, s->out8, s->st);
  double h[8];
  NB_CU(cudaMemcpyAsync(h, s->out8, sizeof(h), cudaMemcpyDeviceToHost, s->st));
  NB_CU(cudaStreamSynchronize(s->st));
  if (E) *E = h[0];
  if (L) { L[0] = h[1]; L[1] = h[2]; L[2] = h[3]; }
  if (P) { P[0] = h[4]; P[1] = h[5]; P[2] = h[6]; }
  if (E_lost) *E_lost = h[7];
  return NB_OK;
}

int nb_get_state(nb_system* s, double* x, double* v, double* m, double* R, double* rc, int* ids,
                 int* n_active, int out_on_device) {
  if (!s) return NB_E_INVALID;
  const Dev& d = s->d;
  int k = 0;
  if (out_on_device) {
    launch_gather(d, x, v, m, R, rc, ids, s->cnt, s->st);
    NB_CU(cudaMemcpyAsync(&k, s->cnt, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
  } else {
    // gather into the snapshot area, then copy the k active bodies out
    double* g = d.snap;
    int* gi = d.snap_i;
    const int n = d.n;
    launch_gather(d, g, g + 3 * n, g + 6 * n, g + 7 * n, g + 8 * n, gi, s->cnt, s->st);
    NB_CU(cudaMemcpyAsync(&k, s->cnt, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
    const size_t b3 = sizeof(double) * 3 * k, b1 = sizeof(double) * k;
    if (x) NB_CU(cudaMemcpyAsync(x, g, b3, cudaMemcpyDeviceToHost, s->st));
    if (v) NB_CU(cudaMemcpyAsync(v, g + 3 * n, b3, cudaMemcpyDeviceToHost, s->st));
    if (m) NB_CU(cudaMemcpyAsync(m, g + 6 * n, b1, cudaMemcpyDeviceToHost, s->st));
    if (R) NB_CU(cudaMemcpyAsync(R, g + 7 * n, b1, cudaMemcpyDeviceToHost, s->st));
    if (rc) NB_CU(cudaMemcpyAsync(rc, g + 8 * n, b1, cudaMemcpyDeviceToHost, s->st));
    if (ids) NB_CU(cudaMemcpyAsync(ids, gi, sizeof(int) * k, cudaMemcpyDeviceToHost, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
  }
  if (n_active) *n_active = k;
  return NB_OK;
}

int nb_get_fsal(nb_system* s, double* a, int* pairs_ij, int cap, int* npairs,
                int out_on_device) {
  if (!s) return NB_E_INVALID;
  const Dev& d = s->d;
  Ctrl c;
  int rc = read_ctrl(s, &c);
  if (rc) return rc;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (a) {
    double* tmp = d.snap;
    launch_a_convert(d, tmp, 0, s->st);
    NB_CU(cudaMemcpyAsync(a, tmp, sizeof(double) * 3 * d.n, kind, s->st));
  }
  const int np = c.n_fprev;
  if (npairs) *npairs = np;
  const int k = np < cap ? np : cap;
  if (pairs_ij && k > 0)
    NB_CU(cudaMemcpyAsync(pairs_ij, d.fprev, sizeof(int2) * k, kind, s->st));
  NB_CU(cudaStreamSynchronize(s->st));
  return np > cap && pairs_ij ? NB_E_OVERFLOW : NB_OK;
}

int nb_encounter_list(nb_system* s, int* step_ij, int cap, int* count) {
  if (!s || cap < 0) return NB_E_INVALID;
  Ctrl c;
  int rc = read_ctrl(s, &c);
  if (rc) return rc;
  const int total = c.n_log;
  const int stored = total < s->d.log_cap ? total : s->d.log_cap;
  if (count) *count = total;
  const int k = stored < cap ? stored : cap;
  if (step_ij && k > 0) {
    NB_CU(cudaMemcpyAsync(step_ij, s->d.log, sizeof(int) * 3 * k, cudaMemcpyDeviceToHost, s->st));
    NB_CU(cudaStreamSynchronize(s->st));
  }
  return total > cap ? NB_E_OVERFLOW : NB_OK;
}

int nb_stats(nb_system* s, nb_stats_t* out) {
  if (!s || !out) return NB_E_INVALID;
  Ctrl c;
  int rc = read_ctrl(s, &c);
  if (rc) return rc;
  out->steps = (long long)c.stats[ST_STEPS];
  out->force_evals = (long long)c.stats[ST_FORCE_EVALS];
  out->encounter_pairs = (long long)c.stats[ST_ENC_PAIRS];
  out->groups = (long long)c.stats[ST_GROUPS];
  out->bs_substeps = (long long)c.stats[ST_BS_SUBSTEPS];
  out->bs_halvings = (long long)c.stats[ST_BS_HALVINGS];
  out->bs_derivs = (long long)c.stats[ST_BS_DERIVS];
  out->merges = (long long)c.stats[ST_MERGES];
  out->kepler_iters = (long long)c.stats[ST_KEPLER_ITERS];
  out->moved_bodies = (long long)c.stats[ST_MOVED];
  out->log_dropped = (long long)c.stats[ST_LOG_DROPPED];
  out->n_active = c.n_active;
  out->last_pairs = c.n_fprev;
  out->ejections = (long long)c.stats[ST_EJECTIONS];
  out->m_ejected = c.m_ejected;
  out->ml_substeps = (long long)c.stats[ST_ML_SUBSTEPS];
  out->ml_groups = (long long)c.stats[ST_ML_GROUPS];
  out->kick_symmetric = s->d.sym;
  return NB_OK;
}

void nb_destroy(nb_system* s) {
  if (!s) return;
  drop_step_graphs(s);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->events) {
    for (cudaEvent_t e : *s->events) cudaEventDestroy(e);
    delete s->events;
  }
  if (s->side) {
    cudaStreamSynchronize(s->side);
    cudaStreamDestroy(s->side);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  free(s);
}

int nb_set_timing(nb_system* s, int enable) {
  if (!s) return NB_E_INVALID;
  s->timing = enable ? 1 : 0;
  s->kick_ms = 0.0;
  s->kick_launches = 0;
  return NB_OK;
}

int nb_timing(nb_system* s, double* kick_ms, long long* kick_launches, long long* launches) {
  if (!s) return NB_E_INVALID;
  if (kick_ms) *kick_ms = s->kick_ms;
  if (kick_launches) *kick_launches = s->kick_launches;
  if (launches) *launches = s->launches;
  return NB_OK;
}

int nb_set_state(nb_system* s, const double* x, const double* v, const double* m,
                 const double* R, const double* rc, const int* ids, const double* a,
                 const int* pairs_ij, int npairs, int on_device) {
  if (!s || !x || !v || !m || !R || !rc || !a || npairs < 0 || (npairs > 0 && !pairs_ij))
    return NB_E_INVALID;
  const Dev& d = s->d;
  if (npairs > d.pair_cap) return NB_E_OVERFLOW;
  const int n = d.n;
  const double *ix = x, *iv = v, *im = m, *iR = R, *irc = rc, *ia = a;
  const int* iid = ids;
  if (!on_device) {
    double* st = d.snap;
    const size_t b3 = sizeof(double) * 3 * n, b1 = sizeof(double) * n;
    NB_CU(cudaMemcpyAsync(st, x, b3, cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaMemcpyAsync(st + 3 * n, v, b3, cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaMemcpyAsync(st + 6 * n, m, b1, cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaMemcpyAsync(st + 7 * n, R, b1, cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaMemcpyAsync(st + 8 * n, rc, b1, cudaMemcpyHostToDevice, s->st));
    NB_CU(cudaMemcpyAsync(st + 9 * n, a, b3, cudaMemcpyHostToDevice, s->st));
    ix = st; iv = st + 3 * n; im = st + 6 * n; iR = st + 7 * n; irc = st + 8 * n;
    ia = st + 9 * n;
    if (ids) {
      NB_CU(cudaMemcpyAsync(d.snap_i, ids, sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
      iid = d.snap_i;
    }
  }
  if (npairs)
    NB_CU(cudaMemcpyAsync(d.fprev, pairs_ij, sizeof(int2) * npairs,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  Ctrl c;
  int rc0 = read_ctrl(s, &c);
  if (rc0) return rc0;
  c.status = 0;
  c.n_fprev = npairs;
  c.n_active = n;
  c.n_prev_members = 0;
  c.n_groups = 0;
  c.n_members = 0;
  NB_CU(cudaMemcpyAsync(d.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->st));
  NB_CU(cudaMemsetAsync(d.member_slot, 0xff, sizeof(int) * n, s->st));
  launch_init_in(d, s->P, ix, iv, im, iR, irc, iid, s->st);
  launch_a_convert(d, const_cast<double*>(ia), 1, s->st);
  s->launches += 2;
  Ctrl c2;
  int rc1 = read_ctrl(s, &c2);
  if (rc1) return rc1;
  if (c2.status) {
    snprintf(s->err, sizeof(s->err), "%s during %s", nb_status_string(c2.status),
             where_name(c2.err_where));
    return c2.status;
  }
  return NB_OK;
}

// ---------------------------------------------------------------------------
size_t nb_kick_scratch_bytes(int n, int split) {
  if (n < 1) return 0;
  const int S = split > 0 ? split : auto_split(n);
  size_t b = 0;
  b += align256(sizeof(double) * 4 * (size_t)n);       // x, y, z, rc2
  b += align256(sizeof(double) * 3 * (size_t)S * n);   // partials
  b += align256(sizeof(Ctrl));
  return b;
}

int nb_kick_rows(int n, int row0, int row1, const double* x, const double* m, const double* rc,
                 double G, int precision, int split, double* a, int* pairs_ij, int cap,
                 int* npairs, void* scratch, size_t scratch_bytes, void* stream) {
  nb_system* s = nullptr;  // for NB_CU
  if (n < 1 || !x || !m || !rc || !a || cap < 0 || (cap > 0 && !pairs_ij)) return NB_E_INVALID;
  if (row0 < 0 || row1 > n || row0 >= row1) return NB_E_INVALID;
  if (precision < NB_PREC_FP64 || precision > NB_PREC_DS) return NB_E_INVALID;
  const int S = split > 0 ? split : auto_split(n);
  if (!scratch || scratch_bytes < nb_kick_scratch_bytes(n, S) || ((uintptr_t)scratch & 255))
    return NB_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)scratch;
  double* sx = (double*)p;
  double* sy = sx + n;
  double* sz = sy + n;
  double* src2 = sz + n;
  p += align256(sizeof(double) * 4 * (size_t)n);
  double* kpart = (double*)p;
  p += align256(sizeof(double) * 3 * (size_t)S * n);
  Ctrl* ctrl = (Ctrl*)p;
  NB_CU(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
  launch_raw_prep(n, x, rc, sx, sy, sz, src2, ctrl, st);
  launch_kick_raw(n, row0, row1, sx, sy, sz, m, rc, src2, S, precision, kpart, (int2*)pairs_ij,
                  cap, ctrl, st);
  launch_raw_finish(n, row0, row1, S, kpart, G, a, st);
  int cnt = 0, stat = 0;
  NB_CU(cudaMemcpyAsync(&cnt, &ctrl->n_ftrial, sizeof(int), cudaMemcpyDeviceToHost, st));
  NB_CU(cudaMemcpyAsync(&stat, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NB_CU(cudaStreamSynchronize(st));
  NB_CU(cudaGetLastError());
  if (npairs) *npairs = cnt;
  if (stat == NB_E_INVALID) return NB_E_INVALID;  // a coordinate beyond 2^37 AU (or NaN)
  return cnt > cap ? NB_E_OVERFLOW : NB_OK;
}

int nb_kick(int n, const double* x, const double* m, const double* rc, double G, int precision,
            int split, double* a, int* pairs_ij, int cap, int* npairs, void* scratch,
            size_t scratch_bytes, void* stream) {
  return nb_kick_rows(n, 0, n, x, m, rc, G, precision, split, a, pairs_ij, cap, npairs, scratch,
                      scratch_bytes, stream);
}

int nb_kepler_drift(int n, double mu, double* x, double* v, double dt, int max_iter,
                    void* scratch, void* stream) {
  nb_system* s = nullptr;
  if (n < 0 || !x || !v || !scratch || max_iter < 1 || !std::isfinite(dt)) return NB_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)scratch;
  NB_CU(cudaMemsetAsync(status, 0, sizeof(int), st));
  launch_kepler_raw(n, mu, x, v, dt, max_iter, status, st);
  int h = 0;
  NB_CU(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NB_CU(cudaStreamSynchronize(st));
  NB_CU(cudaGetLastError());
  return h;
}

size_t nb_peak_scratch_bytes(void) { return (size_t)peak_blocks() * 256 * sizeof(double); }

int nb_measure_peaks(double* fp64_flops, double* fp32_flops, void* scratch, void* stream) {
  if (!scratch) return NB_E_INVALID;
  return measure_peaks(fp64_flops, fp32_flops, scratch, (cudaStream_t)stream);
}

}  // extern "C"
