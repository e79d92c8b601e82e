// Row sharding of the single-system step across ranks (one GPU per rank).
//
// The O(N^2) kick (Eq. Hb) dominates the step; its target rows split without
// any exchange inside the kick, because each row reads every body's position
// and writes only itself. Every rank therefore keeps the whole system (the
// O(N) arrays are small: ~150 B per body) and runs the O(N) phases, the
// encounter set, the groups, the direct solver and the group members' rows on
// identical data, and evaluates the kick and the row-wise force update for
// its own block of rows. Two all-gathers per step (the caller's nb_allgather_fn)
// join the blocks:
//   1. the trial kick's flagged pairs of every block, so that every rank forms
//      the same encounter set (E = F_prev U F_trial is sorted, so the order of
//      the blocks does not matter), and every block's status word;
//   2. the accelerations of every block after the force update.
// With the same n and kick split the rows are bit-identical to those of the
// whole kick, so the sharded step equals nb_step bit for bit.
#include <cstdio>
#include <cstring>

#include "nb_internal.cuh"

namespace nb {

constexpr int XNT = 256;
constexpr int kFlagHeaderInts = 4;  // count, status, unclipped count, 0

struct ShardLayout {
  size_t flag_blk;  // bytes of one rank's flag block
  size_t a_blk;     // bytes of one rank's acceleration block
  size_t send_f, recv_f, send_a, recv_a, total;
};

static size_t a256x(size_t v) { return (v + 255) & ~(size_t)255; }

static ShardLayout shard_layout(const Dev& d, int world, int chunk) {
  ShardLayout L;
  L.flag_blk = a256x(sizeof(int) * kFlagHeaderInts + sizeof(int2) * (size_t)d.pair_cap);
  L.a_blk = a256x(sizeof(double) * 3 * (size_t)chunk);
  L.send_f = 0;
  L.recv_f = L.send_f + L.flag_blk;
  L.send_a = L.recv_f + (size_t)world * L.flag_blk;
  L.recv_a = L.send_a + L.a_blk;
  L.total = L.recv_a + (size_t)world * L.a_blk;
  return L;
}

// This rank's flagged pairs (from the trial kick) into its send block.
__global__ void __launch_bounds__(XNT) k_shard_pack_flags(Dev d, int* send) {
  const int raw = d.ctrl->n_ftrial;
  const int cnt = min(raw, d.pair_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    send[0] = cnt;
    send[1] = d.ctrl->status;
    send[2] = raw;
    send[3] = 0;
  }
  int2* out = (int2*)(send + kFlagHeaderInts);
  for (int k = blockIdx.x * XNT + threadIdx.x; k < cnt; k += gridDim.x * XNT) out[k] = d.ftrial[k];
}

// Every rank's pairs, in rank order, as the trial flag set; a rank's error
// status becomes this rank's (first error wins), so every rank rolls back.
// One CTA per rank block.
__global__ void __launch_bounds__(XNT) k_shard_unpack_flags(Dev d, const char* recv, int world,
                                                            size_t blk) {
  __shared__ int s_off, s_cnt;
  const int r = blockIdx.x;
  if (threadIdx.x == 0) {
    int off = 0;
    unsigned long long total = 0;
    for (int q = 0; q < world; ++q) {
      const int* h = (const int*)(recv + (size_t)q * blk);
      if (q < r) off += h[0];
      total += (unsigned long long)(unsigned)h[2];
    }
    const int* h = (const int*)(recv + (size_t)r * blk);
    s_off = off;
    s_cnt = h[0];
    if (h[1] != 0) set_status(d.ctrl, h[1], 70);
    if (r == 0) {
      if (total > (unsigned long long)d.pair_cap) set_status(d.ctrl, NB_E_OVERFLOW, 71);
      d.ctrl->n_ftrial = (int)min(total, (unsigned long long)d.pair_cap);
    }
  }
  __syncthreads();
  const int2* in = (const int2*)(recv + (size_t)r * blk + sizeof(int) * kFlagHeaderInts);
  for (int k = threadIdx.x; k < s_cnt; k += XNT) {
    const int pos = s_off + k;
    if (pos < d.pair_cap) d.ftrial[pos] = in[k];
  }
}

// This rank's rows of the acceleration into its send block (zero-padded).
__global__ void __launch_bounds__(XNT) k_shard_pack_a(Dev d, double* send, int chunk) {
  const int k = blockIdx.x * XNT + threadIdx.x;
  if (k >= chunk) return;
  const int i = d.row0 + k;
  const bool in = i < d.row1;
  send[k] = in ? d.ax[i] : 0.0;
  send[chunk + k] = in ? d.ay[i] : 0.0;
  send[2 * chunk + k] = in ? d.az[i] : 0.0;
}

// Every rank's rows of the acceleration into the whole force.
__global__ void __launch_bounds__(XNT) k_shard_unpack_a(Dev d, const char* recv, int chunk,
                                                        size_t blk) {
  const int i = blockIdx.x * XNT + threadIdx.x;
  if (i >= d.n) return;
  const int r = i / chunk, k = i - r * chunk;
  const double* b = (const double*)(recv + (size_t)r * blk);
  d.ax[i] = b[k];
  d.ay[i] = b[chunk + k];
  d.az[i] = b[2 * chunk + k];
}

static int chunk_of(int n, int world) { return world > 0 ? (n + world - 1) / world : 0; }

// Exchange 1 (after the trial kick) or 2 (after the force update) of a
// sharded step; nothing for an unsharded system.
int shard_exchange(nb_system* s, int which) {
  if (s->shard_world <= 1) return NB_OK;
  const Dev& d = s->d;
  const int world = s->shard_world, chunk = s->shard_chunk;
  const ShardLayout L = shard_layout(d, world, chunk);
  char* b = s->shard_buf;
  int rc;
  if (which == 1) {
    int grid = (d.pair_cap + XNT - 1) / XNT;
    if (grid > 4 * 148) grid = 4 * 148;
    k_shard_pack_flags<<<grid, XNT, 0, s->st>>>(d, (int*)(b + L.send_f));
    if (cudaGetLastError() != cudaSuccess) return NB_E_CUDA;
    rc = s->shard_fn(s->shard_user, b + L.send_f, b + L.recv_f, L.flag_blk, (void*)s->st);
    if (rc != 0) return NB_E_CUDA;
    k_shard_unpack_flags<<<world, XNT, 0, s->st>>>(d, b + L.recv_f, world, L.flag_blk);
  } else {
    k_shard_pack_a<<<(chunk + XNT - 1) / XNT, XNT, 0, s->st>>>(d, (double*)(b + L.send_a), chunk);
    if (cudaGetLastError() != cudaSuccess) return NB_E_CUDA;
    rc = s->shard_fn(s->shard_user, b + L.send_a, b + L.recv_a, L.a_blk, (void*)s->st);
    if (rc != 0) return NB_E_CUDA;
    k_shard_unpack_a<<<(d.n + XNT - 1) / XNT, XNT, 0, s->st>>>(d, b + L.recv_a, chunk, L.a_blk);
  }
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_E_CUDA;
}

}  // namespace nb

using namespace nb;

extern "C" int nb_shard_rows(int n, int rank, int world, int* row0, int* row1) {
  if (n < 1 || world < 1 || rank < 0 || rank >= world || !row0 || !row1) return NB_E_INVALID;
  const long long c = chunk_of(n, world);
  long long r0 = c * rank, r1 = c * (rank + 1);
  if (r0 > n) r0 = n;
  if (r1 > n) r1 = n;
  *row0 = (int)r0;
  *row1 = (int)r1;
  return NB_OK;
}

extern "C" size_t nb_shard_buffer_bytes(const nb_system* s, int world) {
  if (!s || world < 1) return 0;
  return shard_layout(s->d, world, chunk_of(s->d.n, world)).total;
}

extern "C" int nb_set_shard(nb_system* s, int rank, int world, nb_allgather_fn fn, void* user,
                            void* buf, size_t buf_bytes) {
  if (!s || world < 1 || rank < 0 || rank >= world) return NB_E_INVALID;
  drop_step_graphs(s);  // the kick's rows change
  if (world == 1) {
    s->shard_rank = 0;
    s->shard_world = 1;
    s->shard_chunk = s->d.n;
    s->shard_fn = nullptr;
    s->shard_user = nullptr;
    s->shard_buf = nullptr;
    s->d.row0 = 0;
    s->d.row1 = s->d.n;
    s->d.sym = s->d.sym_ok;  // the unordered-pair kick again where it was chosen
    return NB_OK;
  }
  if (!fn) return NB_E_INVALID;
  if (s->P.rcrit_refresh || s->P.gas || s->P.eject_r > 0.0) {
    snprintf(s->err, sizeof(s->err),
             "row sharding does not cover rcrit_refresh, gas drag or ejection");
    return NB_E_INVALID;
  }
  if (!buf || ((uintptr_t)buf & 255) || buf_bytes < nb_shard_buffer_bytes(s, world))
    return NB_E_WORKSPACE;
  int r0 = 0, r1 = 0;
  nb_shard_rows(s->d.n, rank, world, &r0, &r1);
  s->shard_rank = rank;
  s->shard_world = world;
  s->shard_chunk = chunk_of(s->d.n, world);
  s->shard_fn = fn;
  s->shard_user = user;
  s->shard_buf = (char*)buf;
  s->d.row0 = r0;
  s->d.row1 = r1;
  s->d.sym = 0;  // row blocks: the row kick
  return NB_OK;
}
