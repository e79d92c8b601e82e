// nb_kick_noalloc: the single-launch kick of nb_kick() for callers that
// cannot allocate device memory.
//
// Some callers have no way to obtain scratch memory: code that runs while a
// framework's allocator owns the whole device, real-time or embedded hosts
// that forbid allocation after start-up, or plug-ins that must not touch
// the CUDA allocator at all. This entry point needs only the caller's inputs
// and outputs; its scratch (SoA positions, partial sums and a counter block)
// lives in one file-scope device array below, so the library holds
// kNoallocBytes of device memory on every GPU that loads it, until exit.
//
// Host code must not hand the array's name to a kernel (on the host it only
// stands in for the symbol); the device address is looked up with
// cudaGetSymbolAddress once per device context, by the first call made in
// that context (the device's primary context, or a caller's own context made
// current through the driver API), with that device current. After
// cudaDeviceReset the primary context is a new one and the module is loaded
// again, so the address is looked up again: the cache is keyed on the
// driver's unique context id, never on the device ordinal alone. Make the
// first call in a context before any stream capture. All calls share the one
// array: calls that overlap on the GPU (other streams, other host threads)
// race and corrupt each other's results, so serialise them. Each call clears
// the counters it needs before use.
//
// The accelerations agree with nb_kick() to rounding (the parity suite's
// 1e-13 relative bound), not bit for bit: this variant splits the sources
// into at most kNoallocSplit chunks where nb_kick picks its own split, so
// the partial sums are added in another order. The flagged pair set is the
// same.
#include <cuda.h>

#include <mutex>

#include "nb_internal.cuh"

namespace nb {

constexpr int kNoallocSplit = 4;  // j-chunks of the kick in this variant
constexpr size_t kNoallocDoubles =
    (size_t)(4 + 3 * kNoallocSplit) * NB_NOALLOC_MAX_N;  // x, y, z, rc^2 + partials
constexpr size_t kNoallocBytes = kNoallocDoubles * sizeof(double) + 256 + sizeof(Ctrl);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxContexts = 64;
std::mutex g_mu;
struct CtxAddr {
  unsigned long long ctx_id;
  void* ptr;
};
CtxAddr g_cache[kMaxContexts];
int g_ncache = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

// Unique id of the context current on this thread (0 if none can be had).
// The two driver functions are resolved through the runtime, so the library
// does not link the driver library itself.
unsigned long long current_context_id() {
  if (!g_get_current || !g_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return 0;
    g_get_current = (CtxGetCurrentFn)f1;
    g_get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context: looked up by
// the first call made in each context and cached under the context's id.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NB_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = current_context_id();
  if (id != 0) {
    for (int k = 0; k < g_ncache; ++k)
      if (g_cache[k].ctx_id == id) {
        *out = g_cache[k].ptr;
        return NB_OK;
      }
  }
  // First call in this context (or no context yet: the lookup creates the
  // device's primary context, whose id is read afterwards).
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NB_E_CUDA;
  if (id == 0) id = current_context_id();
  if (id != 0) {
    if (g_ncache < kMaxContexts) {
      g_cache[g_ncache++] = {id, p};
    } else {
      g_cache[id % kMaxContexts] = {id, p};  // evict one: a later call looks it up again
    }
  }
  *out = p;
  return NB_OK;
}
}  // namespace

}  // namespace nb

using namespace nb;

extern "C" int nb_kick_noalloc(int n, const double* x, const double* m, const double* rc,
                               double G, int precision, double* a, int* pairs_ij, int cap,
                               int* npairs, void* stream) {
  if (n < 1 || !x || !m || !rc || !a || cap < 0 || (cap > 0 && !pairs_ij)) return NB_E_INVALID;
  if (n > NB_NOALLOC_MAX_N) return NB_E_INVALID;  // larger systems need nb_kick()
  if (precision < NB_PREC_FP64 || precision > NB_PREC_DS) return NB_E_INVALID;
  void* base = nullptr;
  const int st0 = scratch_address(&base);
  if (st0 != NB_OK) return st0;
  cudaStream_t st = (cudaStream_t)stream;
  int S = kick_blocks(n, 1, precision);  // target tiles
  S = (148 * 8 + S - 1) / S;
  if (S > kNoallocSplit) S = kNoallocSplit;
  if (S > (n + 127) / 128) S = (n + 127) / 128;
  if (S < 1) S = 1;
  double* sx = (double*)base;
  double* sy = sx + n;
  double* sz = sy + n;
  double* src2 = sz + n;
  double* kpart = src2 + n;  // 3 * S * n <= 3 * kNoallocSplit * NB_NOALLOC_MAX_N
  const size_t ctrl_off = (kNoallocDoubles * sizeof(double) + 255) & ~(size_t)255;
  Ctrl* ctrl = (Ctrl*)((char*)base + ctrl_off);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return NB_E_CUDA;
  launch_raw_prep(n, x, rc, sx, sy, sz, src2, ctrl, st);
  launch_kick_raw(n, 0, n, sx, sy, sz, m, rc, src2, S, precision, kpart, (int2*)pairs_ij, cap, ctrl,
                  st);
  launch_raw_finish(n, 0, n, S, kpart, G, a, st);
  int cnt = 0, stat = 0;
  if (cudaMemcpyAsync(&cnt, &ctrl->n_ftrial, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&stat, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return NB_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NB_E_CUDA;
  if (cudaGetLastError() != cudaSuccess) return NB_E_CUDA;
  if (npairs) *npairs = cnt;
  if (stat == NB_E_INVALID) return NB_E_INVALID;  // a coordinate beyond 2^37 AU (or NaN)
  return cnt > cap ? NB_E_OVERFLOW : NB_OK;
}
