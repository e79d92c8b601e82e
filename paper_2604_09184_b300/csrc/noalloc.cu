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
// cudaGetSymbolAddress once per device, by the first call made on that
// device, with that device current. Make that first call before any stream
// capture. All calls share the one array: calls that overlap on the GPU
// (other streams, other host threads) race and corrupt each other's results,
// so serialise them. Each call clears the counters it needs before use.
#include <mutex>

#include "nb_internal.cuh"

namespace nb {

constexpr int kNoallocSplit = 4;  // j-chunks of the kick in this variant
constexpr size_t kNoallocDoubles =
    (size_t)(4 + 3 * kNoallocSplit) * NB_NOALLOC_MAX_N;  // x, y, z, rc^2 + partials
constexpr size_t kNoallocBytes = kNoallocDoubles * sizeof(double) + 256 + sizeof(Ctrl);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NB_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NB_E_CUDA;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
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
