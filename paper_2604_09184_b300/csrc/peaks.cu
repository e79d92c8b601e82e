// Throughput of the FP64 and FP32 FMA pipes, measured with the library's own
// loops: eight independent FMA chains per thread, 8 CTAs of 256 threads per
// SM, timed with CUDA events. These are the denominators of the kick's
// roofline fractions (the chip's FP64 rate is not in any table on the box).
#include "nb_internal.cuh"

namespace nb {

template <typename T, int ILP>
__global__ void __launch_bounds__(256) k_fma_loop(T* out, int iters, T a, T b) {
  T acc[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) acc[k] = (T)(threadIdx.x * 1e-3 + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) acc[k] = acc[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static double time_loop(int dbl, int blocks, int iters, void* scratch, cudaStream_t st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    if (dbl)
      k_fma_loop<double, 8><<<blocks, 256, 0, st>>>((double*)scratch, iters, 0.999999, 1e-7);
    else
      k_fma_loop<float, 8><<<blocks, 256, 0, st>>>((float*)scratch, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 2.0 * 8.0 * (double)blocks * 256.0 * (double)iters / (best * 1e-3);
}

int peak_blocks() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;
}

int measure_peaks(double* fp64, double* fp32, void* scratch, cudaStream_t st) {
  const int blocks = peak_blocks();
  if (fp64) *fp64 = time_loop(1, blocks, 2000, scratch, st);
  if (fp32) *fp32 = time_loop(0, blocks, 20000, scratch, st);
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_E_CUDA;
}

}  // namespace nb
