// Element-wise evaluation of the device arithmetic helpers that the hot loops
// are built from (the seeded reciprocal roots, the table-driven exponential,
// the direct solver's changeover weight, Neville weights and acceptance
// test), so that each can be checked on its own against the oracle and libm.
// Not used by the integrator.
#include "bs.cuh"

namespace nb {

__global__ void k_math_eval(int fn, int n, const double* in, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = fn == NB_MATH_RATIO_LE ? 0.0 : in[i];
  double r = 0.0;
  switch (fn) {
    case NB_MATH_EXP: r = exp_fast(x); break;
    case NB_MATH_RCP: r = rcp_fast(x); break;
    case NB_MATH_RSQRT: r = rinv_fast(x); break;
    case NB_MATH_RPOW32: r = scale_fast<NB_PREC_FP64>(x, 1.0, 1.5, 1.875); break;
    case NB_MATH_RPOW32_MIXED: r = scale_fast<NB_PREC_MIXED>(x, 1.0, 1.5, 0.0); break;
    case NB_MATH_RPOW32_M: r = scale_fast<NB_PREC_FP64>(x, 1.0); break;
    case NB_MATH_CLOSE_WEIGHT: r = close_weight(x, 0.1, 1.0 / 0.9); break;
    case NB_MATH_MASS15: {
      double a, b;
      mass_coeffs(x, a, b);
      r = a;
      break;
    }
    case NB_MATH_MASS1875: {
      double a, b;
      mass_coeffs(x, a, b);
      r = b;
      break;
    }
    case NB_MATH_NEVILLE: {
      const int k = (int)x, j = k >> 4, q = k & 15;
      r = (x == (double)k && j <= kMaxBsK && q >= 1 && q < j) ? kNeville.w[j][q] : 0.0;
      break;
    }
    case NB_MATH_RATIO_LE: {
      const double tol = in[3 * i + 2];
      r = ratio_le(in[3 * i], in[3 * i + 1], tol, next_up(tol)) ? 1.0 : 0.0;
      break;
    }
    case NB_MATH_RINV3: r = rinv3_fast(x); break;
    default: r = 0.0;
  }
  out[i] = r;
}

}  // namespace nb

extern "C" int nb_math_eval(int fn, int n, const double* in, double* out, void* stream) {
  if (n < 0 || fn < 0 || fn > NB_MATH_RINV3) return NB_E_INVALID;
  if (n == 0) return NB_OK;
  if (!in || !out) return NB_E_INVALID;
  nb::k_math_eval<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(fn, n, in, out);
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_E_CUDA;
}
