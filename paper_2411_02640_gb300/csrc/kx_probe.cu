// Arithmetic-pipe probes: the measured per-clock rates that the roofline of
// the generated kernels is quoted against.  Each probe kernel runs eight
// independent dependence chains per thread of one operation (float64 FMA,
// float32 FMA, the float32 base-2 exponential of the special-function unit,
// and CUDA's own float64 exp, log and division as a caller sees them), so
// that with enough resident warps the pipe that executes it saturates.  The
// chains are contractions onto bounded values (no overflow, no denormals)
// and their results are written out so that nothing is folded away.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/kx.h"

namespace {

template <int OP>
__global__ void __launch_bounds__(256) kx_probe_kernel(double* __restrict__ sink, long long iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (OP == 0) {   // float64 fma
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5 + 1e-3 * (t & 7) + 1e-4 * j;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], 0.9999999, 1e-7);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[t] = s;
  } else if (OP == 1) {   // float32 fma
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5f + 1e-3f * (t & 7) + 1e-4f * j;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = __fmaf_rn(a[j], 0.9999f, 1e-4f);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[t] = s;
  } else if (OP == 2) {   // float32 2^x on the special-function unit: x <- 2^-x stays in [0.5, 1]
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5f + 1e-3f * (t & 7) + 1e-4f * j;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a[j]));
        a[j] = y;
      }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[t] = s;
  } else {   // CUDA's float64 exp (x <- e^-x), log (x <- ln(x + 2)), division (x <- 1/(x + 1.5))
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 0.5 + 1e-3 * (t & 7) + 1e-4 * j;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (OP == 3) a[j] = exp(-a[j]);
        else if (OP == 4) a[j] = log(a[j] + 2.0);
        else a[j] = 1.0 / (a[j] + 1.5);
      }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[t] = s;
  }
}

}  // namespace

extern "C" kx_status kx_probe_pipe(int op, int64_t iters, int blocks, int threads, double* sink, void* stream,
                                   double* ops) {
  if (op < 0 || op > 5 || iters < 1 || blocks < 1 || threads < 32 || threads > 256 || threads % 32 || !sink)
    return KX_ERR_ARG;
  const dim3 g(blocks), b(threads);
  cudaStream_t s = (cudaStream_t)stream;
  const long long it = iters;
  switch (op) {
    case 0: kx_probe_kernel<0><<<g, b, 0, s>>>(sink, it); break;
    case 1: kx_probe_kernel<1><<<g, b, 0, s>>>(sink, it); break;
    case 2: kx_probe_kernel<2><<<g, b, 0, s>>>(sink, it); break;
    case 3: kx_probe_kernel<3><<<g, b, 0, s>>>(sink, it); break;
    case 4: kx_probe_kernel<4><<<g, b, 0, s>>>(sink, it); break;
    default: kx_probe_kernel<5><<<g, b, 0, s>>>(sink, it); break;
  }
  if (cudaGetLastError() != cudaSuccess) return KX_ERR_CUDA;
  if (ops) *ops = 8.0 * (double)iters * (double)blocks * (double)threads;
  return KX_OK;
}
