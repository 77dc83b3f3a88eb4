// ugks_probe.cu -- FP64 throughput probe of the GPU the library runs on: the
// FP64 path of the scheme is bound by the FP64 pipe, so its roofline is the
// measured rate of dependent-free FP64 fused multiply-adds and of the FP64
// exponential, not the HBM bandwidth.
#include <cuda_runtime.h>

#include "ugks.h"

namespace {

// 8 independent FMA chains per thread, `iters` rounds: 16 * iters FP64
// flops per thread; the result is stored so nothing is dead code.
__global__ void k_probe_fma(double *out, int iters) {
  double a[8];
  double x = 1.0 + 1e-9 * threadIdx.x, y = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
  for (int m = 0; m < 8; ++m) a[m] = 0.5 + 0.01 * m;
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = fma(a[m], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) s += a[m];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 4 independent exp chains per thread, `iters` rounds: 4 * iters
// exponentials per thread (arguments kept in [-1, 0]).
__global__ void k_probe_exp(double *out, int iters) {
  double a[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) a[m] = -0.25 * m - 1e-7 * threadIdx.x;
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int m = 0; m < 4; ++m) a[m] = -exp(a[m]);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a[0] + a[1] + a[2] + a[3];
}

}  // namespace

extern "C" int ugks_probe_fp64(double *out, int kind, int nblocks, int nthreads, int iters, void *stream) {
  if (!out || nblocks <= 0 || nthreads <= 0 || nthreads > 1024 || iters <= 0 || (kind != 0 && kind != 1))
    return UGKS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (kind == 0) k_probe_fma<<<nblocks, nthreads, 0, s>>>(out, iters);
  else k_probe_exp<<<nblocks, nthreads, 0, s>>>(out, iters);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return UGKS_ERR_CUDA;
  }
  return UGKS_OK;
}
