// ugks_static.cu -- allocation-free receptor interpolation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns every device allocation and hands out only the
// buffers it manages, or code that must not call cudaMalloc while another
// component is capturing or replaying work.  ugks_idw_interpolate_static
// serves them: it takes the fields, receptor list and donor stencils as
// caller buffers and stages the interpolated values in a fixed-size scratch
// array that lives in this file as a static __device__ variable (every GPU
// that loads the library holds it until the process exits).
//
// Host code must not use the array's name as a device address: on the host
// that symbol is only a stand-in.  The device address is obtained once per
// device with cudaGetSymbolAddress (with that device current) and passed to
// the kernels.
#include <cuda_runtime.h>
#include <mutex>

#include "ugks.h"

namespace {

__device__ __align__(256) double g_idw_scratch[UGKS_STATIC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices];
bool g_scratch_ready[kMaxDevices];
std::mutex g_scratch_mutex;

// First call on a device: look up the device address of the scratch array.
int scratch_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return UGKS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ready[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_idw_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return UGKS_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double *>(p);
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_addr[dev];
  return UGKS_OK;
}

// Pass 1: every receptor row from its donors' values before the call
// (Jacobi), into the scratch.  Grid: (receptor, velocity chunk).
__global__ void k_idw_gather_static(double *scratch, const double *f, const double *W,
                                    const double *q, int ncells, int nv, int nrec,
                                    const int32_t *donors, const double *weights) {
  int r = blockIdx.x;
  int k = blockIdx.y * blockDim.x + threadIdx.x;
  const int32_t *dn = donors + 5 * (size_t)r;
  const double *wt = weights + 5 * (size_t)r;
  if (k < nv) {
    double ah = 0.0, ab = 0.0;
    for (int m = 0; m < 5; ++m) {
      int e = dn[m];
      if (e < 0 || e >= ncells) continue;
      const double *fe = f + 2 * ((size_t)e * nv + k);
      ah = ah + wt[m] * fe[0];
      ab = ab + wt[m] * fe[1];
    }
    scratch[2 * ((size_t)r * nv + k)] = ah;
    scratch[2 * ((size_t)r * nv + k) + 1] = ab;
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 0; m < 5; ++m) {
      int e = dn[m];
      if (e < 0 || e >= ncells) continue;
      if (W)
        for (int c = 0; c < 4; ++c) acc[c] = acc[c] + wt[m] * W[4 * (size_t)e + c];
      if (q) {
        acc[4] = acc[4] + wt[m] * q[2 * (size_t)e];
        acc[5] = acc[5] + wt[m] * q[2 * (size_t)e + 1];
      }
    }
    double *sw = scratch + 2 * (size_t)nrec * nv + 6 * (size_t)r;
    for (int c = 0; c < 6; ++c) sw[c] = acc[c];
  }
}

// Pass 2: scatter the staged rows; rows without a donor stay unchanged.
__global__ void k_idw_scatter_static(const double *scratch, double *f, double *W, double *q,
                                     int ncells, int nv, int nrec, const int32_t *receptors,
                                     const int32_t *donors) {
  int r = blockIdx.x;
  int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (donors[5 * (size_t)r] < 0) return;
  int c = receptors[r];
  if (c < 0 || c >= ncells) return;
  if (k < nv) {
    double *fc = f + 2 * ((size_t)c * nv + k);
    fc[0] = scratch[2 * ((size_t)r * nv + k)];
    fc[1] = scratch[2 * ((size_t)r * nv + k) + 1];
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    const double *sw = scratch + 2 * (size_t)nrec * nv + 6 * (size_t)r;
    if (W)
      for (int m = 0; m < 4; ++m) W[4 * (size_t)c + m] = sw[m];
    if (q) {
      q[2 * (size_t)c] = sw[4];
      q[2 * (size_t)c + 1] = sw[5];
    }
  }
}

}  // namespace

extern "C" int ugks_idw_interpolate_static(double *f, double *W, double *q, int ncells, int nv,
                                           const int32_t *receptors, int nrec,
                                           const int32_t *donors, const double *weights,
                                           void *stream) {
  if (!f || ncells <= 0 || nv <= 0 || nrec < 0 || (nrec > 0 && (!receptors || !donors || !weights)))
    return UGKS_ERR_ARG;
  if (nrec == 0) return UGKS_OK;
  // staged values: 2 per (receptor, velocity) plus 6 per receptor
  unsigned long long need = 2ull * nrec * nv + 6ull * nrec;
  if (need > UGKS_STATIC_SCRATCH_DOUBLES) return UGKS_ERR_ARG;
  double *scratch = nullptr;
  int r = scratch_for_current_device(&scratch);
  if (r != UGKS_OK) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int bt = nv >= 256 ? 256 : ((nv + 31) / 32) * 32;
  dim3 grid(nrec, (nv + bt - 1) / bt);
  k_idw_gather_static<<<grid, bt, 0, s>>>(scratch, f, W, q, ncells, nv, nrec, donors, weights);
  k_idw_scatter_static<<<grid, bt, 0, s>>>(scratch, f, W, q, ncells, nv, nrec, receptors, donors);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return UGKS_ERR_CUDA;
  }
  return UGKS_OK;
}
