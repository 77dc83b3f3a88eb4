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
// that symbol is only a stand-in.  The device address is obtained with
// cudaGetSymbolAddress (with the device current) on the first call in each
// CUDA context and passed to the kernels; a new context on a device (after
// cudaDeviceReset, for instance) reloads the module and triggers a new
// lookup on its first call.
#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>

#include "ugks.h"

namespace {

__device__ __align__(256) double g_idw_scratch[UGKS_STATIC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices];
CUcontext g_scratch_ctx[kMaxDevices];     // context the address belongs to
std::mutex g_scratch_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// The calling thread's current CUDA context (driver entry point reached
// through the runtime, so the library needs no link against libcuda).
CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    cudaGetLastError();
    tried = true;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// The scratch array's device address in the current context (looked up on
// the first call in that context).
int scratch_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return UGKS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  // (no context yet: null, which never matches, so the lookup below runs
  // and the next call records the context it created)
  CUcontext ctx = current_context();
  if (!g_scratch_addr[dev] || ctx == nullptr || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_idw_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return UGKS_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double *>(p);
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return UGKS_OK;
}

// Pass 1: every receptor row from its donors' values before the call
// (Jacobi), into the scratch.  Donor ids outside [0, ncells) are skipped and
// the remaining weights of the row renormalised to their sum (a row with no
// donor left keeps its values, flagged by a zero weight sum).  Grid:
// (receptor, velocity chunk).
__global__ void k_idw_gather_static(double *scratch, const double *f, const double *W,
                                    const double *q, int ncells, int nv, int nrec,
                                    const int32_t *donors, const double *weights) {
  int r = blockIdx.x;
  int k = blockIdx.y * blockDim.x + threadIdx.x;
  const int32_t *dn = donors + 5 * (size_t)r;
  const double *wt = weights + 5 * (size_t)r;
  double wv[5], wsum = 0.0;
  bool skipped = false;
  for (int m = 0; m < 5; ++m) {
    int e = dn[m];
    bool ok = e >= 0 && e < ncells;
    skipped = skipped || (e != -1 && !ok);
    wv[m] = ok ? wt[m] : 0.0;
    wsum = wsum + wv[m];
  }
  if (skipped && wsum != 0.0)
    for (int m = 0; m < 5; ++m) wv[m] = wv[m] / wsum;
  double *sw = scratch + 2 * (size_t)nrec * nv + 7 * (size_t)r;
  if (k < nv) {
    double ah = 0.0, ab = 0.0;
    for (int m = 0; m < 5; ++m) {
      int e = dn[m];
      if (e < 0 || e >= ncells) continue;
      const double *fe = f + 2 * ((size_t)e * nv + k);
      ah = ah + wv[m] * fe[0];
      ab = ab + wv[m] * fe[1];
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
        for (int c = 0; c < 4; ++c) acc[c] = acc[c] + wv[m] * W[4 * (size_t)e + c];
      if (q) {
        acc[4] = acc[4] + wv[m] * q[2 * (size_t)e];
        acc[5] = acc[5] + wv[m] * q[2 * (size_t)e + 1];
      }
    }
    for (int c = 0; c < 6; ++c) sw[c] = acc[c];
    sw[6] = wsum;
  }
}

// Pass 2: scatter the staged rows; rows without a donor stay unchanged.
__global__ void k_idw_scatter_static(const double *scratch, double *f, double *W, double *q,
                                     int ncells, int nv, int nrec, const int32_t *receptors,
                                     const int32_t *donors) {
  int r = blockIdx.x;
  int k = blockIdx.y * blockDim.x + threadIdx.x;
  const double *sw = scratch + 2 * (size_t)nrec * nv + 7 * (size_t)r;
  if (donors[5 * (size_t)r] < 0 || sw[6] == 0.0) return;
  int c = receptors[r];
  if (c < 0 || c >= ncells) return;
  if (k < nv) {
    double *fc = f + 2 * ((size_t)c * nv + k);
    fc[0] = scratch[2 * ((size_t)r * nv + k)];
    fc[1] = scratch[2 * ((size_t)r * nv + k) + 1];
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) {
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
  // staged values: 2 per (receptor, velocity) plus 7 per receptor
  unsigned long long need = 2ull * nrec * nv + 7ull * nrec;
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
