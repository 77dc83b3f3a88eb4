// ugks_internal.cuh -- device-side context of libugks and the per-(cell,
// velocity) building blocks shared by the kernels: limited reconstruction
// (Sec. 2.1, second-order initial distribution), the time-averaged interface
// flux of one velocity (Eqs. microscopicFlux, fullSolution; wall condition
// with Eq. maxWalldes) and its sum over the faces of a cell.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "ugks_math.cuh"

namespace ugks {

enum { BC_NONE = 0, BC_WALL = 1, BC_FARFIELD = 2, BC_OUTFLOW = 3, BC_OVERSET = 4 };
enum { ST_FIELD = 0, ST_RECEPTOR = 1, ST_HOLE = 2 };
enum { NB_CELL = 0, NB_GHOST = 1, NB_NONE = 2 };
// slope case per logical direction: none, only minus side, only plus side, both
enum { SL_NONE = 0, SL_M = 1, SL_P = 2, SL_BOTH = 3 };
// face sums of the velocity-reduction pass
enum { FS_W0 = 0, FS_FF = 4, FS_WG = 8, NFS = 12 };
// error flags
enum { EF_GEOMETRY = 1, EF_NONPHYSICAL = 2, EF_BINS = 4, EF_TIMEOUT = 8, EF_ORPHAN = 16, EF_CAPACITY = 32 };

template <typename T> struct Vec2;
template <> struct Vec2<double> { typedef double2 type; };
template <> struct Vec2<float> { typedef float2 type; };

// Everything a kernel needs: sizes, constants and borrowed device pointers
// into the caller's workspace.  Passed by value.
struct Dev {
  int nc, nf, nn, nv, nvp, nblocks;
  int Keff, Kint;
  double Pr, omega, mu_ref, cfl_s, cfl_pseudo;
  double Winf[4];
  double dt, idt;            // physical step and its inverse
  float idt_f;
  // velocity space (double and float copies), length nvp (padding weight 0)
  const double *vx, *vy, *w;
  const float *vxf, *vyf, *wf;
  int nvx, nvy;              // tensor grid: k = iy nvx + ix, w_k = wy1(iy) wx1(ix); nvy of the whole grid
  const float *wx1f, *wy1f;  // 1D trapezoid weights (whole grid)
  const float *vy1f;         // 1D y nodes of the whole grid
  const double *vx1, *vy1, *wx1, *wy1;   // 1D nodes and trapezoid weights of the whole grid (FP64)
  // velocity sharding: this context holds the rows iy0 <= iy < iy0 + nv / nvx
  // of the grid; the arrays above (vx, vy, w and copies) are its own rows, the
  // ones below the whole grid (the same arrays when not sharded)
  int shard, iy0, nv_all;
  const double *vxa, *vya, *wa;
  const float *vxaf, *vyaf, *waf;
  double *msum;              // nc*6: partial moment sums of a sharded step (W fix 4, q 2)
  // static topology
  const int *cell_nodes;     // nc*4
  const int *cell_faces;     // nc*4 (IM, IP, JM, JP)
  const int8_t *cell_sgn;    // nc*4, +1 if the cell is the face's L side
  const int *nb_kind;        // nc*4
  const int *nb_id;          // nc*4 cell id or ghost face id
  const int8_t *nb_shift;    // nc*4 period multiplier
  const int *cell_row;       // nc*2 node ids (0,j), (ni,j)
  const int *cell_block;     // nc
  const int *node_block;     // nn
  const int *face_L, *face_R, *face_a, *face_b, *face_kind, *face_block;
  const int8_t *face_shiftL;
  const double *face_Tw;
  // per-step geometry
  const double *X_ref;
  double *X_old, *X_new;     // nn*2
  float2 *Xf;                // nn: X_new rounded to nearest float (overset filters)
  float4 *cbb;               // nc: cell bounding box at t^{n+1}, rounded outward
  double *vol_old, *vol_new; // nc
  double *xc, *xc_new;       // nc*2
  double *period;            // nc*2
  double *dts;               // nc
  double *Sn, *S, *nrm, *xf, *Uf, *SUn;   // nf*2 / nf
  int *slope_flags;          // nc: 2 bits per direction (i: bits 0-1, j: 2-3)
  int *cmask;                // nc: bit 0 solved cell, bit 1+s solved neighbour across slot s
  double *jinv;              // nc*4 inverse of [[x_xi, y_xi],[x_eta, y_eta]]
  float4 *jinvf;             // nc: the same in FP32
  void *fgeo;                // nf*NFG face geometry record (arithmetic type)
  void *srec;                // nc*NSR sweep record (layout at NSR)
  int *mrec_off;             // nblocks+1: first FP32 macro record of each block (diagonal-major)
  double vbox[4];            // velocity box (vx_min, vx_max, vy_min, vy_max)
  double *affine;            // nblocks*6
  // state
  void *f;                   // nc*nvp (h, b) pairs in the storage type
  double *W, *q;             // nc*4, nc*2
  int *status;               // nc
  // work
  void *Tn, *dfs;            // nc*nvp pairs: level-n term, forward-sweep result
  void *Dbuf;                // nc*nvp pairs: flux divergence of the inner iteration
  void *fval;                // nf*nvp 4-vectors: upwind face value (h, b) and w.grad f (h, b) of the face pass
  const double *stepc;       // [4]: dt, 1/dt, (float)(1/dt) of the pending step, on the device (the step's
                             // kernels read it there, so a captured step graph stays valid when dt changes)
  double *TW;                // nc*4 extensive level-n macro term
  double *Fc;                // nc*4 macro flux divergence of the last flux
  double *dW;                // nc*4 macro increment
  void *mrec;                // nc*41 macro-sweep records (arithmetic type)
  double *Wp;                // nc*4 macro predictor W'
  double *cpar;              // nc*NCP cell parameters (predictor / level n)
  double *cparn;
  void *shp, *shn;           // nc*NSH Shakhov records in the arithmetic type (predictor / level n)
  double *gradW;             // nc*8
  double *ghostW;            // nf*4
  double *fsum;              // nf*NFS
  double *fpar;              // nf*NFP (double)
  void *fparT;               // nf*NFP in the arithmetic type
  double *fflux;             // nf*4 S * macro flux (L -> R / outward)
  double *gam;               // nf spectral radius Gamma
  double *wall_loads;        // nblocks*4
  double *torque_io;         // nblocks*3: torque centres (2 per block), torques
  int *wall_faces;           // ids of the wall faces, ascending
  int nwall;
  // overset
  int *node_active;          // nn
  int *cls;                  // nc scratch classification
  int *donors;               // nc*5
  double *dwgt;              // nc*5
  int fbf;                   // f stored as bf16 pairs (FP32 arithmetic)
  int *rec_list;             // receptor cells, ascending (compacted on the device)
  int *fresh_list;           // cells uncovered by the motion, ascending
  int *conn_cnt;             // 8 counters: receptors, fresh, field, hole, orphans
  int4 *conn_chunk;          // per 1024-cell chunk: receptors, fresh, field, other
  int cap_interp;            // capacity of the lists' interpolation staging
  void *itmp;                // interpolation staging: cap_interp*nvp pairs
  double *itmpW;             // ... *6 doubles
  int *wall_seg;             // segments: node id pairs, grouped per block
  float4 *segf;              // float endpoints of each wall segment (assembly filters)
  int nseg;
  int *wall_seg_off;         // nblocks+1
  int *body_ring;            // body polygon node ids, grouped per block
  int *body_ring_off;        // nblocks+1
  float4 *body_bb;           // nblocks: outward-rounded float box of the body polygon
  const int *cell_off;       // nblocks+1 (device copy)
  const int *node_off;       // nblocks+1
  const int *blk_info;       // nblocks*8: ni, nj, periodic, priority, n_fringe, n_gap, bc-overset mask, body?
  // overset search bins (per block uniform grid, CSR of cell ids)
  double *bin_geo;           // nblocks*4: x0, y0, 1/hx, 1/hy
  int *bin_dim;              // nblocks*3: nbx, nby, first bin
  int *bin_cnt, *bin_start;  // nbins, nbins+1
  int *bin_items;            // bin_cap
  int nbins, bin_cap;
  const int *tiles;          // ntiles*3: block, i0, j0 of the 8x8 cell tiles
  int ntiles;
  int *err;                  // error flags
  int wait_polls;            // bounded waits (sweeps): polls before giving up (EF_TIMEOUT)
  double *mpart;             // MET_NQ*MET_BLOCKS per-block partial sums of the step metrics
  double *mout;              // MET_NQ step metrics of the last metered step
};

// Step metrics (sums over the solved cells, fixed-order reductions):
// squared norms of the macro residual R and the micro residual r of the last
// inner iteration, of the Step-7 moment fix W^{s+1} - W', and the totals of
// Omega^{n+1} W.
enum { MET_R2 = 0, MET_RMICRO2 = 1, MET_FIX2 = 2, MET_TOT = 3, MET_NQ = 7 };
constexpr int MET_BLOCKS = 304, MET_THREADS = 256;

// Polls of a bounded wait before it gives up; the drain of a CTA's own copies
// after a timeout always uses the default.
constexpr int kWaitPolls = 1 << 21;

// face geometry record / per-cell sweep record
enum { FG_SNX = 0, FG_SNY, FG_SUN, FG_UFX, FG_UFY, FG_DXLX, FG_DXLY, FG_DXRX, FG_DXRY, NFG = 12 };
// sweep record: per face slot s, outward (S n_x, S n_y, S U.n) at 3 s; the
// micro-sweep diagonal base at SR_DBASE and the neighbour mask (int bits) at
// SR_MASK; 16 values so a record is a whole number of 16-byte chunks
enum { SR_DBASE = 12, SR_MASK = 13, NSR = 16 };

// values per cell of the macro-sweep record (FP64 packed, FP32 padded to 256 B)
enum { NMR = 41, NMR32 = 64 };

// per-cell parameter record (from W' or W^n)
enum { CP_RHO = 0, CP_UX, CP_UY, CP_LAM, CP_QX, CP_QY, CP_ITAU, CP_DBASE, NCP = 8 };

// Shakhov record in the arithmetic type from a cell record (double)
template <typename T>
__device__ __forceinline__ void write_shrec(const Dev &d, const double *o, double vol, T *r) {
  double il = 1.0 / (2.0 * o[CP_LAM]);
  r[SH_HPRE] = (T)(o[CP_RHO] * o[CP_LAM] * M_1_PI);
  r[SH_UX] = (T)o[CP_UX];
  r[SH_UY] = (T)o[CP_UY];
  r[SH_LAM] = (T)o[CP_LAM];
  r[SH_QX] = (T)o[CP_QX];
  r[SH_QY] = (T)o[CP_QY];
  r[SH_PREF] = (T)(4.0 * (1.0 - d.Pr) * o[CP_LAM] * o[CP_LAM] / (5.0 * o[CP_RHO]));
  r[SH_IL] = (T)il;
  r[SH_ITAU] = (T)o[CP_ITAU];
  r[SH_VOL] = (T)vol;
}

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type ldf(const void *base, size_t idx) {
  return reinterpret_cast<const typename Vec2<T>::type *>(base)[idx];
}
template <typename T>
__device__ __forceinline__ void stf(void *base, size_t idx, T h, T b) {
  typename Vec2<T>::type v;
  v.x = h;
  v.y = b;
  reinterpret_cast<typename Vec2<T>::type *>(base)[idx] = v;
}

// The distribution f in its storage type: the arithmetic type's pair, or on
// the BF16-storage path (FP32 arithmetic) a bf16 pair rounded to nearest on
// store and widened exactly on load.  FB = 1 / 0 fixes the storage at
// compile time (the hot kernels are instantiated for both); FB = -1 reads
// d.fbf at run time.
template <typename T, int FB = -1>
__device__ __forceinline__ typename Vec2<T>::type ldF(const Dev &d, size_t idx) {
  if (sizeof(T) == 4 && (FB == 1 || (FB < 0 && d.fbf))) {
    float2 w = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(d.f)[idx]);
    return typename Vec2<T>::type{(T)w.x, (T)w.y};
  }
  return ldf<T>(d.f, idx);
}
template <typename T, int FB = -1> __device__ __forceinline__ void stF(const Dev &d, size_t idx, T h, T b) {
  if (sizeof(T) == 4 && (FB == 1 || (FB < 0 && d.fbf)))
    reinterpret_cast<__nv_bfloat162 *>(d.f)[idx] = __floats2bfloat162_rn((float)h, (float)b);
  else
    stf<T>(d.f, idx, h, b);
}

// Asynchronous global -> shared copies (cp.async, sm_80+): a per-thread
// prefetch ring for the streaming inputs of the wavefront sweeps.
template <int BYTES> __device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// float -> double on the integer pipes, from the IEEE 754 layouts (sign;
// exponent rebiased by 1023 - 127; 23-bit fraction shifted into the 52-bit
// one): exact for normal numbers, zero and subnormals give signed zero,
// infinities and NaNs are kept.  The FP64 pipe of this GPU retires a warp
// instruction in tens of cycles, so per-face and per-cell conversions go
// through here.
__device__ __forceinline__ double f2d_bits(float x) {
  unsigned u = __float_as_uint(x);
  unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi, lo;
  if (e == 0u) { hi = sign; lo = 0u; }
  else if (e == 0xffu) { hi = sign | 0x7ff00000u | (m >> 3); lo = (m & 7u) << 29; }
  else { hi = sign | ((e + 896u) << 20) | (m >> 3); lo = (m & 7u) << 29; }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_bits(x); }

// mbarrier and bulk (TMA engine) copies, shared::cta addresses
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes)
               : "memory");
}
// raise the expected transaction bytes of the current phase (no arrival)
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mb, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *mb) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mb)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a phase of an mbarrier with at most `polls` polls; false (and
// EF_TIMEOUT in *err) when the limit runs out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mb, unsigned parity, int *err, int polls = kWaitPolls) {
  for (int n = 0; n < polls; ++n)
    if (mbar_try_wait(mb, parity)) return true;
  atomicOr(err, EF_TIMEOUT);
  return false;
}
// global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mb))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

template <typename T> __device__ __forceinline__ T dvx(const Dev &d, int k);
template <> __device__ __forceinline__ double dvx<double>(const Dev &d, int k) { return d.vx[k]; }
template <> __device__ __forceinline__ float dvx<float>(const Dev &d, int k) { return d.vxf[k]; }
template <typename T> __device__ __forceinline__ T dvy(const Dev &d, int k);
template <> __device__ __forceinline__ double dvy<double>(const Dev &d, int k) { return d.vy[k]; }
template <> __device__ __forceinline__ float dvy<float>(const Dev &d, int k) { return d.vyf[k]; }
template <typename T> __device__ __forceinline__ T dw(const Dev &d, int k);
template <> __device__ __forceinline__ double dw<double>(const Dev &d, int k) { return d.w[k]; }
template <> __device__ __forceinline__ float dw<float>(const Dev &d, int k) { return d.wf[k]; }
// the whole velocity grid (k < nv_all), also on a sharded context
template <typename T> __device__ __forceinline__ T dvxa(const Dev &d, int k);
template <> __device__ __forceinline__ double dvxa<double>(const Dev &d, int k) { return d.vxa[k]; }
template <> __device__ __forceinline__ float dvxa<float>(const Dev &d, int k) { return d.vxaf[k]; }
template <typename T> __device__ __forceinline__ T dvya(const Dev &d, int k);
template <> __device__ __forceinline__ double dvya<double>(const Dev &d, int k) { return d.vya[k]; }
template <> __device__ __forceinline__ float dvya<float>(const Dev &d, int k) { return d.vyaf[k]; }
template <typename T> __device__ __forceinline__ T dwa(const Dev &d, int k);
template <> __device__ __forceinline__ double dwa<double>(const Dev &d, int k) { return d.wa[k]; }
template <> __device__ __forceinline__ float dwa<float>(const Dev &d, int k) { return d.waf[k]; }

// value of the cell field f at velocity k for neighbour slot `s` of cell c
// (cell neighbour or ghost Maxwellian of the ghost state)
template <typename T>
__device__ __forceinline__ V2<T> nb_value(const Dev &d, int c, int s, int k) {
  int kind = d.nb_kind[c * 4 + s];
  int id = d.nb_id[c * 4 + s];
  if (kind == NB_CELL) {
    auto v = ldF<T>(d, (size_t)id * d.nvp + k);
    return {v.x, v.y};
  }
  const double *g = d.ghostW + 4 * id;
  Prim p = primitive(g, d.Keff);
  return maxwellian<T>((T)p.rho, (T)p.ux, (T)p.uy, (T)p.lam, dvx<T>(d, k), dvy<T>(d, k),
                       (T)d.Keff);
}

// Limited Cartesian gradient of (h, b) of cell c at velocity k (reading R1:
// van Leer on both-sided centre differences, one-sided where a side has no
// neighbour, mapped with the inverse Jacobian of the centre differences).
template <typename T>
__device__ __forceinline__ void grad_f(const Dev &d, int c, int k, V2<T> fc, V2<T> &gx,
                                       V2<T> &gy) {
  int fl = d.slope_flags[c];
  V2<T> s[2];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    int cs = (fl >> (2 * dir)) & 3;
    V2<T> r = {T(0), T(0)};
    if (cs == SL_BOTH) {
      V2<T> m = nb_value<T>(d, c, 2 * dir, k), p = nb_value<T>(d, c, 2 * dir + 1, k);
      r.h = vanleer<T>(fc.h - m.h, p.h - fc.h);
      r.b = vanleer<T>(fc.b - m.b, p.b - fc.b);
    } else if (cs == SL_P) {
      V2<T> p = nb_value<T>(d, c, 2 * dir + 1, k);
      r.h = p.h - fc.h;
      r.b = p.b - fc.b;
    } else if (cs == SL_M) {
      V2<T> m = nb_value<T>(d, c, 2 * dir, k);
      r.h = fc.h - m.h;
      r.b = fc.b - m.b;
    }
    s[dir] = r;
  }
  const double *J = d.jinv + 4 * c;
  T i11 = (T)J[0], i12 = (T)J[1], i21 = (T)J[2], i22 = (T)J[3];
  gx.h = i11 * s[0].h + i12 * s[1].h;
  gx.b = i11 * s[0].b + i12 * s[1].b;
  gy.h = i21 * s[0].h + i22 * s[1].h;
  gy.b = i21 * s[0].b + i22 * s[1].b;
}

// Copy a record of N values (N * sizeof(T) a multiple of 16, 16-byte aligned)
// into registers with 128-bit loads.
template <typename T, int N> __device__ __forceinline__ void load_rec(const T *src, T *dst) {
  static_assert((N * sizeof(T)) % 16 == 0, "record size");
  const float4 *s = reinterpret_cast<const float4 *>(src);
  float4 *o = reinterpret_cast<float4 *>(dst);
#pragma unroll
  for (int q = 0; q < (int)(N * sizeof(T) / 16); ++q) o[q] = __ldg(s + q);
}

template <typename T> __device__ __forceinline__ const T *fparT(const Dev &d, int f) {
  return reinterpret_cast<const T *>(d.fparT) + (size_t)f * NFP;
}

// Bivariate polynomials sum_{a+b<=D} c_ab cx^a cy^b, coefficients stored
// degree-major (index (a+b)(a+b+1)/2 + b), for the equilibrium parts of the
// interface flux: on the tensor velocity grid every such term is the face
// Maxwellian times a polynomial in c = v - U0.
template <int D, typename R = float> struct Poly2 {
  static constexpr int N = (D + 1) * (D + 2) / 2;
  R c[N];
  __host__ __device__ static constexpr int idx(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }
};
template <int D, typename R = float> __device__ __forceinline__ Poly2<D, R> p2_zero() {
  Poly2<D, R> r;
#pragma unroll
  for (int i = 0; i < Poly2<D, R>::N; ++i) r.c[i] = R(0);
  return r;
}
// a0 + ax cx + ay cy
template <typename R = float> __device__ __forceinline__ Poly2<1, R> p2_lin(R a0, R ax, R ay) {
  Poly2<1, R> r;
  r.c[0] = a0; r.c[Poly2<1, R>::idx(1, 0)] = ax; r.c[Poly2<1, R>::idx(0, 1)] = ay;
  return r;
}
template <int D1, int D2, typename R>
__device__ __forceinline__ Poly2<D1 + D2, R> p2_mul(const Poly2<D1, R> &x, const Poly2<D2, R> &y) {
  Poly2<D1 + D2, R> r = p2_zero<D1 + D2, R>();
#pragma unroll
  for (int s1 = 0; s1 <= D1; ++s1)
#pragma unroll
    for (int b1 = 0; b1 <= s1; ++b1)
#pragma unroll
      for (int s2 = 0; s2 <= D2; ++s2)
#pragma unroll
        for (int b2 = 0; b2 <= s2; ++b2)
          r.c[Poly2<D1 + D2, R>::idx(s1 - b1 + s2 - b2, b1 + b2)] +=
              x.c[Poly2<D1, R>::idx(s1 - b1, b1)] * y.c[Poly2<D2, R>::idx(s2 - b2, b2)];
  return r;
}
// alpha x + beta y (degrees D1 <= D2)
template <int D1, int D2, typename R>
__device__ __forceinline__ Poly2<D2, R> p2_axpby(R alpha, const Poly2<D1, R> &x, R beta, const Poly2<D2, R> &y) {
  Poly2<D2, R> r;
#pragma unroll
  for (int i = 0; i < Poly2<D2, R>::N; ++i) r.c[i] = beta * y.c[i] + (i < Poly2<D1, R>::N ? alpha * x.c[i] : R(0));
  return r;
}
// sum_ab c_ab Mx[a] My[b]
template <int D, typename R>
__device__ __forceinline__ R p2_sum(const Poly2<D, R> &x, const R *Mx, const R *My) {
  R s = R(0);
#pragma unroll
  for (int t = 0; t <= D; ++t)
#pragma unroll
    for (int b = 0; b <= t; ++b) s += x.c[Poly2<D, R>::idx(t - b, b)] * (Mx[t - b] * My[b]);
  return s;
}
// value at (x, y) of a cubic in the layout above (Horner, 9 fused multiply-adds)
template <typename R> __device__ __forceinline__ R poly3_at(const R *c, R x, R y) {
  R yy = c[0] + y * (c[2] + y * (c[5] + y * c[9]));
  R u = c[1] + y * (c[4] + y * c[8]);
  R w = c[3] + y * c[7] + x * c[6];
  return yy + x * (u + x * w);
}

// Equilibrium factors of the time-integrated interface distribution (Eq.
// fullSolution averaged over dt_s, Shakhov g0+ of Sec. 2.1) as cubics in
// c = v - U0 from a face record P: the interface distribution of one
// velocity is
//   h: q1 f + q2 w.grad f + H ih(c),   b: q1 f_b + q2 w.grad f_b + H ib(c),
// with H = rho0 lam0/pi exp(-lam0 c^2): ih = q3 (1 + g0+/g0) + q4 (w.(a.Psi))
// + q5 (A.Psi) in reduced form, ib the same for b (including its B/H =
// Keff/(2 lam0) factor).
template <typename R>
__device__ __forceinline__ void interface_polys(const R *P, R Keff, R Kint, Poly2<3, R> &ih, Poly2<3, R> &ib) {
  R ux = P[FP_UX], uy = P[FP_UY], lam = P[FP_LAM], il = P[FP_IL];
  const R *ax = P + FP_AX, *ay = P + FP_AY, *at = P + FP_AT;
  Poly2<1, R> vxp = p2_lin<R>(ux, R(1), R(0)), vyp = p2_lin<R>(uy, R(0), R(1));
  Poly2<2, R> v2 = p2_axpby(R(1), p2_mul(vxp, vxp), R(1), p2_mul(vyp, vyp));
  Poly2<2, R> c2 = p2_zero<2, R>();
  c2.c[Poly2<2, R>::idx(2, 0)] = R(1);
  c2.c[Poly2<2, R>::idx(0, 2)] = R(1);
  auto slope = [&](const R *s) {     // s0 + s1 vx + s2 vy + s3 v^2 / 2
    Poly2<2, R> r = p2_axpby(s[1], vxp, R(0.5) * s[3], v2);
    r = p2_axpby(s[2], vyp, R(1), r);
    r.c[0] += s[0];
    return r;
  };
  Poly2<2, R> bx = slope(ax), by = slope(ay), bt = slope(at);
  Poly2<1, R> wxp = p2_lin<R>(ux - P[FP_UFX], R(1), R(0)), wyp = p2_lin<R>(uy - P[FP_UFY], R(0), R(1));
  R eh = P[FP_EH], eb = P[FP_EB];
  Poly2<2, R> bxh = bx, byh = by, bxb = bx, byb = by;
  bxh.c[0] += ax[3] * eh; byh.c[0] += ay[3] * eh;
  bxb.c[0] += ax[3] * eb; byb.c[0] += ay[3] * eb;
  Poly2<3, R> sgh = p2_axpby(R(1), p2_mul(wxp, bxh), R(1), p2_mul(wyp, byh));
  Poly2<3, R> sgb = p2_axpby(R(1), p2_mul(wxp, bxb), R(1), p2_mul(wyp, byb));
  Poly2<2, R> sth = bt, stb = bt;
  sth.c[0] += at[3] * eh;
  stb.c[0] += at[3] * eb;
  Poly2<1, R> pc = p2_lin<R>(R(0), P[FP_PREF] * P[FP_QX], P[FP_PREF] * P[FP_QY]);
  Poly2<2, R> th = p2_axpby(R(0), c2, R(2) * lam, c2);
  th.c[0] -= R(4);                                        // 2 lam c^2 - 4
  Poly2<2, R> tb = p2_axpby(R(0), c2, R(2) * lam * Keff * il, c2);
  tb.c[0] += (-R(2) * Keff - R(2) * Kint) * il;           // ((2 lam c^2 - 2) Keff - 2 Kint) / (2 lam)
  R q3 = P[FP_Q3], q4 = P[FP_Q4], q5 = P[FP_Q5];
  ih = p2_axpby(q3, p2_mul(pc, th), q4, sgh);
  ih = p2_axpby(q5, sth, R(1), ih);
  ih.c[0] += q3;
  R kil = Keff * il;
  ib = p2_axpby(q3, p2_mul(pc, tb), q4 * kil, sgb);
  ib = p2_axpby(q5 * kil, stb, R(1), ib);
  ib.c[0] += q3 * kil;
}

// Store the two cubics into a face record (FP_IH, FP_IB).
template <typename R> __device__ __forceinline__ void store_polys(R *P, const Poly2<3, R> &ih, const Poly2<3, R> &ib) {
#pragma unroll
  for (int m = 0; m < 10; ++m) { P[FP_IH + m] = ih.c[m]; P[FP_IB + m] = ib.c[m]; }
}

// S * time-averaged interface flux of velocity k through face fid, oriented
// along the face normal (L -> R, outward for boundary faces).
template <typename T> __device__ V2<T> face_flux(const Dev &d, int fid, int k) {
  T vx = dvx<T>(d, k), vy = dvy<T>(d, k);
  T wS = vx * (T)d.Sn[2 * fid] + vy * (T)d.Sn[2 * fid + 1] - (T)d.SUn[fid];
  const T *P = fparT<T>(d, fid);
  int kind = d.face_kind[fid];
  int L = d.face_L[fid];
  T ufx = P[FP_UFX], ufy = P[FP_UFY];
  T wx = vx - ufx, wy = vy - ufy;
  V2<T> ff, wgf;
  if (kind == BC_WALL) {
    if (!(wS > T(0))) {
      // reflected part: wall Maxwellian at the face velocity (Eq. maxWalldes)
      T lw = P[FP_LAMW];
      T Hw = P[FP_RHOW] * (lw * T(M_1_PI)) * r_exp<T>(-lw * (wx * wx + wy * wy));
      return {wS * Hw, wS * (T)d.Keff / (T(2) * lw) * Hw};
    }
    auto fv = ldF<T>(d, (size_t)L * d.nvp + k);
    V2<T> fc = {fv.x, fv.y}, gx, gy;
    grad_f<T>(d, L, k, fc, gx, gy);
    T dx = (T)(d.xf[2 * fid] - d.xc[2 * L]), dy = (T)(d.xf[2 * fid + 1] - d.xc[2 * L + 1]);
    ff = {fc.h + dx * gx.h + dy * gy.h, fc.b + dx * gx.b + dy * gy.b};
    wgf = {wx * gx.h + wy * gy.h, wx * gx.b + wy * gy.b};
  } else {
    int R = d.face_R[fid];
    bool useL = wS > T(0), useR = wS < T(0);
    V2<T> fL = {0, 0}, fR = {0, 0}, gL = {0, 0}, gR = {0, 0};
    if (!useR) {
      auto fv = ldF<T>(d, (size_t)L * d.nvp + k);
      V2<T> fc = {fv.x, fv.y}, gx, gy;
      grad_f<T>(d, L, k, fc, gx, gy);
      double sh = (double)d.face_shiftL[fid];
      T dx = (T)(d.xf[2 * fid] - (d.xc[2 * L] + sh * d.period[2 * L]));
      T dy = (T)(d.xf[2 * fid + 1] - (d.xc[2 * L + 1] + sh * d.period[2 * L + 1]));
      fL = {fc.h + dx * gx.h + dy * gy.h, fc.b + dx * gx.b + dy * gy.b};
      gL = {wx * gx.h + wy * gy.h, wx * gx.b + wy * gy.b};
    }
    if (!useL) {
      if (R >= 0) {
        auto fv = ldF<T>(d, (size_t)R * d.nvp + k);
        V2<T> fc = {fv.x, fv.y}, gx, gy;
        grad_f<T>(d, R, k, fc, gx, gy);
        T dx = (T)(d.xf[2 * fid] - d.xc[2 * R]), dy = (T)(d.xf[2 * fid + 1] - d.xc[2 * R + 1]);
        fR = {fc.h + dx * gx.h + dy * gy.h, fc.b + dx * gx.b + dy * gy.b};
        gR = {wx * gx.h + wy * gy.h, wx * gx.b + wy * gy.b};
      } else {
        const double *g = d.ghostW + 4 * fid;
        Prim p = primitive(g, d.Keff);
        fR = maxwellian<T>((T)p.rho, (T)p.ux, (T)p.uy, (T)p.lam, vx, vy, (T)d.Keff);
      }
    }
    if (useL) {
      ff = fL; wgf = gL;
    } else if (useR) {
      ff = fR; wgf = gR;
    } else {
      ff = {T(0.5) * (fL.h + fR.h), T(0.5) * (fL.b + fR.b)};
      wgf = {T(0.5) * (gL.h + gR.h), T(0.5) * (gL.b + gR.b)};
    }
  }
  V2<T> I = interface_integral<T>(P, vx, vy, ff, wgf, (T)d.Keff, (T)d.Kint, (T)d.Pr);
  return {wS * I.h, wS * I.b};
}

// D_ik = sum over the faces of cell c of S F_hat (outward positive).
template <typename T> __device__ V2<T> flux_div(const Dev &d, int c, int k) {
  V2<T> acc = {T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int fid = d.cell_faces[c * 4 + s];
    int kind = d.face_kind[fid];
    if (kind == BC_OVERSET) continue;   // outer edge of a component grid: receptors only
    V2<T> F = face_flux<T>(d, fid, k);
    T sg = (T)d.cell_sgn[c * 4 + s];
    acc.h += sg * F.h;
    acc.b += sg * F.b;
  }
  return acc;
}

}  // namespace ugks
